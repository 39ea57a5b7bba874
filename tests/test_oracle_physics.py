"""Pins of the oracle's time step against closed forms and invariants.

Each test fixes part of the oracle by something other than the oracle:
an exact discrete solution obtained independently (DFT), a continuum closed
form (tanh interface, Eshelby inclusion, J2 bilinear response), an invariant
of the equations (mass balance, free-energy decrease) or a result the paper
prints (lever rule, Sec. 4.1).
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import inputs, workloads

NOFLUX = dict(D_O_s=0.0, D_O_g=0.0, D_H_s=0.0, D_H_g=0.0, D_W_s=0.0, D_W_g=0.0)


def _strip(profile_w, ny=2, xO=0.0):
    nx = profile_w.size
    pw = np.tile(profile_w, (ny, 1))
    return {"phi_f": 1.0 - pw, "phi_w": pw, "xO": np.full((ny, nx), xO),
            "xH": np.zeros((ny, nx)), "xW": np.zeros((ny, nx))}


@pytest.mark.parametrize("delta", [2.0, 4.0])
def test_tanh_interface(orc, delta):
    """Binary interface without chemistry relaxes to phi = (1 + tanh(x/delta))/2,
    delta = sqrt(2 eps / w) (Sec. 2.2 interface energy with m(x) = x^2 (1-x)^2);
    the discrete profile error is O(dx^2 / delta^2)."""
    w = 1.2379e-3
    eps = 0.5 * delta ** 2 * w
    nx = int(16 * delta)
    prm = workloads.params(c_chem=0.0, k_for=0.0, mechanics=0, eps_phi=eps, w=w, **NOFLUX)
    x = np.arange(nx) + 0.5
    a, b = nx / 4.0, 3.0 * nx / 4.0
    pf = ((x > a) & (x < b)).astype(float)
    s = orc.Sim(_strip(1.0 - pf), prm)
    relax = delta ** 2 / (prm["L"] * eps)          # relaxation time of the profile
    s.step(int(12 * relax / s.dt))
    prof = s.phi_f[0]
    sel = np.abs(x - a) < 4 * delta
    ex = 0.5 * (1.0 + np.tanh((x - a) / delta))
    err = np.abs(prof[sel] - ex[sel]).max()
    # second-order discretisation error: ~0.03 (dx/delta)^2 measured bound
    assert err < 0.05 / delta ** 2
    from scipy.optimize import curve_fit
    popt, _ = curve_fit(lambda xx, c, d: 0.5 * (1 + np.tanh((xx - c) / d)), x[sel], prof[sel], p0=[a, delta])
    assert abs(popt[1] - delta) / delta < 0.12 / delta ** 2    # second order: ~0.095 / delta^2
    assert abs(popt[0] - a) < 1e-6                 # symmetric profile stays centred
    # gas stays exactly absent
    assert np.abs(1.0 - s.phi_f - s.phi_w).max() < 1e-13


def _interface_error(orc, delta):
    w = 1.2379e-3
    eps = 0.5 * delta ** 2 * w
    nx = int(16 * delta)
    prm = workloads.params(c_chem=0.0, k_for=0.0, mechanics=0, eps_phi=eps, w=w, **NOFLUX)
    x = np.arange(nx) + 0.5
    a, b = nx / 4.0, 3.0 * nx / 4.0
    s = orc.Sim(_strip(1.0 - ((x > a) & (x < b)).astype(float)), prm)
    s.step(int(12 * delta ** 2 / (prm["L"] * eps) / s.dt))
    sel = np.abs(x - a) < 4 * delta
    return np.abs(s.phi_f[0][sel] - 0.5 * (1.0 + np.tanh((x[sel] - a) / delta))).max()


def test_tanh_interface_second_order(orc):
    """The relaxed discrete interface converges to the tanh profile at second
    order in dx / delta: halving dx / delta divides the error by ~4."""
    e = [_interface_error(orc, d) for d in (2.0, 4.0, 8.0)]
    assert all(3.5 < e[i] / e[i + 1] < 4.5 for i in range(2)), e


def _dft_heat(u0, D, dt, n):
    """Exact discrete solution of explicit Euler for u_t = D Lap_h u, periodic."""
    k = [2 * np.pi * np.fft.fftfreq(m) for m in u0.shape]
    grids = np.meshgrid(*k, indexing="ij")
    lam = sum(2.0 - 2.0 * np.cos(g) for g in grids)
    return np.real(np.fft.ifftn(np.fft.fftn(u0) * (1.0 - dt * D * lam) ** n))


@pytest.mark.parametrize("shape", [(48, 64), (12, 14, 16)])
def test_gaussian_diffusion_exact(orc, shape):
    """Hydrogen diffusion with constant D and no reaction is the explicit heat
    equation; every DFT mode decays by (1 - dt D lambda_k)^n exactly."""
    D = 0.3
    rng = np.random.default_rng(1)
    f = inputs.core_shell(shape, 6.0, 2.0)
    axes = [np.arange(m) + 0.5 - m / 2.0 for m in shape]
    g = np.meshgrid(*axes, indexing="ij")
    r2 = sum(a * a for a in g)
    f["xH"] = 0.01 * np.exp(-r2 / (2 * 3.0 ** 2)) + 1e-4 * rng.standard_normal(shape)
    f["mask"] = np.zeros(shape, np.uint8)
    prm = workloads.params(k_for=0.0, mechanics=0, D_H_s=D, D_H_g=D)
    s = orc.Sim(f, prm)
    n = 150
    u0 = f["xH"].copy()
    s.step(n)
    ref = _dft_heat(u0, D, s.dt, n)
    assert np.abs(s.f["xH"] - ref).max() < 1e-12 * np.abs(u0).max()


def test_gaussian_diffusion_continuum(orc):
    """Continuum pin: variance grows by 2 D t per axis (to O(dx^2 / s0^2))."""
    D = 0.25
    shape = (96, 96)
    axes = [np.arange(m) + 0.5 - m / 2.0 for m in shape]
    gy, gx = np.meshgrid(*axes, indexing="ij")
    s0 = 4.0
    f = inputs.core_shell(shape, 6.0, 2.0)
    f["xH"] = np.exp(-(gx ** 2 + gy ** 2) / (2 * s0 ** 2))
    f["mask"] = np.zeros(shape, np.uint8)
    s = orc.Sim(f, workloads.params(k_for=0.0, mechanics=0, D_H_s=D, D_H_g=D))
    n = 400
    s.step(n)
    t = n * s.dt
    u = s.f["xH"]
    var_x = (u * gx ** 2).sum() / u.sum()
    assert abs(var_x - (s0 ** 2 + 2 * D * t)) < 1e-9 * var_x   # exact for the discrete second moment
    peak = u.max() / 1.0
    assert abs(peak - s0 ** 2 / (s0 ** 2 + 2 * D * t)) < 0.01


def _q1_symbol_solve(lam, mu, sig_star, Sbar):
    """Independent periodic solve of the 2D plane-strain Q1 problem with
    homogeneous moduli by Fourier transform (textbook tensor-product symbols):
    1D stiffness 2 - 2 cos k, mass (2 + cos k)/3, first-derivative coupling
    sin kx sin ky; the cell eigenstress enters through the element averages of
    the shape-function gradients."""
    ny, nx = sig_star.shape[:2]
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    s = lambda k: 2 - 2 * np.cos(k)
    m = lambda k: (2 + np.cos(k)) / 3.0
    K11 = (lam + 2 * mu) * s(kx) * m(ky) + mu * m(kx) * s(ky)
    K22 = (lam + 2 * mu) * m(kx) * s(ky) + mu * s(kx) * m(ky)
    K12 = (lam + mu) * np.sin(kx) * np.sin(ky)
    S = [np.fft.fft2(sig_star[..., i]) for i in range(3)]
    ex = np.exp(-1j * kx)
    ey = np.exp(-1j * ky)
    dx = ex - 1.0
    dy = ey - 1.0
    ax = 0.5 * (1.0 + ex)
    ay = 0.5 * (1.0 + ey)
    b1 = dx * ay * S[0] + ax * dy * S[2]
    b2 = ax * dy * S[1] + dx * ay * S[2]
    det = K11 * K22 - K12 * K12
    det[0, 0] = 1.0
    u1 = (K22 * b1 - K12 * b2) / det
    u2 = (K11 * b2 - K12 * b1) / det
    u1[0, 0] = 0.0
    u2[0, 0] = 0.0
    U = np.stack([np.real(np.fft.ifft2(u1)), np.real(np.fft.ifft2(u2))], axis=-1)
    Dm = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    E = np.linalg.solve(Dm, sig_star.reshape(-1, 3).mean(axis=0) + Sbar)
    return U, E


@pytest.mark.parametrize("prestress", [0.0, 0.01])
def test_elasticity_matches_fourier_solution(orc, prestress):
    """Homogeneous moduli: the oracle's Q1 operator, right-hand side, mean-strain
    dofs and PCG agree with an independent Fourier solve to ~rtol * cond."""
    shape = (24, 32)
    rng = np.random.default_rng(7)
    f = inputs.core_shell(shape, 7.0, 3.0)
    f["phi_f"] = np.clip(f["phi_f"] + 0.3 * rng.uniform(size=shape), 0, 1)
    f["phi_w"] = np.zeros(shape)
    prm = workloads.params(E_g_ratio=1.0, cg_rtol=1e-14, cg_maxit=5000, warm_start=0,
                           prestress=prestress)
    s = orc.Sim(f, prm)
    s.mechanics()
    E, nu = 1.0, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    e0 = prm["eig0"] * (f["phi_f"] ** 3 * (6 * f["phi_f"] ** 2 - 15 * f["phi_f"] + 10))
    sig = np.stack([3 * lam * e0 + 2 * mu * e0, 3 * lam * e0 + 2 * mu * e0, np.zeros(shape)], axis=-1)
    U, Eb = _q1_symbol_solve(lam, mu, sig, np.array([-prestress, -prestress, 0.0]))
    u = s.f["u"] - s.f["u"].reshape(-1, 2).mean(axis=0)
    assert np.abs(u - U).max() < 1e-10 * np.abs(U).max()
    assert np.abs(s.f["Ebar"] - Eb).max() < 1e-11


def test_uniform_eigenstrain_prestress_closed_form(orc):
    """Uniform eigenstrain e I (phi_f = 1) and mean stress -p I: u = 0 and the
    plane-strain mean strain solves sigma_xx = sigma_yy = -p with eps_zz = 0."""
    shape = (8, 8)
    f = {"phi_f": np.ones(shape), "phi_w": np.zeros(shape), "xO": np.zeros(shape),
         "xH": np.zeros(shape), "xW": np.zeros(shape)}
    p = 0.013
    prm = workloads.params(prestress=p, cg_rtol=1e-14, warm_start=0)
    s = orc.Sim(f, prm)
    s.mechanics()
    lam = 0.3 / (1.3 * 0.4)
    mu = 1.0 / 2.6
    e = prm["eig0"]
    a = (-p + 3 * lam * e + 2 * mu * e) / (2 * lam + 2 * mu)
    assert np.abs(s.f["u"]).max() < 1e-13
    assert abs(s.f["Ebar"][0] - a) < 1e-13 and abs(s.f["Ebar"][1] - a) < 1e-13
    sg = s.f["sigma"].reshape(-1, 4)
    assert np.abs(sg[:, 0] + p).max() < 1e-13 and np.abs(sg[:, 1] + p).max() < 1e-13


def test_eshelby_disk_plane_strain(orc):
    """Dilatational eigenstrain e in a disk (plane strain, homogeneous moduli):
    uniform interior stress sigma_xx = sigma_yy = -E e / (2 (1 - nu)) in an
    infinite body; with zero mean stress in the periodic box the interior value
    is reduced by the volume fraction f."""
    n = 128
    R = 16.0
    f = inputs.core_shell((n, n), R, 0.0)
    f["phi_f"], f["phi_w"] = f["phi_w"].copy(), np.zeros((n, n))   # inclusion transforms
    prm = workloads.params(E_g_ratio=1.0, cg_rtol=1e-10, warm_start=0)
    s = orc.Sim(f, prm)
    s.mechanics()
    e = prm["eig0"]
    frac = np.pi * R * R / (n * n)
    ref = -1.0 * e / (2 * (1 - 0.3)) * (1 - frac)
    sg = s.f["sigma"]
    c = sg[n // 2 - 3:n // 2 + 3, n // 2 - 3:n // 2 + 3]
    assert np.abs(c[..., 0] - ref).max() < 0.02 * abs(ref)
    assert np.abs(c[..., 1] - ref).max() < 0.02 * abs(ref)
    assert np.abs(c[..., 3]).max() < 1e-3 * abs(ref)


def test_eshelby_sphere(orc):
    """Sphere: uniform interior stress -2 E e / (3 (1 - nu)) I (infinite body),
    reduced by the volume fraction in the periodic box with zero mean stress."""
    n = 32
    R = 6.0
    f = inputs.core_shell((n, n, n), R, 0.0, delta=1.5)
    f["phi_f"], f["phi_w"] = f["phi_w"].copy(), np.zeros((n, n, n))
    prm = workloads.params(E_g_ratio=1.0, cg_rtol=1e-8, warm_start=0)
    s = orc.Sim(f, prm)
    s.mechanics()
    e = prm["eig0"]
    frac = 4.0 / 3.0 * np.pi * R ** 3 / n ** 3
    ref = -2.0 * e / (3 * (1 - 0.3)) * (1 - frac)
    c = s.f["sigma"][n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1]
    for i in range(3):
        assert np.abs(c[..., i] - ref).max() < 0.04 * abs(ref)


def test_free_energy_decreases(orc):
    """Without reaction, supply cells or mechanics the step is a (projected)
    gradient flow of the free energy (Sec. 2.3: non-negative dissipation), so the
    discrete free energy never increases for dt within the stable limit."""
    f = inputs.core_shell((40, 40), 12.0, 4.0)
    f["mask"] = np.zeros((40, 40), np.uint8)
    s = orc.Sim(f, workloads.params(k_for=0.0, mechanics=0))
    F = [s.free_energy()]
    for _ in range(150):
        s.step(1)
        F.append(s.free_energy())
    dF = np.diff(F)
    assert np.all(dF <= 1e-12 * abs(F[0]))
    assert F[-1] < F[0]


def test_mass_balance_periodic(orc):
    """Reaction O + 2H -> H2O with flux-form transport (Sec. 2.4 field relations):
    sum(x_O + x_H2O) and sum(x_H + 2 x_H2O) are conserved to roundoff."""
    f = inputs.core_shell((32, 32), 10.0, 3.0)
    f["mask"] = np.zeros((32, 32), np.uint8)
    s = orc.Sim(f, workloads.params(cg_rtol=1e-8))
    a0 = s.sums()
    s.step(40)
    a1 = s.sums()
    o0, o1 = a0[0] + a0[2], a1[0] + a1[2]
    h0, h1 = a0[1] + 2 * a0[2], a1[1] + 2 * a1[2]
    assert abs(o1 - o0) < 1e-13 * o0
    assert abs(h1 - h0) < 1e-13 * h0
    assert a1[2] > 0.0                       # water was produced


def test_mass_balance_with_supply(orc):
    """With supply cells the balance closes once the removed water and the
    supplied hydrogen are counted (Sec. 4.3 open channels)."""
    f = inputs.core_shell((32, 32), 10.0, 3.0)
    s = orc.Sim(f, workloads.params(cg_rtol=1e-8))
    a0 = s.sums()
    s.step(40)
    a1 = s.sums()
    o0 = a0[0] + a0[2]
    o1 = a1[0] + a1[2] + s.removedW
    h0 = a0[1] + 2 * a0[2]
    h1 = a1[1] + 2 * a1[2] + 2 * s.removedW - s.suppliedH
    assert abs(o1 - o0) < 1e-13 * o0
    assert abs(h1 - h0) < 1e-13 * h0


@pytest.mark.parametrize("x0", [0.25, 0.4])
def test_lever_rule(orc, x0):
    """Sec. 4.1 benchmark: ferrite and wuestite at mean oxygen fraction x0, no
    reaction or mechanics.  At equilibrium the bulk phases sit at the common-
    tangent compositions of the printed polynomials (x_f = 0.010065,
    x_w = 0.517126) and the wuestite fraction follows the lever rule
    (x0 - x_f) / (x_w - x_f), up to the diffuse-interface width over the box
    length.  The interfaces start displaced by 4 cells from the lever
    positions; a wide interface (eps = 1.6) keeps them off the grid scale."""
    xf, xw = 0.010065, 0.517126
    nx = 128
    lever = (x0 - xf) / (xw - xf)
    half = lever * nx / 2 + 4
    x = np.arange(nx) + 0.5
    width = np.sqrt(1.6 / 0.05)
    pw = 0.5 * (np.tanh((x - (nx / 2 - half)) / width) - np.tanh((x - (nx / 2 + half)) / width))
    xO = xf + (xw - xf) * pw
    f = _strip(pw)
    f["xO"] = np.tile(xO + (x0 - xO.mean()), (2, 1))
    prm = workloads.params(k_for=0.0, mechanics=0, D_O_s=1.0, D_O_g=1.0, L=0.05,
                           eps_phi=1.6, kappa_O=1.6 * 1.25e-5)
    s = orc.Sim(f, prm)
    s.step(45000)
    assert abs(s.phi_w.mean() - lever) < 0.03
    assert abs(s.f["xO"][0, 0] - xf) < 0.01           # bulk ferrite
    assert abs(s.f["xO"][0, nx // 2] - xw) < 0.01      # bulk wuestite (printed 0.571 is 0.054 away)


def _shear_state(orc, prm):
    shape = (2, 2, 2)
    f = {"phi_f": np.zeros(shape), "phi_w": np.ones(shape), "xO": np.zeros(shape),
         "xH": np.zeros(shape), "xW": np.zeros(shape)}
    return orc.Sim(f, prm)


def test_j2_shear_ramp_closed_form(orc):
    """Monotonic simple shear with linear hardening (Sec. 2.3 J2 relations,
    small-strain form): |s| = 2G (e - eps_P) = sqrt(2/3)(sigma_Y + H eps_P),
    e = sqrt(2) eps_xy, so eps_P is linear in e after yield; unloading is
    elastic; the yield function is <= 0 after every return."""
    sy, H = 0.01, 0.05
    prm = workloads.params(plasticity=1, sigma_Y=sy, H_hard=H, eig0=0.0)
    s = _shear_state(orc, prm)
    G = 1.0 / 2.6
    for g in np.linspace(0.0, 0.06, 31):
        s.f["Ebar"][:] = 0.0
        s.f["Ebar"][5] = g                       # engineering shear gamma_xy
        orc.return_map(s)
        e = np.sqrt(2.0) * g / 2.0
        epsP = max(0.0, (2 * G * e - np.sqrt(2.0 / 3.0) * sy) / (2 * G + np.sqrt(2.0 / 3.0) * H))
        assert abs(s.f["alpha"].ravel()[0] - epsP) < 1e-13
        tau = s.f["sigma"].reshape(-1, 6)[0, 5]
        snorm = np.sqrt(2.0) * abs(tau)
        assert snorm - np.sqrt(2.0 / 3.0) * (sy + H * s.f["alpha"].ravel()[0]) < 1e-13
    a_max = s.f["alpha"].ravel()[0]
    # elastic unloading: alpha frozen, stress drops by 2 G d(eps_xy)
    tau0 = s.f["sigma"].reshape(-1, 6)[0, 5]
    s.f["Ebar"][5] = 0.05
    orc.return_map(s)
    assert s.f["alpha"].ravel()[0] == a_max
    assert abs(s.f["sigma"].reshape(-1, 6)[0, 5] - (tau0 - G * 0.01)) < 1e-13


def test_j2_plane_strain_plastic_strain_trace_free(orc):
    """Plastic flow is deviatoric (isochoric F_P in Sec. 2.2): tr eps_p = 0."""
    prm = workloads.params(plasticity=1, sigma_Y=0.005, H_hard=0.01)
    f = inputs.core_shell((24, 24), 8.0, 3.0)
    f["phi_f"] = f["phi_w"].copy()
    f["phi_w"] = np.zeros((24, 24))
    s = orc.Sim(f, workloads.params(plasticity=1, sigma_Y=0.005, H_hard=0.01, cg_rtol=1e-9))
    s.mechanics()
    ep = s.f["eps_p"].reshape(-1, 4)
    assert s.f["alpha"].max() > 0.0
    assert np.abs(ep[:, 0] + ep[:, 1] + ep[:, 2]).max() < 1e-15


@pytest.mark.parametrize("ndim", [2, 3])
def test_j2_uniaxial_strain_ramp(orc, ndim):
    """Monotonic uniaxial strain (eps_xx = e, every other component held at
    zero; in 2D plane strain supplies eps_zz = 0): the mean stress stays the
    elastic K e, the plastic strain is deviatoric along (2, -1, -1)/sqrt(6),
    and after yield the von Mises stress sqrt(3/2)|s| = sigma_xx - sigma_yy
    equals sigma_Y + H alpha (Sec. 2.3 J2 relations, small-strain form).
    Shear alone never exercises the trace split; this path does."""
    sy, H = 0.01, 0.05
    prm = workloads.params(plasticity=1, sigma_Y=sy, H_hard=H, eig0=0.0)
    shape = (2,) * ndim
    f = {"phi_f": np.zeros(shape), "phi_w": np.ones(shape), "xO": np.zeros(shape),
         "xH": np.zeros(shape), "xW": np.zeros(shape)}
    s = orc.Sim(f, prm)
    E, nu = 1.0, 0.3
    K, G = E / (3 * (1 - 2 * nu)), E / (2 * (1 + nu))
    r23 = np.sqrt(2.0 / 3.0)
    npl = 4 if ndim == 2 else 6
    for e in np.linspace(0.0, 0.05, 26):
        s.f["Ebar"][:] = 0.0
        s.f["Ebar"][0] = e
        orc.return_map(s)
        a = max(0.0, (2 * G * e * r23 - r23 * sy) / (2 * G + r23 * H))
        assert abs(s.f["alpha"].ravel()[0] - a) < 1e-13
        sig = s.f["sigma"].reshape(-1, npl)[0]
        sxx, syy, szz = sig[0], sig[1], sig[2]
        assert abs((sxx + syy + szz) / 3.0 - K * e) < 1e-13
        assert abs(sxx - (K * e + 2 * G * (2.0 * e / 3.0 - 2.0 * a / np.sqrt(6.0)))) < 1e-13
        assert abs(syy - szz) < 1e-14
        ep = s.f["eps_p"].reshape(-1, npl)[0]
        assert abs(ep[0] - 2.0 * a / np.sqrt(6.0)) < 1e-14
        assert abs(ep[1] + a / np.sqrt(6.0)) < 1e-14 and abs(ep[2] + a / np.sqrt(6.0)) < 1e-14
        if a > 0.0:
            assert abs((sxx - syy) - (sy + H * a)) < 1e-13
        else:
            assert sxx - syy <= sy + 1e-15


@pytest.mark.parametrize("phase,shape", [("wuestite", (40, 48)), ("gas", (40, 48)), ("wuestite", (10, 12, 14))])
def test_oxygen_single_phase_exact(orc, phase, shape):
    """In one phase with a quadratic chemical energy (wuestite: 173.263 x^2
    + ..., gas: 1000 x^2, Sec. 3.1) the oxygen relation with the un-reduced
    flux j_O = -M_O grad mu_O, mu_O = c f'(x_O) - kappa_O Lap x_O and
    M_O = D_O / (c f'') (R3) is linear: x_t = D_O Lap x - (D_O kappa_O /
    (2 a c)) Lap^2 x.  Explicit Euler then scales every DFT mode by
    (1 - dt (D_O lambda + D_O kappa_O lambda^2 / (2 a c)))^n exactly.  A
    dropped gradient-energy term, a mobility without the 1/f'' factor or
    a sign error in either fails this."""
    a = {"wuestite": 173.263, "gas": 1000.0}[phase]
    kappa = 0.5
    rng = np.random.default_rng(7)
    if phase == "wuestite":
        pf, pw = np.zeros(shape), np.ones(shape)
    else:
        pf, pw = np.zeros(shape), np.zeros(shape)
    x0 = 0.3 + 0.02 * rng.standard_normal(shape)
    f = {"phi_f": pf, "phi_w": pw, "xO": x0.copy(), "xH": np.zeros(shape), "xW": np.zeros(shape),
         "mask": np.zeros(shape, np.uint8)}
    prm = workloads.params(k_for=0.0, mechanics=0, kappa_O=kappa, D_O_s=0.05, D_O_g=0.5)
    s = orc.Sim(f, prm)
    D = prm["D_O_s"] if phase == "wuestite" else prm["D_O_g"]
    c = prm["c_chem"]
    n = 300
    s.step(n)
    k = [2 * np.pi * np.fft.fftfreq(m) for m in shape]
    lam = sum(2.0 - 2.0 * np.cos(g) for g in np.meshgrid(*k, indexing="ij"))
    amp = 1.0 - s.dt * (D * lam + D * kappa * lam ** 2 / (2.0 * a * c))
    assert np.abs(amp[lam > 0]).max() < 1.0          # the oracle's dt is stable here
    # the gradient-energy term is not negligible at the shortest wavelengths
    assert (kappa * lam.max() / (2.0 * a * c)) > 0.1
    ref = np.real(np.fft.ifftn(np.fft.fftn(x0) * amp ** n))
    assert np.abs(s.f["xO"] - ref).max() < 1e-12
    # the solid order parameter does not move in a single phase
    assert np.abs(s.phi_f).max() == 0.0
    # the field moved by far more than the tolerance, so the pin is not vacuous
    assert np.abs(s.f["xO"] - x0).max() > 1e-3
