"""Pins of the finite-strain elastic oracle (oracle/finite_strain.py).

Sec. 2.2 of the paper defines the neo-Hooke energy of the elastic part of
the deformation and the transformation stretch d_T^(1/3).  The tests fix
the oracle by: the stress as the derivative of that energy (central
differences), frame indifference, the small-strain moduli K and G at F = I,
homogeneous states (transformation under plane strain, uniaxial mean
stress) against one-dimensional energy minimisations done independently of
the finite-element solver, the small-strain oracle as the volume change
goes to zero, and the mean-stress condition of the periodic box.
"""
import numpy as np
import pytest
from scipy.optimize import brentq, fsolve

from paper_2111_11538_gb300 import inputs, workloads


@pytest.fixture(scope="module")
def fs(orc):
    from oracle import finite_strain
    return finite_strain


def _rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def test_piola_is_the_energy_derivative(fs):
    rng = np.random.default_rng(0)
    for _ in range(5):
        F = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
        K, G, dT = 0.5 + rng.random(), 0.2 + rng.random(), 0.6 + 0.4 * rng.random()
        P = fs.piola(F[None], np.array([K]), np.array([G]), np.array([dT]))[0]
        e = 1e-6
        for i in range(3):
            for j in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[i, j] += e
                Fm[i, j] -= e
                fd = (fs.psi(Fp[None], K, G, np.array([dT]))[0] - fs.psi(Fm[None], K, G, np.array([dT]))[0]) / (2 * e)
                assert abs(fd - P[i, j]) < 1e-8 * max(1.0, abs(P[i, j]))


def test_frame_indifference(fs):
    """psi(Q F) = psi(F) and P(Q F) = Q P(F) for rotations Q."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        if np.linalg.det(F) <= 0:
            continue
        Q = _rot(rng)
        args = (np.array([1.1]), np.array([0.45]), np.array([0.7]))
        assert abs(fs.psi((Q @ F)[None], *args)[0] - fs.psi(F[None], *args)[0]) < 1e-12
        assert np.abs(fs.piola((Q @ F)[None], *args)[0] - Q @ fs.piola(F[None], *args)[0]).max() < 1e-12


def test_small_strain_moduli(fs):
    """At F = I + eps H (d_T = 1): P = K tr(e) I + 2 G dev(e) + O(eps^2),
    e = sym(eps H), i.e. K and G are the bulk and shear moduli (F2)."""
    rng = np.random.default_rng(2)
    K, G = 0.83, 0.38
    for eps in (1e-3, 1e-4):
        H = rng.standard_normal((3, 3))
        e = eps * 0.5 * (H + H.T)
        lin = K * np.trace(e) * np.eye(3) + 2 * G * (e - np.trace(e) / 3 * np.eye(3))
        P = fs.piola((np.eye(3) + eps * H)[None], np.array([K]), np.array([G]), np.array([1.0]))[0]
        assert np.abs(P - lin).max() < 10 * eps * np.abs(lin).max()
    # the stress-free state of a cell is its transformation stretch
    dT = 0.6
    P = fs.piola((dT ** (1 / 3) * np.eye(3))[None], np.array([K]), np.array([G]), np.array([dT]))[0]
    assert np.abs(P).max() < 1e-15


def _energy_stretches(l1, l2, K, G, dT):
    """Energy of F = diag(l1, l2, 1) written with principal stretches."""
    s = dT ** (-1 / 3)
    JE = s ** 3 * l1 * l2
    I1 = s * s * (l1 * l1 + l2 * l2 + 1.0)
    return dT * (0.25 * K * (JE ** 2 - 1 - 2 * np.log(JE)) + 0.5 * G * (JE ** (-2 / 3) * I1 - 3))


def test_uniform_transformation_plane_strain(fs):
    """Uniform ferrite with Omega = 0.4, no mean stress: the box contracts
    uniformly in plane to the minimiser of the one-dimensional energy
    psi(diag(l, l, 1)) (plane strain keeps F_33 = 1, so the state is not
    stress-free)."""
    prm = workloads.params()
    pr = fs.Problem(np.ones((6, 6)), np.zeros((6, 6)), prm, 0.4)
    z = pr.solve()
    u, Fb = pr.unpack(z)
    K, G = pr.K[0], pr.G[0]
    dT = 0.6
    e = 1e-6
    lam = brentq(lambda l: (_energy_stretches(l + e, l + e, K, G, dT) - _energy_stretches(l - e, l - e, K, G, dT)) / (2 * e),
                 0.6, 1.0, xtol=1e-14)
    assert abs(Fb[0, 0] - lam) < 1e-9 and abs(Fb[1, 1] - lam) < 1e-9 and abs(Fb[0, 1]) < 1e-12
    assert np.abs(u).max() < 1e-12
    assert lam < 0.6 ** (1 / 3)          # more in-plane contraction than the free 3D stretch


def test_uniaxial_mean_stress(fs):
    """Homogeneous wuestite under a mean first Piola stress diag(p, 0):
    F = diag(l1, l2, 1) with dpsi/dl1 = p, dpsi/dl2 = 0."""
    prm = workloads.params()
    p = 0.05
    pr = fs.Problem(np.zeros((5, 6)), np.zeros((5, 6)), prm, 0.0, pbar=np.diag([p, 0.0]))
    z = pr.solve(nload=1)
    _, Fb = pr.unpack(z)
    K, G = pr.K[0], pr.G[0]
    e = 1e-6

    def eqs(v):
        l1, l2 = v
        d1 = (_energy_stretches(l1 + e, l2, K, G, 1.0) - _energy_stretches(l1 - e, l2, K, G, 1.0)) / (2 * e)
        d2 = (_energy_stretches(l1, l2 + e, K, G, 1.0) - _energy_stretches(l1, l2 - e, K, G, 1.0)) / (2 * e)
        return [d1 - p, d2]

    l1, l2 = fsolve(eqs, [1.05, 0.98], xtol=1e-14)
    assert abs(Fb[0, 0] - l1) < 1e-8 and abs(Fb[1, 1] - l2) < 1e-8 and abs(Fb[0, 1]) < 1e-12
    assert l1 > 1.0 and l2 < 1.0


def _inclusion(n=10, radius=3.0):
    x = np.arange(n) + 0.5 - n / 2
    gy, gx = np.meshgrid(x, x, indexing="ij")
    r = np.sqrt(gx ** 2 + gy ** 2)
    return 0.5 * (1 - np.tanh((r - radius) / 1.5))        # ferrite disk in wuestite


def test_small_strain_limit(orc, fs):
    """As Omega -> 0 the finite-strain solution of a ferrite disk in wuestite
    approaches the small-strain oracle with eigenstrain -Omega/3 W_f: the
    relative difference of the displacement is O(Omega)."""
    th = _inclusion()
    rel = []
    for om in (0.02, 0.01):
        pr = fs.Problem(th, np.zeros_like(th), workloads.params(), om)
        z = pr.solve(nload=1)
        u, Fb = pr.unpack(z)
        prm = workloads.params(eig0=-om / 3.0, plasticity=0, cg_rtol=1e-13, cg_maxit=100000)
        f = {"phi_f": th, "phi_w": 1.0 - th, "xO": np.zeros_like(th), "xH": np.zeros_like(th),
             "xW": np.zeros_like(th)}
        s = orc.Sim(f, prm)
        s.mechanics()
        us = s.f["u"].reshape(-1, 2)
        du = (u - u.mean(0)) - (us - us.mean(0))
        rel.append(np.abs(du).max() / np.abs(us - us.mean(0)).max())
        E = s.f["Ebar"]
        assert abs((Fb[0, 0] - 1) - E[0]) < 0.01 * abs(E[0]) and abs((Fb[1, 1] - 1) - E[1]) < 0.01 * abs(E[1])
    assert rel[0] < 0.05
    assert 1.7 < rel[0] / rel[1] < 2.3, rel


def test_core_shell_mean_stress_and_equilibrium(fs):
    """Core-shell with gas and the full 40 % volume change: the residual
    vanishes, the whole mean first Piola stress vanishes (its skew part is
    not imposed: it follows from frame indifference with Fbar symmetric),
    and the solution is a local minimum of the total energy."""
    f = inputs.core_shell((8, 8), 2.5, 1.0, delta=1.0)
    from oracle import split_phases
    th, pg = split_phases(f["phi_f"], f["phi_w"])
    pr = fs.Problem(th, pg, workloads.params(), 0.4)
    z = pr.solve(nload=6)
    assert np.abs(pr.residual(z, 0.4)).max() < 1e-11
    assert np.abs(pr.mean_piola(z)[:2, :2]).max() < 1e-12
    E0 = pr.energy(z, 0.4)
    rng = np.random.default_rng(4)
    for _ in range(5):
        dz = 1e-4 * rng.standard_normal(z.size)
        assert pr.energy(z + dz, 0.4) > E0
    _, Fb = pr.unpack(z)
    assert Fb[0, 0] < 1.0 and Fb[1, 1] < 1.0          # the shrinking shell pulls the box in


_KS, _GS = 1.0 / (3 * 0.4), 1.0 / 2.6            # E = 1, nu = 0.3


def _ydev(M):
    return np.linalg.norm(M - np.trace(M) / 3.0 * np.eye(3))


def test_return_map_isochoric_consistent_and_unloads_elastically(fs):
    """After a plastic step det F_P = 1 (F_P isochoric, Sec. 2.2), the
    Mandel stress sits on the yield surface |dev M| = sqrt(2/3)(sigma_Y +
    H eps_P) with dl > 0 (PlaTwoJ); a step back inside the surface is
    elastic and leaves F_P and eps_P unchanged."""
    rng = np.random.default_rng(6)
    sy, H = 0.01, 0.05
    FP, ep = np.eye(3), 0.0
    for _ in range(4):
        F = np.eye(3) + 0.06 * rng.standard_normal((3, 3))
        FP1, ep1, dl, M = fs.return_map(F, FP, ep, _KS, _GS, 0.8, sy, H)
        assert abs(np.linalg.det(FP1) - 1.0) < 1e-13
        if dl > 0.0:
            assert abs(_ydev(M) - np.sqrt(2 / 3) * (sy + H * ep1)) < 1e-13
            assert ep1 > ep
        FP, ep = FP1, ep1
    assert ep > 0.0
    # unloading: the elastic state at the current F_P is stress-free up to d_T
    F0 = 0.8 ** (1 / 3) * FP
    FP2, ep2, dl2, M2 = fs.return_map(F0, FP, ep, _KS, _GS, 0.8, sy, H)
    assert dl2 == 0.0 and ep2 == ep and np.array_equal(FP2, FP) and np.abs(M2).max() < 1e-14


@pytest.mark.parametrize("kind", ["shear", "uniaxial"])
def test_return_map_small_strain_limit(fs, kind):
    """For small strains from F_P = I the multiplier approaches the
    small-strain radial return dl = (2G |dev e| - sqrt(2/3) sigma_Y) /
    (2G + sqrt(2/3) H); the relative difference vanishes with the strain."""
    sy, H = 0.001, 0.05
    errs = []
    for g in (0.01, 0.005):
        F = np.eye(3)
        if kind == "shear":
            F[0, 1] = g
            de = g / np.sqrt(2.0)
        else:
            F[0, 0] = 1.0 + g
            de = g * np.sqrt(2.0 / 3.0)
        _, _, dl, _ = fs.return_map(F, np.eye(3), 0.0, _KS, _GS, 1.0, sy, H)
        ref = (2 * _GS * de - np.sqrt(2 / 3) * sy) / (2 * _GS + np.sqrt(2 / 3) * H)
        errs.append(abs(dl - ref) / ref)
    assert errs[0] < 0.02 and errs[1] < errs[0] / 1.6, errs


def test_return_map_is_objective(fs):
    """A rotation superposed on the current configuration (F -> Q F) leaves
    the plastic deformation, eps_P and the Mandel stress unchanged."""
    rng = np.random.default_rng(8)
    F = np.eye(3) + 0.08 * rng.standard_normal((3, 3))
    a = fs.return_map(F, np.eye(3), 0.0, _KS, _GS, 0.9, 0.005, 0.02)
    Q = _rot(rng)
    b = fs.return_map(Q @ F, np.eye(3), 0.0, _KS, _GS, 0.9, 0.005, 0.02)
    assert a[2] > 0.0 and abs(a[2] - b[2]) < 1e-13
    assert np.abs(a[0] - b[0]).max() < 1e-12 and np.abs(a[3] - b[3]).max() < 1e-12


def test_return_map_monotonic_shear_path(fs):
    """Simple shear to gamma = 0.2 in increments: eps_P grows monotonically
    on the hardening line, det F_P stays 1, and halving the increments
    changes the end state by a first-order amount."""
    sy, H = 0.005, 0.02
    ends = []
    for n in (20, 40, 80):
        FP, ep = np.eye(3), 0.0
        for k in range(1, n + 1):
            F = np.eye(3)
            F[0, 1] = 0.2 * k / n
            FP, ep1, dl, M = fs.return_map(F, FP, ep, _KS, _GS, 1.0, sy, H)
            assert ep1 >= ep and abs(np.linalg.det(FP) - 1.0) < 1e-12
            if dl > 0.0:
                assert abs(_ydev(M) - np.sqrt(2 / 3) * (sy + H * ep1)) < 1e-13
            ep = ep1
        ends.append(ep)
    assert ends[0] > 0.1
    d1, d2 = abs(ends[0] - ends[1]), abs(ends[1] - ends[2])
    assert d2 < d1 and 1.5 < d1 / d2 < 2.6, (ends, d1 / d2)


def test_plastic_step_small_strain_limit(orc, fs):
    """One staggered elasto-plastic mechanics step (F8) of a ferrite disk in
    wuestite approaches the small-strain oracle's step (R6, eigenstrain
    -Omega/3 W_f, the same yield stress relative to Omega): the accumulated
    plastic strain and log F_P against eps_p differ by O(Omega)."""
    from scipy.linalg import logm
    th = _inclusion()
    rel = []
    for om in (0.02, 0.01):
        sy, H = 1e-2 * om, 0.01
        pr = fs.Problem(th, np.zeros_like(th), workloads.params(plasticity=1, sigma_Y=sy, H_hard=H), om)
        pr.mechanics_step()
        s = orc.Sim({"phi_f": th, "phi_w": 1.0 - th, "xO": np.zeros_like(th), "xH": np.zeros_like(th),
                     "xW": np.zeros_like(th)},
                    workloads.params(eig0=-om / 3.0, plasticity=1, sigma_Y=sy, H_hard=H, cg_rtol=1e-13,
                                     cg_maxit=100000))
        s.mechanics()
        a = s.f["alpha"].ravel()
        ep = s.f["eps_p"].reshape(-1, 4)
        lp = np.array([np.real(logm(F)) for F in pr.FP])
        assert (a > 0).all() and (pr.epsP > 0).all()            # every cell yielded in both
        assert np.abs(np.linalg.det(pr.FP) - 1.0).max() < 1e-12
        rel.append(max(np.abs(pr.epsP - a).max() / a.max(),
                       np.abs(lp[:, 0, 0] - ep[:, 0]).max() / np.abs(ep).max(),
                       np.abs(lp[:, 0, 1] - ep[:, 3]).max() / np.abs(ep).max()))
    assert rel[0] < 0.02 and 1.7 < rel[0] / rel[1] < 2.3, rel


def test_elastic_driving_force_small_strain_limit(orc, fs):
    """The finite-strain elastic force on the order parameter (F9) of a
    ferrite disk approaches the elastic part of the small-strain oracle's
    force (its eigenstrain -Omega/3 W_f and coupling scalars) with a
    relative difference O(Omega)."""
    th = _inclusion()
    rel = []
    for om in (0.02, 0.01):
        pr = fs.Problem(th, np.zeros_like(th), workloads.params(), om)
        z = pr.mechanics_step()
        fel = fs.elastic_force(pr, z)
        s = orc.Sim({"phi_f": th, "phi_w": 1.0 - th, "xO": np.zeros_like(th), "xH": np.zeros_like(th),
                     "xW": np.zeros_like(th)},
                    workloads.params(eig0=-om / 3.0, cg_rtol=1e-13, cg_maxit=100000))
        s.mechanics()
        t, s2 = s.f["trE"].ravel(), s.f["devE2"].ravel()
        ths, pgs, xo = s.f["theta"].ravel(), s.f["phig"].ravel(), s.f["xO"].ravel()
        small = np.array([orc.theta_force(s.p, ths[c], pgs[c], xo[c], t[c], s2[c])
                          - orc.theta_force(s.p, ths[c], pgs[c], xo[c], 0.0, 0.0)
                          for c in range(s.N)])
        rel.append(np.abs(fel - small).max() / np.abs(small).max())
    assert rel[0] < 0.05 and 1.7 < rel[0] / rel[1] < 2.3, rel


def test_coupled_step_without_volume_change_is_the_oracle_step(orc, fs):
    """With Omega = 0 and no prestress the finite-strain mechanics is
    stress-free, so the coupled step equals the oracle's step with
    mechanics off, bitwise, including the supply-cell counters."""
    f = inputs.core_shell((12, 12), 3.0, 1.2, delta=1.5)
    assert f["mask"].any()
    prm = workloads.params(plasticity=1)
    c = fs.CoupledSim(f, prm, 0.0)
    o = orc.Sim(f, dict(prm, mechanics=0))
    c.step(3)
    o.step(3)
    for k in ("theta", "xO", "xH", "xW"):
        assert np.array_equal(c.sim.f[k], o.f[k])
    assert c.sim.removedW == o.removedW and c.sim.suppliedH == o.suppliedH
    # with the volume change the mechanics moves the order parameter
    c4 = fs.CoupledSim(f, prm, 0.4)
    c4.step(1)
    o1 = orc.Sim(f, dict(prm, mechanics=0))
    o1.step(1)
    assert np.abs(c4.sim.f["theta"] - o1.f["theta"]).max() > 1e-4


def test_coupled_step_small_strain_limit(orc, fs):
    """The elastic part of one coupled step (CoupledSim: the change of theta
    that the finite-strain mechanics adds to the step without mechanics)
    approaches the same part of one oracle step with the small-strain
    mechanics (eigenstrain -Omega/3 W_f) as Omega -> 0: the relative
    difference is O(Omega).  This fixes the sign and the factor -(L/2) mob
    with which the finite-strain force enters the order parameter's rate."""
    th = _inclusion()
    z = np.zeros_like(th)
    f = {"phi_f": th, "phi_w": 1.0 - th, "xO": z + 0.3, "xH": z + 0.01, "xW": z}
    prm = workloads.params(prestress=0.0, cg_rtol=1e-13, cg_maxit=100000)
    o0 = orc.Sim(f, dict(prm, mechanics=0))
    o0.step(1)
    rel = []
    for om in (0.02, 0.01):
        c = fs.CoupledSim(f, prm, om)
        c.step(1)
        s = orc.Sim(f, dict(prm, eig0=-om / 3.0))
        s.step(1)
        d_fin = c.sim.f["theta"] - o0.f["theta"]
        d_small = s.f["theta"] - o0.f["theta"]
        assert np.abs(d_small).max() > 1e-8        # far above the rounding of theta ~ 1
        rel.append(np.abs(d_fin - d_small).max() / np.abs(d_small).max())
    assert rel[0] < 0.05 and 1.7 < rel[0] / rel[1] < 2.3, rel


def test_3d_uniform_transformation_is_stress_free(fs):
    """In 3D nothing constrains the transformation: uniform ferrite with
    Omega = 0.4 and no mean stress deforms by exactly F = d_T^(1/3) I, where
    F_E = I and every stress vanishes."""
    pr = fs.Problem(np.ones((3, 4, 5)), np.zeros((3, 4, 5)), workloads.params(), 0.4)
    z = pr.solve()
    u, Fb = pr.unpack(z)
    assert np.abs(Fb - 0.6 ** (1 / 3) * np.eye(3)).max() < 1e-12
    assert np.abs(u).max() < 1e-12
    assert np.abs(pr.mean_piola(z)).max() < 1e-12


def test_3d_small_strain_limit(orc, fs):
    """3D: a ferrite ball in wuestite approaches the small-strain oracle
    (eigenstrain -Omega/3 W_f) with a relative displacement difference
    O(Omega); the mean strains agree to the same order."""
    n = 4
    x = np.arange(n) + 0.5 - n / 2
    gz, gy, gx = np.meshgrid(x, x, x, indexing="ij")
    th = 0.5 * (1 - np.tanh((np.sqrt(gx ** 2 + gy ** 2 + gz ** 2) - 1.2) / 1.0))
    rel = []
    for om in (0.02, 0.01):
        pr = fs.Problem(th, np.zeros_like(th), workloads.params(), om)
        u, Fb = pr.unpack(pr.solve(nload=1))
        s = orc.Sim({"phi_f": th, "phi_w": 1.0 - th, "xO": np.zeros_like(th), "xH": np.zeros_like(th),
                     "xW": np.zeros_like(th)},
                    workloads.params(eig0=-om / 3.0, cg_rtol=1e-13, cg_maxit=100000))
        s.mechanics()
        us = s.f["u"].reshape(-1, 3)
        du = (u - u.mean(0)) - (us - us.mean(0))
        rel.append(np.abs(du).max() / np.abs(us - us.mean(0)).max())
        E = s.f["Ebar"]
        for k in range(3):
            assert abs((Fb[k, k] - 1) - E[k]) < 0.02 * abs(E[k])
    assert rel[0] < 0.05 and 1.7 < rel[0] / rel[1] < 2.3, rel


def test_3d_plastic_step_small_strain_limit(orc, fs):
    """3D: one staggered elasto-plastic step of a ferrite ball approaches
    the small-strain oracle's plastic step at O(Omega), in the accumulated
    plastic strain and in every component of log F_P against eps_p
    (xx, yy, zz, yz, xz, xy)."""
    from scipy.linalg import logm
    n = 4
    x = np.arange(n) + 0.5 - n / 2
    gz, gy, gx = np.meshgrid(x, x, x, indexing="ij")
    th = 0.5 * (1 - np.tanh((np.sqrt(gx ** 2 + gy ** 2 + gz ** 2) - 1.2) / 1.0))
    comps = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    rel = []
    for om in (0.02, 0.01):
        sy, H = 1e-2 * om, 0.01
        pr = fs.Problem(th, np.zeros_like(th), workloads.params(plasticity=1, sigma_Y=sy, H_hard=H), om)
        pr.mechanics_step()
        s = orc.Sim({"phi_f": th, "phi_w": 1.0 - th, "xO": np.zeros_like(th), "xH": np.zeros_like(th),
                     "xW": np.zeros_like(th)},
                    workloads.params(eig0=-om / 3.0, plasticity=1, sigma_Y=sy, H_hard=H, cg_rtol=1e-13,
                                     cg_maxit=100000))
        s.mechanics()
        a = s.f["alpha"].ravel()
        ep = s.f["eps_p"].reshape(-1, 6)
        lp = np.array([np.real(logm(F)) for F in pr.FP])
        assert (a > 0).all() and (pr.epsP > 0).all()
        r = [np.abs(pr.epsP - a).max() / a.max()]
        r += [np.abs(lp[:, i, j] - ep[:, k]).max() / np.abs(ep).max() for k, (i, j) in enumerate(comps)]
        rel.append(max(r))
    assert rel[0] < 0.02 and 1.7 < rel[0] / rel[1] < 2.3, rel
