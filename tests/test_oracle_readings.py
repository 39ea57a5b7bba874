"""Pins of the oracle's reaction term, of the phase interpolation of the
species diffusivities and their face means, and the evidence for reading R2.

* Reaction (Sec. 2.3.1, the empirical rate r = m(phi_g) k_for x_O x_H with
  the forward constant; Sec. 4.3, no reaction where the water fraction is 1;
  stoichiometry O + 2 H -> H2O): with every diffusivity zero each cell is a
  closed, well-mixed box whose fractions follow the ODE
      dx_O/dt = -r,  dx_H/dt = -2 r,  dx_H2O/dt = +r.
  The oracle's explicit steps must equal the explicit Euler recurrence of
  that ODE cell by cell for mixed (theta, phi_g), and converge at first order
  to its closed-form solution.  A rate with m(phi_f) instead of m(phi_g), a
  missing k_for or factor 2, or a cut-off on x_H instead of x_H2O fails.
* Diffusivities (Sec. 3.2, Table 1 gives solid and gas values only; reading
  R4: D_i(phi) = (1 - h(phi_g)) D_i,solid + h(phi_g) D_i,gas): in a uniform
  two-phase mixture each Fourier mode of hydrogen and water decays exactly
  as (1 - dt D lambda_k)^n with that D; on a two-cell periodic grid with two
  different gas fractions the antisymmetric mode decays as
  (1 - 4 dt D_face)^n, which fixes the arithmetic face mean.
* Reading R2: the paper's two Allen-Cahn relations for phi_f and phi_w
  (Sec. 2.4, field relations and driving forces) taken literally, with the
  gas fraction dependent (Sec. 2.2), move phi_g away from zero inside a
  ferrite / wuestite interface at the rate L h'(phi)(psi_f + psi_w), which is
  not zero for the absolute CALPHAD energies of Sec. 3.1; the numpy
  restatement below shows it (gas created in the interface, or a blow-up,
  independent of the time step), while the oracle's reading keeps phi_g
  fixed.
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import workloads

NOFLUX = dict(D_O_s=0.0, D_O_g=0.0, D_H_s=0.0, D_H_g=0.0, D_W_s=0.0, D_W_g=0.0)


def h(x):
    """Interpolation function of Sec. 3.1, x^3 (6 x^2 - 15 x + 10)."""
    return x ** 3 * (6.0 * x * x - 15.0 * x + 10.0)


def m(x):
    """Double well x^2 (1 - x)^2 (reading R1)."""
    return x * x * (1.0 - x) ** 2


def _boxes():
    """Cells with different gas fractions, solid splits and fractions; the
    last rows test the cut-off: x_H2O = 1 (no reaction), x_H2O just below 1
    and x_H = 1 (reaction runs)."""
    pg = np.array([0.15, 0.5, 0.85, 0.3, 0.6, 0.7, 0.4, 0.4])
    th = np.array([0.3, 0.8, 0.5, 0.1, 0.9, 0.25, 0.5, 0.5])
    xO = np.array([0.4, 0.55, 0.2, 0.5, 0.3, 0.45, 0.4, 0.3])
    xH = np.array([0.3, 0.1, 0.45, 0.2, 0.25, 0.35, 0.2, 1.0])
    xW = np.array([0.0, 0.2, 0.1, 0.999, 0.05, 1.0, 1.0, 0.0])
    return pg, th, xO, xH, xW


def _box_fields(pg, th, xO, xH, xW):
    sh = (2, pg.size)
    t = lambda v: np.tile(v, (2, 1))
    return {"phi_f": t((1.0 - pg) * th), "phi_w": t((1.0 - pg) * (1.0 - th)), "xO": t(xO), "xH": t(xH),
            "xW": t(xW), "mask": np.zeros(sh, np.uint8)}


def test_reaction_well_mixed_boxes_follow_the_rate_law(orc):
    pg, th, xO, xH, xW = _boxes()
    k, dt, n = 2.5, 0.05, 60
    prm = workloads.params(mechanics=0, k_for=k, dt=dt, **NOFLUX)
    s = orc.Sim(_box_fields(pg, th, xO, xH, xW), prm)
    o, hh, ww = xO.copy(), xH.copy(), xW.copy()
    for _ in range(n):
        s.step(1)
        r = np.where(ww >= 1.0, 0.0, m(pg) * k * o * hh)
        o, hh, ww = o - dt * r, hh - 2.0 * dt * r, ww + dt * r
        for got, exp in ((s.f["xO"], o), (s.f["xH"], hh), (s.f["xW"], ww)):
            assert np.allclose(got[0], exp, rtol=1e-13, atol=1e-15) and np.array_equal(got[0], got[1])
    # the cut-off: boxes that start at x_H2O = 1 keep their fractions, the
    # others react (x_H = 1 does not stop the reaction)
    stop = xW >= 1.0
    assert np.array_equal(s.f["xO"][0][stop], xO[stop]) and np.array_equal(s.f["xH"][0][stop], xH[stop])
    assert np.all(s.f["xO"][0][~stop] < xO[~stop])
    # stoichiometry: O + H2O and H + 2 H2O stay constant per box
    assert np.allclose(s.f["xO"][0] + s.f["xW"][0], xO + xW, rtol=0, atol=1e-14)
    assert np.allclose(s.f["xH"][0] + 2.0 * s.f["xW"][0], xH + 2.0 * xW, rtol=0, atol=1e-14)


def _ode_xO(x0, h0, a, t):
    """Closed form of dx_O/dt = -a x_O x_H, dx_H/dt = -2 a x_O x_H:
    c = x_H - 2 x_O is constant and 1/x_O = (1/x0 + 2/c) e^(a c t) - 2/c."""
    c = h0 - 2.0 * x0
    return c * x0 / ((c + 2.0 * x0) * np.exp(a * c * t) - 2.0 * x0)


def test_reaction_converges_to_the_ode_solution(orc):
    pg, th, xO, xH, xW = _boxes()
    keep = xW < 0.9                      # away from the cut-off
    pg, th, xO, xH, xW = pg[keep], th[keep], xO[keep], xH[keep], xW[keep]
    k, T = 2.5, 4.0
    errs = []
    for dt in (0.04, 0.02, 0.01):
        prm = workloads.params(mechanics=0, k_for=k, dt=dt, **NOFLUX)
        s = orc.Sim(_box_fields(pg, th, xO, xH, xW), prm)
        s.step(int(round(T / dt)))
        exact = _ode_xO(xO, xH, m(pg) * k, T)
        errs.append(np.abs(s.f["xO"][0] - exact).max())
        assert np.allclose(s.f["xH"][0] - 2.0 * s.f["xO"][0], xH - 2.0 * xO, atol=1e-14)
    assert errs[-1] < 2e-3
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(1.8 < q < 2.2 for q in ratios), (errs, ratios)


@pytest.mark.parametrize("pg,th", [(0.3, 0.5), (0.75, 0.2)])
def test_species_diffusivity_in_a_uniform_mixture_exact(orc, pg, th):
    shape = (12, 16)
    rng = np.random.default_rng(7)
    DHs, DHg, DWs, DWg = 0.05, 1.0, 0.02, 0.6
    prm = workloads.params(mechanics=0, k_for=0.0, D_H_s=DHs, D_H_g=DHg, D_W_s=DWs, D_W_g=DWg)
    f = {"phi_f": np.full(shape, (1.0 - pg) * th), "phi_w": np.full(shape, (1.0 - pg) * (1.0 - th)),
         "xO": np.zeros(shape), "xH": rng.uniform(0.0, 0.05, shape), "xW": rng.uniform(0.0, 0.05, shape)}
    s = orc.Sim(f, prm)
    n = 25
    s.step(n)
    ky = 2.0 * np.pi * np.fft.fftfreq(shape[0])[:, None]
    kx = 2.0 * np.pi * np.fft.fftfreq(shape[1])[None, :]
    lam = (2.0 - 2.0 * np.cos(kx)) + (2.0 - 2.0 * np.cos(ky))
    for key, Ds, Dg in (("xH", DHs, DHg), ("xW", DWs, DWg)):
        D = (1.0 - h(pg)) * Ds + h(pg) * Dg
        exact = np.real(np.fft.ifft2(np.fft.fft2(f[key]) * (1.0 - s.dt * D * lam) ** n))
        assert np.abs(s.f[key] - exact).max() < 1e-13, key


def test_face_mean_two_cell_grid(orc):
    pg = np.array([0.2, 0.9])
    th = 0.5
    DHs, DHg = 0.05, 1.0
    prm = workloads.params(mechanics=0, k_for=0.0, D_H_s=DHs, D_H_g=DHg)
    t = lambda v: np.tile(v, (2, 1))
    f = {"phi_f": t((1.0 - pg) * th), "phi_w": t((1.0 - pg) * (1.0 - th)), "xO": np.zeros((2, 2)),
         "xH": t(np.array([0.3, 0.1])), "xW": np.zeros((2, 2))}
    s = orc.Sim(f, prm)
    n = 30
    s.step(n)
    Dc = (1.0 - h(pg)) * DHs + h(pg) * DHg
    Df = 0.5 * (Dc[0] + Dc[1])                 # arithmetic mean of the two cells
    d = (0.3 - 0.1) * (1.0 - 4.0 * s.dt * Df) ** n
    got = s.f["xH"][0]
    assert abs((got[0] - got[1]) - d) < 1e-14
    assert abs(got.sum() - 0.4) < 1e-14
    # the harmonic mean would decay measurably slower
    Dh = 2.0 / (1.0 / Dc[0] + 1.0 / Dc[1])
    assert abs((0.3 - 0.1) * (1.0 - 4.0 * s.dt * Dh) ** n - d) > 1e-3


def _literal_step(pf, pw, xO, dt, P):
    """One explicit Euler step of the paper's Allen-Cahn relations for phi_f
    and phi_w taken literally (mechanics off, uniform x_O): independent
    phi_f, phi_w, dependent phi_g = 1 - phi_f - phi_w, bulk energy
    sum_a h(phi_a) c f_a(x_O), wells w m(phi_a), gradient energies
    (eps / 2) |grad phi_a|^2, periodic 1D grid, dx = 1."""
    c, w, eps, L = P["c_chem"], P["w"], P["eps_phi"], P["L"]
    hp = lambda x: 30.0 * x * x * (1.0 - x) ** 2
    mp = lambda x: 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x)
    ff = 163.708 * xO ** 4 - 182.510 * xO ** 3 + 90.573 * xO ** 2 - 36.031 * xO - 4.372
    fw = 173.263 * xO ** 2 - 213.460 * xO + 41.953
    fg = 1.0e3 * xO ** 2
    lap = lambda v: np.roll(v, 1) + np.roll(v, -1) - 2.0 * v
    pg = 1.0 - pf - pw
    df = hp(pf) * c * ff - hp(pg) * c * fg + w * (mp(pf) - mp(pg)) - eps * (lap(pf) - lap(pg))
    dw = hp(pw) * c * fw - hp(pg) * c * fg + w * (mp(pw) - mp(pg)) - eps * (lap(pw) - lap(pg))
    return pf - dt * L * df, pw - dt * L * dw


def test_literal_relations_create_gas_in_a_ferrite_wuestite_interface(orc):
    P = workloads.params()
    n = 64
    x = np.arange(n) + 0.5
    pf0 = 0.5 * (1.0 + np.tanh((x - n / 4) / 3.0)) - 0.5 * (1.0 + np.tanh((x - 3 * n / 4) / 3.0))
    pw0 = 1.0 - pf0
    # first step: the gas rate is L h'(phi_f) (psi_f + psi_w) exactly
    xO = 0.3
    c = P["c_chem"]
    psum = c * ((163.708 * xO ** 4 - 182.510 * xO ** 3 + 90.573 * xO ** 2 - 36.031 * xO - 4.372)
                + (173.263 * xO ** 2 - 213.460 * xO + 41.953))
    dt = 1e-3
    pf1, pw1 = _literal_step(pf0, pw0, xO, dt, P)
    rate = (1.0 - pf1 - pw1) / dt
    assert np.allclose(rate, P["L"] * 30.0 * pf0 ** 2 * (1.0 - pf0) ** 2 * psum, rtol=1e-9, atol=1e-12)
    assert np.abs(rate).max() > 0.1
    # over time, independent of the step: at x_O = 0.3 the relations blow up
    # before t = 1; at x_O = 0.05 gas fills more than half of the interface
    with np.errstate(all="ignore"):
        for xO, dts in ((0.3, (0.01, 0.005)), (0.05, (0.01, 0.005))):
            res = []
            for dt in dts:
                pf, pw = pf0.copy(), pw0.copy()
                for _ in range(int(round(5.0 / dt))):
                    pf, pw = _literal_step(pf, pw, xO, dt, P)
                    if not np.isfinite(pf).all():
                        break
                res.append(np.abs(1.0 - pf - pw).max() if np.isfinite(pf).all() else np.inf)
            if xO == 0.3:
                assert all(np.isinf(v) for v in res), res
            else:
                assert all(v > 0.5 for v in res) and abs(res[0] - res[1]) < 0.01 * res[0], res
    # the oracle's reading on the same interface: phi_g stays exactly zero and
    # the phases stay within [0, 1] up to rounding
    f = {"phi_f": np.tile(pf0, (2, 1)), "phi_w": np.tile(pw0, (2, 1)), "xO": np.full((2, n), 0.05),
         "xH": np.zeros((2, n)), "xW": np.zeros((2, n))}
    s = orc.Sim(f, workloads.params(mechanics=0, k_for=0.0, **NOFLUX))
    s.step(int(round(5.0 / s.dt)))
    assert np.array_equal(s.f["phig"], np.zeros((2, n)))
    assert s.f["theta"].min() > -1e-6 and s.f["theta"].max() < 1.0 + 1e-6
