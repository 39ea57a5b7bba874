"""Pins of the backward-Euler oracle (oracle/implicit.py) against closed forms.

The paper integrates its field relations by backward Euler (Sec. 2.4,
closing paragraph).  In the linear cases (diffusion of one species,
oxygen in one phase with a quadratic energy) backward Euler has an exact
discrete solution per Fourier mode; in the nonlinear coupled case the
step keeps both balances of the reaction O + 2H -> H2O, converges at first
order in dt, and agrees with the explicit step to O(dt^2) per step; the
Allen-Cahn flow keeps decreasing the free energy at steps the explicit
method cannot take.
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import inputs, workloads

NOFLUX = dict(D_O_s=0.0, D_O_g=0.0, D_H_s=0.0, D_H_g=0.0, D_W_s=0.0, D_W_g=0.0)


@pytest.fixture(scope="module")
def be(orc):
    from oracle import implicit
    return implicit


def _lam(shape):
    k = [2 * np.pi * np.fft.fftfreq(m) for m in shape]
    return sum(2.0 - 2.0 * np.cos(g) for g in np.meshgrid(*k, indexing="ij"))


def _uniform(shape, phase="wuestite", xO=0.3):
    pw = np.ones(shape) if phase == "wuestite" else np.zeros(shape)
    return {"phi_f": np.zeros(shape), "phi_w": pw, "xO": np.full(shape, xO),
            "xH": np.zeros(shape), "xW": np.zeros(shape), "mask": np.zeros(shape, np.uint8)}


@pytest.mark.parametrize("shape", [(16, 20), (6, 6, 8)])
def test_be_hydrogen_diffusion_exact(orc, be, shape):
    """x_t = D Lap_h x: every DFT mode of backward Euler scales by
    1 / (1 + dt D lambda_k) per step, at any dt (here 8x the explicit limit)."""
    D = 0.3
    rng = np.random.default_rng(3)
    f = _uniform(shape)
    f["xH"] = 0.01 + 1e-3 * rng.standard_normal(shape)
    s = orc.Sim(f, workloads.params(k_for=0.0, mechanics=0, D_H_s=D, D_H_g=D))
    dt = 40.0 * s.dt                       # s.dt is 0.2 x the explicit limit
    x0 = f["xH"].copy()
    n = 4
    for _ in range(n):
        be.be_step(s, dt)
    ref = np.real(np.fft.ifftn(np.fft.fftn(x0) / (1.0 + dt * D * _lam(shape)) ** n))
    assert np.abs(s.f["xH"] - ref).max() < 1e-13
    assert np.abs(s.f["xH"] - x0).max() > 1e-4          # the field moved
    assert np.abs(s.f["theta"]).max() == 0.0 and np.abs(s.f["xO"] - 0.3).max() < 1e-15


@pytest.mark.parametrize("phase,shape", [("wuestite", (12, 14)), ("gas", (12, 14)), ("wuestite", (4, 6, 6))])
def test_be_oxygen_single_phase_exact(orc, be, phase, shape):
    """Oxygen in one phase with a quadratic energy (wuestite 173.263 x^2 + ...,
    gas 1000 x^2, Sec. 3.1) is linear: x_t = D Lap x - (D kappa / (2 a c))
    Lap^2 x, so backward Euler scales every mode by
    1 / (1 + dt (D lambda + D kappa lambda^2 / (2 a c)))."""
    a = {"wuestite": 173.263, "gas": 1000.0}[phase]
    kappa = 0.5
    rng = np.random.default_rng(11)
    f = _uniform(shape, phase)
    x0 = 0.3 + 0.02 * rng.standard_normal(shape)
    f["xO"] = x0.copy()
    prm = workloads.params(k_for=0.0, mechanics=0, kappa_O=kappa, D_O_s=0.05, D_O_g=0.5)
    s = orc.Sim(f, prm)
    D = prm["D_O_s"] if phase == "wuestite" else prm["D_O_g"]
    c = prm["c_chem"]
    lam = _lam(shape)
    rate = D * lam + D * kappa * lam ** 2 / (2 * a * c)
    dt = 2.5 / rate.max()                  # explicit Euler's shortest wave: factor -1.5
    n = 3
    for _ in range(n):
        be.be_step(s, dt)
    ref = np.real(np.fft.ifftn(np.fft.fftn(x0) / (1.0 + dt * (D * lam + D * kappa * lam ** 2 / (2 * a * c))) ** n))
    assert np.abs(s.f["xO"] - ref).max() < 1e-13
    assert np.abs(s.f["xO"] - x0).max() > 1e-3
    # the gradient-energy term is not negligible at the shortest wavelengths
    assert kappa * lam.max() / (2.0 * a * c) > 0.1


def _coreshell(shape=(12, 12), mask=True):
    f = inputs.core_shell(shape, 3.5, 1.5, delta=1.5)
    if not mask:
        f["mask"] = np.zeros(shape, np.uint8)
    return f


def test_be_balances_with_reaction_and_supply(orc, be):
    """The reaction O + 2H -> H2O and flux-form transport conserve
    sum(x_O + x_H2O) and sum(x_H + 2 x_H2O) at any state, so backward Euler
    keeps both balances, with the supply cells' counters (S3), to roundoff."""
    f = _coreshell((14, 14))
    assert 0 < f["mask"].sum() < f["mask"].size // 2
    s = orc.Sim(f, workloads.params(cg_rtol=1e-10))
    a0 = s.sums()
    for _ in range(3):
        be.be_step(s, 2.0 * s.dt)
    a1 = s.sums()
    o0, o1 = a0[0] + a0[2], a1[0] + a1[2] + s.removedW
    h0 = a0[1] + 2 * a0[2]
    h1 = a1[1] + 2 * a1[2] + 2 * s.removedW - s.suppliedH
    assert abs(o1 - o0) < 1e-12 * o0
    assert abs(h1 - h0) < 1e-12 * h0
    assert a1[2] > 0.0 and s.suppliedH > 0.0
    m = f["mask"].astype(bool)
    assert np.all(s.f["xH"][m] == s.p.xH_bc) and np.all(s.f["xW"][m] == 0.0)


def _state(s):
    return np.concatenate([s.f[k].ravel() for k in ("theta", "xO", "xH", "xW")])


def test_be_first_order_in_dt(orc, be):
    """Backward Euler with the staggered mechanics is first order: the
    difference between runs at dt and dt/2 to the same time halves with dt."""
    prm = workloads.params(cg_rtol=1e-12)
    T = None
    ys = []
    for k in (2, 4, 8, 16):
        s = orc.Sim(_coreshell(mask=False), prm)
        if T is None:
            T = 8.0 * s.dt
        for _ in range(k):
            be.be_step(s, T / k)
        ys.append(_state(s))
    e = [np.abs(ys[i] - ys[i + 1]).max() for i in range(3)]
    ratios = [e[i] / e[i + 1] for i in range(2)]
    assert all(1.7 < r < 2.3 for r in ratios), (e, ratios)


def test_be_matches_explicit_to_second_order_per_step(orc, be):
    """One backward-Euler step and one explicit step from the same state
    differ by O(dt^2): dt^2 R'(y) R(y) to leading order."""
    prm = workloads.params(cg_rtol=1e-12)
    d = []
    for frac in (1.0, 0.5, 0.25):
        sb = orc.Sim(_coreshell(mask=False), prm)
        se = orc.Sim(_coreshell(mask=False), prm, dt=frac * sb.dt)
        be.be_step(sb, frac * sb.dt)
        se.step(1)
        d.append(np.abs(_state(sb) - _state(se)).max())
    assert 3.5 < d[0] / d[1] < 4.5 and 3.5 < d[1] / d[2] < 4.5, d


def test_be_allen_cahn_energy_decreases_at_large_steps(orc, be):
    """Without chemistry, transport, reaction and mechanics the order
    parameter follows the Allen-Cahn gradient flow; backward Euler is then the
    minimising-movement step, so the free energy decreases at every step, here
    at 1.5x the explicit limit of the gradient term (explicit Euler's
    shortest wave grows by a factor 2 per step)."""
    nx = 24
    x = np.arange(nx) + 0.5
    pf = ((x > nx / 4) & (x < 3 * nx / 4)).astype(float)
    noise = 1e-3 * np.random.default_rng(5).random((2, nx))   # seeds every mode
    th0 = np.tile(pf, (2, 1)) * (1.0 - noise) + np.tile(1.0 - pf, (2, 1)) * noise
    f = {"phi_f": th0, "phi_w": 1.0 - th0,
         "xO": np.zeros((2, nx)), "xH": np.zeros((2, nx)), "xW": np.zeros((2, nx)),
         "mask": np.zeros((2, nx), np.uint8)}
    prm = workloads.params(c_chem=0.0, k_for=0.0, mechanics=0, **NOFLUX)
    s = orc.Sim(f, prm)
    # theta_t = -(L/2)(2 w m'(theta) - 2 eps Lap theta): the shortest wave
    # decays at rate L eps 4d, so explicit Euler needs dt < 2 / (4d L eps)
    dt = 3.0 / (8.0 * prm["L"] * prm["eps_phi"])
    F = [s.free_energy()]
    for _ in range(8):
        be.be_step(s, dt)
        F.append(s.free_energy())
    assert np.all(np.diff(F) < 0.0), F
    assert s.f["theta"].min() > -1e-9 and s.f["theta"].max() < 1.0 + 1e-9
    # explicit Euler at the same dt leaves [0, 1]
    se = orc.Sim(f, prm, dt=dt)
    se.step(8)
    assert se.f["theta"].min() < -1e-3 or se.f["theta"].max() > 1.0 + 1e-3


def test_be_paper_scaled_parameters(orc, be):
    """With the diffusivities and reaction rate of the paper's Table 1
    (workloads.paper_params) explicit Euler needs dt ~ 7.5e-8 (gas
    diffusion); backward Euler takes steps of 0.05 and 0.5, six to seven
    orders larger, and keeps both balances with the supply cells."""
    prm = workloads.paper_params(cg_rtol=1e-10)
    f = _coreshell((14, 14))
    s = orc.Sim(f, prm)
    assert abs(s.dt - 0.2 / (2 * 2 * prm["D_O_g"])) < 1e-3 * s.dt
    a0 = s.sums()
    for dt in (0.05, 0.05, 0.5):
        be.be_step(s, dt)
    a1 = s.sums()
    o0, o1 = a0[0] + a0[2], a1[0] + a1[2] + s.removedW
    h0 = a0[1] + 2 * a0[2]
    h1 = a1[1] + 2 * a1[2] + 2 * s.removedW - s.suppliedH
    assert abs(o1 - o0) < 1e-12 * o0
    assert abs(h1 - h0) < 1e-11 * h0
    for k in ("theta", "xO", "xH", "xW"):
        assert np.isfinite(s.f[k]).all()
    assert s.f["xH"].min() > -1e-9 and a1[2] > 0.0


def test_be_3d_coupled_balances_with_plasticity(orc, be):
    """3D core-shell with mechanics, J2 plasticity, reaction and supply
    cells: backward-Euler steps keep both balances to roundoff."""
    f = inputs.core_shell((6, 6, 6), 1.5, 0.7, delta=0.8)
    assert f["mask"].any()
    s = orc.Sim(f, workloads.params(cg_rtol=1e-10, plasticity=1, sigma_Y=0.002, H_hard=0.01))
    a0 = s.sums()
    for _ in range(2):
        be.be_step(s, 2.0 * s.dt)
    a1 = s.sums()
    o0, o1 = a0[0] + a0[2], a1[0] + a1[2] + s.removedW
    h0 = a0[1] + 2 * a0[2]
    h1 = a1[1] + 2 * a1[2] + 2 * s.removedW - s.suppliedH
    assert abs(o1 - o0) < 1e-12 * o0 and abs(h1 - h0) < 1e-12 * h0
    assert s.f["alpha"].max() > 0.0 and a1[2] > 0.0
