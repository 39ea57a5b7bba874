"""GPU backward-Euler steps (pf_step_implicit) against the oracle's
backward-Euler step (oracle/implicit.py).

The paper integrates its field relations by backward Euler and solves each
step by Newton's method (Sec. 2.4, closing paragraph).  Both sides solve
F(y) = y - y_n - dt R(y) with the staggered mechanics and held supply cells,
the oracle by Newton with a dense finite-difference Jacobian, the library by
matrix-free Newton-Krylov (Jacobian-vector products in forward mode); both stop at the same rule (max |F| <= 1e-12,
or an update below 1e-12 of the largest field value), so the states agree to
the Newton tolerance amplified by the step's conditioning: 1e-9 (relative L2)
at the bench parameters, 1e-8 at the paper's diffusivities, where dt R
carries terms ~1e4 times the fields.  The library's block preconditioner
runs in FP32 by default (pc_precision "mixed") or FP64; F is FP64 either
way, so both meet the same bounds.
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import PFError, Simulation, inputs, native, workloads

pytestmark = pytest.mark.gpu

KEYS = ("theta", "xO", "xH", "xW")


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


@pytest.fixture(scope="module")
def be(orc):
    from oracle import implicit
    return implicit


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _coreshell(shape=(14, 14), mask=True):
    f = inputs.core_shell(shape, 3.5, 1.5, delta=1.5)
    if not mask:
        f["mask"] = np.zeros(shape, np.uint8)
    return f


def _run(orc, be, f, prm, dts, **kw):
    ref = orc.Sim(f, prm)
    sim = Simulation(f["phi_f"].shape, prm, precision="fp64")
    sim.set_fields(f)
    stats = []
    for dt in dts:
        be.be_step(ref, dt)
        stats.append(sim.step_implicit(1, dt, **kw))
    g = sim.get_fields(keys=KEYS + ("sigma", "alpha"))
    d = sim.diagnostics()
    sim.close()
    return ref, g, d, stats


def _balances(d, f, tol):
    O0 = f["xO"].sum() + f["xW"].sum()
    H0 = f["xH"].sum() + 2 * f["xW"].sum()
    assert abs(d["sum_O"] + d["sum_H2O"] + d["removed_H2O"] - O0) < tol * O0
    assert abs(d["sum_H"] + 2 * d["sum_H2O"] + 2 * d["removed_H2O"] - d["supplied_H"] - H0) < tol * H0


@pytest.mark.parametrize("pc_precision", ["mixed", "fp64"])
def test_backward_euler_2d_matches_oracle(orc, be, pc_precision):
    """14x14 core-shell with supply cells, mechanics, reaction: three steps
    at 4x the explicit stability limit."""
    f = _coreshell()
    prm = workloads.params(cg_rtol=1e-12)
    dt = 20.0 * orc.Sim(f, prm).dt                  # Sim.dt is 0.2 x the explicit limit
    ref, g, d, stats = _run(orc, be, f, prm, [dt] * 3, pc_precision=pc_precision)
    for k in KEYS:
        assert rel(g[k], ref.f[k]) < 1e-9, (k, rel(g[k], ref.f[k]))
    assert rel(g["sigma"], ref.f["sigma"]) < 1e-8
    s = ref.sums()
    assert abs(d["sum_O"] - s[0]) < 1e-10 * s[0] and abs(d["sum_H2O"] - s[2]) < 1e-9 * max(s[2], 1e-12)
    assert abs(d["removed_H2O"] - ref.removedW) < 1e-9 * max(ref.removedW, 1e-12)
    assert abs(d["supplied_H"] - ref.suppliedH) < 1e-9 * max(ref.suppliedH, 1e-12)
    _balances(d, f, 1e-12)
    assert d["steps"] == 3 and d["dt"] == dt
    assert all(st["newton_iters"] >= 1 and st["rc"] == native.PF_OK for st in stats)
    m = f["mask"].astype(bool)
    assert np.all(g["xH"][m] == workloads.params()["xH_bc"]) and np.all(g["xW"][m] == 0.0)


def test_backward_euler_3d_plasticity_matches_oracle(orc, be):
    """3D core-shell with J2 plasticity, reaction and supply cells."""
    f = inputs.core_shell((6, 6, 6), 1.5, 0.7, delta=0.8)
    prm = workloads.params(cg_rtol=1e-12, plasticity=1, sigma_Y=0.002, H_hard=0.01)
    dt = 10.0 * orc.Sim(f, prm).dt
    ref, g, d, _ = _run(orc, be, f, prm, [dt, dt])
    for k in KEYS:
        assert rel(g[k], ref.f[k]) < 1e-9, (k, rel(g[k], ref.f[k]))
    assert rel(g["alpha"], ref.f["alpha"]) < 1e-8
    _balances(d, f, 1e-12)


def test_backward_euler_paper_parameters(orc, be):
    """The paper's Table 1 diffusivities and reaction rate
    (workloads.paper_params): explicit Euler needs dt ~ 7.5e-8; backward
    Euler takes 0.05, 0.05 and 0.5 on both sides."""
    f = _coreshell()
    prm = workloads.paper_params(cg_rtol=1e-12)
    ref, g, d, stats = _run(orc, be, f, prm, [0.05, 0.05, 0.5])
    for k in KEYS:
        assert rel(g[k], ref.f[k]) < 1e-8, (k, rel(g[k], ref.f[k]))
    _balances(d, f, 1e-11)
    assert all(np.isfinite(g[k]).all() for k in KEYS)


def test_backward_euler_preconditioner_is_needed_at_paper_stiffness():
    """At the paper's diffusivities (dt D_gas ~ 3e4 per cell) GMRES without
    the block preconditioner does not solve a Newton system within 1000
    iterations, and Newton does not converge in two; with 32 Chebyshev steps
    per block every system is solved in far fewer, and Newton converges."""
    f = _coreshell()
    prm = workloads.paper_params(cg_rtol=1e-12)
    sim = Simulation(f["phi_f"].shape, prm, precision="fp64")
    sim.set_fields(f)
    st = sim.step_implicit(1, 0.05, newton_maxit=2, gmres_maxit=1000, pc_degree=0, check=False)
    assert st["rc"] == native.PF_ENOTCONV and st["gmres_iters"] == 2000, st
    sim.set_fields(f)
    st = sim.step_implicit(1, 0.05, newton_maxit=30, gmres_maxit=1000, pc_degree=32)
    assert st["rc"] == native.PF_OK and st["gmres_iters"] < 1000 * st["newton_iters"] // 2, st
    assert st["residual"] <= 1e-11
    sim.close()


def test_backward_euler_rejects_mixed_and_bad_options():
    f = _coreshell()
    prm = workloads.params()
    sim = Simulation(f["phi_f"].shape, prm, precision="mixed")
    sim.set_fields(f)
    with pytest.raises(PFError) as e:
        sim.step_implicit(1, 0.1)
    assert e.value.code == native.PF_EINVAL
    sim.close()
    sim = Simulation(f["phi_f"].shape, prm, precision="fp64")
    with pytest.raises(PFError) as e:
        sim.step_implicit(1, 0.1)                     # no fields yet
    assert e.value.code == native.PF_ESTATE
    sim.set_fields(f)
    o = native.pf_implicit_opts(dt=0.1, newton_tol=1e-12, newton_maxit=5, gmres_rtol=1e-6, gmres_restart=20,
                                gmres_maxit=100, pc_degree=8, pc_precision=2)
    rc, _ = native.pf_step_implicit(sim.h, 1, o)
    assert rc == native.PF_EINVAL
    for bad in ({"dt": -1.0}, {"gmres_restart": 61}, {"pc_degree": -1}, {"gmres_rtol": 1.0}):
        kw = dict(dt=0.1)
        kw.update(bad)
        dt = kw.pop("dt")
        with pytest.raises(PFError) as e:
            sim.step_implicit(1, dt, **kw)
        assert e.value.code == native.PF_EINVAL
    sim.close()
