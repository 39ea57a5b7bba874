"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative L2 over the grid):
  * plain FP64 method: 1e-10 on the phase fields and fractions after the full
    500-step 64x64 core-shell run.  The stress inherits the CG stopping rule
    ||r|| <= 1e-10 ||b||: two correct solves differ by up to cond(A) * 1e-10
    in the solution, and the gas/solid stiffness contrast (1.93e-3) puts
    cond(A) near 1e3, so sigma is held to 1e-7;
  * mixed method (FP32 fields and operator, FP64-grade reductions): 1e-4 on
    the phase fields and fractions, 1e-3 on the stress.
"""
import os

import numpy as np
import pytest

from paper_2111_11538_gb300 import PFError, Simulation, inputs, native, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


def _compare(g, s, tol, tol_sigma=None, keys=("phi_f", "phi_w", "xO", "xH", "xW")):
    ref = {"phi_f": s.phi_f, "phi_w": s.phi_w, "xO": s.f["xO"], "xH": s.f["xH"], "xW": s.f["xW"]}
    errs = {k: rel(g[k], ref[k]) for k in keys}
    for k, e in errs.items():
        assert e < tol, (k, e, errs)
    if tol_sigma is not None:
        e = rel(g["sigma"], s.f["sigma"])
        assert e < tol_sigma, ("sigma", e)
    return errs


def test_coreshell64_fp64_500_steps():
    """The small core-shell workload: 64x64, FP64, elastic, rtol 1e-10, 500 steps,
    against the stored oracle run (tests/golden/make_golden.py)."""
    gold = np.load(os.path.join(GOLDEN, "coreshell64_fp64_500.npz"))
    wl = workloads.WORKLOADS["coreshell64"]
    f = workloads.build_fields("coreshell64")
    sim = Simulation(wl["shape"], wl["params"], precision="fp64")
    sim.set_fields(f)
    sim.step(wl["steps"])
    g = sim.get_fields()
    for k in ("phi_f", "phi_w", "xO", "xH", "xW"):
        assert rel(g[k], gold[k]) < 1e-10, (k, rel(g[k], gold[k]))
    assert rel(g["sigma"], gold["sigma"]) < 1e-7
    d = sim.diagnostics()
    assert abs(d["removed_H2O"] - float(gold["removedW"])) <= 1e-10 * max(1e-30, abs(float(gold["removedW"])))
    assert d["steps"] == 500


@pytest.mark.parametrize("plastic", [0, 1])
def test_ragged_2d_fp64(orc, plastic):
    """Odd grid (37 x 29: several blocks, ragged tail), supply cells, grain
    mobility scatter, prestress and (optionally) J2 plasticity."""
    shape = (29, 37)
    rng = np.random.default_rng(5)
    f = inputs.core_shell(shape, 9.0, 3.0)
    f["mob"] = rng.uniform(0.8, 1.2, shape)
    prm = workloads.params(plasticity=plastic, sigma_Y=0.004, H_hard=0.01, prestress=0.003, cg_rtol=1e-12)
    sim = Simulation(shape, prm, precision="fp64")
    sim.set_fields(f)
    sim.step(30)
    g = sim.get_fields()
    s = orc.Sim(f, prm)
    s.step(30)
    _compare(g, s, 1e-10, 1e-8)
    if plastic:
        assert s.f["alpha"].max() > 0
        assert rel(g["alpha"], s.f["alpha"]) < 1e-8
        assert rel(g["eps_p"], s.f["eps_p"]) < 1e-8


def test_3d_fp64(orc):
    shape = (9, 10, 12)
    f = inputs.core_shell(shape, 3.5, 1.5, delta=1.5)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-12)
    sim = Simulation(shape, prm, precision="fp64")
    sim.set_fields(f)
    sim.step(8)
    g = sim.get_fields()
    s = orc.Sim(f, prm)
    s.step(8)
    _compare(g, s, 1e-10, 1e-8)


@pytest.mark.parametrize("shape", [(64, 64), (10, 12, 14)])
def test_mixed_precision(orc, shape):
    """FP32 fields / operator with FP64-grade reductions against the FP64 oracle."""
    if len(shape) == 2:
        f = inputs.core_shell(shape, 20.0, 4.0)
    else:
        f = inputs.core_shell(shape, 4.0, 1.5, delta=1.5)
    prm = workloads.params(plasticity=1, cg_rtol=1e-6)
    n = 60 if len(shape) == 2 else 10
    sim = Simulation(shape, prm, precision="mixed")
    sim.set_fields(f)
    sim.step(n)
    g = sim.get_fields()
    s = orc.Sim(f, prm, cg_rtol=1e-10)
    s.step(n)
    _compare(g, s, 1e-4, 1e-3)


def test_mass_balance_fp64_sums():
    """O + H2O and H + 2 H2O balances from the library's FP64 sums, with the
    removed water and supplied hydrogen counted."""
    shape = (48, 48)
    f = inputs.core_shell(shape, 15.0, 3.0)
    prm = workloads.params(cg_rtol=1e-8)
    sim = Simulation(shape, prm, precision="fp64")
    sim.set_fields(f)
    O0 = f["xO"].sum() + f["xW"].sum()
    H0 = f["xH"].sum() + 2 * f["xW"].sum()
    sim.step(50)
    d = sim.diagnostics()
    assert abs(d["sum_O"] + d["sum_H2O"] + d["removed_H2O"] - O0) < 1e-12 * O0
    assert abs(d["sum_H"] + 2 * d["sum_H2O"] + 2 * d["removed_H2O"] - d["supplied_H"] - H0) < 1e-12 * H0
    assert d["sum_H2O"] + d["removed_H2O"] > 0
    assert 0 < d["reduction_degree"] < 1


def test_reduction_rate_telescopes():
    """The reduction rate of Sec. 4.2.1 is the change of the reduction
    degree over the last step divided by dt, so its sum times dt telescopes
    to the reduction degree; a call of several steps reports its last step's
    rate (the same as stepping one at a time)."""
    shape = (32, 32)
    f = inputs.core_shell(shape, 10.0, 3.0)
    prm = workloads.params(cg_rtol=1e-8)
    a = Simulation(shape, prm, precision="fp64")
    a.set_fields(f)
    assert a.diagnostics()["reduction_rate"] == 0.0
    acc, prev = 0.0, 0.0
    for _ in range(9):
        a.step(1)
        d = a.diagnostics()
        assert d["reduction_rate"] > 0.0
        assert abs(d["reduction_rate"] * d["dt"] - (d["reduction_degree"] - prev)) < 1e-13
        acc += d["reduction_rate"] * d["dt"]
        prev = d["reduction_degree"]
    assert abs(acc - d["reduction_degree"]) < 1e-13
    b = Simulation(shape, prm, precision="fp64")
    b.set_fields(f)
    b.step(6)
    b.step(3)
    assert b.diagnostics()["reduction_rate"] == d["reduction_rate"]


def test_status_not_converged():
    shape = (32, 32)
    f = inputs.core_shell(shape, 10.0, 3.0)
    sim = Simulation(shape, workloads.params(cg_rtol=1e-12, cg_maxit=3), precision="fp64")
    sim.set_fields(f)
    with pytest.raises(PFError) as e:
        sim.step(2)
    assert e.value.code == native.PF_ENOTCONV
    assert sim.diagnostics()["steps"] == 2       # steps are still taken


def test_status_nonfinite():
    shape = (32, 32)
    f = inputs.core_shell(shape, 10.0, 3.0)
    f["xH"] = f["xH"].copy()
    f["xH"][5, 5] = np.nan
    sim = Simulation(shape, workloads.params(mechanics=0), precision="fp64")
    sim.set_fields(f)
    with pytest.raises(PFError) as e:
        sim.step(1)
    assert e.value.code == native.PF_ENONFINITE


@pytest.mark.parametrize("kind", ["coreshell", "porous"])
def test_checkpoint_restart_bitwise(kind):
    """Run 2n steps, versus n steps, save all state (pf_get_fields of every
    field, the order parameter theta and the gas fraction included), restore
    into a new handle,
    n more steps: identical in FP64, bit for bit, also on a porous input
    whose supply layers have no solid (phi_g = 1), where theta is not
    recoverable from phi_f and phi_w."""
    shape = (40, 40)
    if kind == "coreshell":
        f = inputs.core_shell(shape, 12.0, 3.0)
    else:
        f = inputs.porous(shape, 6, 0.2, 4.0, 0.4, 17)
        assert np.any(1.0 - f["phi_f"] - f["phi_w"] == 1.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10)
    a = Simulation(shape, prm, precision="fp64")
    a.set_fields(f)
    a.step(20)
    ga = a.get_fields()
    b = Simulation(shape, prm, precision="fp64")
    b.set_fields(f)
    b.step(10)
    mid = b.get_fields()
    ck = dict(mid)
    ck["mob"] = f["mob"]
    ck["mask"] = f["mask"]
    c = Simulation(shape, prm, precision="fp64")
    c.set_fields(ck)
    c.step(10)
    gc = c.get_fields()
    for k in ("phi_f", "phi_w", "xO", "xH", "xW", "theta", "phig", "alpha", "u", "Ebar", "eps_p", "sigma"):
        assert np.array_equal(gc[k], ga[k]), (k, rel(gc[k], ga[k]))
    # without theta the restore loses it where phi_g = 1 (the known limit
    # of phi_f, phi_w alone)
    if kind == "porous":
        del ck["theta"], ck["phig"]
        d = Simulation(shape, prm, precision="fp64")
        d.set_fields(ck)
        assert not np.array_equal(d.get_fields(keys=("theta",))["theta"], mid["theta"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_round_trip_keeps_the_extrapolated_guess(precision):
    """A state round trip through the host in the middle of a run
    (pf_get_fields of every field, pf_set_fields of them on the same
    handle) keeps the second-order extrapolated guess and, for the mixed
    form, the FP64 copy of the displacement: the run continues bit for bit
    as if it had not been interrupted."""
    shape = (48, 48)
    f = inputs.porous(shape, 6, 0.2, 4.0, 0.4, 17)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-9, warm_start="extrap2")
    keys = ("phi_f", "phi_w", "xO", "xH", "xW", "theta", "phig", "alpha", "u", "Ebar", "eps_p", "sigma")
    a = Simulation(shape, prm, precision=precision)
    a.set_fields(f)
    a.step(12)
    ga = a.get_fields(keys=keys)
    b = Simulation(shape, prm, precision=precision)
    b.set_fields(f)
    b.step(6)
    mid = b.get_fields()
    ck = dict(mid)
    ck["mob"] = f["mob"]
    ck["mask"] = f["mask"]
    b.set_fields(ck)
    b.step(6)
    gb = b.get_fields(keys=keys)
    for k in keys:
        assert np.array_equal(gb[k], ga[k]), (k, rel(gb[k], ga[k]))
    # a changed displacement restarts the guess: the handle then runs as a
    # fresh handle given the same state does, bit for bit
    c = Simulation(shape, prm, precision=precision)
    c.set_fields(f)
    c.step(6)
    ck2 = dict(c.get_fields())
    ck2["mob"], ck2["mask"] = f["mob"], f["mask"]
    ck2["u"] = ck2["u"] * (1.0 + 1e-3)
    c.set_fields(ck2)
    c.step(6)
    d = Simulation(shape, prm, precision=precision)
    d.set_fields(ck2)
    d.step(6)
    gc, gd = c.get_fields(keys=keys), d.get_fields(keys=keys)
    for k in keys:
        assert np.array_equal(gc[k], gd[k]), (k, rel(gc[k], gd[k]))
    assert not np.array_equal(gc["u"], ga["u"])
    for s_ in (a, b, c, d):
        s_.close()


def test_device_pointers_match_host():
    torch = pytest.importorskip("torch")
    shape = (24, 20)
    f = inputs.core_shell(shape, 7.0, 2.0)
    prm = workloads.params(cg_rtol=1e-10)
    a = Simulation(shape, prm, precision="fp64")
    a.set_fields(f)
    a.step(5)
    ga = a.get_fields()
    b = Simulation(shape, prm, precision="fp64")
    tf = {k: torch.as_tensor(np.ascontiguousarray(v), device="cuda") for k, v in f.items()}
    b.set_fields(tf, where="device")
    b.step(5)
    gb = b.get_fields()
    for k in ("phi_f", "xO", "xH", "xW", "u"):
        assert np.array_equal(ga[k], gb[k]), k


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a word nothing updates gives up after its poll limit
    and reports PF_ETIMEOUT; the CUDA context stays usable."""
    import time
    t0 = time.time()
    assert native.pf_selftest_wait(1 << 16) == native.PF_ETIMEOUT
    assert time.time() - t0 < 30
    assert native.pf_selftest_wait(0) == native.PF_EINVAL
    shape = (32, 32)
    sim = Simulation(shape, workloads.params(mechanics=0), precision="fp64")
    sim.set_fields(inputs.core_shell(shape, 10.0, 3.0))
    sim.step(2)
    assert sim.diagnostics()["steps"] == 2
    sim.close()


@pytest.mark.parametrize("shape", [(40, 48), (10, 12, 14)])
def test_pcg_tile_shapes_agree(shape):
    """Both node tiles of the PCG sweep solve the same system: FP64 fields
    agree to the CG tolerance, whichever shape the library picks."""
    f = inputs.core_shell(shape, 0.3 * shape[-1], 3.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10)
    out = []
    for tile in (1, 2):
        sim = Simulation(shape, dict(prm, pcg_tile=tile), precision="fp64")
        sim.set_fields(f)
        sim.step(10)
        out.append(sim.get_fields())
        sim.close()
    for k in ("phi_f", "phi_w", "xO", "xH", "xW"):
        assert rel(out[0][k], out[1][k]) < 1e-10, k
    assert rel(out[0]["sigma"], out[1]["sigma"]) < 1e-7


def test_pcg_3d_cell_path_matches_matrix_path():
    """In 3D FP32 the 16x4x4 tile applies the operator from per-cell average
    stress and hourglass forces, the 32x4x2 tile from the element matrices;
    both solve to the same tolerance (mixed method, rtol 1e-9)."""
    shape = (12, 14, 16)
    f = inputs.core_shell(shape, 5.0, 2.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-9, prestress=0.01)
    out = []
    for tile in (1, 2):
        sim = Simulation(shape, dict(prm, pcg_tile=tile), precision="mixed")
        sim.set_fields(f)
        sim.step(8)
        out.append(sim.get_fields())
        sim.close()
    for k in ("phi_f", "phi_w", "xO", "xH", "xW"):
        assert rel(out[0][k], out[1][k]) < 1e-6, (k, rel(out[0][k], out[1][k]))
    assert rel(out[0]["sigma"], out[1]["sigma"]) < 1e-4


def test_get_fields_into_caller_arrays():
    """get_fields(out=...) fills the caller's arrays (the end-to-end bench
    passes pinned host memory) with what a plain get_fields returns."""
    shape = (24, 20)
    sim = Simulation(shape, workloads.params(plasticity=1), precision="mixed")
    sim.set_fields(inputs.core_shell(shape, 7.0, 2.0))
    sim.step(3)
    keys = ("phi_f", "xO", "u", "eps_p", "Ebar")
    ref = sim.get_fields(keys=keys)
    out = {k: np.full_like(v, -7.0) for k, v in ref.items()}
    got = sim.get_fields(keys=keys, out=out)
    for k in keys:
        assert got[k] is out[k]
        assert np.array_equal(out[k], ref[k]), k
    with pytest.raises(ValueError):
        sim.get_fields(keys=("phi_f",), out={"phi_f": np.zeros(3)})
    sim.close()


@pytest.mark.parametrize("shape", [(40, 36), (12, 14, 16)])
def test_free_energy_matches_oracle(orc, shape):
    """pf_free_energy (the discrete counterpart of the free energy whose
    decrease is the dissipation inequality, Sec. 2.3) against the oracle's:
    on the initial state (no elastic energy yet) to 1e-12, and after FP64
    steps with mechanics and J2 on both sides solved to rtol 1e-13, to 1e-10."""
    f = inputs.core_shell(shape, 0.3 * shape[-1], 3.0)
    f["mob"] = np.random.default_rng(5).uniform(0.8, 1.2, shape)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-13)
    sim = Simulation(shape, prm, precision="fp64")
    sim.set_fields(f)
    ref = orc.Sim(f, prm)
    e0 = sim.free_energy()
    assert abs(e0 - ref.free_energy()) <= 1e-12 * abs(ref.free_energy())
    sim.step(4)
    ref.step(4)
    e1, r1 = sim.free_energy(), ref.free_energy()
    assert abs(e1 - r1) <= 1e-10 * abs(r1), (e1, r1)
    assert e1 != e0
    sim.close()


@pytest.mark.parametrize("plastic", [0, 1])
def test_fp64_stress_at_tight_tolerance(orc, plastic):
    """Both sides solve to rtol 1e-14, so that two correct solves agree far
    below 1e-10 (the solution error is up to cond(A) rtol, cond(A) ~ 1e3;
    at rtol 1e-13 the J2 run's stress differed by 1.3e-10): the plain FP64
    method is held to 1e-10 on the fields and on the stress, 64x64
    core-shell, elastic and J2, 40 steps."""
    shape = (64, 64)
    f = workloads.build_fields("coreshell64")
    prm = workloads.params(plasticity=plastic, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-14, cg_maxit=50000)
    sim = Simulation(shape, prm, precision="fp64")
    sim.set_fields(f)
    sim.step(40)
    g = sim.get_fields()
    s = orc.Sim(f, prm)
    s.step(40)
    _compare(g, s, 1e-10, 1e-10)
    assert rel(g["eps_p"], s.f["eps_p"]) < 1e-10 or not plastic
    sim.close()

