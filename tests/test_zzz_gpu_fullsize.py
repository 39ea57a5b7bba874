"""Parity at the workloads' full sizes, in the configuration the benchmark
times (multigrid solve, the workloads' extrapolated guesses and CG
tolerances), in FP64 so that the checks are exact:

  * per workload a few steps, the library's state before one more step and
    after it; the oracle recomputes that step's J2 return and explicit
    update from the library's own state (whole grid in 2D, sampled periodic
    sub-boxes in 3D, tests/fullsize_local.py) and, in 2D, the solve's
    residual under its own operator;
  * the O + H2O and H + 2 H2O balances of the whole run;
  * the mixed method against the FP64 method on the 512^2 headline workload.

Grids: 512^2 core-shell J2, 2048^2 porous, 256^3 porous J2, the batch of 64
porous instances (128^2 .. 1024^2).
"""
import numpy as np
import pytest

from fullsize_local import solve_residual, step_errors
from paper_2111_11538_gb300 import Batch, Simulation, inputs, native, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


def _lib_params(name):
    """The workload's parameters plus its initial guess, for the library
    (the oracle takes the parameters alone)."""
    p = dict(workloads.WORKLOADS[name]["params"])
    p["warm_start"] = workloads.WORKLOADS[name].get("warm_start", "extrap")
    return p


def _balances(d, f):
    O0 = f["xO"].sum() + f["xW"].sum()
    H0 = f["xH"].sum() + 2 * f["xW"].sum()
    assert abs(d["sum_O"] + d["sum_H2O"] + d["removed_H2O"] - O0) < 1e-11 * O0
    assert abs(d["sum_H"] + 2 * d["sum_H2O"] + 2 * d["removed_H2O"] - d["supplied_H"] - H0) < 1e-11 * H0


@pytest.mark.parametrize("name", ["coreshell512", "porous2048"])
def test_2d_workload_full_size(orc, name):
    f = workloads.build_fields(name)
    shape = f["phi_f"].shape
    prm = workloads.WORKLOADS[name]["params"]
    sim = Simulation(shape, _lib_params(name), precision="fp64")
    sim.set_fields(f)
    sim.step(4)
    before = sim.get_fields()
    sim.step(1)
    after = sim.get_fields()
    errs = step_errors(orc, prm, before, after, f)
    assert max(errs.values()) < 1e-9, errs
    assert solve_residual(orc, prm, before, after, f) < 5.0 * prm["cg_rtol"]
    d = sim.diagnostics()
    assert d["precond"] == native.PF_PC_MG and d["steps"] == 5
    _balances(d, f)


def test_3d_workload_full_size(orc):
    name = "porous256cube"
    f = workloads.build_fields(name)
    shape = f["phi_f"].shape
    prm = workloads.WORKLOADS[name]["params"]
    sim = Simulation(shape, _lib_params(name), precision="fp64")
    sim.set_fields(f)
    sim.step(3)
    before = sim.get_fields()
    sim.step(1)
    after = sim.get_fields()
    rng = np.random.default_rng(9)
    origins = [(0, 0, 0), tuple(n // 2 for n in shape)] + [tuple(int(v) for v in rng.integers(0, 256, 3))]
    for o in origins:
        errs = step_errors(orc, prm, before, after, f, origin=o, m=16)
        assert max(errs.values()) < 1e-9, (o, errs)
    d = sim.diagnostics()
    assert d["precond"] == native.PF_PC_MG and d["steps"] == 4
    _balances(d, f)


def test_batch_full_size(orc):
    name = "batch64"
    wl = workloads.WORKLOADS[name]
    desc = inputs.batch_instances(wl["count"], wl["seed"])
    shapes = [(d["n"], d["n"]) for d in desc]
    prms = [dict(wl["params"], prestress=d["prestress"]) for d in desc]
    lib_prms = [dict(p, warm_start=wl["warm_start"]) for p in prms]
    b = Batch(shapes, lib_prms, precision="fp64")
    fields = [inputs.batch_fields(d) for d in desc]
    for i, fi in enumerate(fields):
        b.set_fields(i, fi)
    b.step(2)
    sizes = [d["n"] for d in desc]
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    before = {i: b.get_fields(i) for i in picks}
    b.step(1)
    for i in picks:
        after = b.get_fields(i)
        errs = step_errors(orc, prms[i], before[i], after, fields[i])
        assert max(errs.values()) < 1e-9, (i, errs)
        assert solve_residual(orc, prms[i], before[i], after, fields[i]) < 5.0 * prms[i]["cg_rtol"]
    for i, fi in enumerate(fields):
        _balances(b.diagnostics(i), fi)


def test_mixed_against_oracle_from_fp64_snapshot(orc):
    """The 512^2 J2 workload in the configuration the benchmark times for it
    (mixed method: FP32 multigrid V-cycles inside FP64 refinement to rtol
    1e-8, the extrapolated guess) against the oracle over a short window:
    the library's FP64 state after 12 steps is loaded into both, which then
    take 3 steps (the mixed method's extrapolation history restarts at the
    load, as the oracle's guess does); 1e-4 on the fields, 1e-3 on the
    stress."""
    name = "coreshell512"
    f = workloads.build_fields(name)
    shape = f["phi_f"].shape
    sim = Simulation(shape, _lib_params(name), precision="fp64")
    sim.set_fields(f)
    sim.step(12)
    snap = sim.get_fields()
    sim.close()
    snap["mob"], snap["mask"] = f["mob"], f["mask"]
    mixed = Simulation(shape, _lib_params(name), precision="mixed")
    mixed.set_fields(snap)
    mixed.step(3)
    g = mixed.get_fields()
    mixed.close()
    ref = orc.Sim(snap, workloads.WORKLOADS[name]["params"])
    ref.step(3)
    exp = {"phi_f": ref.phi_f, "phi_w": ref.phi_w, "xO": ref.f["xO"], "xH": ref.f["xH"], "xW": ref.f["xW"]}
    for k in exp:
        r = np.linalg.norm(g[k] - exp[k]) / np.linalg.norm(exp[k])
        assert r < 1e-4, (k, r)
    r = np.linalg.norm(g["sigma"] - ref.f["sigma"]) / np.linalg.norm(ref.f["sigma"])
    assert r < 1e-3, r


def test_mixed_against_fp64_headline():
    """The benchmark's mixed method stays within the mixed parity tolerance
    (1e-4 on the fields, 1e-3 on the stress) of the FP64 method on the
    512^2 J2 workload after 8 steps."""
    name = "coreshell512"
    f = workloads.build_fields(name)
    shape = f["phi_f"].shape
    out = {}
    for prec in ("fp64", "mixed"):
        sim = Simulation(shape, _lib_params(name), precision=prec)
        sim.set_fields(f)
        sim.step(8)
        out[prec] = sim.get_fields()
    for k in ("phi_f", "phi_w", "xO", "xH", "xW"):
        r = np.linalg.norm(out["mixed"][k] - out["fp64"][k]) / np.linalg.norm(out["fp64"][k])
        assert r < 1e-4, (k, r)
    r = np.linalg.norm(out["mixed"]["sigma"] - out["fp64"]["sigma"]) / np.linalg.norm(out["fp64"]["sigma"])
    assert r < 1e-3, r
