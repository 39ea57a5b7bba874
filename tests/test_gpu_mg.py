"""Multigrid-preconditioned CG (2D, precond="mg"): it solves the same systems
as the Jacobi preconditioner, to the same stopping rule, in far fewer
iterations.

* the 500-step 64x64 core-shell run against the stored oracle run, with the
  tolerances of the Jacobi path (1e-10 on the fields, 1e-7 on the stress);
* MG against Jacobi on hierarchies of every kind: one level (odd sizes:
  the V-cycle reduces to a Chebyshev polynomial preconditioner), grid-wide
  coarse levels followed by levels run by one block (96x80 -> ... -> 6x5),
  several grid-wide levels (256x256), both storage types.  Two solves that
  both meet ||r|| <= rtol ||b|| differ by up to cond(A) rtol (cond ~ 1e3
  here), so after a few steps the fields agree to 1e-8 (FP64, rtol 1e-10)
  or 1e-5 (mixed, rtol 1e-8), the stress to 1e3 times that;
* a cold-start solve at 128x128 takes at most a fifth of Jacobi's iterations;
* batches and CUDA-graph replay behave as with Jacobi;
* 3D (every level on the whole grid): against the oracle at 16^3 with the
  tolerances of the 3D Jacobi parity test (1e-10 fields, 1e-8 stress), and
  against Jacobi on 3-, 2- and 1-level hierarchies in both storage types.
"""
import os

import numpy as np
import pytest

from paper_2111_11538_gb300 import Batch, Simulation, inputs, native, workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KEYS = ("phi_f", "phi_w", "xO", "xH", "xW")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


def _run(shape, prm, f, steps, precision, precond, tile=None):
    p = dict(prm, precond=precond)
    if tile is not None:
        p["pcg_tile"] = tile
    sim = Simulation(shape, p, precision=precision)
    sim.set_fields(f)
    sim.step(steps)
    g = sim.get_fields()
    d = sim.diagnostics()
    sim.close()
    return g, d


def test_coreshell64_fp64_500_steps_mg():
    gold = np.load(os.path.join(GOLDEN, "coreshell64_fp64_500.npz"))
    wl = workloads.WORKLOADS["coreshell64"]
    g, d = _run(wl["shape"], wl["params"], workloads.build_fields("coreshell64"), wl["steps"], "fp64", "mg")
    for k in KEYS:
        assert rel(g[k], gold[k]) < 1e-10, (k, rel(g[k], gold[k]))
    assert rel(g["sigma"], gold["sigma"]) < 1e-7
    assert d["cg_iters_total"] > 0


@pytest.mark.parametrize("shape", [(33, 29), (96, 80), (256, 256)])
@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-10, 1e-8), ("mixed", 1e-8, 1e-5)])
def test_mg_matches_jacobi(shape, precision, rtol, tol):
    f = inputs.core_shell(shape, 0.3 * min(shape), 0.06 * min(shape) + 1.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=rtol, prestress=0.01)
    gj, dj = _run(shape, prm, f, 6, precision, "jacobi")
    gm, dm = _run(shape, prm, f, 6, precision, "mg")
    for k in KEYS:
        assert rel(gm[k], gj[k]) < tol, (k, rel(gm[k], gj[k]))
    assert rel(gm["sigma"], gj["sigma"]) < 1e3 * tol, rel(gm["sigma"], gj["sigma"])
    assert rel(gm["Ebar"], gj["Ebar"]) < 1e3 * tol
    assert dm["cg_iters_total"] < dj["cg_iters_total"], (dm["cg_iters_total"], dj["cg_iters_total"])


@pytest.mark.parametrize("tile", [1, 2])
def test_mg_both_tiles(tile):
    shape = (64, 96)
    f = inputs.core_shell(shape, 18.0, 4.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10)
    gj, _ = _run(shape, prm, f, 5, "fp64", "jacobi")
    gm, _ = _run(shape, prm, f, 5, "fp64", "mg", tile=tile)
    for k in KEYS:
        assert rel(gm[k], gj[k]) < 1e-8, (k, rel(gm[k], gj[k]))
    assert rel(gm["sigma"], gj["sigma"]) < 1e-5


def test_mg_cold_solve_iterations():
    shape = (128, 128)
    f = inputs.core_shell(shape, 40.0, 8.0)
    prm = workloads.params(plasticity=0, cg_rtol=1e-8, warm_start="zero")
    _, dj = _run(shape, prm, f, 1, "fp64", "jacobi")
    _, dm = _run(shape, prm, f, 1, "fp64", "mg")
    assert dm["cg_iters_last"] * 5 <= dj["cg_iters_last"], (dm["cg_iters_last"], dj["cg_iters_last"])


def test_mg_batch_matches_single():
    shapes = [(40, 48), (64, 64), (33, 29)]
    fields = [inputs.core_shell(shapes[0], 12.0, 3.0), inputs.core_shell(shapes[1], 20.0, 4.0),
              inputs.porous(shapes[2], 4, 0.2, 4.0, 0.4, seed=7)]
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10, precond="mg")
    b = Batch(shapes, prm, precision="fp64")
    for i, f in enumerate(fields):
        b.set_fields(i, f)
    b.step(8)
    for i, (s, f) in enumerate(zip(shapes, fields)):
        ref, _ = _run(s, prm, f, 8, "fp64", "mg")
        got = b.get_fields(i)
        for k in KEYS:
            assert rel(got[k], ref[k]) < 1e-10, (i, k, rel(got[k], ref[k]))
        assert rel(got["sigma"], ref["sigma"]) < 1e-7
    b.close()


def test_mg_graph_replay_equals_eager():
    shape = (48, 40)
    f = inputs.core_shell(shape, 14.0, 3.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10, precond="mg")
    out = []
    for prof in (True, False):
        sim = Simulation(shape, prm, precision="fp64")
        if prof:
            sim.profile(True)
        sim.set_fields(f)
        sim.step(9)
        out.append(sim.get_fields())
        sim.close()
    for k in KEYS + ("u", "sigma", "eps_p"):
        assert np.array_equal(out[0][k], out[1][k]), (k, rel(out[1][k], out[0][k]))


def test_mg3_fp64_against_oracle(orc):
    shape = (16, 16, 16)
    f = inputs.core_shell(shape, 5.0, 2.0, delta=1.5)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-12)
    g, d = _run(shape, prm, f, 6, "fp64", "mg")
    assert d["precond"] == native.PF_PC_MG and d["mg_levels"] == 2
    s = orc.Sim(f, prm)
    s.step(6)
    ref = {"phi_f": s.phi_f, "phi_w": s.phi_w, "xO": s.f["xO"], "xH": s.f["xH"], "xW": s.f["xW"]}
    for k in KEYS:
        assert rel(g[k], ref[k]) < 1e-10, (k, rel(g[k], ref[k]))
    assert rel(g["sigma"], s.f["sigma"]) < 1e-8


def test_mg3_mixed_against_oracle(orc):
    """The configuration the 3D bench times, on a grid the oracle finishes:
    mixed precision (FP32 V-cycles inside FP64 refinement), multigrid with
    three levels (32^3 -> 16^3 -> 8^3), J2 plasticity, the extrapolated
    guess, CG rtol 1e-8, a porous input with supply layers; against the
    oracle's FP64 Jacobi solves at the same rtol: 1e-4 on the fields, 1e-3
    on the stress."""
    shape = (32, 32, 32)
    f = inputs.porous(shape, 20, 0.15, 3.0, 0.4, 31)
    prm = workloads.params(plasticity=1, cg_rtol=1e-8)
    g, d = _run(shape, dict(prm, warm_start="extrap"), f, 3, "mixed", "mg")
    assert d["precond"] == native.PF_PC_MG and d["mg_levels"] == 3
    s = orc.Sim(f, prm)
    s.step(3)
    ref = {"phi_f": s.phi_f, "phi_w": s.phi_w, "xO": s.f["xO"], "xH": s.f["xH"], "xW": s.f["xW"]}
    for k in KEYS:
        assert rel(g[k], ref[k]) < 1e-4, (k, rel(g[k], ref[k]))
    assert rel(g["sigma"], s.f["sigma"]) < 1e-3, rel(g["sigma"], s.f["sigma"])


@pytest.mark.parametrize("shape,levels", [((32, 32, 32), 3), ((16, 24, 32), 2), ((9, 10, 12), 1)])
@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-10, 1e-8), ("mixed", 1e-8, 1e-5)])
def test_mg3_matches_jacobi(shape, levels, precision, rtol, tol):
    f = inputs.core_shell(shape, 0.3 * min(shape), 0.1 * min(shape) + 1.0, delta=1.5)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=rtol, prestress=0.01)
    gj, dj = _run(shape, prm, f, 4, precision, "jacobi")
    gm, dm = _run(shape, prm, f, 4, precision, "mg")
    assert dm["mg_levels"] == levels and dj["precond"] == native.PF_PC_JACOBI
    for k in KEYS:
        assert rel(gm[k], gj[k]) < tol, (k, rel(gm[k], gj[k]))
    assert rel(gm["sigma"], gj["sigma"]) < 1e3 * tol, rel(gm["sigma"], gj["sigma"])
    assert rel(gm["Ebar"], gj["Ebar"]) < 1e3 * tol
    if levels > 1:
        assert dm["cg_iters_total"] < dj["cg_iters_total"], (dm["cg_iters_total"], dj["cg_iters_total"])


def test_mg3_batch_matches_single():
    shapes = [(32, 32, 32), (16, 32, 48)]
    fields = [inputs.core_shell(shapes[0], 9.0, 3.0, delta=1.5), inputs.core_shell(shapes[1], 6.0, 2.0, delta=1.5)]
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10, precond="mg")
    b = Batch(shapes, prm, precision="fp64")
    for i, f in enumerate(fields):
        b.set_fields(i, f)
    b.step(4)
    for i, (s, f) in enumerate(zip(shapes, fields)):
        ref, d = _run(s, prm, f, 4, "fp64", "mg")
        got = b.get_fields(i)
        assert b.diagnostics(i)["mg_levels"] == d["mg_levels"] >= 2
        for k in KEYS:
            assert rel(got[k], ref[k]) < 1e-10, (i, k, rel(got[k], ref[k]))
        assert rel(got["sigma"], ref["sigma"]) < 1e-7
    b.close()
