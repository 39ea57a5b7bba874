"""Batches: many independent instances advanced by the same launches.

* a batch gives each instance the result it gets alone: bit for bit when
  only the cell kernels run (their block split per instance is the one of a
  single handle), within the FP64 CG tolerance with the mechanics on (the
  PCG blocks of a launch are split between the instances, so its sums are
  taken in another order);
* steps replayed from the CUDA graph equal steps launched one by one;
* the status of a batch step is the worst over its instances.
"""
import numpy as np
import pytest

from paper_2111_11538_gb300 import Batch, PFError, Simulation, inputs, native, workloads

pytestmark = pytest.mark.gpu

KEYS = ("phi_f", "phi_w", "xO", "xH", "xW")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    native.build_library()
    native.lib()


def _instances():
    """Three uneven 2D instances: two core-shell particles and a porous patch."""
    shapes = [(40, 48), (64, 64), (33, 29)]
    fields = [inputs.core_shell(shapes[0], 12.0, 3.0),
              inputs.core_shell(shapes[1], 20.0, 4.0),
              inputs.porous(shapes[2], 4, 0.2, 4.0, 0.4, seed=7)]
    return shapes, fields


def _single(shape, prm, f, steps, precision="fp64", profile=False):
    sim = Simulation(shape, prm, precision=precision)
    if profile:
        sim.profile(True)
    sim.set_fields(f)
    sim.step(steps)
    g = sim.get_fields()
    sim.close()
    return g


def test_batch_cells_only_bitwise_equal_to_single():
    shapes, fields = _instances()
    prm = workloads.params(mechanics=0)
    b = Batch(shapes, prm, precision="fp64")
    assert len(b) == 3
    for i, f in enumerate(fields):
        b.set_fields(i, f)
    b.step(7)
    for i, (s, f) in enumerate(zip(shapes, fields)):
        ref = _single(s, prm, f, 7)
        got = b.get_fields(i, keys=KEYS)
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (i, k, rel(got[k], ref[k]))
        assert b.diagnostics(i)["steps"] == 7
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_batch_mechanics_matches_single(precision, tol):
    shapes, fields = _instances()
    # the batch resolves the library's preconditioner choice once for all its
    # instances (the 33x29 one keeps it at Jacobi): singles use the same
    prms = [workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10 if precision == "fp64" else 1e-8,
                             prestress=p, precond="jacobi") for p in (0.0, 0.01, 0.02)]
    b = Batch(shapes, prms, precision=precision)
    for i, f in enumerate(fields):
        b.set_fields(i, f)
    b.step(12)
    for i, (s, f) in enumerate(zip(shapes, fields)):
        ref = _single(s, prms[i], f, 12, precision=precision)
        got = b.get_fields(i)
        for k in KEYS:
            assert rel(got[k], ref[k]) < tol, (i, k, rel(got[k], ref[k]))
        assert rel(got["sigma"], ref["sigma"]) < 1e3 * tol, (i, rel(got["sigma"], ref["sigma"]))
        d = b.diagnostics(i)
        assert d["steps"] == 12 and d["cg_iters_total"] > 0
    b.close()


def test_graph_replay_equals_eager_launches():
    """With per-kernel timing on, every kernel is launched directly; without
    it, pairs of steps replay a captured graph.  Same launches, same bits."""
    shape = (48, 40)
    f = inputs.core_shell(shape, 14.0, 3.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.004, H_hard=0.01, cg_rtol=1e-10)
    eager = _single(shape, prm, f, 9, profile=True)
    graph = _single(shape, prm, f, 9, profile=False)
    for k in KEYS + ("u", "sigma", "eps_p"):
        assert np.array_equal(eager[k], graph[k]), (k, rel(graph[k], eager[k]))


def test_batch_graph_replay_equals_eager_launches():
    shapes, fields = _instances()
    prm = workloads.params(plasticity=0, cg_rtol=1e-10)
    out = []
    for prof in (True, False):
        b = Batch(shapes, prm, precision="fp64")
        if prof:
            b.profile(True)
        for i, f in enumerate(fields):
            b.set_fields(i, f)
        b.step(6)
        if prof:
            p = b.profile_read()
            assert p["count"]["cg"] == 6 and p["count"]["update"] == 6   # one launch per class and step
        out.append([b.get_fields(i, keys=KEYS + ("u",)) for i in range(len(shapes))])
        b.close()
    for i in range(len(shapes)):
        for k in KEYS + ("u",):
            assert np.array_equal(out[0][i][k], out[1][i][k]), (i, k)


def test_batch_status_is_worst_over_instances():
    shapes, fields = _instances()
    bad = dict(fields[1])
    bad["xH"] = bad["xH"].copy()
    bad["xH"][3, 3] = np.nan
    b = Batch(shapes, workloads.params(mechanics=0), precision="fp64")
    for i, f in enumerate([fields[0], bad, fields[2]]):
        b.set_fields(i, f)
    with pytest.raises(PFError) as e:
        b.step(1)
    assert e.value.code == native.PF_ENONFINITE
    b.close()


def test_batch_rejects_single_instance_calls_and_bad_index():
    shapes, fields = _instances()
    b = Batch(shapes, workloads.params(mechanics=0), precision="fp64")
    f = native.pf_fields()
    assert native.pf_set_fields(b.h, f, native.PF_HOST) == native.PF_EINVAL
    assert native.pf_get_fields(b.h, f, native.PF_HOST) == native.PF_EINVAL
    assert native.pf_batch_set_fields(b.h, 3, f, native.PF_HOST) == native.PF_EINVAL
    assert native.pf_batch_get_diagnostics(b.h, -1)[0] == native.PF_EINVAL
    with pytest.raises(PFError) as e:
        b.step(1)                      # no fields yet
    assert e.value.code == native.PF_ESTATE
    b.close()
