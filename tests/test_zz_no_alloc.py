"""The allocation-free field update, pf_fields_update_static.

Callers that cannot allocate device memory at the point of use (runtimes
with a fixed device-memory budget, hosts that must leave the allocator alone)
use this entry point instead of a handle: it keeps its working arrays in a
fixed device array of the library.  Its results must equal those of the
regular entry point (pf_step with the mechanics off) on two calls in a row,
within the FP64 tolerance of the other GPU tests, in 2D and 3D; with given
coupling scalars (tr eps_e, |dev eps_e|^2) they must equal the oracle's
field update on the same inputs.  This file is collected last so that a
failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2111_11538_gb300 import Simulation, inputs, make_config, native, workloads
from paper_2111_11538_gb300.native import pf_fields

pytestmark = pytest.mark.gpu

KEYS = ("phi_f", "phi_w", "xO", "xH", "xW")
NAMES = {"phi_f": "phi_f", "phi_w": "phi_w", "xO": "x_O", "xH": "x_H", "xW": "x_H2O"}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _dp(t):
    return ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_double))


def _static_call(cfg, cur, mob, mask, stream, trE=None, devE2=None):
    """One call through the C ABI on caller-owned device buffers; returns the
    new fields (device tensors)."""
    torch = pytest.importorskip("torch")
    nxt = {k: torch.empty_like(cur[k]) for k in KEYS}
    fin, fout = pf_fields(), pf_fields()
    for k in KEYS:
        setattr(fin, NAMES[k], _dp(cur[k]))
        setattr(fout, NAMES[k], _dp(nxt[k]))
    fin.mobility = _dp(mob)
    fin.dirichlet = ctypes.cast(mask.data_ptr(), ctypes.POINTER(ctypes.c_ubyte))
    rc = native.pf_fields_update_static(cfg, fin, None if trE is None else _dp(trE),
                                        None if devE2 is None else _dp(devE2), fout, stream)
    assert rc == native.PF_OK, native.pf_static_last_error()
    return nxt


@pytest.mark.parametrize("shape", [(40, 48), (16, 16, 16)])
def test_static_update_matches_regular_entry_point_twice(shape):
    torch = pytest.importorskip("torch")
    native.build_library()
    native.lib()
    f = inputs.core_shell(shape, 12.0 if len(shape) == 2 else 5.0, 3.0)
    f["mob"] = np.random.default_rng(3).uniform(0.8, 1.2, shape)
    prm = workloads.params(mechanics=0)

    # regular entry point: handle, mechanics off, two steps
    sim = Simulation(shape, prm, precision="fp64", mechanics=0)
    sim.set_fields(f)
    sim.step(1)
    ref1 = sim.get_fields(keys=KEYS)
    sim.step(1)
    ref2 = sim.get_fields(keys=KEYS)
    sim.close()

    # allocation-free entry point on caller-owned device buffers
    cfg = make_config(shape, prm, precision="fp64", mechanics=0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    cur = {k: dev(f[k]) for k in KEYS}
    mob = dev(f["mob"])
    mask = torch.as_tensor(np.ascontiguousarray(f["mask"], dtype=np.uint8), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for ref in (ref1, ref2):
        nxt = _static_call(cfg, cur, mob, mask, stream)
        for k in KEYS:
            got = nxt[k].cpu().numpy()
            assert _rel(got, ref[k]) < 1e-12, (k, _rel(got, ref[k]))
        cur = nxt


def test_static_update_with_coupling_scalars_matches_oracle_twice():
    """Nonzero tr eps_e and |dev eps_e|^2 per cell (the elastic driving force
    of the order parameter): two calls against the oracle's field update on
    the same inputs."""
    torch = pytest.importorskip("torch")
    import oracle
    native.build_library()
    shape = (36, 44)
    f = inputs.core_shell(shape, 11.0, 3.0)
    rng = np.random.default_rng(11)
    f["mob"] = rng.uniform(0.8, 1.2, shape)
    trE = rng.uniform(-0.06, 0.02, shape)
    devE2 = rng.uniform(0.0, 4e-3, shape)
    prm = workloads.params(mechanics=0)
    ref = oracle.Sim(f, prm)
    ref.f["trE"][...] = trE
    ref.f["devE2"][...] = devE2
    cfg = make_config(shape, prm, precision="fp64", mechanics=0)
    cfg.dt = ref.dt
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    cur = {k: dev(f[k]) for k in KEYS}
    mob = dev(f["mob"])
    mask = torch.as_tensor(np.ascontiguousarray(f["mask"], dtype=np.uint8), device="cuda")
    tE, dE = dev(trE), dev(devE2)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        ref.fields_update()
        exp = {"phi_f": ref.phi_f, "phi_w": ref.phi_w, "xO": ref.f["xO"], "xH": ref.f["xH"], "xW": ref.f["xW"]}
        cur = _static_call(cfg, cur, mob, mask, stream, tE, dE)
        for k in KEYS:
            got = cur[k].cpu().numpy()
            assert _rel(got, exp[k]) < 1e-12, (k, _rel(got, exp[k]))


def test_static_update_rejects_oversize_grid():
    native.build_library()
    cfg = make_config((512, 512), workloads.params(mechanics=0))
    fin, fout = pf_fields(), pf_fields()
    rc = native.pf_fields_update_static(cfg, fin, None, None, fout, None)
    assert rc == native.PF_EINVAL
    rc = native.pf_fields_update_static(cfg, fin, None, None, fout, None)
    assert rc == native.PF_EINVAL
    assert "PF_STATIC_MAX_CELLS" in native.pf_static_last_error()
