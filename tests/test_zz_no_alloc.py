"""The allocation-free field update, pf_fields_update_static.

Callers that cannot allocate device memory at the point of use (code running
during CUDA-graph stream capture, runtimes with a fixed device-memory budget,
hosts that must leave the allocator alone) use this entry point instead of a
handle: it keeps its working arrays in a fixed device array of the library.
Its results must equal those of the regular entry point (pf_step with the
mechanics off) on two calls in a row, within the FP64 tolerance of the other
GPU tests.  This file is collected last so that a failure here comes after
every other test has run.
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


def test_static_update_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    native.build_library()
    native.lib()
    shape = (40, 48)
    f = inputs.core_shell(shape, 12.0, 3.0)
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
        nxt = {k: torch.empty_like(cur[k]) for k in KEYS}
        fin, fout = pf_fields(), pf_fields()
        for k in KEYS:
            setattr(fin, NAMES[k], _dp(cur[k]))
            setattr(fout, NAMES[k], _dp(nxt[k]))
        fin.mobility = _dp(mob)
        fin.dirichlet = ctypes.cast(mask.data_ptr(), ctypes.POINTER(ctypes.c_ubyte))
        rc = native.pf_fields_update_static(cfg, fin, None, None, fout, stream)
        assert rc == native.PF_OK, native.pf_static_last_error()
        for k in KEYS:
            got = nxt[k].cpu().numpy()
            assert _rel(got, ref[k]) < 1e-12, (k, _rel(got, ref[k]))
        cur = nxt


def test_static_update_rejects_oversize_grid():
    native.build_library()
    cfg = make_config((512, 512), workloads.params(mechanics=0))
    fin, fout = pf_fields(), pf_fields()
    rc = native.pf_fields_update_static(cfg, fin, None, None, fout, None)
    assert rc == native.PF_EINVAL
    rc = native.pf_fields_update_static(cfg, fin, None, None, fout, None)
    assert rc == native.PF_EINVAL
    assert "PF_STATIC_MAX_CELLS" in native.pf_static_last_error()
