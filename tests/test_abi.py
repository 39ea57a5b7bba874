"""C-ABI library: builds, loads without a GPU, exports every symbol of
include/pf.h, and its host-only functions agree with the oracle."""
import ctypes
import os
import re

import pytest

from paper_2111_11538_gb300 import make_config, native, workloads

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")


@pytest.fixture(scope="module")
def lib():
    native.build_library()
    return native.lib()


def _declared():
    txt = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", txt)))


def test_header_declares_binding_symbols():
    assert _declared() == sorted(native.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("shape", [(16, 16), (8, 8, 8), (40, 24)])
@pytest.mark.parametrize("over", [{}, {"D_O_g": 0.0, "D_H_g": 0.3, "D_W_g": 0.0}, {"eps_phi": 3.0}, {"k_for": 50.0}])
def test_dt_stable_matches_oracle(lib, orc, shape, over):
    prm = workloads.params(**over)
    cfg = make_config(shape, prm)
    assert abs(native.pf_dt_stable(cfg) - orc.dt_stable(shape, prm)) <= 1e-15 * orc.dt_stable(shape, prm)


def test_create_rejects_bad_config(lib):
    prm = workloads.params()
    cfg = make_config((16, 16), prm)
    cfg.ndim = 4
    rc, h = native.pf_create(cfg)
    assert rc == native.PF_EINVAL and not h.value
    assert "ndim" in native.pf_last_error(None)
    cfg = make_config((16, 16), prm)
    cfg.nx = 1
    rc, h = native.pf_create(cfg)
    assert rc == native.PF_EINVAL


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    rc, h = native.pf_create(make_config((16, 16), workloads.params()))
    assert rc == native.PF_ECUDA and not h.value
    assert native.pf_last_error(None)


def test_null_handle_calls(lib):
    assert lib.pf_step(None, 1, None) == native.PF_EINVAL
    assert lib.pf_step_implicit(None, 1, None, None, None) == native.PF_EINVAL
    assert lib.pf_set_fields(None, None, 0) == native.PF_EINVAL
    assert lib.pf_set_coupling(None, None, None, 0) == native.PF_EINVAL
    lib.pf_destroy(None)


def test_fs_coupling_validates_before_touching_the_gpu(lib):
    """eig0 = 0 leaves no equivalent coupling scalar; NULL arrays are
    argument errors (both answered before any CUDA call)."""
    import numpy as np
    th = np.ones((4, 4))
    cfg = make_config((4, 4), dict(workloads.params(), eig0=0.0))
    rc, _ = native.pf_fs_coupling(cfg, th, th * 0, 0.1, np.zeros((16, 2)), np.eye(2))
    assert rc == native.PF_EINVAL and b"eig0" in lib.pf_fs_last_error()
    assert lib.pf_fs_coupling(None, None, None, 0.1, None, None, None, None) == native.PF_EINVAL


def test_finite_strain_validates_before_touching_the_gpu(lib):
    """pf_finite_strain_solve answers bad options, precisions, grid sizes
    and material constants with PF_EINVAL and a message before any CUDA
    call."""
    import numpy as np
    th = np.ones((4, 4))
    good = dict(nload=1, newton_maxit=5, newton_tol=1e-10, cg_maxit=10, cg_rtol=1e-6, precision=native.PF_MIXED)
    cases = [(dict(good, nload=0), b"pf_fs_opts"), (dict(good, cg_rtol=1.0), b"pf_fs_opts"),
             (dict(good, newton_tol=0.0), b"pf_fs_opts"), (dict(good, precision=7), b"precision")]
    cfg = make_config((4, 4), workloads.params())
    for o, msg in cases:
        rc, _, _, _ = native.pf_finite_strain_solve(cfg, th, th * 0, 0.1, None, native.pf_fs_opts(**o))
        assert rc == native.PF_EINVAL and msg in lib.pf_fs_last_error(), (o, lib.pf_fs_last_error())
    bad = make_config((4, 4), dict(workloads.params(), nu=0.5))
    rc, _, _, _ = native.pf_finite_strain_solve(bad, th, th * 0, 0.1, None, native.pf_fs_opts(**good))
    assert rc == native.PF_EINVAL and b"nu" in lib.pf_fs_last_error()
    one = make_config((4, 4), workloads.params())
    one.nx = 1
    rc, _, _, _ = native.pf_finite_strain_solve(one, th, th * 0, 0.1, None, native.pf_fs_opts(**good))
    assert rc == native.PF_EINVAL and b"grid sizes" in lib.pf_fs_last_error()


def test_batch_create_validates_before_touching_the_gpu(lib):
    prm = workloads.params()
    two = make_config((16, 16), prm)
    three = make_config((8, 8, 8), prm)
    rc, h = native.pf_batch_create([two, three])
    assert rc == native.PF_EINVAL and not h.value
    assert "share ndim" in native.pf_last_error(None)
    mixed = make_config((16, 16), prm, precision="mixed")
    rc, h = native.pf_batch_create([two, mixed])
    assert rc == native.PF_EINVAL
    bad = make_config((16, 16), prm)
    bad.nx = 1
    rc, h = native.pf_batch_create([two, bad])
    assert rc in (native.PF_EINVAL, native.PF_ECUDA) and not h.value
    assert lib.pf_batch_create(None, 0, ctypes.byref(ctypes.c_void_p())) == native.PF_EINVAL
    assert native.pf_batch_size(None) == 0


def test_create_rejects_unknown_pcg_tile(lib):
    cfg = make_config((16, 16), workloads.params(), pcg_tile=3)
    rc, h = native.pf_create(cfg)
    assert rc == native.PF_EINVAL and "pcg_tile" in native.pf_last_error(None)


def test_create_rejects_bad_precond(lib):
    cfg = make_config((16, 16), workloads.params(), precond=3)
    rc, h = native.pf_create(cfg)
    assert rc == native.PF_EINVAL and "precond" in native.pf_last_error(None)
    cfg = make_config((8, 8, 8), workloads.params(), precond=-1)
    rc, h = native.pf_create(cfg)
    assert rc == native.PF_EINVAL and "precond" in native.pf_last_error(None)


def _c_layout(structs):
    """sizeof and offsetof of every field, as the C compiler lays out the
    structs of include/*.h (compiled here with gcc, plain C)."""
    import subprocess
    import tempfile
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pf.h"', '#include "pf_unet.h"',
             'int main(void) {']
    for name, cls in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append('return 0; }')
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c11", "-I" + INCLUDE, "-o", exe, src])
        out = subprocess.check_output([exe], text=True)
    return dict((k, int(v)) for k, v in (l.split() for l in out.splitlines()))


def test_ctypes_structs_match_the_c_layout():
    """The Python binding's ctypes records have the field names, order,
    offsets and sizes of the C structs in the headers."""
    structs = [("pf_params", native.pf_params), ("pf_config", native.pf_config), ("pf_fields", native.pf_fields),
               ("pf_diag", native.pf_diag), ("pf_profile", native.pf_profile),
               ("pf_implicit_opts", native.pf_implicit_opts), ("pf_implicit_stats", native.pf_implicit_stats),
               ("pf_fs_opts", native.pf_fs_opts), ("pf_fs_stats", native.pf_fs_stats),
               ("pf_unet_config", native.pf_unet_config)]
    c = _c_layout(structs)
    for name, cls in structs:
        assert c[name] == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert c["%s.%s" % (name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_enum_constants_match_the_headers():
    """Every PF_* integer constant of the binding has the header's value."""
    import subprocess
    import tempfile
    names = [n for n in dir(native) if n.startswith("PF_") and isinstance(getattr(native, n), int)]
    txt = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    names = [n for n in names if re.search(r"\b%s\b" % n, txt)]
    assert len(names) >= 25
    lines = ['#include <stdio.h>', '#include "pf.h"', '#include "pf_unet.h"', 'int main(void) {']
    lines += ['printf("%s %%lld\\n", (long long)(%s));' % (n, n) for n in names]
    lines.append('return 0; }')
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "enums.c"), os.path.join(d, "enums")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c11", "-I" + INCLUDE, "-o", exe, src])
        out = subprocess.check_output([exe], text=True)
    for line in out.splitlines():
        k, v = line.split()
        assert getattr(native, k) == int(v), k
