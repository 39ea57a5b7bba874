"""ctypes binding of the C ABI in include/pf.h (argument marshalling only).

Every step of the method runs in the CUDA library ``libpf.so`` built from
``csrc/``; there is no Python or CPU fallback.  If the library is missing the
functions raise ``RuntimeError``.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
LIB_PATH = os.path.join(_HERE, "libpf.so")
CSRC = os.path.join(_HERE, "csrc")
UNITS = [os.path.join(CSRC, n) for n in ("pf_lib.cu", "pcg_2d.cu", "pcg_3d.cu", "unet.cu", "finite.cu")]   # translation units
BUILD_DIR = os.path.join(_HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENOTCONV, PF_ENONFINITE, PF_ETIMEOUT, PF_ESTATE = range(8)
PF_FP64, PF_MIXED = 0, 1
PF_WS_ZERO, PF_WS_PREV, PF_WS_LEARNED, PF_WS_EXTRAP, PF_WS_EXTRAP2 = 0, 1, 2, 3, 4
PF_PC_AUTO, PF_PC_JACOBI, PF_PC_MG = 0, 1, 2
PF_HOST, PF_DEVICE = 0, 1

STATUS_NAMES = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_ENOMEM", 3: "PF_ECUDA", 4: "PF_ENOTCONV",
                5: "PF_ENONFINITE", 6: "PF_ETIMEOUT", 7: "PF_ESTATE"}


class pf_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "c_chem", "w", "eps_phi", "kappa_O", "L", "D_O_s", "D_O_g", "D_H_s", "D_H_g", "D_W_s", "D_W_g",
        "k_for", "xH_bc", "E_s", "nu", "E_g_ratio", "eig0", "sigma_Y", "H_hard", "prestress")]


class pf_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int), ("mechanics", ctypes.c_int), ("plasticity", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("cg_maxit", ctypes.c_int), ("cg_rtol", ctypes.c_double),
                ("dt", ctypes.c_double), ("p", pf_params), ("pcg_tile", ctypes.c_int),
                ("precond", ctypes.c_int), ("fused_chunk", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)


class pf_fields(ctypes.Structure):
    _fields_ = [("phi_f", _DP), ("phi_w", _DP), ("x_O", _DP), ("x_H", _DP), ("x_H2O", _DP),
                ("u", _DP), ("Ebar", _DP), ("eps_p", _DP), ("alpha", _DP), ("sigma", _DP),
                ("mobility", _DP), ("dirichlet", ctypes.POINTER(ctypes.c_ubyte)), ("theta", _DP),
                ("phi_g", _DP)]


class pf_diag(ctypes.Structure):
    _fields_ = [("sum_O", ctypes.c_double), ("sum_H", ctypes.c_double), ("sum_H2O", ctypes.c_double),
                ("removed_H2O", ctypes.c_double), ("supplied_H", ctypes.c_double),
                ("sum_O_init", ctypes.c_double), ("reduction_degree", ctypes.c_double),
                ("cg_rel_residual", ctypes.c_double), ("cg_iters_last", ctypes.c_int),
                ("cg_iters_max", ctypes.c_int), ("cg_iters_total", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("dt", ctypes.c_double), ("status", ctypes.c_int),
                ("precond", ctypes.c_int), ("mg_levels", ctypes.c_int),
                ("reduction_rate", ctypes.c_double)]


PF_K_SETUP, PF_K_CG, PF_K_RETURN, PF_K_UPDATE, PF_K_WARM, PF_K_NCLASS = range(6)
KERNEL_CLASSES = ["setup", "cg", "return", "update", "warm"]


class pf_implicit_opts(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
                ("gmres_rtol", ctypes.c_double), ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("pc_degree", ctypes.c_int), ("pc_precision", ctypes.c_int)]


class pf_implicit_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("newton_iters_total", ctypes.c_int),
                ("gmres_iters", ctypes.c_longlong), ("residual", ctypes.c_double)]


class pf_fs_opts(ctypes.Structure):
    _fields_ = [("nload", ctypes.c_int), ("newton_maxit", ctypes.c_int), ("newton_tol", ctypes.c_double),
                ("cg_maxit", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("precision", ctypes.c_int)]


class pf_fs_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("cg_iters", ctypes.c_longlong), ("residual", ctypes.c_double),
                ("hvp_ms", ctypes.c_double), ("hvp_launches", ctypes.c_longlong)]


class pf_profile(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("launches", ctypes.c_longlong),
                ("count", ctypes.c_longlong * PF_K_NCLASS), ("ms", ctypes.c_double * PF_K_NCLASS),
                ("cg_iters", ctypes.c_longlong), ("graph_steps", ctypes.c_longlong)]


class pf_unet_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("cin", ctypes.c_int), ("levels", ctypes.c_int),
                ("channels", ctypes.c_int * 5)]


# exported symbols, in the order of include/pf.h then include/pf_unet.h
SYMBOLS = ["pf_create", "pf_set_fields", "pf_step", "pf_step_implicit", "pf_finite_strain_solve", "pf_finite_strain_step",
           "pf_fs_return_map", "pf_fs_elastic_force", "pf_fs_coupling", "pf_fs_last_error",
           "pf_set_coupling", "pf_get_fields", "pf_get_diagnostics",
           "pf_free_energy", "pf_dt_stable", "pf_profile_enable", "pf_profile_read",
           "pf_batch_create", "pf_batch_size", "pf_batch_set_fields", "pf_batch_get_fields",
           "pf_batch_get_diagnostics", "pf_attach_unet", "pf_selftest_wait",
           "pf_device_bytes", "pf_last_error", "pf_destroy",
           "pf_fields_update_static", "pf_static_last_error",
           "pf_unet_create", "pf_unet_param_count", "pf_unet_set_loss", "pf_unet_set_params", "pf_unet_get_params",
           "pf_unet_forward", "pf_unet_loss_grad", "pf_unet_adam_step", "pf_unet_last_error",
           "pf_unet_destroy"]
PF_STATIC_MAX_CELLS = 65536

_lock = threading.Lock()
_lib = None


def _stale():
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(s) > t for s in deps)


def build_library(force=False, verbose=False):
    """Compile csrc/ into libpf.so for sm_103a with nvcc (in-tree): each
    translation unit in parallel, then one link."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tag = "%d" % os.getpid()
    objs, procs = [], []
    for u in UNITS:
        o = os.path.join(BUILD_DIR, os.path.basename(u) + "." + tag + ".o")
        cmd = ["nvcc", "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
               "-I" + INCLUDE, "-c", "-o", o, u]
        if verbose:
            print(" ".join(cmd))
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(o)
    for p, cmd in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
    tmp = LIB_PATH + ".tmp" + tag
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    """Load libpf.so (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpf.so is not built: run __graft_entry__.build() or "
                               "paper_2111_11538_gb300.native.build_library()")
        l = ctypes.CDLL(LIB_PATH)
        l.pf_create.argtypes = [ctypes.POINTER(pf_config), ctypes.POINTER(ctypes.c_void_p)]
        l.pf_create.restype = ctypes.c_int
        l.pf_set_fields.argtypes = [ctypes.c_void_p, ctypes.POINTER(pf_fields), ctypes.c_int]
        l.pf_set_fields.restype = ctypes.c_int
        l.pf_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        l.pf_step.restype = ctypes.c_int
        l.pf_step_implicit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pf_implicit_opts),
                                       ctypes.POINTER(pf_implicit_stats), ctypes.c_void_p]
        l.pf_step_implicit.restype = ctypes.c_int
        l.pf_finite_strain_solve.argtypes = [ctypes.POINTER(pf_config), _DP, _DP, ctypes.c_double, _DP,
                                             ctypes.POINTER(pf_fs_opts), _DP, _DP, ctypes.POINTER(pf_fs_stats)]
        l.pf_finite_strain_solve.restype = ctypes.c_int
        l.pf_finite_strain_step.argtypes = [ctypes.POINTER(pf_config), _DP, _DP, ctypes.c_double, _DP,
                                            ctypes.POINTER(pf_fs_opts), _DP, _DP, _DP, _DP,
                                            ctypes.POINTER(pf_fs_stats)]
        l.pf_finite_strain_step.restype = ctypes.c_int
        l.pf_fs_return_map.argtypes = [ctypes.c_int, _DP, _DP, _DP, _DP, _DP, _DP, ctypes.c_double, ctypes.c_double]
        l.pf_fs_return_map.restype = ctypes.c_int
        l.pf_fs_elastic_force.argtypes = [ctypes.POINTER(pf_config), _DP, _DP, ctypes.c_double, _DP, _DP, _DP, _DP]
        l.pf_fs_elastic_force.restype = ctypes.c_int
        l.pf_fs_coupling.argtypes = [ctypes.POINTER(pf_config), _DP, _DP, ctypes.c_double, _DP, _DP, _DP, _DP]
        l.pf_fs_coupling.restype = ctypes.c_int
        l.pf_set_coupling.argtypes = [ctypes.c_void_p, _DP, _DP, ctypes.c_int]
        l.pf_set_coupling.restype = ctypes.c_int
        l.pf_fs_last_error.argtypes = []
        l.pf_fs_last_error.restype = ctypes.c_char_p
        l.pf_get_fields.argtypes = [ctypes.c_void_p, ctypes.POINTER(pf_fields), ctypes.c_int]
        l.pf_get_fields.restype = ctypes.c_int
        l.pf_get_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(pf_diag)]
        l.pf_get_diagnostics.restype = ctypes.c_int
        l.pf_free_energy.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        l.pf_free_energy.restype = ctypes.c_int
        l.pf_dt_stable.argtypes = [ctypes.POINTER(pf_config)]
        l.pf_dt_stable.restype = ctypes.c_double
        l.pf_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
        l.pf_profile_enable.restype = ctypes.c_int
        l.pf_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(pf_profile)]
        l.pf_profile_read.restype = ctypes.c_int
        l.pf_batch_create.argtypes = [ctypes.POINTER(pf_config), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        l.pf_batch_create.restype = ctypes.c_int
        l.pf_batch_size.argtypes = [ctypes.c_void_p]
        l.pf_batch_size.restype = ctypes.c_int
        l.pf_batch_set_fields.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pf_fields), ctypes.c_int]
        l.pf_batch_set_fields.restype = ctypes.c_int
        l.pf_batch_get_fields.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pf_fields), ctypes.c_int]
        l.pf_batch_get_fields.restype = ctypes.c_int
        l.pf_batch_get_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pf_diag)]
        l.pf_batch_get_diagnostics.restype = ctypes.c_int
        l.pf_selftest_wait.argtypes = [ctypes.c_longlong]
        l.pf_selftest_wait.restype = ctypes.c_int
        l.pf_attach_unet.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        l.pf_attach_unet.restype = ctypes.c_int
        l.pf_device_bytes.argtypes = [ctypes.c_void_p]
        l.pf_device_bytes.restype = ctypes.c_longlong
        l.pf_last_error.argtypes = [ctypes.c_void_p]
        l.pf_last_error.restype = ctypes.c_char_p
        l.pf_destroy.argtypes = [ctypes.c_void_p]
        l.pf_destroy.restype = None
        l.pf_fields_update_static.argtypes = [ctypes.POINTER(pf_config), ctypes.POINTER(pf_fields), _DP, _DP,
                                              ctypes.POINTER(pf_fields), ctypes.c_void_p]
        l.pf_fields_update_static.restype = ctypes.c_int
        _FP = ctypes.POINTER(ctypes.c_float)
        l.pf_unet_create.argtypes = [ctypes.POINTER(pf_unet_config), ctypes.POINTER(ctypes.c_void_p)]
        l.pf_unet_create.restype = ctypes.c_int
        l.pf_unet_param_count.argtypes = [ctypes.c_void_p]
        l.pf_unet_param_count.restype = ctypes.c_longlong
        l.pf_unet_set_loss.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        l.pf_unet_set_loss.restype = ctypes.c_int
        l.pf_unet_set_params.argtypes = [ctypes.c_void_p, _FP]
        l.pf_unet_set_params.restype = ctypes.c_int
        l.pf_unet_get_params.argtypes = [ctypes.c_void_p, _FP]
        l.pf_unet_get_params.restype = ctypes.c_int
        l.pf_unet_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        l.pf_unet_forward.restype = ctypes.c_int
        l.pf_unet_loss_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), _FP, ctypes.c_void_p]
        l.pf_unet_loss_grad.restype = ctypes.c_int
        l.pf_unet_adam_step.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        l.pf_unet_adam_step.restype = ctypes.c_int
        l.pf_unet_last_error.argtypes = [ctypes.c_void_p]
        l.pf_unet_last_error.restype = ctypes.c_char_p
        l.pf_unet_destroy.argtypes = [ctypes.c_void_p]
        l.pf_unet_destroy.restype = None
        l.pf_static_last_error.argtypes = []
        l.pf_static_last_error.restype = ctypes.c_char_p
        _lib = l
        return l


# ---- thin same-name wrappers ------------------------------------------------
def pf_create(cfg):
    h = ctypes.c_void_p()
    rc = lib().pf_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, h


def pf_set_fields(h, fields, where=PF_HOST):
    return lib().pf_set_fields(h, ctypes.byref(fields), where)


def pf_step(h, nsteps, stream=None):
    return lib().pf_step(h, int(nsteps), ctypes.c_void_p(stream) if stream else None)


def pf_step_implicit(h, nsteps, opts, stream=None):
    st = pf_implicit_stats()
    rc = lib().pf_step_implicit(h, int(nsteps), ctypes.byref(opts), ctypes.byref(st),
                                ctypes.c_void_p(stream) if stream else None)
    return rc, st


def pf_finite_strain_solve(cfg, theta, phig, omega, pbar, opts):
    """Host arrays in, (rc, u, Fbar, stats) out (see include/pf.h)."""
    import numpy as np
    th = np.ascontiguousarray(theta, dtype=np.float64)
    pg = np.ascontiguousarray(phig, dtype=np.float64)
    d = cfg.ndim
    u = np.zeros(th.size * d)
    fb = np.zeros(d * d)
    pb = None if pbar is None else np.ascontiguousarray(pbar, dtype=np.float64).ravel()
    st = pf_fs_stats()
    ptr = lambda a: a.ctypes.data_as(_DP)                                   # noqa: E731
    rc = lib().pf_finite_strain_solve(ctypes.byref(cfg), ptr(th), ptr(pg), float(omega),
                                      ptr(pb) if pb is not None else None, ctypes.byref(opts), ptr(u), ptr(fb),
                                      ctypes.byref(st))
    return rc, u.reshape(-1, d), fb.reshape(d, d), st


def pf_finite_strain_step(cfg, theta, phig, omega, pbar, opts, FP, epsP):
    """One staggered step; FP (N, 3, 3) and epsP (N,) are updated in place
    (contiguous float64 arrays); returns (rc, u, Fbar, stats)."""
    import numpy as np
    th = np.ascontiguousarray(theta, dtype=np.float64)
    pg = np.ascontiguousarray(phig, dtype=np.float64)
    assert FP.dtype == np.float64 and FP.flags.c_contiguous and epsP.dtype == np.float64 and epsP.flags.c_contiguous
    d = cfg.ndim
    u = np.zeros(th.size * d)
    fb = np.zeros(d * d)
    pb = None if pbar is None else np.ascontiguousarray(pbar, dtype=np.float64).ravel()
    st = pf_fs_stats()
    ptr = lambda a: a.ctypes.data_as(_DP)                                   # noqa: E731
    rc = lib().pf_finite_strain_step(ctypes.byref(cfg), ptr(th), ptr(pg), float(omega),
                                     ptr(pb) if pb is not None else None, ctypes.byref(opts), ptr(u), ptr(fb),
                                     ptr(FP), ptr(epsP), ctypes.byref(st))
    return rc, u.reshape(-1, d), fb.reshape(d, d), st


def pf_fs_return_map(F, FP, epsP, K, G, dT, sigma_Y, H):
    """Pointwise multiplicative J2 update; FP, epsP updated in place."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (F, K, G, dT)]
    assert FP.dtype == np.float64 and FP.flags.c_contiguous and epsP.dtype == np.float64 and epsP.flags.c_contiguous
    ptr = lambda a: a.ctypes.data_as(_DP)                                   # noqa: E731
    return lib().pf_fs_return_map(int(epsP.size), ptr(arrs[0]), ptr(FP), ptr(epsP), ptr(arrs[1]), ptr(arrs[2]),
                                  ptr(arrs[3]), float(sigma_Y), float(H))


def _fs_cellwise(fn, cfg, theta, phig, omega, u, Fbar, FP):
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (theta, phig, u, Fbar)]
    fp = None if FP is None else np.ascontiguousarray(FP, dtype=np.float64).ravel()
    out = np.zeros(arrs[0].size)
    ptr = lambda a: a.ctypes.data_as(_DP)                                   # noqa: E731
    rc = fn(ctypes.byref(cfg), ptr(arrs[0]), ptr(arrs[1]), float(omega), ptr(arrs[2]),
            ptr(arrs[3]), ptr(fp) if fp is not None else None, ptr(out))
    return rc, out


def pf_fs_elastic_force(cfg, theta, phig, omega, u, Fbar, FP=None):
    """(rc, d psi / d theta per cell); host arrays."""
    return _fs_cellwise(lib().pf_fs_elastic_force, cfg, theta, phig, omega, u, Fbar, FP)


def pf_fs_coupling(cfg, theta, phig, omega, u, Fbar, FP=None):
    """(rc, the equivalent small-strain coupling scalar per cell); host arrays."""
    return _fs_cellwise(lib().pf_fs_coupling, cfg, theta, phig, omega, u, Fbar, FP)


def pf_set_coupling(h, trE, devE2=None, where=PF_HOST):
    """Set a mechanics-free handle's coupling scalars from FP64 arrays (None: zero)."""
    import numpy as np
    keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (trE, devE2)]
    ptr = [None if a is None else a.ctypes.data_as(_DP) for a in keep]
    return lib().pf_set_coupling(h, ptr[0], ptr[1], where)


def pf_get_fields(h, fields, where=PF_HOST):
    return lib().pf_get_fields(h, ctypes.byref(fields), where)


def pf_get_diagnostics(h):
    d = pf_diag()
    rc = lib().pf_get_diagnostics(h, ctypes.byref(d))
    return rc, d


def pf_free_energy(h):
    v = ctypes.c_double()
    rc = lib().pf_free_energy(h, ctypes.byref(v))
    return rc, v.value


def pf_dt_stable(cfg):
    return lib().pf_dt_stable(ctypes.byref(cfg))


def pf_profile_enable(h, on=True):
    return lib().pf_profile_enable(h, 1 if on else 0)


def pf_profile_read(h):
    p = pf_profile()
    rc = lib().pf_profile_read(h, ctypes.byref(p))
    return rc, p


def pf_batch_create(cfgs):
    arr = (pf_config * len(cfgs))(*cfgs)
    h = ctypes.c_void_p()
    rc = lib().pf_batch_create(arr, len(cfgs), ctypes.byref(h))
    return rc, h


def pf_batch_size(h):
    return lib().pf_batch_size(h)


def pf_batch_set_fields(h, i, fields, where=PF_HOST):
    return lib().pf_batch_set_fields(h, int(i), ctypes.byref(fields), where)


def pf_batch_get_fields(h, i, fields, where=PF_HOST):
    return lib().pf_batch_get_fields(h, int(i), ctypes.byref(fields), where)


def pf_batch_get_diagnostics(h, i):
    d = pf_diag()
    rc = lib().pf_batch_get_diagnostics(h, int(i), ctypes.byref(d))
    return rc, d


def pf_selftest_wait(spin_limit):
    return lib().pf_selftest_wait(int(spin_limit))


def pf_attach_unet(h, net):
    return lib().pf_attach_unet(h, net)


def pf_device_bytes(h):
    return lib().pf_device_bytes(h)


def pf_last_error(h=None):
    s = lib().pf_last_error(h)
    return s.decode() if s else ""


def pf_destroy(h):
    lib().pf_destroy(h)


def pf_fields_update_static(cfg, fin, trE, devE2, fout, stream=None):
    """Allocation-free field update; every pointer is device memory (see pf.h)."""
    return lib().pf_fields_update_static(ctypes.byref(cfg), ctypes.byref(fin), trE, devE2,
                                         ctypes.byref(fout), ctypes.c_void_p(stream) if stream else None)


def pf_static_last_error():
    s = lib().pf_static_last_error()
    return s.decode() if s else ""


def pf_unet_create(cfg):
    h = ctypes.c_void_p()
    rc = lib().pf_unet_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, h


def pf_unet_param_count(h):
    return lib().pf_unet_param_count(h)


PF_UNET_LOSS_MSE, PF_UNET_LOSS_GRAD = 0, 1


def pf_unet_set_loss(h, kind, weight_channel=1, floor=0.01):
    return lib().pf_unet_set_loss(h, int(kind), int(weight_channel), float(floor))


def pf_unet_set_params(h, host):
    return lib().pf_unet_set_params(h, host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def pf_unet_get_params(h, host):
    return lib().pf_unet_get_params(h, host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def pf_unet_forward(h, inp, out, nb, nx, ny, nz, stream=None):
    """inp / out: device addresses (int) of FP32 channels-last arrays."""
    return lib().pf_unet_forward(h, ctypes.c_void_p(inp), ctypes.c_void_p(out), nb, nx, ny, nz,
                                 ctypes.c_void_p(stream) if stream else None)


def pf_unet_loss_grad(h, inp, target, nb, nx, ny, nz, grad_host=None, stream=None):
    loss = ctypes.c_double()
    g = grad_host.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if grad_host is not None else None
    rc = lib().pf_unet_loss_grad(h, ctypes.c_void_p(inp), ctypes.c_void_p(target), nb, nx, ny, nz,
                                 ctypes.byref(loss), g, ctypes.c_void_p(stream) if stream else None)
    return rc, loss.value


def pf_unet_adam_step(h, lr, stream=None):
    return lib().pf_unet_adam_step(h, float(lr), ctypes.c_void_p(stream) if stream else None)


def pf_unet_last_error(h=None):
    s = lib().pf_unet_last_error(h)
    return s.decode() if s else ""


def pf_unet_destroy(h):
    lib().pf_unet_destroy(h)
