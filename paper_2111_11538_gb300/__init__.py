"""GB300-native coupled phase-field step for wuestite-to-iron reduction by
hydrogen (arXiv 2111.11538): Python front end of the C ABI in include/pf.h.

    from paper_2111_11538_gb300 import Simulation, workloads, inputs
    fields = inputs.core_shell((64, 64), 20.0, 4.0)
    sim = Simulation((64, 64), workloads.params(), precision="fp64")
    sim.set_fields(fields)
    sim.step(500)
    out = sim.get_fields()

All arithmetic of the step runs in the CUDA library; this module only moves
arrays across the boundary.
"""
import ctypes

import numpy as np

from . import native
from .native import (PF_DEVICE, PF_FP64, PF_HOST, PF_MIXED, PF_OK, PF_PC_AUTO, PF_PC_JACOBI, PF_PC_MG,
                     PF_WS_EXTRAP, PF_WS_EXTRAP2, PF_WS_LEARNED, PF_WS_PREV, PF_WS_ZERO,
                     STATUS_NAMES, pf_config, pf_diag, pf_fields, pf_params)

__all__ = ["Simulation", "FiniteStrainSimulation", "Batch", "PFError", "make_config", "native"]

PARAM_NAMES = [f[0] for f in pf_params._fields_]


class PFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


def make_config(shape, prm, precision="fp64", mechanics=None, plasticity=None, warm_start=None,
                cg_rtol=None, cg_maxit=None, dt=None, pcg_tile=None, precond=None, fused_chunk=None):
    """Build a pf_config from a grid shape ((ny, nx) or (nz, ny, nx)) and a
    parameter dict (see workloads.params)."""
    c = pf_config()
    c.ndim = len(shape)
    if c.ndim == 2:
        c.ny, c.nx = shape
        c.nz = 1
    elif c.ndim == 3:
        c.nz, c.ny, c.nx = shape
    else:
        raise ValueError("shape must have 2 or 3 entries")
    c.precision = {"fp64": PF_FP64, "mixed": PF_MIXED}[precision]
    c.mechanics = int(prm.get("mechanics", 1) if mechanics is None else mechanics)
    c.plasticity = int(prm.get("plasticity", 0) if plasticity is None else plasticity)
    ws = prm.get("warm_start", 1) if warm_start is None else warm_start
    c.warm_start = {"zero": PF_WS_ZERO, "prev": PF_WS_PREV, "learned": PF_WS_LEARNED,
                    "extrap": PF_WS_EXTRAP, "extrap2": PF_WS_EXTRAP2}.get(ws, ws)
    c.cg_rtol = float(prm.get("cg_rtol", 1e-10) if cg_rtol is None else cg_rtol)
    c.cg_maxit = int(prm.get("cg_maxit", 20000) if cg_maxit is None else cg_maxit)
    c.dt = float(prm.get("dt", 0.0) if dt is None else dt)
    c.pcg_tile = int(prm.get("pcg_tile", 0) if pcg_tile is None else pcg_tile)
    c.fused_chunk = int(prm.get("fused_chunk", 0) if fused_chunk is None else fused_chunk)
    pc = prm.get("precond", "auto") if precond is None else precond
    c.precond = {"auto": PF_PC_AUTO, "jacobi": PF_PC_JACOBI, "mg": PF_PC_MG}.get(pc, pc)
    for k in PARAM_NAMES:
        setattr(c.p, k, float(prm[k]))
    return c


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


FIELD_KEYS = ("phi_f", "phi_w", "xO", "xH", "xW", "u", "Ebar", "eps_p", "alpha", "sigma", "theta", "phig")
_NAMES = {"phi_f": "phi_f", "phi_w": "phi_w", "xO": "x_O", "xH": "x_H", "xW": "x_H2O",
          "u": "u", "Ebar": "Ebar", "eps_p": "eps_p", "alpha": "alpha", "sigma": "sigma",
          "mob": "mobility", "theta": "theta", "phig": "phi_g"}


def _in_fields(fields, where, N, ndim):
    """pf_fields pointing at the caller's arrays (numpy on the host, torch
    CUDA tensors on the device) and the list of objects that must stay alive
    until the call returns."""
    f = pf_fields()
    keep = []
    npl = 4 if ndim == 2 else 6
    nv = 3 if ndim == 2 else 6
    if where == "host":
        sizes = {"u": N * ndim, "eps_p": N * npl, "Ebar": nv}
        for key in ("phi_f", "phi_w", "xO", "xH", "xW", "alpha", "mob", "u", "eps_p", "Ebar", "theta", "phig"):
            v = fields.get(key)
            if v is None:
                continue
            a = np.ascontiguousarray(v, dtype=np.float64)
            if a.size != sizes.get(key, N):
                raise ValueError("%s has %d values, expected %d" % (key, a.size, sizes.get(key, N)))
            keep.append(a)
            setattr(f, _NAMES[key], _dptr(a))
        v = fields.get("mask")
        if v is not None:
            a = np.ascontiguousarray(v, dtype=np.uint8)
            if a.size != N:
                raise ValueError("mask has %d values, expected %d" % (a.size, N))
            keep.append(a)
            f.dirichlet = a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    elif where == "device":
        for key in ("phi_f", "phi_w", "xO", "xH", "xW", "alpha", "mob", "u", "eps_p", "Ebar", "theta", "phig"):
            t = fields.get(key)
            if t is not None:
                t = t.contiguous()
                keep.append(t)
                setattr(f, _NAMES[key], ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_double)))
        t = fields.get("mask")
        if t is not None:
            t = t.contiguous()
            keep.append(t)
            f.dirichlet = ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_ubyte))
    else:
        raise ValueError("where must be 'host' or 'device'")
    return f, keep


def _out_fields(keys, shape, out=None):
    """pf_fields pointing at arrays for the requested keys: the caller's
    (float64, C-contiguous, of the field's shape; pinned host memory makes
    the copies direct) where `out` has them, fresh numpy arrays otherwise."""
    ndim = len(shape)
    npl = 4 if ndim == 2 else 6
    nv = 3 if ndim == 2 else 6
    shp = {"u": shape + (ndim,), "eps_p": shape + (npl,), "sigma": shape + (npl,), "Ebar": (nv,)}
    f = pf_fields()
    res = {}
    for k in keys:
        want = shp.get(k, shape)
        a = out.get(k) if out is not None else None
        if a is None:
            a = np.zeros(want)
        elif a.dtype != np.float64 or not a.flags.c_contiguous or a.size != int(np.prod(want)):
            raise ValueError("out[%r] must be a C-contiguous float64 array of %d values" % (k, int(np.prod(want))))
        res[k] = a
        setattr(f, _NAMES[k], _dptr(a))
    return f, res


class Simulation:
    """One grid advanced by the CUDA library.

    Host arrays are numpy float64 (cell-major, x fastest).  ``set_fields`` and
    ``get_fields`` also accept / fill torch CUDA float64 tensors when
    ``where="device"``.
    """

    def __init__(self, shape, prm, precision="fp64", **kw):
        self.shape = tuple(shape)
        self.ndim = len(self.shape)
        self.N = int(np.prod(self.shape))
        self.cfg = make_config(self.shape, prm, precision=precision, **kw)
        rc, h = native.pf_create(self.cfg)
        if rc != PF_OK:
            raise PFError(rc, native.pf_last_error(None))
        self.h = h
        self.np_ = 4 if self.ndim == 2 else 6
        self.nv = 3 if self.ndim == 2 else 6

    # ------------------------------------------------------------------
    def _check(self, rc):
        if rc != PF_OK:
            raise PFError(rc, native.pf_last_error(self.h))
        return rc

    def set_fields(self, fields, where="host"):
        f, keep = _in_fields(fields, where, self.N, self.ndim)
        rc = native.pf_set_fields(self.h, f, PF_HOST if where == "host" else PF_DEVICE)
        del keep
        return self._check(rc)

    def step(self, n=1, stream=None, check=True):
        rc = native.pf_step(self.h, n, stream)
        if check:
            self._check(rc)
        return rc

    def step_implicit(self, n, dt, newton_tol=1e-12, newton_maxit=30, gmres_rtol=1e-6, gmres_restart=60,
                      gmres_maxit=5000, pc_degree=32, pc_precision="mixed", stream=None, check=True):
        """n backward-Euler steps of length dt (pf_step_implicit); returns the
        Newton and GMRES counts as a dict.  pc_precision: the block
        preconditioner in FP32 ("mixed") or FP64 ("fp64")."""
        if pc_precision not in ("mixed", "fp64"):
            raise ValueError("pc_precision must be 'mixed' or 'fp64'")
        o = native.pf_implicit_opts(dt=float(dt), newton_tol=float(newton_tol), newton_maxit=int(newton_maxit),
                                    gmres_rtol=float(gmres_rtol), gmres_restart=int(gmres_restart),
                                    gmres_maxit=int(gmres_maxit), pc_degree=int(pc_degree),
                                    pc_precision=PF_MIXED if pc_precision == "mixed" else PF_FP64)
        rc, st = native.pf_step_implicit(self.h, n, o, stream)
        if check:
            self._check(rc)
        out = {k: getattr(st, k) for k, _ in native.pf_implicit_stats._fields_}
        out["rc"] = rc
        return out

    def get_fields(self, keys=FIELD_KEYS, out=None):
        """Fields as numpy arrays; with `out` (a dict of preallocated arrays,
        e.g. pinned host memory) the copies land there."""
        f, res = _out_fields(keys, self.shape, out)
        self._check(native.pf_get_fields(self.h, f, PF_HOST))
        return res

    def diagnostics(self):
        rc, d = native.pf_get_diagnostics(self.h)
        self._check(rc)
        return {k: getattr(d, k) for k, _ in pf_diag._fields_}

    def free_energy(self):
        rc, v = native.pf_free_energy(self.h)
        self._check(rc)
        return v

    @property
    def dt(self):
        return self.diagnostics()["dt"]

    def set_coupling(self, trE, devE2=None, where="host"):
        """Coupling scalars of a mechanics = 0 handle's field update
        (pf_set_coupling); None: zero."""
        self._check(native.pf_set_coupling(self.h, trE, devE2, PF_HOST if where == "host" else PF_DEVICE))

    def profile(self, on=True):
        self._check(native.pf_profile_enable(self.h, on))

    def profile_read(self):
        rc, p = native.pf_profile_read(self.h)
        self._check(rc)
        return {"launches": p.launches, "cg_iters": p.cg_iters, "graph_steps": p.graph_steps,
                "count": {k: p.count[i] for i, k in enumerate(native.KERNEL_CLASSES)},
                "ms": {k: p.ms[i] for i, k in enumerate(native.KERNEL_CLASSES)}}

    def attach_unet(self, net):
        """Use a trained warm-start network (warmstart.WarmStartNet) for the
        initial guess of every solve (config warm_start="learned"); None
        detaches."""
        self._check(native.pf_attach_unet(self.h, net.h if net is not None else None))
        self._net = net            # keep it alive while attached

    def device_bytes(self):
        return native.pf_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            native.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class FiniteStrainSimulation:
    """The explicit step coupled to finite-strain mechanics (Sec. 2.2 neo-Hooke
    mixture with the transformation stretch, Sec. 2.3/2.4 multiplicative J2
    flow).  Each step: the staggered finite-strain mechanics step at the
    current order parameter (pf_finite_strain_step, F_P updated in place),
    its elastic force on the order parameter as the equivalent small-strain
    coupling scalar (pf_fs_coupling), then one field update of a
    mechanics = 0 handle with that coupling (pf_set_coupling, pf_step):
    transport, reaction, chemical and double-well forces, the supply-cell
    reset.  The field update and the mechanics' residual are FP64; the
    Hessian-vector products FP32 (precision="mixed") or FP64.  The
    equilibrium is solved from zero over `nload` load steps every step."""

    def __init__(self, shape, prm, omega, prestress=0.0, pbar=None, nload=4, newton_tol=1e-13, cg_rtol=1e-12,
                 precision="mixed"):
        self.shape = tuple(shape)
        self.N = int(np.prod(self.shape))
        self.sim = Simulation(self.shape, dict(prm, mechanics=0), precision="fp64")
        self.cfg = make_config(self.shape, dict(prm, prestress=prestress))
        if self.cfg.p.eig0 == 0.0:
            raise ValueError("the coupling needs a nonzero eig0 (any value: it cancels)")
        self.omega = float(omega)
        self.pbar = pbar
        self.opts = native.pf_fs_opts(nload=int(nload), newton_maxit=40, newton_tol=float(newton_tol),
                                      cg_maxit=20000, cg_rtol=float(cg_rtol),
                                      precision=PF_MIXED if precision == "mixed" else PF_FP64)
        self.FP = np.tile(np.eye(3), (self.N, 1, 1))
        self.epsP = np.zeros(self.N)
        self.u = None
        self.Fbar = None
        self.stats = None

    def _fs(self, rc):
        if rc != PF_OK:
            raise PFError(rc, native.lib().pf_fs_last_error().decode())

    def set_fields(self, fields):
        self.sim.set_fields(fields)
        self.FP[:] = np.eye(3)
        self.epsP[:] = 0.0

    def step(self, n=1):
        for _ in range(int(n)):
            g = self.sim.get_fields(keys=("theta", "phig"))
            th, pg = g["theta"].ravel(), g["phig"].ravel()
            rc, self.u, self.Fbar, self.stats = native.pf_finite_strain_step(
                self.cfg, th, pg, self.omega, self.pbar, self.opts, self.FP, self.epsP)
            self._fs(rc)
            rc, tE = native.pf_fs_coupling(self.cfg, th, pg, self.omega, self.u, self.Fbar, self.FP)
            self._fs(rc)
            self.sim.set_coupling(tE)
            self.sim.step(1)

    def get_fields(self, keys=FIELD_KEYS):
        return self.sim.get_fields(keys=keys)

    def diagnostics(self):
        return self.sim.diagnostics()

    def close(self):
        self.sim.close()


class Batch:
    """Many independent instances stepped by the same launches.

    ``shapes`` and ``prms`` give one grid shape and parameter dict per
    instance; the instances share ndim, precision and whether mechanics is
    on.  Fields go in and out per instance (index ``i``); ``step`` advances
    all of them.
    """

    def __init__(self, shapes, prms, precision="fp64", **kw):
        if isinstance(prms, dict):
            prms = [prms] * len(shapes)
        self.shapes = [tuple(s) for s in shapes]
        self.cfgs = [make_config(s, p, precision=precision, **kw) for s, p in zip(self.shapes, prms)]
        rc, h = native.pf_batch_create(self.cfgs)
        if rc != PF_OK:
            raise PFError(rc, native.pf_last_error(None))
        self.h = h

    def __len__(self):
        return native.pf_batch_size(self.h)

    def _check(self, rc):
        if rc != PF_OK:
            raise PFError(rc, native.pf_last_error(self.h))
        return rc

    def set_fields(self, i, fields, where="host"):
        shape = self.shapes[i]
        f, keep = _in_fields(fields, where, int(np.prod(shape)), len(shape))
        rc = native.pf_batch_set_fields(self.h, i, f, PF_HOST if where == "host" else PF_DEVICE)
        del keep
        return self._check(rc)

    def step(self, n=1, stream=None, check=True):
        rc = native.pf_step(self.h, n, stream)
        if check:
            self._check(rc)
        return rc

    def get_fields(self, i, keys=FIELD_KEYS, out=None):
        f, res = _out_fields(keys, self.shapes[i], out)
        self._check(native.pf_batch_get_fields(self.h, i, f, PF_HOST))
        return res

    def diagnostics(self, i):
        rc, d = native.pf_batch_get_diagnostics(self.h, i)
        self._check(rc)
        return {k: getattr(d, k) for k, _ in pf_diag._fields_}

    def profile(self, on=True):
        self._check(native.pf_profile_enable(self.h, on))

    def profile_read(self):
        rc, p = native.pf_profile_read(self.h)
        self._check(rc)
        return {"launches": p.launches, "cg_iters": p.cg_iters, "graph_steps": p.graph_steps,
                "count": {k: p.count[i] for i, k in enumerate(native.KERNEL_CLASSES)},
                "ms": {k: p.ms[i] for i, k in enumerate(native.KERNEL_CLASSES)}}

    def attach_unet(self, net):
        """Use a trained warm-start network (warmstart.WarmStartNet) for the
        initial guess of every solve (config warm_start="learned"); None
        detaches."""
        self._check(native.pf_attach_unet(self.h, net.h if net is not None else None))
        self._net = net            # keep it alive while attached

    def device_bytes(self):
        return native.pf_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            native.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
