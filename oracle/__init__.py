"""Plain FP64 CPU oracle of the coupled phase-field step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It compiles ``oracle.c`` with the host
C compiler into ``oracle/_build/liboracle.so`` and wraps it with ctypes.  It
shares no code with the CUDA library.

Submodules: ``implicit`` (backward-Euler time step of the field relations)
and ``finite_strain`` (neo-Hooke mechanics with the transformation stretch
and multiplicative J2, and the coupled explicit step that uses it).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")


def build(force=False):
    """Compile the oracle (plain C, -O2, no fast-math) if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dt", ctypes.c_double),
                ("c_chem", ctypes.c_double), ("w", ctypes.c_double), ("eps_phi", ctypes.c_double),
                ("kappa_O", ctypes.c_double), ("L", ctypes.c_double),
                ("D_O_s", ctypes.c_double), ("D_O_g", ctypes.c_double),
                ("D_H_s", ctypes.c_double), ("D_H_g", ctypes.c_double),
                ("D_W_s", ctypes.c_double), ("D_W_g", ctypes.c_double),
                ("k_for", ctypes.c_double), ("xH_bc", ctypes.c_double),
                ("E_s", ctypes.c_double), ("nu", ctypes.c_double), ("E_g_ratio", ctypes.c_double),
                ("eig0", ctypes.c_double), ("sigma_Y", ctypes.c_double), ("H_hard", ctypes.c_double),
                ("prestress", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("cg_maxit", ctypes.c_int), ("mechanics", ctypes.c_int), ("plasticity", ctypes.c_int),
                ("warm_start", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)
_UP = ctypes.POINTER(ctypes.c_ubyte)


class State(ctypes.Structure):
    _fields_ = [("theta", _DP), ("phig", _DP), ("xO", _DP), ("xH", _DP), ("xW", _DP),
                ("u", _DP), ("Ebar", _DP), ("eps_p", _DP), ("alpha", _DP),
                ("mob", _DP), ("mask", _UP), ("trE", _DP), ("devE2", _DP), ("sigma", _DP),
                ("removedW", ctypes.c_double), ("suppliedH", ctypes.c_double),
                ("cg_iters", ctypes.c_int), ("cg_relres", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        l = ctypes.CDLL(build())
        for name in ("or_h", "or_hp", "or_m", "or_mp"):
            getattr(l, name).restype = ctypes.c_double
            getattr(l, name).argtypes = [ctypes.c_double]
        for name in ("or_f", "or_fp", "or_fpp"):
            getattr(l, name).restype = ctypes.c_double
            getattr(l, name).argtypes = [ctypes.c_int, ctypes.c_double]
        l.or_dt_stable.restype = ctypes.c_double
        l.or_dt_stable.argtypes = [ctypes.POINTER(Params)]
        l.or_step.restype = ctypes.c_int
        l.or_step.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State), ctypes.c_int]
        l.or_mechanics.restype = ctypes.c_int
        l.or_mechanics.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State)]
        l.or_fields_update.restype = None
        l.or_fields_update.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State)]
        l.or_rates.restype = None
        l.or_rates.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State), _DP]
        l.or_return_map.restype = None
        l.or_return_map.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State)]
        l.or_free_energy.restype = ctypes.c_double
        l.or_free_energy.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State)]
        l.or_sums.restype = None
        l.or_sums.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State), _DP]
        l.or_mech_apply.restype = None
        l.or_mech_apply.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP, _DP]
        l.or_mech_diag.restype = None
        l.or_mech_diag.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP]
        l.or_mech_rhs.restype = None
        l.or_mech_rhs.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(State), _DP, _DP, _DP]
        l.or_cell_lame.restype = None
        l.or_cell_lame.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP, _DP]
        l.or_pcg.restype = ctypes.c_int
        l.or_pcg.argtypes = [ctypes.POINTER(Params), _DP, _DP, _DP, _DP, _DP]
        l.or_theta_force.restype = ctypes.c_double
        l.or_theta_force.argtypes = [ctypes.POINTER(Params)] + [ctypes.c_double] * 5
        l.or_local_energy.restype = ctypes.c_double
        l.or_local_energy.argtypes = [ctypes.POINTER(Params)] + [ctypes.c_double] * 5
        _lib = l
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


PARAM_KEYS = [f[0] for f in Params._fields_]


def make_params(shape, prm, **over):
    """Build the ctypes parameter record from a grid shape and a parameter dict.

    ``shape`` is (ny, nx) or (nz, ny, nx) (row-major, x fastest).
    """
    d = dict(prm)
    d.update(over)
    p = Params()
    p.ndim = len(shape)
    if p.ndim == 2:
        p.ny, p.nx = shape
        p.nz = 1
    else:
        p.nz, p.ny, p.nx = shape
    for k in PARAM_KEYS:
        if k in ("ndim", "nx", "ny", "nz"):
            continue
        if k in d:
            setattr(p, k, d[k])
    if d.get("dt", 0.0) <= 0.0:
        p.dt = d.get("dt_factor", 0.2) * lib().or_dt_stable(ctypes.byref(p))
    return p


def split_phases(phi_f, phi_w):
    """(phi_f, phi_w) -> (theta, phi_g): gas fraction and ferrite share of the solid."""
    phi_f = np.asarray(phi_f, dtype=np.float64)
    phi_w = np.asarray(phi_w, dtype=np.float64)
    solid = phi_f + phi_w
    theta = np.where(solid > 0.0, phi_f / np.where(solid > 0.0, solid, 1.0), 0.0)
    return theta, 1.0 - solid


class Sim:
    """Holds FP64 numpy copies of every field and steps them with the oracle.

    Inputs use the paper's phase fields phi_f, phi_w; the oracle evolves the
    solid order parameter theta with the gas fraction phi_g fixed.
    """

    def __init__(self, fields, prm, **over):
        phi_f = np.ascontiguousarray(fields["phi_f"], dtype=np.float64)
        self.shape = phi_f.shape
        self.p = make_params(self.shape, prm, **over)
        d = self.p.ndim
        N = phi_f.size
        nv = 3 if d == 2 else 6
        npl = 4 if d == 2 else 6
        self.f = {}
        th, pg = split_phases(fields["phi_f"], fields["phi_w"])
        self.f["theta"] = np.ascontiguousarray(fields.get("theta", th), dtype=np.float64).copy()
        self.f["phig"] = np.ascontiguousarray(fields.get("phig", pg), dtype=np.float64).copy()
        for k in ("xO", "xH", "xW"):
            self.f[k] = np.ascontiguousarray(fields[k], dtype=np.float64).copy()
        self.f["mob"] = np.ascontiguousarray(fields.get("mob", np.ones(self.shape)), dtype=np.float64).copy()
        self.f["mask"] = np.ascontiguousarray(fields.get("mask", np.zeros(self.shape, np.uint8)), dtype=np.uint8).copy()
        self.f["u"] = np.ascontiguousarray(fields.get("u", np.zeros(self.shape + (d,))), dtype=np.float64).copy()
        self.f["Ebar"] = np.ascontiguousarray(fields.get("Ebar", np.zeros(nv)), dtype=np.float64).copy()
        self.f["eps_p"] = np.ascontiguousarray(fields.get("eps_p", np.zeros(self.shape + (npl,))), dtype=np.float64).copy()
        self.f["alpha"] = np.ascontiguousarray(fields.get("alpha", np.zeros(self.shape)), dtype=np.float64).copy()
        self.f["trE"] = np.zeros(self.shape)
        self.f["devE2"] = np.zeros(self.shape)
        self.f["sigma"] = np.zeros(self.shape + (npl,))
        self.s = State()
        for k in ("theta", "phig", "xO", "xH", "xW", "u", "Ebar", "eps_p", "alpha", "mob", "trE", "devE2", "sigma"):
            setattr(self.s, k, _dp(self.f[k]))
        self.s.mask = self.f["mask"].ctypes.data_as(_UP)
        self.s.removedW = 0.0
        self.s.suppliedH = 0.0
        self.N = N

    @property
    def phi_f(self):
        return (1.0 - self.f["phig"]) * self.f["theta"]

    @property
    def phi_w(self):
        return (1.0 - self.f["phig"]) * (1.0 - self.f["theta"])

    def step(self, n=1):
        return lib().or_step(ctypes.byref(self.p), ctypes.byref(self.s), int(n))

    def mechanics(self):
        return lib().or_mechanics(ctypes.byref(self.p), ctypes.byref(self.s))

    def fields_update(self):
        lib().or_fields_update(ctypes.byref(self.p), ctypes.byref(self.s))

    def rates(self):
        """d/dt of (theta, x_O, x_H, x_H2O) at the current fields, shape (4, N)."""
        out = np.zeros(4 * self.N)
        lib().or_rates(ctypes.byref(self.p), ctypes.byref(self.s), _dp(out))
        return out.reshape(4, self.N)

    def free_energy(self):
        return lib().or_free_energy(ctypes.byref(self.p), ctypes.byref(self.s))

    def sums(self):
        out = np.zeros(3)
        lib().or_sums(ctypes.byref(self.p), ctypes.byref(self.s), _dp(out))
        return out  # sum xO, sum xH, sum xW

    @property
    def removedW(self):
        return self.s.removedW

    @property
    def suppliedH(self):
        return self.s.suppliedH

    @property
    def dt(self):
        return self.p.dt


def dt_stable(shape, prm):
    p = make_params(shape, prm, dt=1.0)
    return lib().or_dt_stable(ctypes.byref(p))


def lame(p, theta, phig):
    lam = np.zeros(theta.size)
    mu = np.zeros(theta.size)
    lib().or_cell_lame(ctypes.byref(p), _dp(np.ascontiguousarray(theta, np.float64)),
                       _dp(np.ascontiguousarray(phig, np.float64)), _dp(lam), _dp(mu))
    return lam, mu


def mech_apply(p, lam, mu, x):
    y = np.zeros_like(x)
    lib().or_mech_apply(ctypes.byref(p), _dp(lam), _dp(mu), _dp(np.ascontiguousarray(x, np.float64)), _dp(y))
    return y


def mech_diag(p, lam, mu, n):
    y = np.zeros(n)
    lib().or_mech_diag(ctypes.byref(p), _dp(lam), _dp(mu), _dp(y))
    return y


def pcg(p, lam, mu, b, x0=None):
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    rel = np.zeros(1)
    it = lib().or_pcg(ctypes.byref(p), _dp(lam), _dp(mu), _dp(np.ascontiguousarray(b)), _dp(x), _dp(rel))
    return x, it, float(rel[0])


def theta_force(p, theta, phig, xO, t, s2):
    return lib().or_theta_force(ctypes.byref(p), theta, phig, xO, t, s2)


def local_energy(p, theta, phig, xO, t, s2):
    return lib().or_local_energy(ctypes.byref(p), theta, phig, xO, t, s2)


def h(x):
    return lib().or_h(x)


def hp(x):
    return lib().or_hp(x)


def m(x):
    return lib().or_m(x)


def mp(x):
    return lib().or_mp(x)


def f(a, x):
    return lib().or_f(a, x)


def fp(a, x):
    return lib().or_fp(a, x)


def fpp(a, x):
    return lib().or_fpp(a, x)


def return_map(sim):
    """Run only the per-cell stress update / J2 return on the current u, Ebar."""
    lib().or_return_map(ctypes.byref(sim.p), ctypes.byref(sim.s))


def mech_rhs(sim, lam, mu):
    n = sim.N * sim.p.ndim + (3 if sim.p.ndim == 2 else 6)
    b = np.zeros(n)
    lib().or_mech_rhs(ctypes.byref(sim.p), ctypes.byref(sim.s), _dp(lam), _dp(mu), _dp(b))
    return b
