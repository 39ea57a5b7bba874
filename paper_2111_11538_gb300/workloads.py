"""Nondimensional parameter sets and the benchmark workloads.

Units: energy density in units of the solid Young's modulus E_s, length in
grid spacings (dx = 1), time in units of 1 / (L E_s) (phase mobility L = 1).

Derivation of the default ("bench") set from the paper's Table 1 (Sec. 3.2)
at theta = 973.15 K:
  * R theta / V_mol = 8.3145 * 973.15 / 1.224e-5 = 0.661 GPa; the wuestite
    Young's modulus from K = 88, G = 24 GPa is 66.0 GPa, so the CALPHAD
    polynomials of Sec. 3.1 enter scaled by c_chem = 0.661 / 66.0 = 0.0100.
  * w_alpha = 1e3 / V_mol = 0.0817 GPa -> w = 0.0817 / 66.0 = 1.2379e-3.
  * interface resolution: at the common-tangent potential the interpolated
    CALPHAD energies raise a barrier of c_chem * 5.0 = 0.05 between ferrite
    and wuestite, ~300x the double-well height 2 w m(1/2); this barrier, not
    w, sets the ferrite/wuestite interface width.  epsilon_alpha = 0.4 makes
    that interface span about three cells (10-90 %), the width the
    workloads' initial tanh profiles have; kappa_O keeps the paper's ratio
    kappa_O / epsilon_alpha = 5e-10 / 4e-5.
  * gas / solid stiffness ratio E_g / E_s = K_g / K_w = 0.17 / 88 = 1.93e-3.
  * The paper's diffusivities and mobility make the explicit scheme stiff by
    ~1e6 (D_gas / (L epsilon)); the bench set compresses them:
    D_O,s = D_H,s = 0.05, D_gas = 1.0 for all species, D_H2O,s = 1e-10,
    k_for = 1.0, x_H on supply cells 0.01 (Sec. 4.2).
"""

BENCH_PARAMS = {
    "c_chem": 0.0100,
    "w": 1.2379e-3,
    "eps_phi": 0.4,
    "kappa_O": 0.4 * (5.0e-10 / 4.0e-5),
    "L": 1.0,
    "D_O_s": 0.05, "D_O_g": 1.0,
    "D_H_s": 0.05, "D_H_g": 1.0,
    "D_W_s": 1.0e-10, "D_W_g": 1.0,
    "k_for": 1.0,
    "xH_bc": 0.01,
    "E_s": 1.0, "nu": 0.3, "E_g_ratio": 1.93e-3,
    "eig0": -0.05,
    "sigma_Y": 0.01, "H_hard": 0.001,
    "prestress": 0.0,
    "cg_rtol": 1e-10, "cg_maxit": 20000,
    "mechanics": 1, "plasticity": 0, "warm_start": 1,
    "dt": 0.0,          # 0 -> 0.2 x stable limit
}


def params(**over):
    p = dict(BENCH_PARAMS)
    p.update(over)
    return p


def paper_params(**over):
    """Table 1 of the paper (Sec. 3.2) in the units of BENCH_PARAMS, for
    time integration by backward Euler (explicit Euler needs dt ~ 7e-8 here).

    The time unit is 1 / (L E_s) = 1 / (1.5e-10 * 66.0e9) = 0.101 s; the
    grid spacing that eps = 0.4 stands for is dx^2 = eps_phys / (E_s eps) =
    4.0e-5 / (66.0e9 * 0.4) = 1.515e-15 m^2 (dx = 39 nm).  A diffusivity D
    [m^2/s] becomes D * 0.101 / 1.515e-15 = 6.67e13 D, a rate k [1/s] becomes
    0.101 k, a stress [GPa] becomes its ratio to 66.0 GPa:
      * D_O: 2.16e-11 (solids) -> 1440, 1.0e-8 (gas) -> 6.67e5;
      * D_H: 2.5e-11 -> 1667, 1.0e-8 -> 6.67e5;
      * D_H2O: 2.5e-20 -> 1.67e-6, 1.0e-8 -> 6.67e5;
      * k_for: 4.5e4 -> 4545;
      * sigma_Y = 0.3 GPa -> 4.55e-3, H = 1.29 GPa -> 1.95e-2.
    The energies (c_chem, w, eps_phi, kappa_O) and the elastic set are those
    of BENCH_PARAMS, which already follow Table 1.
    """
    p = dict(BENCH_PARAMS)
    p.update({
        "D_O_s": 1440.0, "D_O_g": 6.67e5,
        "D_H_s": 1667.0, "D_H_g": 6.67e5,
        "D_W_s": 1.67e-6, "D_W_g": 6.67e5,
        "k_for": 4545.0,
        "sigma_Y": 4.55e-3, "H_hard": 1.95e-2,
    })
    p.update(over)
    return p


# The five workloads (grid, steps, precision, numerics).  Geometry builders
# live in inputs.py.
WORKLOADS = {
    "coreshell64": {
        "shape": (64, 64), "steps": 500, "precision": "fp64",
        "geometry": ("core_shell", {"radius": 20.0, "shell": 4.0}),
        "params": params(plasticity=0, cg_rtol=1e-10),
    },
    "coreshell512": {
        "shape": (512, 512), "steps": 20000, "precision": "fp64|mixed",
        "geometry": ("core_shell", {"radius": 160.0, "shell": 32.0}),
        # both methods solve to 1e-8: with Jacobi preconditioning this grid's
        # cond(A) times the FP32 unit roundoff is near 1, so the FP32 passes of
        # the mixed method cannot resolve residuals much below 1e-9
        "params": params(plasticity=1, sigma_Y=0.01, H_hard=0.001, cg_rtol=1e-8),
        # plastic flow makes the history less smooth: linear extrapolation
        # (1.30 ms/step; second order 1.42)
        "warm_start": "extrap",
    },
    "porous2048": {
        "shape": (2048, 2048), "steps": 10000, "precision": "mixed",
        "geometry": ("porous", {"n_grains": 200, "pore_fraction": 0.2, "pore_median": 12.0,
                                "pore_sigma": 0.5, "seed": 2}),
        "params": params(plasticity=0, cg_rtol=1e-8),
        # CG initial guess the bench uses (measured on GB300): the elastic
        # solution evolves smoothly, so second-order extrapolation pays
        # (18.0 vs 32.0 ms/step with the linear one)
        "warm_start": "extrap2",
    },
    "porous256cube": {
        "shape": (256, 256, 256), "steps": 2000, "precision": "mixed",
        "geometry": ("porous", {"n_grains": 500, "pore_fraction": 0.15, "pore_median": 6.0,
                                "pore_sigma": 0.4, "seed": 3}),
        "params": params(plasticity=1, cg_rtol=1e-8),
    },
    "batch64": {
        "count": 64, "steps": 5000, "precision": "mixed", "seed": 4,
        "params": params(plasticity=0, cg_rtol=1e-8),
        # elastic: second-order extrapolation (259 vs 325 ms/step on GB300)
        "warm_start": "extrap2",
    },
}


def build_fields(name, shape=None):
    from . import inputs
    wl = WORKLOADS[name]
    kind, kw = wl["geometry"]
    shape = tuple(shape or wl["shape"])
    if kind == "core_shell":
        scale = shape[-1] / float(wl["shape"][-1])
        return inputs.core_shell(shape, kw["radius"] * scale, kw["shell"] * scale)
    return inputs.porous(shape, **kw)
