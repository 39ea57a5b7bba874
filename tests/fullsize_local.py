"""Oracle checks of one time step at any grid size (test helper).

The oracle recomputes the per-cell part of a step from the state the
library had before it: given the fields, plastic state and solved
displacement, the J2 return (Sec. 2.3) and the explicit update (Sec. 2.4)
are local, so they can be redone on the whole grid, or on a periodic
sub-box whose interior cells have all their inputs inside the box.  The
solve itself is checked by its residual under the oracle's operator.
"""
import numpy as np

STATE_KEYS = ("phi_f", "phi_w", "xO", "xH", "xW", "u", "Ebar", "eps_p", "alpha")
OUT_KEYS = ("alpha", "eps_p", "sigma", "phi_f", "phi_w", "xO", "xH", "xW")


def oracle_state(sim):
    """The state of an oracle.Sim in the layout of Simulation.get_fields."""
    out = {"phi_f": sim.phi_f.copy(), "phi_w": sim.phi_w.copy()}
    for k in ("xO", "xH", "xW", "u", "Ebar", "eps_p", "alpha", "sigma", "theta", "phig"):
        out[k] = sim.f[k].copy()
    return out


def _box(a, origin, m, nd):
    for ax in range(nd):
        a = np.take(a, np.arange(origin[ax], origin[ax] + m), axis=ax, mode="wrap")
    return a


def step_errors(orc, prm, before, after, static, origin=None, m=None):
    """Largest differences, relative to each output's largest magnitude (at
    least 1e-6), between the outputs of one step (`after`) and the oracle's
    return map and explicit update recomputed from `before` (fields, eps_p,
    alpha) and the step's solved displacement (`after`'s u and Ebar).  With `origin` and
    `m` the check runs on the periodic m-cell box at `origin` and compares
    the cells at least 3 from its faces; otherwise on the whole grid.
    `static` holds the mobility and the supply mask."""
    nd = before["phi_f"].ndim
    if origin is None:
        cut = lambda a: a                                       # noqa: E731
        inner = (slice(None),) * nd
    else:
        cut = lambda a: _box(a, origin, m, nd)                   # noqa: E731
        inner = (slice(3, m - 3),) * nd
    exact = "theta" in before and "phig" in before
    keys = ("phi_f", "phi_w", "xO", "xH", "xW", "eps_p", "alpha") + (("theta", "phig") if exact else ())
    f = {k: cut(before[k]) for k in keys}
    f["mob"] = cut(static["mob"])
    f["mask"] = cut(static["mask"])
    f["u"] = cut(after["u"])
    f["Ebar"] = np.asarray(after["Ebar"], dtype=np.float64)
    s = orc.Sim(f, prm)
    orc.return_map(s)
    ref = {"alpha": s.f["alpha"].copy(), "eps_p": s.f["eps_p"].copy(), "sigma": s.f["sigma"].copy()}
    s.fields_update()
    ref.update({"phi_f": s.phi_f, "phi_w": s.phi_w, "xO": s.f["xO"], "xH": s.f["xH"], "xW": s.f["xW"],
                "theta": s.f["theta"]})
    # With the exported order parameter and gas fraction the state is exact
    # and every cell is compared (theta too).  From phi_f, phi_w alone the
    # order parameter of cells with no solid (phi_g = 1) is lost; its value
    # there enters the Laplacian of the neighbours, so the phase outputs are
    # then compared away from such cells.
    gas = (f["phi_f"] + f["phi_w"]) == 0.0
    near_gas = gas.copy()
    for ax in range(nd):
        near_gas |= np.roll(gas, 1, axis=ax) | np.roll(gas, -1, axis=ax)
    errs = {}
    for k in OUT_KEYS + (("theta",) if exact else ()):
        g = cut(after[k])[inner]
        r = ref[k][inner]
        if k in ("phi_f", "phi_w") and not exact:
            keep = ~near_gas[inner]
            g, r = g[keep], r[keep]
        # relative to the output's magnitude, floored at 1e-6 so that a field
        # still near zero (early water, elastic plastic strain) is held to an
        # absolute bound
        errs[k] = float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-6)) if g.size else 0.0
    return errs


def solve_residual(orc, prm, before, after, static):
    """||b - A x|| / ||b|| of the step's solved displacement (`after`'s u
    and Ebar) for the operator and right-hand side the oracle builds from
    the state before the step (whole grid)."""
    f = {k: before[k] for k in ("phi_f", "phi_w", "xO", "xH", "xW", "eps_p", "alpha", "theta", "phig")
         if k in before}
    f["mob"] = static["mob"]
    f["mask"] = static["mask"]
    s = orc.Sim(f, prm)
    lam, mu = orc.lame(s.p, s.f["theta"].ravel(), s.f["phig"].ravel())
    b = orc.mech_rhs(s, lam, mu)
    x = np.concatenate([np.asarray(after["u"], dtype=np.float64).ravel(),
                        np.asarray(after["Ebar"], dtype=np.float64).ravel()])
    r = b - orc.mech_apply(s.p, lam, mu, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))
