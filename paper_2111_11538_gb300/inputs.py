"""Seeded synthetic initial microstructures.

This module only builds initial fields (geometry, random grains and pores).
It contains none of the time-step arithmetic and is shared by the CUDA path,
the oracle tests and the benchmark so that both sides see identical inputs.

Every generator returns a dict of float64 numpy arrays (row-major, x fastest;
shape (ny, nx) or (nz, ny, nx)):

    phi_f, phi_w      ferrite / wuestite order parameters (gas = 1 - phi_f - phi_w)
    xO, xH, xW        oxygen, hydrogen, water molar fractions
    mob               per-cell factor on the phase mobility (grain scatter)
    mask              uint8, 1 on cells whose x_H / x_H2O are held (gas supply)

The paper's core-shell geometry (Sec. 4.2: wuestite core, iron shell, gas
box with 1 % hydrogen, x_O of the oxide at the wuestite equilibrium value)
and its SEM-derived porous microstructure (Sec. 4.3; the image is not
available) are replaced by these seeded stand-ins.
"""
import numpy as np

X_W_INIT = 0.571   # oxygen fraction of the oxide (Sec. 3.1 figure caption, Sec. 4.2)
X_F_INIT = 0.01    # oxygen fraction of the iron shell (Sec. 3.1)
XH_GAS = 0.01      # hydrogen fraction of the gas (Sec. 4.2)


def _tanh_step(d, delta):
    """0 -> 1 across d = 0 with width parameter delta (phi = (1 + tanh(d/delta))/2)."""
    return 0.5 * (1.0 + np.tanh(d / delta))


def _centre_dist(shape):
    axes = [np.arange(n, dtype=np.float64) + 0.5 - n / 2.0 for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    return np.sqrt(sum(g * g for g in grids))


def core_shell(shape, radius, shell, delta=3.0, supply_gap=None):
    """Wuestite core (radius) with an iron shell (thickness shell) in a gas box.

    shape: (ny, nx) or (nz, ny, nx).  The Dirichlet (hydrogen supply) mask is
    every cell farther than radius + shell + supply_gap from the centre
    (default gap 2 * delta), i.e. the gas away from the shell.
    """
    r = _centre_dist(shape)
    phi_w = 1.0 - _tanh_step(r - radius, delta)
    phi_f = _tanh_step(r - radius, delta) - _tanh_step(r - radius - shell, delta)
    phi_g = 1.0 - phi_f - phi_w
    if supply_gap is None:
        supply_gap = 2.0 * delta
    return {
        "phi_f": phi_f,
        "phi_w": phi_w,
        "xO": X_W_INIT * phi_w + X_F_INIT * phi_f,
        "xH": XH_GAS * phi_g,
        "xW": np.zeros(shape),
        "mob": np.ones(shape),
        "mask": (r > radius + shell + supply_gap).astype(np.uint8),
    }


def _periodic_nearest(points, shape):
    """Index of the nearest seed point for every cell (periodic box)."""
    from scipy.spatial import cKDTree
    box = np.array(shape[::-1], dtype=np.float64)            # x, y(, z)
    tree = cKDTree(points, boxsize=box)
    axes = [np.arange(n, dtype=np.float64) + 0.5 for n in shape[::-1]]
    grids = np.meshgrid(*axes, indexing="ij")               # x, y(, z) order
    q = np.stack([g.ravel() for g in grids], axis=1)
    _, ids = tree.query(q, workers=-1)
    # grids were built x-major; reshape to (x, y, z) then transpose to (z, y, x)
    return ids.reshape(tuple(shape[::-1])).transpose(tuple(range(len(shape)))[::-1])


def porous(shape, n_grains, pore_fraction, pore_median, pore_sigma, seed,
           delta=3.0, supply_layers=2, mob_range=(0.8, 1.2), rim=3.0):
    """Voronoi wuestite grains with lognormal gas pores (periodic box).

    * n_grains seed points uniform in the box; every grain gets a mobility
      factor drawn uniformly from mob_range.
    * pores: balls with radii ~ lognormal(ln(pore_median), pore_sigma) at
      uniform centres, added until the gas volume fraction reaches
      pore_fraction; their edges are smoothed with the tanh profile.
    * a ferrite rim of width `rim` cells lines every pore.
    * the outermost supply_layers cell layers of the box are gas and form the
      hydrogen supply (mask), as an open channel to the surroundings.
    """
    rng = np.random.default_rng(seed)
    d = len(shape)
    box = np.array(shape[::-1], dtype=np.float64)
    seeds = rng.uniform(0.0, 1.0, size=(n_grains, d)) * box
    grain = _periodic_nearest(seeds, shape)
    gmob = rng.uniform(mob_range[0], mob_range[1], size=n_grains)
    mob = gmob[grain]

    # signed distance to the nearest pore surface (negative inside)
    dist = np.full(shape, np.inf)
    total = float(np.prod(shape))
    filled = 0.0
    while filled < pore_fraction * total:
        rad = float(np.exp(np.log(pore_median) + pore_sigma * rng.standard_normal()))
        c = rng.uniform(0.0, 1.0, size=d) * np.array(shape, dtype=np.float64)
        reach = int(np.ceil(rad + 3.0 * delta)) + 1
        sl = []
        offs = []
        for ax in range(d):
            n = shape[ax]
            lo = int(np.floor(c[ax])) - reach
            ids = np.arange(lo, lo + 2 * reach + 1)
            sl.append(np.mod(ids, n))
            offs.append(ids.astype(np.float64) + 0.5 - c[ax])
        og = np.meshgrid(*offs, indexing="ij")
        rr = np.sqrt(sum(o * o for o in og)) - rad
        ix = np.ix_(*sl)
        old = dist[ix]
        new = np.minimum(old, rr)
        dist[ix] = new
        # cells that turned gas with this pore (the count of dist < 0 over
        # the box, kept incrementally; the ball's box never wraps onto itself
        # on the grids used here, and where it does the sum below is exact)
        if all(2 * reach + 1 <= n for n in shape):
            filled += float(np.count_nonzero(new < 0.0) - np.count_nonzero(old < 0.0))
        else:
            filled = float(np.sum(dist < 0.0))
    phi_g = 1.0 - _tanh_step(dist, delta)
    mask = np.zeros(shape, dtype=np.uint8)
    for ax in range(d):
        idx = [slice(None)] * d
        idx[ax] = slice(0, supply_layers)
        mask[tuple(idx)] = 1
        idx[ax] = slice(shape[ax] - supply_layers, shape[ax])
        mask[tuple(idx)] = 1
    phi_g = np.where(mask == 1, 1.0, phi_g)
    # the oxide next to every pore starts as a thin iron rim (the reduced
    # surface layer, as the shell of the core-shell geometry)
    theta = 1.0 - _tanh_step(dist - rim, delta)
    solid = 1.0 - phi_g
    phi_f = solid * theta
    phi_w = solid * (1.0 - theta)
    return {
        "phi_f": phi_f,
        "phi_w": phi_w,
        "xO": X_W_INIT * phi_w + X_F_INIT * phi_f,
        "xH": XH_GAS * phi_g,
        "xW": np.zeros(shape),
        "mob": mob,
        "mask": mask,
    }


def batch_instances(count, seed, sizes=(128, 256, 512, 1024), pore_range=(0.05, 0.3),
                    prestress_range=(0.0, 0.02)):
    """Descriptors of independent 2D porous instances with uneven sizes.

    Returns a list of dicts {n, pore_fraction, prestress, seed}; the fields of
    instance i come from porous((n, n), ...) with seed * 1000 + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        out.append({
            "n": n,
            "pore_fraction": float(rng.uniform(*pore_range)),
            "prestress": float(rng.uniform(*prestress_range)),
            "seed": seed * 1000 + i,
        })
    return out


def batch_fields(desc, delta=3.0):
    n = desc["n"]
    grains = max(4, int(round(200 * (n * n) / (2048.0 * 2048.0))))
    return porous((n, n), grains, desc["pore_fraction"], 12.0, 0.5, desc["seed"], delta=delta)
