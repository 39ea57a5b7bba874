"""Sharding of independent instances over ranks (one GPU each).

The instances of a batch are independent problems (separate particles and
pore networks, Sec. 4.3), so a multi-GPU run splits the instance list and
needs no exchange on the data path: rank r advances only its instances.
Work per instance and step is taken as its cells under the multigrid
solve (V-cycles per step do not grow with the grid) and as cells x linear
size under the Jacobi solve (its iteration count grows with the linear
size); instances are dealt largest first to the least-loaded rank.
"""


def instance_cost(shape, precond="mg"):
    """Relative work of one instance per step: "mg" (the library's choice
    for batches of multigrid-sized grids) or "jacobi"."""
    cells = 1
    for n in shape:
        cells *= n
    if precond == "mg":
        return cells
    if precond == "jacobi":
        return cells * max(shape)
    raise ValueError("precond must be 'mg' or 'jacobi'")


def shard(costs, world):
    """Indices of the instances of each rank: list of `world` sorted lists."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(o) for o in out]
