"""Measure the PCG sweep's node tiles per size class on the GPU and print
the table the library compiles in (PCG_TABLE_* in csrc/pf_lib.cu).

    python -m paper_2111_11538_gb300.autotune [--json OUT]

For every size class (2D up to 2^18 nodes, 2D above, 3D) and storage type
it steps a core-shell grid of that class with each tile shape (pf_config
.pcg_tile = 1, 2) and reports the solve time per PCG iteration from the
library's CUDA-event profile; the fastest shape wins.  Every shape gives
the same result to rounding, so the choice changes speed only.
"""
import argparse
import json

CLASSES = [
    ("2D_SMALL", (512, 512)),        # <= 2^18 nodes
    ("2D_LARGE", (1024, 1024)),
    ("3D", (96, 96, 96)),
]


def measure(shape, precision, tile, steps=3):
    from . import Simulation, inputs, workloads
    n = shape[-1]
    f = inputs.core_shell(shape, 0.31 * n, 0.06 * n)
    prm = workloads.params(plasticity=1, cg_rtol=1e-8, pcg_tile=tile)
    sim = Simulation(shape, prm, precision=precision)
    sim.set_fields(f)
    sim.step(2)
    sim.profile(True)
    sim.step(steps)
    p = sim.profile_read()
    sim.close()
    return 1e3 * p["ms"]["cg"] / max(1, p["cg_iters"])


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    table, rows = {}, []
    for name, shape in CLASSES:
        for prec, tag in (("mixed", "F32"), ("fp64", "F64")):
            times = [measure(shape, prec, t) for t in (1, 2)]
            best = min(range(2), key=lambda k: times[k])
            key = "PCG_TABLE_%s_%s" % (name.replace("3D", "3D").split("_")[0], tag)
            if name.startswith("2D"):
                key = "PCG_TABLE_2D_%s_%s" % (tag, name.split("_")[1])
            table[key] = best
            rows.append({"class": name, "shape": list(shape), "precision": prec,
                         "us_per_iteration": times, "best": best})
            print("%-9s %-16s %-5s us/iter tile1 %8.2f tile2 %8.2f -> %s = %d" % (
                name, "x".join(map(str, shape)), prec, times[0], times[1], key, best), flush=True)
    if a.json:
        with open(a.json, "w") as fh:
            json.dump({"table": table, "rows": rows}, fh, indent=1)


if __name__ == "__main__":
    main()
