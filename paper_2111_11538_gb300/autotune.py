"""Measure the launch shapes the library picks per size class on the GPU,
record the measurements and write the table the library compiles in.

    python -m paper_2111_11538_gb300.autotune [--json OUT] [--header OUT]

Tuned choices (every one changes speed only: the results agree to rounding,
or are identical for the marching update):

  * PCG node tile (pf_config.pcg_tile = 1, 2) of the Jacobi-preconditioned
    solve, per size class (2D up to 2^18 nodes, 2D above, 3D) and storage
    type: a core-shell grid of the class is stepped with each tile and the
    solve time per CG iteration (the library's CUDA-event profile) decides;
  * the same tiles for the 2D multigrid-preconditioned solve (its V-cycle
    sweeps use the tile), per 2D size class and storage type, decided by
    the solve time per step on a porous grid of the class;
  * the start-up weight w of the marching field update's chunk choice (the
    cost model (items per block) x (planes per item + w)), per dimension:
    for each candidate w the chunk length the model then picks is run on
    the 2048^2 and 256^3 porous grids with the mechanics off
    (pf_config.fused_chunk), and the fastest update wins.

The table goes to data/autotune_gb300.json (with the measurements) and to
csrc/tuning.h (the defines the library compiles); a CPU test checks that
the two agree and that every entry is the argmin of its measurements.
"""
import argparse
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
JSON_PATH = os.path.join(HERE, "data", "autotune_gb300.json")
HEADER_PATH = os.path.join(HERE, "csrc", "tuning.h")

PCG_CLASSES = [
    ("2D", "SMALL", (512, 512)),        # <= 2^18 nodes
    ("2D", "LARGE", (1024, 1024)),
    ("3D", None, (96, 96, 96)),
]
MG_CLASSES = [("SMALL", (512, 512)), ("LARGE", (2048, 2048))]
STARTUP_CANDIDATES = (0, 1, 2, 3, 5, 8, 16, 32, 64)
FUSED_CASES = {2: (2048, 2048), 3: (256, 256, 256)}


def _sim(shape, prm, precision):
    from . import Simulation
    return Simulation(shape, prm, precision=precision)


def measure_pcg(shape, precision, tile, steps=3):
    """Solve time per CG iteration (us), Jacobi preconditioner."""
    from . import inputs, workloads
    n = shape[-1]
    f = inputs.core_shell(shape, 0.31 * n, 0.06 * n)
    prm = workloads.params(plasticity=1, cg_rtol=1e-8, pcg_tile=tile, precond="jacobi")
    sim = _sim(shape, prm, precision)
    sim.set_fields(f)
    sim.step(2)
    sim.profile(True)
    sim.step(steps)
    p = sim.profile_read()
    sim.close()
    return 1e3 * p["ms"]["cg"] / max(1, p["cg_iters"])


def measure_mg2d(shape, precision, tile, steps=4):
    """Solve time per step (ms), multigrid preconditioner, porous grid."""
    from . import inputs, workloads
    f = inputs.porous(shape, 200, 0.2, 12.0, 0.5, 2)
    prm = workloads.params(plasticity=0, cg_rtol=1e-8, pcg_tile=tile, precond="mg", warm_start="extrap")
    sim = _sim(shape, prm, precision)
    sim.set_fields(f)
    sim.step(3)
    sim.profile(True)
    sim.step(steps)
    p = sim.profile_read()
    sim.close()
    return p["ms"]["cg"] / steps


def model_chunk(cols, nm, cap, w):
    """The library's chunk choice for start-up weight w (host logic of the
    marching update, the same cost model)."""
    best, bcost = nm, None
    for zc in range(1, nm + 1):
        items = cols * ((nm + zc - 1) // zc)
        nb = min(items, cap)
        cost = ((items + nb - 1) // nb) * (zc + w)
        if bcost is None or cost < bcost:
            bcost, best = cost, zc
    return best


def measure_fused(f, chunk, steps=20):
    """Update time per launch (us) with an explicit chunk length."""
    from . import workloads
    shape = f["phi_f"].shape
    sim = _sim(shape, workloads.params(mechanics=0, fused_chunk=chunk), "mixed")
    sim.set_fields(f)
    sim.step(3)
    sim.profile(True)
    sim.step(steps)
    p = sim.profile_read()
    sim.close()
    return 1e3 * p["ms"]["update"] / max(1, p["count"]["update"])


def write_header(table, path=HEADER_PATH):
    lines = ["// Launch shapes per size class, measured on GB300 by",
             "// paper_2111_11538_gb300/autotune.py (which writes this file from the table",
             "// in paper_2111_11538_gb300/data/autotune_gb300.json).",
             "#pragma once"]
    for k in sorted(table):
        lines.append("#define %s %d" % (k, table[k]))
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--json", default=JSON_PATH)
    ap.add_argument("--header", default=HEADER_PATH)
    a = ap.parse_args(argv)
    from . import native
    native.build_library()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    table, rows = {}, []
    for dim, cls, shape in PCG_CLASSES:
        for prec, tag in (("mixed", "F32"), ("fp64", "F64")):
            times = [measure_pcg(shape, prec, t) for t in (1, 2)]
            best = min(range(2), key=lambda k: times[k])
            key = "PCG_TABLE_%s_%s%s" % (dim, tag, "_" + cls if cls else "")
            table[key] = best
            rows.append({"key": key, "kind": "pcg_jacobi", "shape": list(shape), "precision": prec,
                         "unit": "us per CG iteration", "candidates": [0, 1], "times": times, "best": best})
            print("%-26s %-14s tile0 %9.2f tile1 %9.2f -> %d" % (key, "x".join(map(str, shape)), times[0],
                                                                times[1], best), flush=True)
    for cls, shape in MG_CLASSES:
        for prec, tag in (("mixed", "F32"), ("fp64", "F64")):
            times = [measure_mg2d(shape, prec, t) for t in (1, 2)]
            best = min(range(2), key=lambda k: times[k])
            key = "PCG_TABLE_MG2D_%s_%s" % (tag, cls)
            table[key] = best
            rows.append({"key": key, "kind": "pcg_mg2d", "shape": list(shape), "precision": prec,
                         "unit": "ms of solve per step", "candidates": [0, 1], "times": times, "best": best})
            print("%-26s %-14s tile0 %9.3f tile1 %9.3f -> %d" % (key, "x".join(map(str, shape)), times[0],
                                                                times[1], best), flush=True)
    for dim, shape in FUSED_CASES.items():
        from . import workloads
        f = workloads.build_fields("porous256cube" if dim == 3 else "porous2048")
        tx, ty = (32, 8) if dim == 3 else (256, 1)
        cols = -(-shape[-1] // tx) * (-(-shape[-2] // ty) if dim == 3 else 1)
        nm = shape[0]
        per_sm = 3
        cap = sms * per_sm
        chunks = [model_chunk(cols, nm, cap, w) for w in STARTUP_CANDIDATES]
        cache = {}
        times = []
        for c in chunks:
            if c not in cache:
                cache[c] = measure_fused(f, c)
            times.append(cache[c])
        best = min(range(len(STARTUP_CANDIDATES)), key=lambda k: (times[k], STARTUP_CANDIDATES[k]))
        key = "FUSED_STARTUP_%dD" % dim
        table[key] = STARTUP_CANDIDATES[best]
        rows.append({"key": key, "kind": "fused_startup", "shape": list(shape), "precision": "mixed",
                     "unit": "us per update launch", "candidates": list(STARTUP_CANDIDATES), "chunks": chunks,
                     "times": times, "best": STARTUP_CANDIDATES[best]})
        print("%-26s %-14s %s -> w %d" % (key, "x".join(map(str, shape)),
                                          " ".join("w%d:%d:%.1f" % (w, c, t) for w, c, t in
                                                   zip(STARTUP_CANDIDATES, chunks, times)),
                                          STARTUP_CANDIDATES[best]), flush=True)
    with open(a.json, "w") as fh:
        json.dump({"table": table, "rows": rows, "sms": sms}, fh, indent=1)
    write_header(table, a.header)


if __name__ == "__main__":
    main()
