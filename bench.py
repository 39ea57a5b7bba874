"""Benchmark of the coupled phase-field step on GB300.

Workload (default): 3D porous microstructure, 256 x 256 x 256 cells (~500
Voronoi grains, pore fraction 0.15, lognormal pore radii with median 6 cells
and sigma 0.4, two supply layers on every face), J2 plasticity (sigma_Y =
0.01 E, H = 0.001 E), CG residual 1e-8.  One "step" is the whole hot path:
mechanics right-hand side, initial guess, PCG solve, J2 return, field
update.  The chosen form (FP32 fields and operator, FP64-grade reductions,
FP64 iterative refinement of the solve) gives ``value``; the plain FP64
method is measured beside it on the same GPU and the same input.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload porous256cube|coreshell512|porous2048|batch64|stencil|implicit|finite]

Under torchrun (N > 1) every rank advances its own replica of the workload
(the single-grid step does not shard; see the design notes) and ``value`` is
the sum over ranks.  Rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s, coupled PF+diffusion+mechanics, at stated FP64 error; % HBM peak"
L2_BYTES = 129 * 1024 * 1024

# Algorithmic bytes per node and PCG iteration (the minimum traffic of one
# Jacobi-preconditioned iteration: x, r, p read and written, w / s and the
# diagonal and the two Lame parameters read): 2D 16 words, 3D 24 words.
CG_ITER_WORDS = {2: 16, 3: 24}
CG_INIT_WORDS = {2: 10, 3: 15}
# The compulsory traffic of one multigrid-preconditioned iteration (a V-cycle)
# per finest-level node, in FP32 words (model, reported beside the figure
# above).  2D: finest level 29 (CG update fused into the first smoothing
# sweep) + 9.5 (post-smoothing) + 8 (w = A u); coarse grid levels ~18;
# shared-memory levels none.  3D (three components per vector): first sweep
# 46 (r, w, s, p, x, xpost and dinv, lam, mu read; p, x, s, r, xpre, r1, d1
# written), post-smoothing sweep 19 (xpre, r, xpost-correction, dinv, lam,
# mu read; xpost written), w = A u 17 (xpost, r, lam, mu read; w written),
# every coarse level 1/8 of the nodes with four sweeps of ~20 words: ~11.
MG_ITER_WORDS = {2: 64, 3: 93}
MG_INIT_WORDS = {2: 28, 3: 40}
# DRAM bytes per k_pcg launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from one ncu capture of the current kernel on the named workload, per
# finest node and V-cycle (so that it scales with the launch's iterations);
# None where the current kernel has not been captured.  porous256cube: the
# first timed solve of `bench.py --only mixed --steps 1 --warmup 4` (44
# V-cycles), 139.35 GB read + 85.84 GB written = 305.1 B per node and V-cycle
# (profiles/launches_porous256_mixed.md).
PCG_TRAFFIC_PER_NODE_ITER = {"porous256cube": 305.05}
# Algorithmic bytes per cell of the fused explicit update (k_fusedz): theta,
# phi_g, x_O, x_H, x_H2O, tr eps_e, |dev eps_e|^2, mobility read, the 1-byte
# supply mask read, theta, x_O, x_H, x_H2O written.
FUSED_BYTES = {"mixed": 8 * 4 + 1 + 4 * 4, "fp64": 8 * 8 + 1 + 4 * 8}
# ncu DRAM bytes per cell of the fused update, mechanics off, None where the
# current kernel has not been captured.  3D: one launch on the 256^3 porous
# input, 576.0 MB read + 244.0 MB written = 48.9 B per cell
# (profiles/k_fusedz_porous256_mechanics_off.md).
FUSED_TRAFFIC_PER_CELL = {2: None, 3: 48.875}


def _load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOAD = "porous256cube"
PRECOND = "auto"
SHAPE = None        # grid override for the short profiling lines (--shape)
WARM = None         # CG initial guess (--warm-start); default: the workload's "warm_start", else "extrap"

DESCR = {
    "porous256cube": "porous256cube_j2: 3D porous 256x256x256, ~500 Voronoi grains, pore fraction 0.15, "
                     "lognormal pore radii (median 6, sigma 0.4), supply layers on every face, J2 plasticity "
                     "sigma_Y=0.01E H=0.001E, CG rtol 1e-8",
    "coreshell512": "coreshell512_j2: 2D core-shell 512x512, radius 160, shell 32, J2 plasticity "
                    "sigma_Y=0.01E H=0.001E, CG rtol 1e-8",
    "porous2048": "porous2048: 2D porous 2048x2048, ~200 Voronoi grains, pore fraction 0.2, lognormal pore radii "
                  "(median 12, sigma 0.5), elastic, CG rtol 1e-8",
    "coreshell64": "coreshell64: 2D core-shell 64x64, radius 20, shell 4, elastic, CG rtol 1e-10",
}
WARM_TEXT = {"extrap": "2 u_n - u_(n-1) (previous solution for the first two steps)",
             "extrap2": "3 u_n - 3 u_(n-1) + u_(n-2) (lower orders for the first three steps)",
             "prev": "previous solution", "zero": "zero", "learned": "learned (U-Net)"}


def workload_fields(name=None):
    """Seeded initial fields of a workload: the bench's own (on the --shape
    grid if given), or another workload on its own grid."""
    from paper_2111_11538_gb300 import workloads
    if name is None:
        return workloads.build_fields(WORKLOAD, shape=SHAPE)
    return workloads.build_fields(name)


def workload_params(precision, name=None):
    from paper_2111_11538_gb300 import workloads
    # both forms solve to the workload's CG residual: the mixed form reaches
    # it through FP64 iterative refinement around its FP32 iteration
    p = dict(workloads.WORKLOADS[name or WORKLOAD]["params"], precond=PRECOND)
    p["warm_start"] = warm_mode(name)
    return p


def warm_mode(name=None):
    from paper_2111_11538_gb300 import workloads
    return WARM or workloads.WORKLOADS[name or WORKLOAD].get("warm_start", "extrap")


def run_gpu(precision, steps, warmup, fields, profile=True, warm=None, net=None, name=None, prm=None,
            keys=("phi_f", "phi_w", "xO", "xH", "xW", "sigma")):
    """Advance `fields` for warmup + steps steps, timing the last `steps`
    with CUDA events on the launch stream (the L2 flushed before each)."""
    import torch
    from paper_2111_11538_gb300 import Simulation
    shape = fields["phi_f"].shape
    prm = dict(prm) if prm is not None else workload_params(precision, name)
    if warm is not None:
        prm["warm_start"] = warm
    sim = Simulation(shape, prm, precision=precision)
    if net is not None:
        sim.attach_unet(net)
    sim.set_fields(fields)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    for _ in range(warmup):
        sim.step(1, stream=sh)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    sim.profile(profile)
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(steps):
        flush.zero_()                       # evict the working set from L2
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(1, stream=sh)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
    prof = sim.profile_read() if profile else None
    diag = sim.diagnostics()
    if prof is not None:
        prof["precond"] = "mg" if diag["precond"] == 2 else "jacobi"
        prof["mg_levels"] = diag["mg_levels"]
    out = sim.get_fields(keys=keys) if keys else None
    sim.close()
    del flush
    return total_ms, prof, diag, out


def run_e2e(precision, steps, fields, warmup=2):
    """Same metric through the public API with host buffers: every step copies
    the full state in from pinned host memory and the fields back out.  The
    first `warmup` steps run untimed, as in the device timing, so that both
    time the same steps of the run (its early steps take more V-cycles)."""
    import torch
    from paper_2111_11538_gb300 import Simulation
    shape = fields["phi_f"].shape
    sim = Simulation(shape, workload_params(precision), precision=precision)

    def pinned(a, dtype=np.float64):
        t = torch.empty(a.shape, dtype=torch.float64 if dtype == np.float64 else torch.uint8, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()
    state = {k: pinned(v, np.uint8 if k == "mask" else np.float64) for k, v in fields.items()}
    sim.set_fields(state)
    sim.step(warmup)
    keys = ("phi_f", "phi_w", "xO", "xH", "xW", "theta", "phig", "u", "Ebar", "eps_p", "alpha")
    cur = sim.get_fields(keys=keys)
    state.update({k: pinned(v) for k, v in cur.items()})
    h2d = sum(v.nbytes for v in state.values())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.set_fields(state)
        sim.step(1)
        cur = sim.get_fields(keys=keys, out=state)     # straight into the pinned state
    dt = time.perf_counter() - t0
    d2h = sum(cur[k].nbytes for k in keys)
    sim.close()
    return dt, h2d, d2h


def run_batch(precision, steps, warmup, count=64, seed=4, profile=True, rank=0, world=1):
    """The batched workload: `count` independent 2D porous instances of uneven
    sizes (128^2 .. 1024^2), seeded pore fractions and prestresses, advanced
    together by one launch per kernel class and step.  With several ranks
    each advances its cost-balanced share of the instances."""
    import torch
    from paper_2111_11538_gb300 import Batch, inputs, sharding, workloads
    desc = inputs.batch_instances(count, seed)
    mine = sharding.shard([sharding.instance_cost((d["n"], d["n"])) for d in desc], world)[rank]
    desc = [desc[i] for i in mine]
    count = len(desc)
    base = dict(workloads.WORKLOADS["batch64"]["params"], precond=PRECOND,
                warm_start=WARM or workloads.WORKLOADS["batch64"].get("warm_start", "extrap"))
    shapes = [(d["n"], d["n"]) for d in desc]
    prms = [dict(base, prestress=d["prestress"]) for d in desc]
    b = Batch(shapes, prms, precision=precision)
    for i, d in enumerate(desc):
        b.set_fields(i, inputs.batch_fields(d))
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    b.step(warmup, stream=sh)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    b.profile(profile)
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(1, stream=sh)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    prof = b.profile_read()
    cells = sum(n[0] * n[1] for n in shapes)
    iters = [b.diagnostics(i)["cg_iters_last"] for i in range(count)]
    b.close()
    return total_ms, prof, cells, iters


WARMSTART_WEIGHTS = os.path.join(ROOT, "paper_2111_11538_gb300", "data", "warmstart2d.npz")


def learned_warm_start(steps, warmup, fields, prev_ms, prev_iters, name):
    """The chosen form with the learned warm start (the trained 2D network
    shipped with the package) beside the default guess of the timed run
    (the "default_guess_*" keys), same steps."""
    if len(fields["phi_f"].shape) != 2:
        return {"status": "no trained 3D network ships with the package; the 2D network is reported on "
                          "the 512x512 core-shell line"}
    if not os.path.exists(WARMSTART_WEIGHTS):
        return {"status": "no trained network at paper_2111_11538_gb300/data/warmstart2d.npz"}
    from paper_2111_11538_gb300 import warmstart
    net = warmstart.load(WARMSTART_WEIGHTS)
    ms, prof, diag, _ = run_gpu("mixed", steps, warmup, fields, warm="learned", net=net, name=name, keys=())
    info = {}
    if os.path.exists(WARMSTART_WEIGHTS + ".json"):
        info = json.load(open(WARMSTART_WEIGHTS + ".json"))
    N = fields["phi_f"].size
    net.close()
    return {"value": N * steps / (ms / 1e3), "unit": "cell-steps/s", "ms_per_step": ms / steps,
            "cg_iters_per_step": prof["cg_iters"] / steps, "default_guess": warm_mode(name),
            "default_guess_cg_iters_per_step": prev_iters / steps,
            "default_guess_ms_per_step": prev_ms / steps,
            "network_ms": prof["ms"]["warm"] / max(1, prof["count"]["warm"]), "training": info}


def stencil_roofline(fields, name, steps=20, warmup=3):
    """Achieved HBM bandwidth of the fused explicit update alone: the
    workload's microstructure stepped with the mechanics off, so that every
    launch is k_fusedz; per-launch CUDA events on the launch stream."""
    from paper_2111_11538_gb300 import Simulation, workloads
    shape = fields["phi_f"].shape
    sim = Simulation(shape, workloads.params(mechanics=0), precision="mixed")
    sim.set_fields(fields)
    sim.step(warmup)
    sim.profile(True)
    sim.step(steps)
    prof = sim.profile_read()
    sim.close()
    launches = prof["count"]["update"]
    ms = prof["ms"]["update"] / launches
    hbm, kind = _load_peaks()
    N = int(np.prod(shape))
    algo = FUSED_BYTES["mixed"] * N
    gbs = algo / (ms / 1e3) / 1e9
    nd = len(shape)
    tr = FUSED_TRAFFIC_PER_CELL.get(nd)
    return {"kernel": "k_fusedz (mu_O + explicit update, %dD)" % nd,
            "workload": "%s, %s cells, mechanics off" % (name, "x".join(str(v) for v in shape[::-1])),
            "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "traffic": tr * N if tr else None, "peak_kind": kind + " (hbm_gbs, burst copy)",
            "algorithmic_bytes_per_launch": algo, "us_per_launch": ms * 1e3, "launches": launches}


def oracle_sample(fields, n=20):
    """The 256^3 workload's own fields cropped to their n^3 corner (the corner
    holds the supply layers of three faces; the crop is periodic like the
    whole box), for the oracle's CPU timing."""
    return {k: np.ascontiguousarray(v[:n, :n, :n]) for k, v in fields.items()}


def time_oracle(fields, prm, warmup, steps=None, seconds=None):
    """Single-threaded FP64 oracle steps on the host: `warmup` untimed steps,
    then `steps` timed steps (or timed steps until `seconds` have passed)."""
    import oracle
    s = oracle.Sim(fields, prm)
    for _ in range(warmup):
        s.step(1)
    n, its = 0, []
    t0 = time.perf_counter()
    while (steps is not None and n < steps) or (steps is None and time.perf_counter() - t0 < seconds):
        its.append(s.step(1))
        n += 1
    dt = time.perf_counter() - t0
    return fields["phi_f"].size * n / dt, n, dt, its


def cpu_baseline(crop, seconds=12.0):
    """The FP64 oracle on the host (single thread) over a bounded sample of the
    workload: its own fields cropped to the 20^3 corner, one untimed step,
    then timed steps until about `seconds` have passed."""
    from paper_2111_11538_gb300 import workloads
    prm = workloads.WORKLOADS[WORKLOAD]["params"]
    v, n, dt, its = time_oracle(crop, prm, 1, seconds=seconds)
    edge = crop["phi_f"].shape[0]
    return {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d^3 corner of the 256^3 porous workload's own fields (periodic crop, same parameters, "
                      "J2, CG rtol 1e-8), %d timed steps after 1 untimed, single-threaded FP64 C; the oracle's "
                      "Jacobi PCG took %s iterations per step on the crop" % (edge, n, its)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def reduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pcg_roofline(prof, N, nd, steps, name):
    """k_pcg against the HBM roofline: achieved = (24 words per node and
    iteration in 3D, 16 in 2D: the minimum traffic of one PCG iteration)
    x N x the launch's iterations / the launch's event time, beside the
    multigrid V-cycle's own compulsory traffic (model)."""
    hbm, peak_kind = _load_peaks()
    mg = prof.get("precond") == "mg"
    launches = prof["count"]["cg"]
    cg_ms = prof["ms"]["cg"]
    iters = prof["cg_iters"]
    if not launches or cg_ms <= 0:
        return None
    us_launch = cg_ms / launches * 1e3
    it_launch = iters / launches
    algo = CG_ITER_WORDS[nd] * 4 * N * it_launch
    achieved = algo / (us_launch / 1e6) / 1e9
    model = (MG_ITER_WORDS[nd] if mg else CG_ITER_WORDS[nd]) * 4 * N * it_launch + \
            (MG_INIT_WORDS[nd] if mg else CG_INIT_WORDS[nd]) * 4 * N
    tr = PCG_TRAFFIC_PER_NODE_ITER.get(name)
    return {"kernel": "k_pcg (persistent PCG, %s, %dD)" % ("multigrid V-cycle" if mg else "Jacobi", nd),
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": tr * N * it_launch if tr else None,
            "peak_kind": peak_kind + " (hbm_gbs, burst copy)",
            "unit_bytes": "%d B per node and PCG iteration x %d nodes x %.2f iterations per launch"
                          % (CG_ITER_WORDS[nd] * 4, N, it_launch),
            "algorithmic_bytes_per_launch": algo, "us_per_launch": us_launch, "iters_per_launch": it_launch,
            "vcycle_model_bytes_per_launch": model, "vcycle_model_frac": model / (us_launch / 1e6) / 1e9 / hbm}


def short_line(name, steps, warmup):
    """Another workload on its own grid, the chosen form beside the plain FP64
    method (short runs), for the extra keys of the headline line."""
    f = workload_fields(name)
    if f is None:
        return None
    N = f["phi_f"].size
    ms, prof, diag, out = run_gpu("mixed", steps, warmup, f, name=name)
    s64 = max(2, steps // 4)
    ms64, prof64, _, out64 = run_gpu("fp64", s64, warmup + steps - s64, f, name=name)
    line = {"workload": DESCR.get(name, name), "cells": N, "steps": steps, "warmup": warmup,
            "value": N * steps / (ms / 1e3), "unit": "cell-steps/s", "ms_per_step": ms / steps,
            "cg_iters_per_step": prof["cg_iters"] / steps, "warm_start": WARM_TEXT.get(warm_mode(name)),
            "fp64_plain": {"value": N * s64 / (ms64 / 1e3), "ms_per_step": ms64 / s64,
                           "cg_iters_per_step": prof64["cg_iters"] / s64},
            "error_vs_fp64": {k: relerr(out[k], out64[k]) for k in out},
            "kernel_ms": prof["ms"]}
    line["speedup_vs_fp64_plain"] = line["value"] / line["fp64_plain"]["value"]
    line["roofline"] = pcg_roofline(prof, N, len(f["phi_f"].shape), steps, name)
    if len(f["phi_f"].shape) == 2:
        line["learned_warm_start"] = learned_warm_start(steps, warmup, f, ms, prof["cg_iters"], name)
    return line


def backward_euler_line(n=256, steps=3, dt=0.05, explicit_steps=20):
    """Backward-Euler steps (pf_step_implicit, FP64) at the paper's Table 1
    diffusivities and reaction rate (workloads.paper_params) on the n x n
    core-shell of the 512^2 recipe, beside explicit steps of the same model
    (the library's dt: 0.2 x the explicit limit): physical time advanced per
    wall-clock second both ways.  Wall clock (the Newton-Krylov loop is
    driven from the host)."""
    import time
    import torch
    from paper_2111_11538_gb300 import Simulation, inputs, workloads
    f = inputs.core_shell((n, n), 0.3125 * n, 0.0625 * n)
    prm = workloads.paper_params(cg_rtol=1e-10)
    sim = Simulation((n, n), prm, precision="fp64")
    sim.set_fields(f)
    sim.step_implicit(1, dt)                   # allocations, first solve
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    newton = gmres = 0
    for _ in range(steps):
        st = sim.step_implicit(1, dt)
        newton += st["newton_iters"]
        gmres += st["gmres_iters"]
    t_imp = (time.perf_counter() - t0) / steps
    d = sim.diagnostics()
    # the same steps with the block preconditioner in FP64
    sim.set_fields(f)
    sim.step_implicit(1, dt, pc_precision="fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gmres64 = 0
    for _ in range(steps):
        gmres64 += sim.step_implicit(1, dt, pc_precision="fp64")["gmres_iters"]
    t_imp64 = (time.perf_counter() - t0) / steps
    sim.close()
    ex = Simulation((n, n), prm, precision="fp64")
    ex.set_fields(f)
    ex.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ex.step(explicit_steps)
    t_exp = (time.perf_counter() - t0) / explicit_steps
    dt_e = ex.diagnostics()["dt"]
    ex.close()
    return {"workload": "core-shell %dx%d, paper Table 1 diffusivities and k_for (explicit limit %.2e), FP64"
                        % (n, n, dt_e / 0.2),
            "dt": dt, "s_per_step": t_imp, "newton_iters_per_step": newton / steps,
            "gmres_iters_per_step": gmres / steps, "preconditioner": "FP32 (FP64 GMRES, products, residual)",
            "s_per_step_fp64_preconditioner": t_imp64, "gmres_iters_per_step_fp64_preconditioner": gmres64 / steps,
            "explicit_dt": dt_e, "explicit_s_per_step": t_exp,
            "explicit_steps_per_step": dt / dt_e,
            "physical_time_per_s": dt / t_imp, "explicit_physical_time_per_s": dt_e / t_exp,
            "speedup_vs_explicit": (dt / t_imp) / (dt_e / t_exp),
            "balances": {"O": d["sum_O"] + d["sum_H2O"] + d["removed_H2O"],
                         "H": d["sum_H"] + 2 * d["sum_H2O"] + 2 * d["removed_H2O"] - d["supplied_H"]}}


# The finite-strain Hessian-vector product kernel (k_fs_hvp<3, FDf>, FP32
# forward mode) from one ncu capture of the current kernel on the 64^3
# workload (profiles/k_fs_hvp_coreshell64_finite_strain.md): FP32 flops per
# cell = 2 FFMA + FADD + FMUL thread instructions / cells, and DRAM bytes
# per cell (the 64^3 working set sits in L2, so they are below the
# compulsory bytes).  Its bound is the FP32 pipe: the peak is 152 SMs x 128
# FP32 lanes x 2 flops x 2.07 GHz (the counters' FFMA peak of 128 per cycle
# and SM; the maximum SM clock).
FS_HVP_FLOPS_PER_CELL = 10036.4
FS_HVP_DRAM_PER_CELL = 114.4
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def finite_strain_line(n=64, omega=0.2, nload=2, only="both"):
    """One staggered elasto-plastic finite-strain mechanics step
    (pf_finite_strain_step: neo-Hooke mixture with the transformation
    stretch, Newton-CG to max |residual| <= 1e-10, then the multiplicative J2
    update per cell) on the n^3 core-shell with gas, with FP32 and with FP64
    Hessian-vector products: wall time, Newton and CG counts, and the
    product kernel's device time (CUDA events around each launch on its
    stream, pf_fs_stats.hvp_ms).  The call allocates its own memory, so the
    wall time includes that; the first call (untimed) loads the kernels."""
    import time
    import torch
    from paper_2111_11538_gb300 import Simulation, inputs, make_config, native, workloads
    shape = (n, n, n)
    f = inputs.core_shell(shape, 0.3 * n, 0.15 * n, delta=1.0)
    prm = workloads.params(plasticity=1, sigma_Y=0.002, H_hard=0.01)
    sim = Simulation(shape, dict(prm, mechanics=0), precision="fp64")
    sim.set_fields(f)
    g = sim.get_fields(keys=("theta", "phig"))
    sim.close()
    th, pg = g["theta"].ravel(), g["phig"].ravel()
    cfg = make_config(shape, prm)
    N = th.size
    out = {"workload": "finite-strain elasto-plastic step, core-shell %d^3 with gas (E_g/E_s = %.3g), Omega = %g, "
                       "%d load steps, FP64 residual" % (n, prm["E_g_ratio"], omega, nload), "cells": N}
    small = (8, 8, 8)
    for name, prec in (("fp32_products", native.PF_MIXED), ("fp64_products", native.PF_FP64)):
        if only != "both" and (prec == native.PF_MIXED) != (only == "mixed"):
            continue
        o = native.pf_fs_opts(nload=nload, newton_maxit=40, newton_tol=1e-10, cg_maxit=100000, cg_rtol=1e-10,
                              precision=prec)
        FP = np.tile(np.eye(3), (int(np.prod(small)), 1, 1))
        native.pf_finite_strain_step(make_config(small, prm), np.full(small, 0.5), np.zeros(small), omega, None, o,
                                     FP, np.zeros(int(np.prod(small))))
        FP = np.tile(np.eye(3), (N, 1, 1))
        ep = np.zeros(N)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, u, Fb, st = native.pf_finite_strain_step(cfg, th, pg, omega, None, o, FP, ep)
        t = time.perf_counter() - t0
        out[name] = {"rc": rc, "s_per_step": t, "newton_iters": st.newton_iters, "cg_iters": st.cg_iters,
                     "residual": st.residual, "hvp_launches": st.hvp_launches,
                     "hvp_ms_per_launch": st.hvp_ms / max(st.hvp_launches, 1),
                     "hvp_share_of_wall": st.hvp_ms / 1e3 / t,
                     "cell_products_per_s": N * st.hvp_launches / t, "plastic_cells": int((ep > 0).sum()),
                     "max_u": float(np.abs(u).max())}
    if "fp32_products" in out:
        a = out["fp32_products"]
        tf = FS_HVP_FLOPS_PER_CELL * N / (a["hvp_ms_per_launch"] * 1e-3) / 1e12
        out["roofline"] = {"kernel": "k_fs_hvp<3, FDf> (FP32 Hessian-vector product)", "bound": "alu",
                           "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": tf / FP32_PEAK_TFLOPS,
                           "traffic": FS_HVP_DRAM_PER_CELL * N if n == 64 else None,
                           "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                           "unit_flops": "%.1f FP32 flops per cell (ncu instruction counts) x %d cells per launch"
                                         % (FS_HVP_FLOPS_PER_CELL, N)}
    if only == "both":
        a, b = out["fp32_products"], out["fp64_products"]
        out["speedup_fp32_products"] = b["s_per_step"] / a["s_per_step"]
        out["hvp_speedup_per_launch"] = b["hvp_ms_per_launch"] / max(a["hvp_ms_per_launch"], 1e-12)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (default: --steps, after the same --warmup)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads' keys")
    ap.add_argument("--workload", default="porous256cube",
                    help="porous256cube (default, the headline); coreshell512, porous2048, coreshell64, "
                         "batch64, stencil, implicit (backward-Euler steps at the paper's "
                         "diffusivities) or finite (a finite-strain elasto-plastic step, 64^3) print a "
                         "short line")
    ap.add_argument("--only", default="both", choices=["both", "mixed", "fp64"],
                    help="profiling aid: run one method only and print a short line")
    ap.add_argument("--precond", default="auto", choices=["auto", "jacobi", "mg"],
                    help="CG preconditioner (auto: the library's choice for the grid)")
    ap.add_argument("--warm-start", default=None, choices=["zero", "prev", "extrap", "extrap2"],
                    help="CG initial guess: extrapolation from the previous solutions (first or "
                         "second order), the previous solution, or zero; default: the workload's choice")
    ap.add_argument("--shape", default=None,
                    help="profiling aid with --only: the workload's geometry on another grid, "
                         "e.g. 128,128,128 (nz,ny,nx)")
    args = ap.parse_args()
    global WORKLOAD, PRECOND, SHAPE, WARM
    WORKLOAD = args.workload
    PRECOND = args.precond
    WARM = args.warm_start
    if args.shape:
        if args.only == "both" and args.workload != "finite":
            ap.error("--shape needs --only (the headline line is measured on the workload's own grid)")
        SHAPE = tuple(int(v) for v in args.shape.split(","))
    if args.warmup < 3:
        args.warmup = 3

    ws, rank, local = dist_setup()
    cfg = {"workload": DESCR.get(WORKLOAD, WORKLOAD),
           "warm_start": WARM_TEXT.get(warm_mode()) if WORKLOAD in DESCR else None,
           "precond": args.precond + (" (library choice: multigrid V-cycle for this grid)" if args.precond == "auto" else ""),
           "l2": "flushed before every timed step (256 MB write); the 256^3 working set (~2 GB) exceeds L2",
           "parallelism": "replicas" if ws > 1 else "single"}

    if args.impl == "reference":
        # the reference arm: the FP64 oracle on the host cores, on a bounded
        # sample of the same workload (there is no reference implementation
        # to install: the paper publishes no code)
        if rank != 0:
            return
        import oracle
        oracle.build()
        from paper_2111_11538_gb300 import workloads
        crop = oracle_sample(workload_fields("porous256cube"), 20)
        v, n, dt, its = time_oracle(crop, workloads.WORKLOADS["porous256cube"]["params"], args.warmup,
                                    steps=args.steps)
        sample = ("each step: one oracle step of the 20^3 corner of the 256^3 porous workload's own fields "
                  "(periodic crop, same parameters, J2, CG rtol 1e-8), single-threaded FP64 C")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-steps/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": cfg,
                          "cpu_baseline": {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2111_11538_gb300 import native
    native.build_library()
    if WORKLOAD == "stencil":
        out = [stencil_roofline(workload_fields("porous256cube"), "porous256cube", args.steps,
                                args.warmup),
               stencil_roofline(workload_fields("porous2048"), "porous2048", args.steps, args.warmup)]
        print(json.dumps(out))
        return
    if WORKLOAD == "implicit":
        print(json.dumps(backward_euler_line()))
        return
    if WORKLOAD == "finite":
        print(json.dumps(finite_strain_line(n=SHAPE[0] if SHAPE else 64, only=args.only)))
        return
    if WORKLOAD == "batch64":
        meth = "mixed" if args.only == "both" else args.only
        for prof_on in (False, True):
            msb, profb, cells, iters = run_batch(meth, args.steps, args.warmup, profile=prof_on, rank=rank, world=ws)
            msb = reduce_max(msb, ws)
            cells = int(reduce_sum(cells, ws))
            if rank == 0:
                print(json.dumps({"workload": WORKLOAD, "method": meth, "cells": cells, "steps": args.steps,
                                  "n_gpus": ws, "scaling": "strong (the 64 instances split over ranks, no collective)",
                                  "timing": "per-kernel events" if prof_on else "graph replay",
                                  "ms_per_step": msb / args.steps, "value": cells * args.steps / (msb / 1e3),
                                  "kernel_ms": profb["ms"], "cg_iters": profb["cg_iters"],
                                  "graph_steps": profb["graph_steps"],
                                  "cg_iters_last_min_max": [min(iters), max(iters)]}))
        return
    fields = workload_fields()
    N = fields["phi_f"].size
    nd = len(fields["phi_f"].shape)
    if args.only != "both":
        ms1, prof1, diag1, _ = run_gpu(args.only, args.steps, args.warmup, fields, keys=())
        if rank == 0:
            print(json.dumps({"workload": WORKLOAD, "shape": list(fields["phi_f"].shape), "method": args.only,
                              "cells": N, "steps": args.steps,
                              "ms_per_step": ms1 / args.steps, "value": N * args.steps / (ms1 / 1e3),
                              "kernel_ms": prof1["ms"], "cg_iters": prof1["cg_iters"],
                              "precond": prof1.get("precond"), "mg_levels": prof1.get("mg_levels"),
                              "roofline": pcg_roofline(prof1, N, nd, args.steps, WORKLOAD)}))
        return

    # plain FP64 method on the same input (reported beside the chosen form);
    # its state after fp64_warm + steps64 steps is the reference of the
    # chosen form's per-field error
    steps64 = max(2, args.fp64_steps)
    warm64 = 3
    barrier(ws)
    ms64, prof64, diag64, out64 = run_gpu("fp64", steps64, warm64, fields)

    # the chosen form, timed (clocks sampled during the timed region)
    barrier(ws)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ms, prof, diag, out = run_gpu("mixed", args.steps, args.warmup, fields)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    ms_max = reduce_max(ms, ws)
    value = N * args.steps * ws / (ms_max / 1e3)

    # per-field error of the chosen form against the plain FP64 method after
    # the same number of steps (the FP64 path is held to the oracle by the
    # parity tests)
    if args.steps + args.warmup == steps64 + warm64:
        outm = out
    else:
        _, _, _, outm = run_gpu("mixed", steps64, warm64, fields, profile=False)
    err = {k: relerr(outm[k], out64[k]) for k in out64}
    del out, outm, out64

    roof = pcg_roofline(prof, N, nd, args.steps, WORKLOAD)
    stencil = stencil_roofline(fields, WORKLOAD, steps=20, warmup=3)
    e2e_steps = args.e2e_steps or args.steps
    e2e_dt, h2d, d2h = run_e2e("mixed", e2e_steps, fields, warmup=args.warmup)
    e2e_val = N * e2e_steps * ws / reduce_max(e2e_dt, ws)

    extra = {}
    if not args.no_extra and ws == 1:
        try:
            extra["coreshell512"] = short_line("coreshell512", 20, 5)
        except Exception as e:  # noqa: BLE001
            extra["coreshell512"] = {"error": str(e)[:200]}
        try:
            extra["roofline_stencil_2d"] = stencil_roofline(workload_fields("porous2048"), "porous2048")
        except Exception as e:  # noqa: BLE001
            extra["roofline_stencil_2d"] = {"error": str(e)[:200]}
        try:
            extra["backward_euler"] = backward_euler_line()
        except Exception as e:  # noqa: BLE001
            extra["backward_euler"] = {"error": str(e)[:200]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        try:
            cpu = cpu_baseline(oracle_sample(fields, 20))
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "error": str(e)[:200]}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 fields+operator, f64 reductions and f64 refinement of the solve "
                 "(error vs plain f64 in error_vs_fp64)",
        "data": "synthetic", "config": dict(cfg, cells=N),
        "fp64_plain": {"value": N * steps64 * ws / (reduce_max(ms64, ws) / 1e3), "unit": "cell-steps/s",
                       "steps": steps64, "warmup": warm64, "ms_per_step": ms64 / steps64,
                       "cg_iters_per_step": prof64["cg_iters"] / steps64, "kernel_ms": prof64["ms"]},
        "speedup_vs_fp64_plain": None,
        "error_vs_fp64": dict(err, after_steps=steps64 + warm64),
        "cg": {"rtol": workload_params("mixed")["cg_rtol"],
               "mixed": "FP32 Chronopoulos-Gear PCG passes inside FP64 iterative refinement",
               "precond": prof.get("precond"), "mg_levels": prof.get("mg_levels"),
               "iters_timed": prof["cg_iters"], "iters_per_step": prof["cg_iters"] / args.steps},
        "kernel_ms": prof["ms"], "kernel_count": prof["count"],
        "roofline": roof,
        "roofline_stencil": stencil,
        "learned_warm_start": learned_warm_start(0, 0, fields, 0, 0, WORKLOAD),
        "e2e": {"value": e2e_val, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "warmup": args.warmup,
                "note": "pf_set_fields / pf_step / pf_get_fields of the full state with pinned host buffers "
                        "every step, over the same steps of the run as the device timing; a round trip "
                        "leaves the solver's trajectory unchanged (same V-cycles per step)"},
        "gpu_launches": prof["launches"],
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    line["speedup_vs_fp64_plain"] = value / line["fp64_plain"]["value"] if line["fp64_plain"]["value"] else None
    print(json.dumps(line))


if __name__ == "__main__":
    main()
