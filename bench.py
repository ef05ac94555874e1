"""Benchmark of the space-time MLMC monodomain path on GB300.

One step = one complete MLMC estimate of the mean activation map of the
3-level 2D workload (32^2/64^2/128^2 Q1 grids, 64/128/256 implicit-Euler
steps, 64 KL modes, N_l = 512/128/32 level pairs): xi, KL fields, both solves
of every pair, activation maps, level differences, accumulation and the
estimate, all through ``mlmc_run`` of the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                    [--impl ours|reference]

Prints one JSON line.  ``value`` is device time per estimate (CUDA events on
the launching stream, L2 flushed between steps); ``e2e`` is the wall time of
the same public call with host inputs and host outputs; ``roofline`` is for
the per-sample solve kernel, from CUDA events around its launches inside the
timed region and the iteration counts it reports; ``cpu_baseline`` times the
oracle on this host's cores on a bounded sample of the same workload.
``--impl reference`` times the oracle alone as the reference arm.
"""
import argparse
import concurrent.futures
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-RMSE eps (s) for MLMC mean activation map; stencil HBM GB/s; p99 latency"
# The ALU peaks are measured in-line by the library's FMA-chain probe
# (mlmc_probe_fma_rate: 8 independent FMA chains per thread, 16 x 256 threads
# per SM, CUDA events) and reported in the line; FP64 runs far below FP32 on
# this part, so FP64 and FP32 work are each set against their own peak.
# Algorithmic flops per node: one CG iteration (9-coupling stencil and Hessian
# diagonal 20, two dots 4, four vector updates 7) and one nonlinear iteration
# (residual: stencil 18, mass and reaction terms 12; update 2), in the CG's
# precision and in FP64 respectively.
FLOP_CG_NODE = 31
FLOP_NEWTON_NODE = 32
# Algorithmic HBM bytes per node of the 3D global-memory sweep (couplings are
# streamed from HBM every pass, each symmetric pair stored once: 14 per node):
# an FP32 CG iteration reads 14 FP32 couplings and touches 14 FP32 vector words
# (112 B); an FP64 one 14 FP64 couplings and 14 FP64 words (224 B); a Newton
# iteration runs the residual and the line-search passes, each 14 FP64
# couplings and 8 FP64 words (2 x 176 B).
BYTES_CG32_NODE_3D = 14 * 4 + 14 * 4
BYTES_CG64_NODE_3D = 14 * 8 + 14 * 8
BYTES_NEWTON_NODE_3D = 2 * (14 * 8 + 8 * 8)
# iteration cap per time step on the 3D slab: its level 1 steps take up to
# thousands of continuation iterations
SLAB3D_NEWTON_MAX = 40000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d", choices=["2d", "3d"],
                    help="2d: the 3-level 2D MLMC workload (default); 3d: the 4-level 3D slab "
                         "(32x32x8 .. 256x256x64, N_l = 256/64/16/4; minutes per estimate, no "
                         "CPU baseline by default: its finest levels take hours on the host)")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the automatic solve layouts instead of the autotuner's choice")
    ap.add_argument("--layouts", default=None, metavar="L0,L1,...",
                    help="use these per-level layout codes (mlmc_set_layout) instead of tuning")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch each estimate's kernels directly instead of as one CUDA graph")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-eps run and the serving run (reported beside the step time)")
    ap.add_argument("--profile-case", type=int, default=None, metavar="LEVEL",
                    help="run one small solve of LEVEL (2 samples, after one warm-up solve) for "
                         "an ncu capture of the solve kernel, instead of the benchmark")
    ap.add_argument("--profile-workload", default="2d", choices=["2d", "3d"],
                    help="--profile-case on the 3-level 2D workload or the 4-level 3D slab")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="--profile-case: only the first STEPS time steps of the level (same dt)")
    ap.add_argument("--profile-precond", default="jacobi", choices=["jacobi", "gmg"])
    ap.add_argument("--profile-kl", type=int, default=None, metavar="LEVEL",
                    help="run the tensor-core KL synthesis of LEVEL of the 3D slab twice for 256 "
                         "samples (the second launch is the one to capture), instead of the benchmark")
    return ap.parse_args()


# ------------------------------------------------------------------ oracle timing
def oracle_sample_cost(w, pairs, seed=1000, threads=None):
    """Single-thread seconds per level pair, measured on `pairs[l]` pairs of each
    level run concurrently on `threads` host threads (the C oracle releases the GIL)."""
    import oracle as O
    from paper_1911_06066_gb300 import workloads as W
    threads = threads or (os.cpu_count() or 1)
    levels = []
    extra = {k: w[k] for k in ("scheme", "stim_kind", "stim_amp", "stim_sigma", "stim_t1", "qoi")
             if k in w}
    for l in range(w["levels"]):
        n, m = W.level_shape(w, l)
        levels.append(O.make_level(w["dim"], n, m, w["L"], w["T"], w["c"], w["a"], w["s_t"],
                                   w["s_l0"], w["theta0"], w["theta1"], w["stim_r"], w["stim_c"],
                                   **extra))
    jobs = [(l, i) for l in range(w["levels"]) for i in range(pairs[l])]
    # longest first so the pool drains evenly
    jobs.sort(key=lambda j: -j[0])

    def one(job):
        l, i = job
        t0 = time.perf_counter()
        O.sample_pair(levels[l], levels[l - 1] if l else None, levels[0], w["sigma2"], w["ell"],
                      w["M"], seed, l, i)
        return l, time.perf_counter() - t0

    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, jobs))
    wall = time.perf_counter() - t0
    per = []
    for l in range(w["levels"]):
        ts = [t for ll, t in res if ll == l]
        per.append(sum(ts) / len(ts) if ts else 0.0)
    return per, wall, min(threads, len(jobs))


def cpu_estimate_seconds(w, per_pair, cores):
    """All-core time of one full estimate: sum_l N_l C_l / cores."""
    return sum(n * c for n, c in zip(w["N"], per_pair)) / cores


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ arms
def run_reference(args, w):
    """The oracle (CPU, FP64) as the reference arm: each step times a bounded
    sample of level pairs on all host cores and extrapolates to one estimate."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample = [16, 4, 1]
    for _ in range(args.warmup):
        oracle_sample_cost(w, [2, 0, 0])
    vals = []
    for k in range(args.steps):
        per, wall, used = oracle_sample_cost(w, sample, seed=2000 + k, threads=cores)
        vals.append(cpu_estimate_seconds(w, per, cores))
    v = sum(vals) / len(vals)
    desc = "L0/L1/L2 pairs %s per step, single-thread time per pair x N_l / %d cores" % (sample, cores)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "N_l": w["N"]},
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_ours(args, w):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU baseline first: host threads only, before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        sample = [32, 8, 2]
        per, wall, used = oracle_sample_cost(w, sample, threads=cores)
        cpu = {"value": cpu_estimate_seconds(w, per, cores), "unit": "s", "cores": cores,
               "kind": "oracle",
               "sample": "level pairs %s of the workload on %d host threads (%.1f s wall); "
                         "single-thread s/pair %s, extrapolated to N_l=%s on %d cores"
                         % (sample, used, wall, [round(x, 4) for x in per], w["N"], cores)}

    from __graft_entry__ import build
    build()
    from paper_1911_06066_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = B.MLMC_PREC_MIXED if args.precision == "mixed" else B.MLMC_PREC_FP64
    graph = not args.no_graph
    ctx = B.Context(B.make_config(w, prec, use_graph=graph,
                                  newton_max=SLAB3D_NEWTON_MAX if w["dim"] == 3 else 5000))
    seed = 1 + rank      # disjoint streams per rank: each rank runs its own estimate
    batch = max(w["N"])
    # a side stream: the legacy default stream cannot be captured into a graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device="cuda")
    # the project's autotuner picks each level's solve layout (block kernel,
    # shared- or global-memory clusters of 1-16 CTAs) on that level's batch,
    # before the warm-up
    # The levels then share the device inside an estimate, so the per-level
    # choice is kept only if a whole estimate is faster with it than with the
    # automatic layouts (each timed on its second run).
    layouts = {}
    if args.layouts:
        codes = [int(x) for x in args.layouts.split(",")]
        for l, c in enumerate(codes[:w["levels"]]):
            ctx.set_layout(l, c)
        layouts = {"given": codes}
    elif not args.no_tune:
        for l in range(w["levels"]):
            best, ms = ctx.autotune(l, min(w["N"][l], batch), seed=seed + 1000)
            layouts[l] = {"layout": best, "ms": {str(k): round(v, 2) for k, v in ms.items()}}

        def estimate_ms():
            # as the timed steps: one untimed run, then the mean of two runs,
            # each after an L2 flush
            ctx.run(w["N"], seed=seed + 2000, batch=batch)
            tot = 0.0
            for _ in range(2):
                flush.zero_()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                ctx.run(w["N"], seed=seed + 2000, batch=batch)
                ev1.record(stream)
                torch.cuda.synchronize()
                tot += ev0.elapsed_time(ev1)
            return tot / 2

        # every combination of (automatic, tuned) per level for up to three
        # levels, else greedy over the levels from the automatic layouts
        import itertools
        L = w["levels"]
        tuned = [layouts[l]["layout"] for l in range(L)]
        trail = []

        def trial(choice):
            for l in range(L):
                ctx.set_layout(l, tuned[l] if choice[l] else 0)
            t = estimate_ms()
            trail.append({"layouts": [ctx.layout(k) for k in range(L)], "ms": round(t, 1)})
            return t

        if L <= 3:
            combos = [c for c in itertools.product((0, 1), repeat=L)
                      if all(tuned[l] != 0 or not c[l] for l in range(L))]
            times = {c: trial(c) for c in combos}
            best = min(times, key=times.get)
            # the automatic layouts unless another combination is >= 1 % faster
            auto = tuple([0] * L)
            if times[best] > 0.99 * times[auto]:
                best = auto
        else:
            best = [0] * L
            t_best = trial(best)
            for l in range(L):
                if tuned[l] == 0:
                    continue
                cand = list(best)
                cand[l] = 1
                t = trial(cand)
                if t < 0.99 * t_best:
                    best, t_best = cand, t
        for l in range(L):
            ctx.set_layout(l, tuned[l] if best[l] else 0)
        layouts["whole_estimate_ms"] = trail

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ALU peaks of this device, measured in-line (FMA-chain probe)
    peaks = {"fp64_tflops": B.fma_rate(True, stream), "fp32_tflops": B.fma_rate(False, stream)}

    from paper_1911_06066_gb300 import distributed as D

    def one_estimate():
        """One step: one whole MLMC estimate.  One rank: mlmc_run.  N ranks:
        each rank runs its shard of every level's ids (mlmc_run_more), the
        per-level states are all-gathered over NCCL and merged in rank order
        (mlmc_merge_states); every rank ends with the estimate of all N_l."""
        if world == 1:
            return ctx.run(w["N"], seed=seed, batch=batch)
        out = D.run_sharded(ctx, w["N"], seed=seed, batch=batch)
        out["stats"] = None
        return out

    warmup = max(args.warmup, 3) if w["dim"] == 2 else args.warmup
    for _ in range(warmup):
        one_estimate()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    dev_ms, wall_s, solve_ms, launches, nsolve, rmse = 0.0, 0.0, 0.0, 0.0, 0.0, []
    per_level = None
    for k in range(args.steps):
        flush.zero_()                       # L2 flush (512 MB > 126 MB L2) outside the timed span
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        res = one_estimate()                # host in, host out (synchronising)
        e1.record(stream)
        t1 = time.perf_counter()
        torch.cuda.synchronize()
        dev_ms += e0.elapsed_time(e1)
        wall_s += t1 - t0
        st = res["stats"]
        if st is not None:
            solve_ms += st["solve_ms"]
            launches += st["launches"]
            nsolve += st["solve_launches"]
        rmse.append(res["rmse"])
        # per grid level: the solve launches of this run and the counters since
        # its reset (mlmc_run resets), i.e. this estimate's work
        lv_stats = ctx.level_stats()
        if per_level is None:
            per_level = [dict(v) for v in lv_stats]
        else:
            for acc, v in zip(per_level, lv_stats):
                for key in acc:
                    acc[key] += v[key]
    torch.cuda.synchronize()
    clk = clocks.stop()

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(w, B, prec, seed, stream, peaks)

    ms = dev_ms / args.steps
    e2e_s = wall_s / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e_s = t[0].item(), t[1].item()
    if rank != 0:
        return
    L = w["levels"]
    n0 = (w["n0"][0] + 1) * (w["n0"][1] + 1) * ((w["n0"][2] + 1) if w["dim"] == 3 else 1)
    d2h = 8 * (2 * n0 + 2 * L * n0 + L + 2) + 8 * 5
    levels = level_bounds(per_level, args.steps, peaks)
    if w["dim"] == 3:
        add_hbm_bytes(levels, per_level, args.steps)
    out = {
        "metric": METRIC, "value": ms * 1e-3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == B.MLMC_PREC_FP64 else
                 "f64 nonlinear iteration/residual/QoI + f32 CG (f64 KL field on the 32^2 level)",
        "data": "synthetic",
        "config": {"workload": w["name"], "N_l": w["N"], "grids": grids_of(w),
                   "steps_per_level": [w["m0"] * 2 ** l for l in range(w["levels"])],
                   "kl_modes": w["M"],
                   "precision": args.precision, "l2": "flushed between steps (512 MB write)",
                   "launch": "one CUDA graph per estimate" if graph else "direct launches",
                   "layouts": ({str(l): ctx.layout(l) for l in range(w["levels"])}
                               if layouts else "automatic"),
                   "rmse_achieved": statistics.mean(rmse),
                   "parallelism": ("one thread-block cluster per sample; levels on concurrent "
                                   "streams" + ("" if world == 1 else
                                                "; level ids sharded over %d ranks, one NCCL "
                                                "all-gather + Chan merge per estimate" % world))},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * L,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches / args.steps) if launches else None,
        "roofline": roofline_3d(levels, ms, peaks) if w["dim"] == 3 else
                    roofline_2d(levels, ms, peaks, all(ctx.layout(l) == 0 for l in range(L))),
        "levels": levels,
        "peaks_measured": peaks,
        "clocks": clk,
        "cpu_baseline": cpu,
        "autotune": layouts or None,
    }
    out.update(extras)
    print(json.dumps(out))


def level_bounds(per_level, steps, peaks):
    """Each grid level's solve launches against their own bound: FP64 work
    (nonlinear iterations, FP64 CG) over the measured FP64 FMA rate plus FP32
    CG work over the FP32 rate gives the ALU-bound time; frac = that time /
    the launches' measured time.  Per step (one estimate)."""
    out = []
    for l, v in enumerate(per_level):
        ms = v["solve_ms"] / steps
        f64 = (FLOP_NEWTON_NODE * v["newton_node_iters"] + FLOP_CG_NODE * v["cg64_node_iters"]) / steps
        f32 = FLOP_CG_NODE * (v["cg_node_iters"] - v["cg64_node_iters"]) / steps
        t_bound = f64 / (peaks["fp64_tflops"] * 1e12) + f32 / (peaks["fp32_tflops"] * 1e12)
        out.append({"level": l, "solve_ms": ms, "launches": v["solve_launches"] / steps,
                    "fp64_gflop": f64 * 1e-9, "fp32_gflop": f32 * 1e-9,
                    "alu_bound_ms": t_bound * 1e3,
                    "frac": t_bound * 1e3 / ms if ms > 0 else None,
                    "retried_pseudo_steps_or_halvings": v["halvings"] / steps,
                    "not_converged": v["not_converged"] / steps})
    return out


def roofline_2d(levels, step_ms, peaks, auto_layouts):
    """The dominant kernel is the per-sample sweep; its bound is the ALU (FP64
    for the nonlinear iterations and the FP64 CG, FP32 for the FP32 CG).
    achieved = FP64-equivalent algorithmic flops (FP32 flops scaled by
    peak64 / peak32) of the dominant grid level's launches over their
    measured time; peak = the measured FP64 rate, so frac = ALU-bound time /
    measured time of that level."""
    dom = max(levels, key=lambda v: v["solve_ms"])
    p64, p32 = peaks["fp64_tflops"], peaks["fp32_tflops"]
    eq = (dom["fp64_gflop"] + dom["fp32_gflop"] * p64 / p32) * 1e9
    achieved = eq / (dom["solve_ms"] * 1e-3) / 1e12 if dom["solve_ms"] > 0 else 0.0
    tot_bound = sum(v["alu_bound_ms"] for v in levels)
    return {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s",
            "frac": achieved / p64,
            # no DRAM capture of the current sweep at this size: the samples live
            # on chip (shared memory / L2), see the 2D profile summary
            "traffic": None,
            "kernel": "solve_cluster_kernel (per-sample sweep), grid level %d: FP64 + FP32 work "
                      "as FP64-equivalent flops" % dom["level"],
            "peak_source": "FP64 FMA-chain probe in this run (mlmc_probe_fma_rate), of measured",
            "whole_estimate_frac": tot_bound / step_ms if step_ms > 0 else None}


def measured_hbm_peak():
    """HBM copy bandwidth measured on the GB300s (GB/s), else the
    earlier single-GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def roofline_3d(levels, step_ms, peaks):
    """HBM roofline of the global-memory sweep (3D levels >= 1): algorithmic
    bytes of the dominant grid level's launches (from its node-weighted
    iteration counts) over their summed CUDA-event time (launches overlap on
    concurrent streams), against the measured copy bandwidth."""
    peak, src = measured_hbm_peak()
    dom = max(levels, key=lambda v: v["solve_ms"])
    achieved = dom["hbm_gb"] / (dom["solve_ms"] * 1e-3) if dom["solve_ms"] > 0 else 0.0
    tot_gb = sum(v["hbm_gb"] for v in levels)
    # every level's fraction too: the finest grid is the one whose sweep
    # streams its couplings from HBM (the coarser ones fit the L2)
    for v in levels:
        v["hbm_frac"] = v["hbm_gbs"] / peak if v.get("hbm_gbs") else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "solve_cluster_kernel, global-memory layout (couplings streamed per pass), "
                      "grid level %d" % dom["level"],
            "peak_source": src, "aggregate_gbs": tot_gb / (step_ms * 1e-3) if step_ms > 0 else None,
            "aggregate_frac": tot_gb / (step_ms * 1e-3) / peak if step_ms > 0 else None,
            "finest_level_frac": levels[-1].get("hbm_frac")}


def add_hbm_bytes(levels, per_level, steps):
    for v, c in zip(levels, per_level):
        nb = (BYTES_CG32_NODE_3D * (c["cg_node_iters"] - c["cg64_node_iters"]) +
              BYTES_CG64_NODE_3D * c["cg64_node_iters"] + BYTES_NEWTON_NODE_3D * c["newton_node_iters"])
        v["hbm_gb"] = nb / steps * 1e-9
        v["hbm_gbs"] = v["hbm_gb"] / (v["solve_ms"] * 1e-3) if v["solve_ms"] > 0 else None
    return levels


def timed_run(ctx, N, seed, batch, stream):
    """One estimate through mlmc_run, timed with CUDA events on `stream`."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = ctx.run(N, seed=seed, batch=batch)
    e1.record(stream)
    torch.cuda.synchronize()
    return res, e0.elapsed_time(e1) * 1e-3


def run_extras(w, B, prec, seed, stream, peaks):
    """Measurements beside the step time, on the same workload.

    fp64_check: the same estimate (same seed and N_l) in FP64, its time and
    the largest difference of its mean activation map from the timed
    precision's, against the 0.1 eps the mixed form must stay within.

    adaptive: the driver (mlmc_run_to_rmse) from pilot counts with eps = 1e-3 T;
    it drives the sampling error to eps / sqrt(2) and reports whether the
    bias estimate allows eps at all on this hierarchy (``reached``); only a
    run that reached eps has a ``time_to_eps_s``.  Beside it, the plain FP64
    one-sample-per-launch form's time for the same N_l, extrapolated from a
    few timed pairs per level; the per-level diagnostics of the estimate; and
    the same diagnostics with a fourth, finer level (256^2, 512 steps).

    serving: an open-loop Poisson stream of level-pair requests at 2000/s with
    per-request seeds and stimulus centres uniform in [0, 0.2]^2, the levels
    mixed in the proportions of the adaptive N_l, through the request server.

    slab3d: one estimate of the 4-level 3D slab (N_l = 256/64/16/4) with the
    HBM roofline of its global-memory sweep.
    """
    import numpy as np
    import torch
    from paper_1911_06066_gb300 import serving as S
    from paper_1911_06066_gb300 import workloads as W

    out = {}
    eps = 1e-3 * w["T"]
    batch = max(w["N"])
    # ---- the same estimate in FP64
    ctx = B.Context(B.make_config(w, prec, use_graph=True))
    ctx64 = B.Context(B.make_config(w, B.MLMC_PREC_FP64, use_graph=True))
    ctx64.run(w["N"], seed=seed, batch=batch)
    r64, s64 = timed_run(ctx64, w["N"], seed, batch, stream)
    rp, sp = timed_run(ctx, w["N"], seed, batch, stream)
    dmean = float(np.abs(rp["mean"] - r64["mean"]).max())
    out["fp64_check"] = {"fp64_seconds": s64, "timed_precision_seconds": sp,
                         "max_abs_dmean": dmean, "tolerance": 0.1 * eps,
                         "within": dmean <= 0.1 * eps,
                         "workload": w["name"], "N_l": w["N"], "seed": seed}
    del ctx64
    # ---- adaptive driver, bias diagnostics
    ctx.run([64, 16, 4], seed=seed + 100, batch=64)          # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ctx.run_to_rmse(eps, [64, 16, 4], max_rounds=8, max_per_level=1 << 20, seed=seed + 200,
                          batch=512)
    t_run = time.perf_counter() - t0
    N = res["N_l"]
    diag = ctx.diagnostics()
    stat = float(np.sqrt(np.sum(res["V_l"] / N)))
    plain = B.Context(B.make_config(w, B.MLMC_PREC_FP64, solver=B.MLMC_SOLVER_BLOCK))
    plain.run([1, 1, 1], seed=seed + 300, batch=1)
    per = []
    for l, k in enumerate([8, 4, 2]):
        cnt = [0] * w["levels"]
        cnt[l] = k
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        plain.reset()
        plain.run_more([0] * w["levels"], cnt, seed=seed + 400, batch=1)
        per.append((time.perf_counter() - t1) / k)
    plain_s = float(np.sum(np.asarray(per) * N))
    out["adaptive"] = {
        "eps": eps, "reached": bool(res["reached"]),
        "time_to_eps_s": t_run if res["reached"] else None,
        "seconds": t_run, "target_sampling_rmse": eps / math.sqrt(2.0), "sampling_rmse": stat,
        "bias": res["bias"], "rmse": res["rmse"], "message": res["message"],
        "N_l": N.tolist(), "V_l": res["V_l"].tolist(), "C_l": res["C_l"].tolist(),
        "mean_correction_norm_l": diag["mean_norm"].tolist(), "weak_rate_alpha": diag["alpha"],
        "censored_fraction_l": diag["censored"].tolist(),
        "plain_fp64_one_sample_per_launch": {
            "seconds_per_pair": per, "seconds_for_same_N_l": plain_s,
            "how": "8/4/2 pairs per level timed, x N_l (extrapolated)"},
        "same_N_l_ratio_plain_over_this": plain_s / t_run if t_run > 0 else None}
    del plain
    # a fourth, finer level (256^2, 512 steps) for the weak rate
    w4 = dict(w, levels=4, N=[256, 64, 16, 8], name=w["name"] + "+256")
    ctx4 = B.Context(B.make_config(w4, prec, use_graph=True))
    r4, s4 = timed_run(ctx4, w4["N"], seed + 500, 256, stream)
    d4 = ctx4.diagnostics()
    out["bias_diagnostic_4_levels"] = {
        "grids": grids_of(w4), "N_l": w4["N"], "seconds": s4,
        "mean_correction_norm_l": d4["mean_norm"].tolist(), "weak_rate_alpha": d4["alpha"],
        "censored_fraction_l": d4["censored"].tolist(), "V_l": r4["V_l"].tolist()}
    del ctx4
    # the paper's work model (Sec. 4.2) from this workload's measured costs
    out["work_report"] = work_report_of(ctx, w["levels"], 32, stream)
    # ---- serving
    mix = N / N.sum()
    srv_ctx = B.Context(B.make_config(w, prec))
    srv = B.Server(srv_ctx, max_batch=256, slots=6, mem_budget=8 << 30, max_wait_s=0.005)
    sched = S.poisson_schedule(2000.0, 2000, mix, rng_seed=seed, per_request_seed=True,
                               stim_box=(0.0, 0.2))
    rep = S.run_open_loop(srv, sched, timeout=600)
    srv.close()
    serving = {k: rep[k] for k in ("offered_rate", "completed", "seconds", "throughput", "p50_ms",
                                   "p99_ms", "max_queue", "batches", "arena_peak_bytes", "failed")}
    serving.update({"rate": 2000.0, "requests": 2000, "level_mix": mix.tolist(),
                    "variant": "per-request seeds, stimulus centre ~ U[0,0.2]^2",
                    "max_batch": 256, "slots": 6})
    # the offered 2000/s exceeds what one GPU sustains on this mix, so those
    # latencies are queueing; a second stream at half the measured throughput
    # gives the service latency of a sustainable load
    rate2 = 0.5 * rep["throughput"]
    srv = B.Server(srv_ctx, max_batch=256, slots=6, mem_budget=8 << 30, max_wait_s=0.005)
    n2 = int(max(200, min(2000, 3.0 * rate2)))
    sched = S.poisson_schedule(rate2, n2, mix, rng_seed=seed + 1, per_request_seed=True,
                               stim_box=(0.0, 0.2))
    rep2 = S.run_open_loop(srv, sched, timeout=600)
    srv.close()
    serving["sustainable"] = {k: rep2[k] for k in ("offered_rate", "completed", "seconds",
                                                   "throughput", "p50_ms", "p99_ms", "max_queue",
                                                   "batches", "failed")}
    serving["sustainable"].update({"rate": rate2, "requests": n2})
    out["serving"] = serving
    del srv_ctx
    # ---- the 4-level 3D slab, at reduced counts: its level 1 (64x64x16,
    # c dt max r' = 2.37) needs thousands of continuation iterations per late
    # step as the front widens, so the full N_l = 256/64/16/4 takes many
    # minutes (python bench.py --workload 3d runs it)
    w3 = dict(W.SLAB3D_4LVL, N=[16, 8, 4, 2])
    ctx3 = B.Context(B.make_config(w3, prec, use_graph=True, newton_max=SLAB3D_NEWTON_MAX))
    ctx3.run([2, 1, 1, 1], seed=seed + 600, batch=2)         # warm: modules, graph shapes
    r3, s3 = timed_run(ctx3, w3["N"], seed + 700, max(w3["N"]), stream)
    ls3 = ctx3.level_stats()
    lv3 = add_hbm_bytes(level_bounds(ls3, 1, peaks), ls3, 1)
    out["slab3d"] = {"workload": W.SLAB3D_4LVL["name"], "N_l": w3["N"], "grids": grids_of(w3),
                     "seconds": s3, "rmse": r3["rmse"], "C_l": r3["C_l"].tolist(),
                     "levels": lv3, "roofline": roofline_3d(lv3, s3 * 1e3, peaks),
                     "work_report": work_report_of(ctx3, 4, 2, stream)}
    return out


def per_sample_costs(ctx, levels, n, stream, seed=777):
    """W'_l of Sec. 4.2: device seconds per sample of grid level l, from one
    batch of n samples solved alone (CUDA events, after a warm-up solve)."""
    import torch
    out = []
    for l in range(levels):
        Z = ctx.kl_field(l, ctx.xi(seed, l, torch.arange(n)))
        ctx.solve(l, Z[:1])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.solve(l, Z)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) * 1e-3 / n)
    return out


def work_report_of(ctx, levels, n, stream):
    """Sec. 4.2's gamma_d (Eq. complexity) and work model (Eq. work,
    Eq. Work-MC, Eq. Work-MLMC) from measured per-sample costs."""
    from paper_1911_06066_gb300 import experiments as E
    rep = E.work_report(per_sample_costs(ctx, levels, n, stream))
    rep["how"] = "W'_l: device seconds per sample of level l, %d samples solved alone" % n
    return rep


def run_profile_case(args, w):
    """Two samples of one level of the benchmark workload through mlmc_solve:
    launch 1 is a warm-up, launch 2 the one to capture (ncu -s 1 -c 1).
    --profile-steps S keeps the level's time step and runs only its first S
    steps (a shorter end time), so that a capture of a large level ends soon."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_1911_06066_gb300 import binding as B
    level = args.profile_case
    if args.profile_steps:
        m_full = w["m0"] * 2 ** level
        steps = args.profile_steps
        if steps % (2 ** level) or steps > m_full:
            raise SystemExit("--profile-steps must be a multiple of 2^level, at most the level's steps")
        w = dict(w, m0=steps // 2 ** level, T=w["T"] * steps / m_full)
    prec = B.MLMC_PREC_MIXED if args.precision == "mixed" else B.MLMC_PREC_FP64
    pc = B.MLMC_PRECOND_GMG if args.profile_precond == "gmg" else B.MLMC_PRECOND_JACOBI
    ctx = B.Context(B.make_config(w, prec, precond=pc))
    Z = ctx.kl_field(level, ctx.xi(0, level, torch.arange(2)))
    ctx.solve(level, Z[:1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, info = ctx.solve(level, Z)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": level, "workload": w["name"], "steps": w["m0"] * 2 ** level,
                      "precision": args.precision, "precond": args.profile_precond, "samples": 2,
                      "seconds": time.perf_counter() - t0, "info": B.info_dicts(info)}))


def run_profile_kl(args):
    """The tensor-core KL synthesis of one level of the 3D slab for 256 samples,
    twice: launch 1 warms up, launch 2 is the one to capture (ncu -s 1 -c 1)."""
    import torch
    from __graft_entry__ import build
    build()
    from paper_1911_06066_gb300 import binding as B
    from paper_1911_06066_gb300 import workloads as W
    w = W.SLAB3D_4LVL
    level = args.profile_kl
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    xi = ctx.xi(0, level, torch.arange(256))
    ctx.kl_field_tc(level, xi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Z = ctx.kl_field_tc(level, xi)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, cells, _ = ctx.level_info(level)
    flops = 2.0 * 3 * cells * 256 * ((w["M"] + 31) // 32 * 32)
    print(json.dumps({"profile_kl": level, "cells": cells, "samples": 256, "modes": w["M"],
                      "ms": ms, "tensor_tflops_3xtf32": flops / ms * 1e-9,
                      "z_bytes_gbs": cells * 256 * 8 / ms * 1e-6, "z_absmax": float(Z.abs().max())}))


def grids_of(w):
    from paper_1911_06066_gb300 import workloads as W
    return "/".join("x".join(str(n) for n in W.level_shape(w, l)[0][:w["dim"]])
                    for l in range(w["levels"]))


def main():
    args = parse()
    from paper_1911_06066_gb300 import workloads as W
    w = W.MLMC2D_3LVL
    if args.workload == "3d":
        w = W.SLAB3D_4LVL
        args.no_cpu_baseline = True
        args.no_extras = True
    if args.profile_kl is not None:
        run_profile_kl(args)
    elif args.profile_case is not None:
        run_profile_case(args, W.SLAB3D_4LVL if args.profile_workload == "3d" else w)
    elif args.impl == "reference" and w["dim"] == 3:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's 3D levels 2-3 take hours "
                          "per sample on the host cores; the reference arm times the 2D workload"}))
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
