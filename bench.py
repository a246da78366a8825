#!/usr/bin/env python3
"""NSGA-III generation throughput on GB300.

One step = one generation of a plain NSGA-III run: variation + objective,
then the environmental selection over the merged 2N x m objectives
(dominance matrix, front peel, normalization, association, niching) and the
gather of the next population, as one CUDA-graph launch of the C-ABI
library.

Default (no --workload): the headline line on the largest single-GPU
configuration, m = 10, two-layer directions p1 = 3 + p2 = 2 (275), N =
100,000, d = 200, 200 generations timed from generation 0 after warm-up
generations on the same context (re-initialised), with sub-records for the
m = 5, N = 10,628 run ("secondary"), the 64 batched runs ("batched"), a
prefix of the served request stream ("served"), the measured issue ceiling
of the dominance build ("issue_probe") and the oracle on the host cores
("cpu_baseline").

Metric: selected solutions per second (N x generations / device time), plus
generations per second.  The L2 cache is flushed (256 MB write) before every
timed step; each step is timed by CUDA events on the launching stream.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
        [--workload headline|small|scale|large|huge|knapsack|batched|served|sweep|popsweep|select]
Multi-GPU (torchrun): each rank advances an independent replica (seed + rank),
"scaling": "weak"; rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# Runs on separate streams (the run server: one stream per admitted run) share
# the device's hardware work queues, 8 unless the process asks for more
# before CUDA starts; with 64 runs in flight, 8 queues serialise kernels of
# unrelated runs (the served prefix: 14.4 -> 15.4 runs/s with 32).  Graph
# branches (batched runs) and single-stream runs are not affected.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2504_06067_gb300 import workloads as wl  # noqa: E402

METRIC = "selected sols/s & gens/s (% HBM roofline); batched/served runs/s, p50/p99 vs plain"
WORKLOADS = {"small": wl.SMALL, "scale": wl.SCALE, "large": wl.LARGE, "huge": wl.HUGE,
             "knapsack": wl.KNAPSACK}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
NUM_SMS = 152
LANES_PER_SM = 128


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed generations (default: the workload's run length)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["headline"] + sorted(WORKLOADS) +
                   ["batched", "served", "sweep", "popsweep", "select", "custom", "shapes"], default="headline")
    p.add_argument("--runs", type=int, default=64, help="batched: independent runs")
    p.add_argument("--m", type=int, default=10, help="custom: objectives")
    p.add_argument("--N", type=int, default=30000, help="custom: population")
    p.add_argument("--d", type=int, default=200, help="custom: variables")
    p.add_argument("--p1", type=int, default=3, help="custom: Das-Dennis divisions")
    p.add_argument("--p2", type=int, default=2, help="custom: inner-layer divisions (0: one layer)")
    p.add_argument("--sweep-m", type=str, default=None,
                   help="sweep / popsweep: comma-separated subset of m (or of N)")
    p.add_argument("--requests", type=int, default=None, help="served: requests of the stream")
    p.add_argument("--served-prefix", type=int, default=100,
                   help="headline: requests of the served stream in the served record")
    p.add_argument("--no-batched", action="store_true", help="headline: skip the batched record")
    p.add_argument("--no-served", action="store_true", help="headline: skip the served record")
    p.add_argument("--cpu-budget", type=float, default=20.0,
                   help="seconds of oracle work for the cpu_baseline sample (at least one generation)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--streaming", action="store_true",
                   help="no dominance matrix: the peel recomputes dominance (required for huge)")
    return p.parse_args(argv)


# ------------------------------------------------------------ distributed --
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def reduce_max(dist, x, device="cpu"):
    """Max of a float over ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(dist, world, units_per_rank, seconds, device="cpu"):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time.  Returns (rate, max seconds)."""
    t = reduce_max(dist, seconds, device)
    return world * units_per_rank / t, t


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return dict(PEAKS_FALLBACK), "fallback"


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` on `workload` from the committed ncu
    summary, or None when absent or taken on a different kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) != 4 or line.startswith("#"):
            continue
        k, wk, traffic, sha = parts
        if k != kernel or wk != workload:
            continue
        src = os.path.join(ROOT, "paper_2504_06067_gb300", "csrc", sha.split(":")[0])
        want = sha.split(":")[1]
        try:
            got = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            return None
        return float(traffic) if got == want else None
    return None


def ncu_issue_active(kernel):
    """smsp__issue_active of `kernel` from the committed full-set capture
    (profiles/issue.txt: kernel, workload of the capture, fraction, source
    hash), or None when absent or taken on a different kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "issue.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) != 4 or line.startswith("#") or parts[0] != kernel:
            continue
        src = os.path.join(ROOT, "paper_2504_06067_gb300", "csrc", parts[3].split(":")[0])
        try:
            got = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            return None
        if got == parts[3].split(":")[1]:
            return {"value": float(parts[2]), "capture": parts[1], "source": "profiles/issue.txt"}
    return None


# ------------------------------------------------------------- our impl ----
PHASE_NAMES = ["variation", "reset", "dominance", "peel", "niching", "gather", "total"]


def phase_breakdown(n, make_ctx, K, warmup, flush, stream):
    """Average device time (ms) of each phase over K generations from
    generation 0, L2 flushed before each, of a context whose graphs carry an
    event around every phase (phase_timing 2).  A pass of its own, outside
    the timed region: those event nodes lengthen every generation."""
    sh = stream.cuda_stream
    ctx = make_ctx(2)
    phases = (C.c_float * 7)()
    tot = [0.0] * 7
    try:
        def ok(st):
            return n.check(st, ctx)

        ok(n.nsga3_init(ctx, sh))
        for _ in range(warmup):
            ok(n.nsga3_step(ctx, sh))
        ok(n.nsga3_init(ctx, sh))
        ok(n.nsga3_sync(ctx, sh))
        for _ in range(K):
            flush.zero_()
            ok(n.nsga3_step(ctx, sh))
            ok(n.nsga3_phase_times(ctx, phases, 7))  # waits for the generation
            for t in range(7):
                tot[t] += phases[t]
        st = n.nsga3_sync(ctx, sh)
        if st != n.OK:
            raise RuntimeError("device status %d in the phase pass" % st)
    finally:
        n.nsga3_destroy(ctx)
    return {nm: round(tot[i] / K, 5) for i, nm in enumerate(PHASE_NAMES)}


def plain_measure(n, torch, cfg, K, warmup, stream, flush, seed, events, e2e_steps, dist, world,
                  kp=None, streaming=0):
    """Times K generations of one plain run of `cfg` from generation 0 (after
    `warmup` generations on the same context, re-initialised), L2 flushed
    before each, CUDA events on the launching stream around each step.  The
    timed graph carries events around the dominance build and the peel when
    `events` is 1 (none when 0).  Then `e2e_steps` generations through the C
    ABI with the parents uploaded from and the next population read back to
    pinned host memory inside the timed region.  Returns a dict; the phase
    breakdown is a separate pass (phase_breakdown)."""
    W = wl.objective_weights(cfg.m, cfg.seed)

    def make_ctx(level):
        if kp is not None:
            opts = n.default_opts(seed=seed, problem=1, kp_profit=kp[0].ctypes.data,
                                  kp_weight=kp[1].ctypes.data, kp_capacity=kp[2].ctypes.data,
                                  streaming=streaming, phase_timing=level)
        else:
            opts = n.default_opts(seed=seed, p2=cfg.p2, tau=cfg.tau, W=W.ctypes.data,
                                  streaming=streaming, phase_timing=level)
        return n.create(cfg.m, cfg.d, cfg.N, cfg.p1, opts)

    ctx = make_ctx(events)
    sh = stream.cuda_stream
    info = (C.c_int32 * 13)()
    phases = (C.c_float * 7)()
    launches = C.c_int32()

    def ok(st):
        return n.check(st, ctx)

    try:
        ok(n.nsga3_init(ctx, sh))
        for _ in range(warmup):
            ok(n.nsga3_step(ctx, sh))
        ok(n.nsga3_sync(ctx, sh))
        ok(n.nsga3_init(ctx, sh))
        ok(n.nsga3_sync(ctx, sh))
        dom_ms = peel_ms = 0.0
        peel_rows = passes = niche_steps = n_launch = 0
        dstat = (C.c_int64 * 8)()
        dsum = [0] * 8
        step_ms = []
        barrier(dist)
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ok(n.nsga3_step(ctx, sh))
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if events:
                ok(n.nsga3_phase_times(ctx, phases, 7))
                dom_ms += phases[2]
                peel_ms += phases[3]
            ok(n.nsga3_get_selection_info(ctx, info))
            ok(n.nsga3_last_launches(ctx, C.byref(launches)))
            ok(n.nsga3_get_dominance_stats(ctx, dstat))
            for t in range(8):
                dsum[t] += dstat[t]
            passes += info[6]
            peel_rows += info[12]
            n_launch += launches.value
            if info[4]:
                niche_steps += 1
        torch.cuda.synchronize()
        barrier(dist)
        st = n.nsga3_sync(ctx, sh)
        if st != n.OK:
            raise RuntimeError("device status %d after the timed run of %s" % (st, cfg.name))
        total_s = sum(step_ms) / 1e3
        value, total_s_max = job_rate(dist, world, cfg.N * K, total_s, "cuda")
        out = {"value": value, "gens_per_s": world * K / total_s_max, "ms_per_step": total_s_max * 1e3 / K,
               "steps": K, "peel_passes_per_step": passes / K, "peel_rows": peel_rows,
               "niching_steps": niche_steps, "gpu_launches": n_launch,
               "domstat": [x / K for x in dsum] if cfg.m <= 10 else None,
               "timed_events": "dominance build and peel" if events else "none"}
        if events:
            out["timed_region_ms"] = {"dominance": dom_ms / K, "peel": peel_ms / K}
        if e2e_steps:
            Xh = torch.empty((cfg.N, cfg.d), dtype=torch.float32).pin_memory()
            Fh = torch.empty((cfg.N, cfg.m), dtype=torch.float32).pin_memory()
            Rh = torch.empty(cfg.N, dtype=torch.int32).pin_memory()
            ok(n.nsga3_init(ctx, sh))
            ok(n.nsga3_get_population(ctx, Xh.data_ptr(), Fh.data_ptr(), Rh.data_ptr(), sh))
            ok(n.nsga3_sync(ctx, sh))
            e2e_ms = []
            Ke = min(K, e2e_steps)
            for k in range(Ke):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ok(n.nsga3_set_population(ctx, Xh.data_ptr(), Fh.data_ptr(), Rh.data_ptr(), sh))
                ok(n.nsga3_step(ctx, sh))
                ok(n.nsga3_get_population(ctx, Xh.data_ptr(), Fh.data_ptr(), Rh.data_ptr(), sh))
                e1.record(stream)
                e1.synchronize()
                e2e_ms.append(e0.elapsed_time(e1))
            ok(n.nsga3_sync(ctx, sh))
            e_s = reduce_max(dist, sum(e2e_ms) / 1e3, "cuda")
            per_step = cfg.N * (cfg.d + cfg.m + 1) * 4
            out["e2e"] = {"value": world * cfg.N * Ke / e_s, "unit": "sols/s", "h2d_bytes_per_step": per_step,
                          "d2h_bytes_per_step": per_step, "steps": Ke, "gens_per_s": world * Ke / e_s}
    finally:
        n.nsga3_destroy(ctx)
    return out, make_ctx


def issue_probe(n, torch, stream):
    """The measured issue ceiling of the dominance test's FADD / LOP3 mix
    (nsga3_issue_probe), with the SM clock sampled while it runs."""
    scratch = torch.rand(64, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    rate, ms = n.issue_probe(scratch.data_ptr(), blocks_per_sm=8, iters=400000, reps=5,
                             stream=stream.cuda_stream)
    clocks = sampler.stop()
    return {"instr_per_s": rate, "unit": "thread-instructions/s", "best_launch_ms": ms,
            "mix": "2 FP32 subtractions + 1 three-input LOP3 per step, 8 chains per thread, "
                   "8 CTAs of 256 threads per SM, no memory traffic; fastest of 5 launches",
            "clocks": clocks,
            "per_sm_per_clock": (rate / NUM_SMS / (clocks["sm_mhz"] * 1e6)) if clocks.get("sm_mhz") else None}


def roofline_of(cfg, avg_ms, peel_rows_per_step, probe, peaks, peak_kind, domstat=None):
    """Roofline of the dominant kernel (the dominance build, bound by issue,
    or the peel, bound by memory) from its average launch time.  The
    dominance build (m <= 10) tests only the pairs that its block boxes and
    its per-entry row and column tests cannot rule out: the units one launch
    processes are the (lane, column) pairs it tests (2m compares each, as
    for every pair), counted by the kernel (nsga3_get_dominance_stats); the
    rate over all n2(n2-1)/2 pairs is reported beside it."""
    n2 = 2 * cfg.N
    pairs = n2 * (n2 - 1) / 2
    if avg_ms["dominance"] >= avg_ms["peel"]:
        all_ops = pairs * 2 * cfg.m  # FP32 compares: all(f_i <= f_j) and all(f_j <= f_i)
        tested = None
        if domstat is not None and sum(domstat[:5]) > 0:
            tested = min(pairs, float(domstat[6]))
        ops = (tested if tested is not None else pairs) * 2 * cfg.m
        sec = avg_ms["dominance"] / 1e3
        achieved = ops / sec / 1e12
        if probe is not None:
            peak = probe["instr_per_s"] / 1e12
            src = "measured: nsga3_issue_probe (the FADD / LOP3 mix of the test, all SMs, no memory)"
        else:
            clk = peaks.get("sm_max_mhz", 2070.0) * 1e6
            peak = NUM_SMS * LANES_PER_SM * clk / 1e12
            src = "152 SMs x 128 lanes x %.0f MHz (max SM clock, %s)" % (clk / 1e6, peak_kind)
        roof = {"kernel": "k_dominance<%d>" % cfg.m if cfg.m <= 10 else "k_dominance_gen", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "T/s (compares; issue slots)",
                "frac": achieved / peak, "peak_source": src,
                "algorithmic": ("tested pairs x 2m FP32 compares per launch (%.4g; the (lane, column) "
                                "pairs the kernel tests, counted by it)" % ops) if tested is not None else
                               "n2(n2-1)/2 pairs x 2m FP32 compares per launch (%.4g)" % ops,
                "launch_ms": avg_ms["dominance"],
                "traffic": ncu_traffic("k_dominance", cfg.name)}
        if tested is not None:
            tot = float(sum(domstat[:5]))
            roof["pairs_tested_frac"] = tested / pairs
            roof["block_pair_pairs_frac"] = min(pairs, 1024.0 * sum(domstat[1:5])) / pairs
            roof["live_pairs_frac"] = float(domstat[7]) / pairs
            roof["block_pairs"] = {"zero": domstat[0] / tot, "one_direction_f0": domstat[1] / tot,
                                   "row_dom_col": domstat[2] / tot, "col_dom_row": domstat[3] / tot,
                                   "both": domstat[4] / tot, "tiles_skipped": int(domstat[5])}
            roof["all_pairs_compare_rate"] = all_ops / sec / 1e12
            roof["issue_active_ncu"] = ncu_issue_active("k_dominance")
            roof["dense_matrix_gbs"] = (n2 * n2 / 8 + n2 * cfg.m * 4) / sec / 1e9
        return roof
    bytes_read = peel_rows_per_step * 128 * 4.0  # row segments of 128 columns
    achieved = bytes_read / (avg_ms["peel"] / 1e3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"kernel": "k_peel (all passes of one selection)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": "hbm_gbs (%s)" % peak_kind,
            "algorithmic": "dominator row segments read (128 columns x 4 B each), all passes",
            "launch_ms": avg_ms["peel"], "traffic": ncu_traffic("k_peel", cfg.name)}


def plain_record(n, torch, cfg, K, args, stream, flush, seed, events, dist, world, probe, kp=None,
                 streaming=0, phases=True):
    """plain_measure + the phase pass + the roofline, as one record."""
    res, make_ctx = plain_measure(n, torch, cfg, K, args.warmup, stream, flush, seed, events,
                                  0 if args.no_e2e else 200, dist, world, kp=kp, streaming=streaming)
    breakdown = phase_breakdown(n, make_ctx, K, args.warmup, flush, stream) if phases else None
    peaks, peak_kind = measured_peaks()
    avg = res.get("timed_region_ms") or {"dominance": breakdown["dominance"], "peel": breakdown["peel"]}
    src = "CUDA events inside the timed graph" if "timed_region_ms" in res else \
        "the phase pass (events around every phase)"
    roof = roofline_of(cfg, avg, res["peel_rows"] / K, probe, peaks, peak_kind, res.get("domstat"))
    roof["launch_ms_source"] = src
    res["phase_ms"] = breakdown
    res["roofline"] = roof
    return res


def cfg_dict(cfg, streaming=0):
    return {"workload": cfg.name + ("_streaming" if streaming else ""), "m": cfg.m, "N": cfg.N,
            "d": cfg.d, "refs": cfg.w}


def run_ours(args, world, rank, local):
    """A single plain workload (--workload small|scale|large|huge|knapsack)."""
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n

    if args.workload == "custom":
        cfg = wl.RunConfig("custom_m%d_N%d_d%d_p%d%s" % (args.m, args.N, args.d, args.p1,
                                                         "+%d" % args.p2 if args.p2 else ""),
                           m=args.m, d=args.d, N=args.N, p1=args.p1, p2=args.p2, tau=0.5,
                           generations=args.steps)
    else:
        cfg = WORKLOADS[args.workload]
    seed = cfg.seed + rank
    streaming = 1 if (args.streaming or args.workload == "huge") else 0
    kp = wl.knapsack_instance(cfg.m, cfg.d, cfg.seed) if args.workload == "knapsack" else None
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    probe = issue_probe(n, torch, stream)
    K = args.steps
    sampler = ClockSampler(local)
    sampler.start()
    res = plain_record(n, torch, cfg, K, args, stream, flush, seed, 1, dist, world, probe, kp=kp,
                       streaming=streaming)
    clocks = sampler.stop()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    line = {
        "metric": METRIC,
        "value": res["value"],
        "unit": "sols/s",
        "gens_per_s": res["gens_per_s"],
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": res["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": ("synthetic 0-1 knapsack instance (profits, weights U[10, 100], capacity half the "
                 "weight; stands in for MOKnapsack)" if args.workload == "knapsack" else
                 "synthetic (seeded softmax-simplex objective, W ~ N(0,1); stands in for DTLZ)"),
        "config": dict(cfg_dict(cfg, streaming), generations="timed %d from generation 0" % K,
                       l2="flushed (256 MB write) before every timed step",
                       timing="events around the dominance build and the peel inside the timed "
                              "graph; phase_ms from a second pass with an event around every phase",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "phase_ms": res["phase_ms"],
        "timed_region_ms": res.get("timed_region_ms"),
        "peel_passes_per_step": res["peel_passes_per_step"],
        "niching_steps": res["niching_steps"],
        "roofline": res["roofline"],
        "issue_probe": probe,
        "e2e": res.get("e2e"),
        "gpu_launches": res["gpu_launches"],
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1 and args.workload != "custom":
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_budget)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_headline(args, world, rank, local):
    """The default line: m = 10, N = 100,000 (the largest single-GPU
    configuration) as the headline, with the m = 5, N = 10,628 run, the 64
    batched runs, a prefix of the served request stream, the issue probe and
    the oracle on the host cores as sub-records."""
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    progress("issue probe")
    probe = issue_probe(n, torch, stream)
    cfg = wl.LARGE
    K = args.steps
    progress("headline %s: %d generations" % (cfg.name, K))
    sampler = ClockSampler(local)
    sampler.start()
    # events around the dominance build and the peel in the timed graph: about
    # 15 us of a 13.6 ms generation, and they time the dominant kernel live
    head = plain_record(n, torch, cfg, K, args, stream, flush, cfg.seed + rank, 1, dist, world, probe)
    clocks = sampler.stop()
    progress("secondary %s" % wl.SCALE.name)
    sec_cfg = wl.SCALE
    sec = plain_record(n, torch, sec_cfg, sec_cfg.generations, args, stream, flush, sec_cfg.seed + rank, 0,
                       dist, world, probe)
    sec_line = {"value": sec["value"], "unit": "sols/s", "gens_per_s": sec["gens_per_s"],
                "ms_per_step": sec["ms_per_step"], "steps": sec["steps"],
                "config": dict(cfg_dict(sec_cfg), l2="flushed (256 MB write) before every timed step",
                               timing="no event nodes in the timed graph; phase_ms and the roofline's "
                                      "launch time from a second pass with an event around every phase"),
                "phase_ms": sec["phase_ms"], "roofline": sec["roofline"], "e2e": sec.get("e2e"),
                "peel_passes_per_step": sec["peel_passes_per_step"], "gpu_launches": sec["gpu_launches"]}
    del flush
    torch.cuda.empty_cache()
    batched = None
    if not args.no_batched:
        progress("batched")
        batched = batched_core(n, torch, stream, args.runs, 300, max(args.warmup, 1), dist, world, rank)
    served = None
    if not args.no_served:
        progress("served")
        served = served_core(n, torch, args.served_prefix, dist, world, rank)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "sols/s",
        "gens_per_s": head["gens_per_s"],
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded softmax-simplex objective, W ~ N(0,1); stands in for DTLZ)",
        "config": dict(cfg_dict(cfg), generations="timed %d from generation 0" % K,
                       l2="flushed (256 MB write) before every timed step",
                       timing="events around the dominance build and the peel inside the timed "
                              "graph; phase_ms from a second pass with an event around every phase",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "phase_ms": head["phase_ms"],
        "timed_region_ms": head.get("timed_region_ms"),
        "peel_passes_per_step": head["peel_passes_per_step"],
        "niching_steps": head["niching_steps"],
        "roofline": head["roofline"],
        "issue_probe": probe,
        "e2e": head.get("e2e"),
        "gpu_launches": head["gpu_launches"],
        "clocks": clocks,
        "secondary": sec_line,
        "batched": batched,
        "served": served,
    }
    if not args.no_cpu_baseline and world == 1:
        progress("cpu baseline")
        line["cpu_baseline"] = cpu_baseline(cfg, args.cpu_budget)
        line["secondary"]["cpu_baseline"] = cpu_baseline(sec_cfg, args.cpu_budget)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


# ---------------------------------------------------------------- batched ----
def batched_core(n, torch, stream, n_runs, gens, warmup, dist, world, rank):
    """64 uneven independent runs (N log-uniform in [100, 20000], m in
    {3, 5, 8}, d = m + 19): one batched CUDA graph per generation against the
    plain path (each run alone, one graph launch per generation, runs one
    after another).  Both arms time initialisation + `gens` generations of
    all runs, and the read-back of every final population (e2e); the same
    runs then go through the run server (one stream per run).  Returns the
    record (rank 0) or None."""
    cfgs = wl.batched_configs(n_runs=n_runs, seed=0, generations=gens)
    Ws = [wl.objective_weights(c.m, c.seed) for c in cfgs]
    ctxs = []
    progress("creating %d contexts" % len(cfgs))
    for c, W in zip(cfgs, Ws):
        o = n.default_opts(seed=c.seed + 1000003 * rank, W=W.ctypes.data)
        ctxs.append(n.create(c.m, c.d, c.N, c.p1, o))
    sh = stream.cuda_stream
    hosts = [(torch.empty((c.N, c.d), dtype=torch.float32).pin_memory(),
              torch.empty((c.N, c.m), dtype=torch.float32).pin_memory(),
              torch.empty(c.N, dtype=torch.int32).pin_memory()) for c in cfgs]

    def launches():
        tot = C.c_int64()
        s = 0
        for x in ctxs:
            n.check(n.nsga3_total_launches(x, C.byref(tot)), x)
            s += tot.value
        return s

    run_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in ctxs]

    def plain():
        for x, (a, b) in zip(ctxs, run_ev):
            a.record(stream)
            n.check(n.nsga3_init(x, sh), x)
            n.check(n.nsga3_run(x, gens, sh), x)
            b.record(stream)

    def batched():
        for x in ctxs:
            n.check(n.nsga3_init(x, sh), x)
        n.check(n.run_batch(ctxs, gens, sh), ctxs[0])

    def read_back():
        for x, (X, F, R) in zip(ctxs, hosts):
            n.check(n.nsga3_get_population(x, X.data_ptr(), F.data_ptr(), R.data_ptr(), sh), x)

    try:
        # warm-up: build every graph (the batched one included)
        progress("warm-up")
        for x in ctxs:
            n.check(n.nsga3_init(x, sh), x)
        n.check(n.run_batch(ctxs, warmup, sh), ctxs[0])
        for x in ctxs:
            n.check(n.nsga3_run(x, warmup, sh), x)
        torch.cuda.synchronize()
        res = {}
        for arm, fn in (("plain", plain), ("batched", batched)):
            progress("%s arm" % arm)
            barrier(dist)
            torch.cuda.synchronize()
            l0 = launches()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            w0 = time.perf_counter()
            e0.record(stream)
            fn()
            e1.record(stream)
            read_back()
            e2.record(stream)
            e2.synchronize()
            wall = time.perf_counter() - w0
            res[arm] = {"s": reduce_max(dist, e0.elapsed_time(e1) / 1e3, "cuda"),
                        "e2e_s": reduce_max(dist, e0.elapsed_time(e2) / 1e3, "cuda"),
                        "wall_s": wall, "launches": launches() - l0,
                        "pop": [tuple(t.clone() for t in h) for h in hosts]}
            for x in ctxs:
                st = n.nsga3_sync(x, sh)
                if st != n.OK:
                    raise RuntimeError("device status %d in the %s arm" % (st, arm))
    finally:
        for x in ctxs:
            n.nsga3_destroy(x)
    # the same runs through the run server: every run on its own stream,
    # no per-generation join between runs
    torch.cuda.synchronize()
    progress("server arm")
    reqs = [(0.0, c) for c in cfgs]
    budget = int(min(0.7 * torch.cuda.mem_get_info()[0], 160e9))
    w0 = time.perf_counter()
    sinf, _ = _serve(n, reqs, budget, len(cfgs), 8)
    server_s = time.perf_counter() - w0
    server_span = max(i.t_done for i in sinf.values()) - min(i.t_submit for i in sinf.values())
    same = all(all(torch.equal(a, b) for a, b in zip(p, q))
               for p, q in zip(res["plain"]["pop"], res["batched"]["pop"]))
    # each run's device time alone (plain arm): how the batched time compares
    # with the largest run (a lower bound) and with the sum of all runs
    solo = [a.elapsed_time(b) / 1e3 for a, b in run_ev]
    big = [t for t, c in zip(solo, cfgs) if c.N >= 3000]
    if rank != 0:
        return None
    R = len(cfgs)
    b, p = res["batched"], res["plain"]
    dom_bytes = sum((2 * c.N) ** 2 / 8 for c in cfgs)
    return {
        "value": world * R / b["s"],
        "unit": "runs/s",
        "steps": gens,
        "warmup": warmup,
        "ms_per_step": b["s"] * 1e3 / gens,
        "config": {"workload": "batched_%druns_%dgens" % (R, gens), "runs": R,
                   "N": [c.N for c in cfgs], "m": [c.m for c in cfgs],
                   "d": "m + 19", "seeds": "0..%d" % (R - 1),
                   "l2": "not flushed: the runs' bit matrices alone hold %.2f GB, above the "
                         "129 MB L2" % (dom_bytes / 1e9)},
        "plain": {"value": world * R / p["s"], "unit": "runs/s", "ms": p["s"] * 1e3,
                  "gpu_launches": p["launches"]},
        "batched_vs_plain": p["s"] / b["s"],
        "plain_solo_s": {"largest_run": max(solo), "runs_N_ge_3000": sum(big), "runs_N_lt_3000": sum(solo) - sum(big),
                         "largest5": sorted((round(t, 4) for t in solo), reverse=True)[:5]},
        "server_streams": {"value": world * R / server_span, "unit": "runs/s", "wall_s": server_s,
                           "note": "the same runs submitted at once to the run server (one stream "
                                   "per run, 8 generations per launch batch, no join per generation)"},
        "identical_populations": bool(same),
        "gens_per_s": world * R * gens / b["s"],
        "sols_per_s": world * sum(c.N for c in cfgs) * gens / b["s"],
        "e2e": {"value": world * R / b["e2e_s"], "unit": "runs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": sum(c.N * (c.d + c.m + 1) * 4 for c in cfgs) / gens,
                "note": "inputs are (m, d, N, seed, W) set at creation; the final populations "
                        "are read back into pinned host memory inside the timed region"},
        "gpu_launches": b["launches"],
    }


def run_batched(args, world, rank, local):
    """--workload batched: the batched record as its own line."""
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n

    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    rec = batched_core(n, torch, stream, args.runs, args.steps, max(args.warmup, 1), dist, world, rank)
    clocks = sampler.stop()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded softmax-simplex objectives)"}
    line.update(rec)
    line["config"]["parallelism"] = "replicas" if world > 1 else "single GPU"
    line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def _serve(n, reqs, budget, max_active, gens_per_launch):
    """Replays a request stream against one server: requests are submitted
    at their arrival times (relative to the first), results fetched as they
    complete.  Returns per-request infos and the server statistics."""
    import threading
    srv = n.Server(budget, max_active=max_active, gens_per_launch=gens_per_launch)
    infos = {}
    errors = []

    def producer():
        t0 = time.perf_counter()
        for t, c in reqs:
            dt = t - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            try:
                srv.submit(c.m, c.d, c.N, c.p1, c.generations, wl.objective_weights(c.m, c.seed),
                           seed=c.seed, p2=c.p2)
            except Exception as e:  # noqa: BLE001 - reported below
                errors.append(repr(e))

    th = threading.Thread(target=producer)
    th.start()
    progress("serving %d requests (%d slots)" % (len(reqs), max_active))
    while len(infos) < len(reqs) and not errors:
        rid = srv.wait(1000)
        if rid < 0:
            continue
        st, info = srv.fetch(rid)
        infos[rid] = info
        if len(infos) % 50 == 0:
            progress("%d / %d runs done" % (len(infos), len(reqs)))
    th.join()
    stats = srv.stats()
    srv.close()
    if errors:
        raise RuntimeError(errors[0])
    bad = [i for i in infos.values() if i.status != n.OK]
    if bad:
        raise RuntimeError("run failed: status %d %s" % (bad[0].status, bad[0].message.decode()))
    return infos, stats


def _latency_summary(infos, reqs):
    import numpy as np
    lat = np.array([i.t_done - i.t_submit for i in infos.values()])
    t_first = min(i.t_submit for i in infos.values())
    t_last = max(i.t_done for i in infos.values())
    work = sum(c.N * c.generations for _, c in reqs)
    return {"runs_per_s": len(infos) / (t_last - t_first), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "makespan_s": t_last - t_first,
            "sols_per_s": work / (t_last - t_first), "requests": len(infos)}


def served_core(n, torch, n_req, dist, world, rank, n_plain=None):
    """A Poisson stream of run requests (40 per second; N log-uniform in
    [100, 50000], m in 3..10, 50..1000 generations, d = m + 29): its first
    `n_req` requests served by the continuous-batching server (64 slots, 8
    generations per launch batch), against the plain path on the first
    `n_plain` (default all) requests (the same server with one slot: one run
    at a time, in arrival order).  Latency = completion - arrival on the
    server clock; runs/s = requests / (last completion - first arrival).
    Returns the record (rank 0) or None."""
    reqs_all = wl.served_requests(n_req=n_req, rate_hz=40.0, seed=rank)
    n_plain = n_req if n_plain is None else min(n_plain, n_req)
    free, total = torch.cuda.mem_get_info()
    budget = int(min(0.7 * free, 160e9))
    # warm-up: one small run through each kind of server
    warm = [(0.0, wl.RunConfig("w", m=3, d=32, N=100, p1=12, generations=5, seed=0))]
    _serve(n, warm, budget // 8, 2, 8)
    barrier(dist)
    plain_inf, _ = _serve(n, reqs_all[:n_plain], budget, 1, 8)
    served_small = None
    if n_plain < n_req:
        served_small, _ = _serve(n, reqs_all[:n_plain], budget, 64, 8)
    served_inf, served_stats = _serve(n, reqs_all, budget, 64, 8)
    if served_small is None:
        served_small = served_inf
    barrier(dist)
    plain = _latency_summary(plain_inf, reqs_all[:n_plain])
    # each run's time alone (one slot: admitted when the previous run left)
    solo = sorted((i.t_done - i.t_admit for i in plain_inf.values()), reverse=True)
    arrive = {rid: t for rid, (t, _) in enumerate(reqs_all[:n_plain])}
    bound = max(arrive[rid] + (i.t_done - i.t_admit) for rid, i in plain_inf.items())
    plain["solo_s_total"] = sum(solo)
    plain["solo_s_largest10"] = [round(x, 3) for x in solo[:10]]
    plain["largest10_work_share"] = sum(solo[:10]) / sum(solo)
    plain["makespan_lower_bound_s"] = bound
    same = _latency_summary(served_small, reqs_all[:n_plain])
    full = _latency_summary(served_inf, reqs_all)
    makespan = reduce_max(dist, full["makespan_s"], "cuda")
    if rank != 0:
        return None
    rec = {
        "value": world * full["requests"] / makespan,
        "unit": "runs/s",
        "steps": full["requests"],
        "config": {"workload": "served_%dreq_40hz" % n_req, "requests": n_req, "rate_hz": 40.0,
                   "stream": "the first %d requests of the seeded 2,000-request stream" % n_req,
                   "N": "log-uniform [100, 50000]", "m": "3..10", "generations": "50..1000",
                   "d": "m + 29", "slots": 64, "gens_per_launch": 8, "budget_bytes": budget,
                   "l2": "not flushed: concurrent runs' working sets exceed the 129 MB L2"},
        "served": full,
        "plain": plain,
        "served_vs_plain_runs_per_s": same["runs_per_s"] / plain["runs_per_s"],
        "p50_s": full["p50_s"],
        "p99_s": full["p99_s"],
        "plain_p50_s": plain["p50_s"],
        "plain_p99_s": plain["p99_s"],
        "peak_active": served_stats["peak_active"],
        "peak_bytes": served_stats["peak_bytes"],
        "e2e": {"value": world * full["requests"] / makespan, "unit": "runs/s",
                "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": sum(c.N * (c.d + c.m + 1) * 4 for _, c in reqs_all) / n_req,
                "note": "the server API is host-to-host: requests in, final populations out in host "
                        "memory; value and e2e are the same measurement"},
        "gpu_launches": served_stats["launches"],
    }
    if n_plain < n_req:
        rec["served_first_%d" % n_plain] = same
    return rec


def run_served(args, world, rank, local):
    """--workload served: the served record as its own line (plain path on
    the first 100 requests)."""
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n

    n_req = args.requests or 400
    sampler = ClockSampler(local)
    sampler.start()
    rec = served_core(n, torch, n_req, dist, world, rank, n_plain=100)
    clocks = sampler.stop()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    line = {"metric": METRIC, "n_gpus": world, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded softmax-simplex objectives, Poisson arrivals)"}
    line.update(rec)
    line["ms_per_step"] = 1e3 / rec["value"]
    line["config"]["parallelism"] = "replicas" if world > 1 else "single GPU"
    line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


# ------------------------------------------------------ objective sweep ----
# TensorNSGA-III's seconds per generation in the paper's Table II (DTLZ3,
# N = 800, d = 1000, 100 generations, on the paper's GPU): context only.
PAPER_TABLE2_S = {4: 4.334e-3, 8: 4.624e-3, 16: 5.083e-3, 32: 6.514e-3, 64: 8.103e-3,
                  128: 1.016e-2, 256: 2.348e-2, 512: 3.199e-2}
# ... and in Table I (DTLZ3, m = 6, d = 500, population N)
PAPER_TABLE1_S = {50: 1.120e-3, 100: 1.135e-3, 200: 1.121e-3, 400: 1.243e-3, 800: 1.493e-3,
                  1600: 2.063e-3, 3200: 4.886e-3, 6400: 1.575e-2, 12800: 5.966e-2}


def run_sweep(args, world, rank, local):
    """Generations per second over m = 4 ... 512 at N = 800, d = 1000 (the
    shape of Table II; --workload sweep) or over N = 50 ... 12,800 at m = 6,
    d = 500 (Table I; --workload popsweep); each point is its own run:
    warm-up, then K timed generations from generation 0, L2 flushed before
    each."""
    import torch
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n

    K = args.steps
    sh = torch.cuda.current_stream().cuda_stream
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    launches = C.c_int32()
    rows = []
    n_launch = 0
    sampler = ClockSampler(local)
    sampler.start()
    pop = args.workload == "popsweep"
    cfgs = wl.population_sweep() if pop else wl.objective_sweep()
    only = None if not args.sweep_m else {int(x) for x in args.sweep_m.split(",")}
    for cfg in cfgs:
        if only is not None and (cfg.N if pop else cfg.m) not in only:
            continue
        progress("sweep m=%d N=%d" % (cfg.m, cfg.N))
        W = wl.objective_weights(cfg.m, cfg.seed)

        def make_ctx(level, cfg=cfg, W=W):
            return n.create(cfg.m, cfg.d, cfg.N, cfg.p1,
                            n.default_opts(seed=cfg.seed + rank, W=W.ctypes.data, phase_timing=level))

        ctx = make_ctx(0)

        def ok(st):
            return n.check(st, ctx)

        ok(n.nsga3_init(ctx, sh))
        for _ in range(args.warmup):
            ok(n.nsga3_step(ctx, sh))
        ok(n.nsga3_init(ctx, sh))
        ok(n.nsga3_sync(ctx, sh))
        barrier(dist)
        ms = []
        for k in range(K):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ok(n.nsga3_step(ctx, sh))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            ok(n.nsga3_last_launches(ctx, C.byref(launches)))
            n_launch += launches.value
        st = n.nsga3_sync(ctx, sh)
        n.nsga3_destroy(ctx)
        if st != n.OK:
            raise RuntimeError("device status %d (m = %d)" % (st, cfg.m))
        breakdown = phase_breakdown(n, make_ctx, K, args.warmup, flush, stream)
        s_max = reduce_max(dist, sum(ms) / 1e3, "cuda")
        row = {"m": cfg.m, "N": cfg.N, "refs": cfg.w, "ms_per_gen": s_max * 1e3 / K,
               "gens_per_s": world * K / s_max, "sols_per_s": world * K * cfg.N / s_max,
               "phase_ms": breakdown}
        if pop:
            row["paper_table1_ms"] = PAPER_TABLE1_S[cfg.N] * 1e3
        else:
            row["paper_table2_ms"] = PAPER_TABLE2_S[cfg.m] * 1e3
        rows.append(row)
    clocks = sampler.stop()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    top = rows[-1]
    line = {
        "metric": ("gens/s over the population sweep (Table I shape: m 6, d 500, N 50..12800)" if pop else
                   "gens/s over the objective sweep (Table II shape: N 800, d 1000, m 4..512)"),
        "value": top["gens_per_s"],
        "unit": ("gens/s at N = %d" % top["N"]) if pop else ("gens/s at m = %d" % top["m"]),
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": top["ms_per_gen"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded softmax-simplex objective, W ~ N(0,1); stands in for DTLZ3)",
        "config": {"workload": "popsweep_m6_d500_N50-12800" if pop else "sweep_N800_d1000_m4-512",
                   "l2": "flushed (256 MB write) before every timed step",
                   "generations": "timed %d from generation 0 per m" % K,
                   "timing": "no event nodes in the timed graphs; phase_ms from a second pass "
                             "per point with an event around every phase",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "sweep": rows,
        "roofline": None,
        "e2e": None,
        "gpu_launches": n_launch,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        cfg = cfgs[-1]
        import oracle
        spg, nst = oracle_generations(cfg, args.cpu_budget)
        line["cpu_baseline"] = {"value": 1.0 / spg, "unit": line["unit"], "cores": oracle.threads(),
                                "kind": "oracle",
                                "sample": "%d generation(s) of %s (FP64 C oracle, OpenMP on %d threads)"
                                          % (nst, cfg.name, oracle.threads())}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


# ----------------------------------------------------------------- oracle ----
def oracle_generations(cfg, budget_s, max_steps=None, warmup=0):
    """Times oracle generations of `cfg` from a seeded initial population until
    the budget is spent (at least one).  Returns (seconds per generation, n)."""
    import numpy as np

    import oracle
    oracle.build()
    if cfg is wl.KNAPSACK:
        kp = wl.knapsack_instance(cfg.m, cfg.d, cfg.seed)
        order = oracle.kp_order(kp[0], kp[1])
        Z = oracle.refdirs(cfg.m, cfg.p1)
        X, F = oracle.kp_eval(oracle.kp_init(cfg.N, cfg.d, cfg.seed), *kp)
        rank = np.zeros(cfg.N, np.int32)
        times = []
        t_start = time.perf_counter()
        g = 0
        while True:
            t0 = time.perf_counter()
            X, F, rank = oracle.kp_generation(X, F, rank, *kp, order, Z, cfg.seed, g)
            times.append(time.perf_counter() - t0)
            g += 1
            if (max_steps is not None and len(times) >= max_steps) or time.perf_counter() - t_start >= budget_s:
                break
        return sum(times) / len(times), len(times)
    W = wl.objective_weights(cfg.m, cfg.seed)
    Z = oracle.refdirs(cfg.m, cfg.p1, cfg.p2, cfg.tau)
    X = oracle.init_population(cfg.N, cfg.d, cfg.seed)
    F = oracle.evaluate(X, W)
    rank = np.zeros(cfg.N, np.int32)
    g = 0
    for _ in range(warmup):
        X, F, rank = oracle.generation(X, F, rank, W, Z, cfg.seed, g)
        g += 1
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        X, F, rank = oracle.generation(X, F, rank, W, Z, cfg.seed, g)
        times.append(time.perf_counter() - t0)
        g += 1
        if max_steps is not None and len(times) >= max_steps:
            break
        if time.perf_counter() - t_start >= budget_s:
            break
    return sum(times) / len(times), len(times)


def cpu_baseline(cfg, budget_s):
    import oracle
    spg, n = oracle_generations(cfg, budget_s)
    return {"value": cfg.N / spg, "unit": "sols/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d generation(s) of %s from generation 0 (FP64 C oracle; OpenMP over the "
                      "sort's and the association's independent loops on %d threads, %d host "
                      "cores on the box)" % (n, cfg.name, oracle.threads(), os.cpu_count() or 0)}


def reference_cfg(args):
    if args.workload in ("sweep", "popsweep"):
        return {"sweep": wl.objective_sweep, "popsweep": wl.population_sweep}[args.workload]()[-1]
    if args.workload in ("headline", "select"):
        return wl.LARGE
    if args.workload in ("batched", "served"):
        return wl.SCALE
    return WORKLOADS[args.workload]


def run_reference(args, world, rank):
    """The oracle as the reference arm, on this workload's metric: whole
    generations from generation 0 of the same seeded run, as many of the
    requested steps as a 150 s budget allows (at least one)."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    cfg = reference_cfg(args)
    budget = 150.0
    spg, nsteps = oracle_generations(cfg, budget, max_steps=args.steps, warmup=0)
    value = cfg.N / spg
    cores = oracle.threads()
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "sols/s",
        "gens_per_s": 1.0 / spg,
        "n_gpus": world,
        "steps": nsteps,
        "warmup": 0,
        "ms_per_step": spg * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded softmax-simplex objective, W ~ N(0,1); stands in for DTLZ)",
        "config": dict(cfg_dict(cfg), generations="timed %d from generation 0" % args.steps,
                       l2="flushed (256 MB write) before every timed step",
                       timing="events around the dominance build and the peel inside the timed "
                              "graph; phase_ms from a second pass with an event around every phase",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "reference_steps": "%d generation(s) from generation 0 of the requested %d (150 s budget); "
                           "the oracle keeps no state between runs, so no warm-up generation" %
                           (nsteps, args.steps),
        "cpu_baseline": {"value": value, "unit": "sols/s", "cores": cores, "kind": "oracle",
                         "sample": "%d generation(s) of %s from generation 0 (FP64 C oracle, OpenMP "
                                   "on %d threads)" % (nsteps, cfg.name, cores)},
        "e2e": {"value": value, "unit": "sols/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


# ------------------------------------------------------ selection alone ----
SELECT_KINDS = ("equal", "dups", "chain", "simplex")


def run_shapes(args, world, rank, local):
    """Launch-shape sweep (--workload shapes): for (m, 2N) buckets of the
    configurations' shapes, every persistent-CTA count of the dominance
    build and of the cooperative peel (nsga3_opts.dom_ctas_per_sm,
    peel_ctas_per_sm), each its own run from generation 0: warm-up, then K
    generations with events around the dominance build and the peel, L2
    flushed before each.  The final populations of every setting of a bucket
    must be identical (the shapes change no result); the fastest setting is
    reported beside the default (0: all resident)."""
    import hashlib
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_2504_06067_gb300 import native as n

    K = args.steps
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    phases = (C.c_float * 7)()
    buckets = [wl.RunConfig("shape_m3_N2000", m=3, d=22, N=2000, p1=wl.largest_p(3, 2000), generations=K),
               wl.SCALE,
               wl.RunConfig("shape_m8_N10000", m=8, d=27, N=10000, p1=wl.largest_p(8, 10000), generations=K),
               wl.RunConfig("shape_m10_N30000", m=10, d=200, N=30000, p1=3, p2=2, generations=K),
               wl.LARGE]
    sampler = ClockSampler(local)
    sampler.start()
    out = []
    for cfg in buckets:
        W = wl.objective_weights(cfg.m, cfg.seed)
        res = {}
        digests = set()
        dom_max = 5 if cfg.m <= 8 else 4
        settings = [(dc, 0) for dc in range(0, dom_max + 1)] + [(0, pc) for pc in (1, 2)]
        for dc, pc in settings:
            progress("shapes %s dom_ctas=%d peel_ctas=%d" % (cfg.name, dc, pc))
            opts = n.default_opts(seed=cfg.seed, p2=cfg.p2, tau=cfg.tau, W=W.ctypes.data, phase_timing=1,
                                  dom_ctas_per_sm=dc, peel_ctas_per_sm=pc)
            ctx = n.create(cfg.m, cfg.d, cfg.N, cfg.p1, opts)
            try:
                n.check(n.nsga3_init(ctx, sh), ctx)
                for _ in range(args.warmup):
                    n.check(n.nsga3_step(ctx, sh), ctx)
                n.check(n.nsga3_init(ctx, sh), ctx)
                dom = peel = step = 0.0
                for _ in range(K):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    n.check(n.nsga3_step(ctx, sh), ctx)
                    e1.record(stream)
                    e1.synchronize()
                    step += e0.elapsed_time(e1)
                    n.check(n.nsga3_phase_times(ctx, phases, 7), ctx)
                    dom += phases[2]
                    peel += phases[3]
                X = np.zeros((cfg.N, cfg.d), np.float32)
                F = np.zeros((cfg.N, cfg.m), np.float32)
                R = np.zeros(cfg.N, np.int32)
                n.check(n.nsga3_get_population(ctx, X.ctypes.data, F.ctypes.data, R.ctypes.data, sh), ctx)
                n.check(n.nsga3_sync(ctx, sh), ctx)
                digests.add(hashlib.sha256(X.tobytes() + F.tobytes() + R.tobytes()).hexdigest())
            finally:
                n.nsga3_destroy(ctx)
            res["dom%d_peel%d" % (dc, pc)] = {"dominance_ms": dom / K, "peel_ms": peel / K, "step_ms": step / K}
        best_dom = min((k for k in res if k.endswith("_peel0")), key=lambda k: res[k]["dominance_ms"])
        best_peel = min(("dom0_peel0", "dom0_peel1", "dom0_peel2"), key=lambda k: res[k]["peel_ms"])
        out.append({"workload": cfg.name, "m": cfg.m, "N": cfg.N, "settings": res,
                    "fastest_dominance": best_dom, "fastest_peel": best_peel,
                    "identical_populations": len(digests) == 1})
    clocks = sampler.stop()
    if rank == 0:
        print(json.dumps({"metric": "launch-shape sweep (dominance build and front peel CTAs per SM)",
                          "steps": K, "warmup": args.warmup, "buckets": out, "clocks": clocks,
                          "note": "dom0 / peel0 = the default (every CTA that fits at once); times are the "
                                  "phase events of generations 0..K-1, L2 flushed before each"}))


def run_select(args, world, rank, local):
    """Selection microbenchmark: nsga3_select alone (selected sols/s = N /
    the time of one selection, objectives already on the device) on merged
    objective matrices saved from the plain runs of m3_N92, m5_N10628 and
    m10_N100000 at generations 0, mid and last, and on adversarial sets
    (all equal, many duplicates, a chain of one point per front, a single
    simplex front) of the m5_N10628 and m10_N100000 shapes; beside it the
    oracle's selection of the same matrices on the host cores (where it
    fits the budget), which must select the same indices."""
    import numpy as np
    import torch

    import oracle
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    from paper_2504_06067_gb300 import native as n
    oracle.build()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    K = args.steps
    rows = []
    n_launch = 0
    sampler = ClockSampler(local)
    sampler.start()
    cpu_left = args.cpu_budget * 6
    for cfg in (wl.SMALL, wl.SCALE, wl.LARGE):
        W = wl.objective_weights(cfg.m, cfg.seed)
        mats = []
        progress("select: saving %s objectives" % cfg.name)
        ctx = n.create(cfg.m, cfg.d, cfg.N, cfg.p1,
                       n.default_opts(seed=cfg.seed, p2=cfg.p2, tau=cfg.tau, W=W.ctypes.data))
        try:
            Fp = np.zeros((cfg.N, cfg.m), np.float32)
            Fc = np.zeros((cfg.N, cfg.m), np.float32)
            n.check(n.nsga3_init(ctx, sh), ctx)
            g = 0
            for want in (0, cfg.generations // 2, cfg.generations):
                n.check(n.nsga3_run(ctx, want - g, sh), ctx)
                g = want
                n.check(n.nsga3_get_population(ctx, None, Fp.ctypes.data, None, sh), ctx)
                n.check(n.nsga3_vary(ctx, sh), ctx)
                n.check(n.nsga3_get_children(ctx, None, Fc.ctypes.data, sh), ctx)
                n.check(n.nsga3_sync(ctx, sh), ctx)
                mats.append(("generation %d" % want, want, np.vstack([Fp, Fc]).copy()))
        finally:
            n.nsga3_destroy(ctx)
        if cfg is not wl.SMALL:
            for kind in SELECT_KINDS:
                mats.append((kind, 0, wl.objectives(kind, 2 * cfg.N, cfg.m, seed=cfg.seed)))
        Z = oracle.refdirs(cfg.m, cfg.p1, cfg.p2, cfg.tau)
        ctx = n.create(cfg.m, cfg.d, cfg.N, cfg.p1, n.default_opts(seed=cfg.seed, p2=cfg.p2, tau=cfg.tau))
        try:
            dF = torch.empty((2 * cfg.N, cfg.m), dtype=torch.float32, device="cuda")
            dr = torch.empty(2 * cfg.N, dtype=torch.int32, device="cuda")
            ds = torch.empty(cfg.N, dtype=torch.int32, device="cuda")
            info = (C.c_int32 * 13)()
            launches = C.c_int32()
            for label, gen, F in mats:
                progress("select: %s %s" % (cfg.name, label))
                dF.copy_(torch.from_numpy(F))
                for _ in range(3):
                    n.check(n.nsga3_set_counter(ctx, gen, sh), ctx)
                    n.check(n.nsga3_select(ctx, dF.data_ptr(), dr.data_ptr(), ds.data_ptr(), sh), ctx)
                n.check(n.nsga3_sync(ctx, sh), ctx)
                ms = []
                for _ in range(K):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    n.check(n.nsga3_select(ctx, dF.data_ptr(), dr.data_ptr(), ds.data_ptr(), sh), ctx)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                    n.check(n.nsga3_last_launches(ctx, C.byref(launches)), ctx)
                    n_launch += launches.value
                st = n.nsga3_sync(ctx, sh)
                if st != n.OK:
                    raise RuntimeError("device status %d (%s %s)" % (st, cfg.name, label))
                n.check(n.nsga3_get_selection_info(ctx, info), ctx)
                t = reduce_max(dist, statistics.median(ms) / 1e3, "cuda")
                row = {"workload": cfg.name, "objectives": label, "N": cfg.N, "m": cfg.m,
                       "ms": t * 1e3, "selected_sols_per_s": world * cfg.N / t,
                       "fronts_to_l": info[0] + 1, "niching": bool(info[4]), "peel_passes": info[6]}
                # the oracle beside it while the budget lasts (the m10 sort takes about a minute)
                if rank == 0 and world == 1 and (cpu_left > 0 or cfg is wl.SMALL):
                    t0 = time.perf_counter()
                    ref = oracle.select(F, cfg.N, Z, seed=cfg.seed, gen=gen)
                    ot = time.perf_counter() - t0
                    cpu_left -= ot
                    same = (np.array_equal(dr.cpu().numpy(), ref["rank"]) and
                            np.array_equal(ds.cpu().numpy(), ref["selected"]))
                    row["oracle"] = {"s": ot, "selected_sols_per_s": cfg.N / ot, "cores": oracle.threads(),
                                     "identical": bool(same)}
                rows.append(row)
        finally:
            n.nsga3_destroy(ctx)
    clocks = sampler.stop()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    head = [r for r in rows if r["workload"] == wl.LARGE.name and r["objectives"].startswith("generation")]
    top = head[-1]
    line = {
        "metric": "selected sols/s of nsga3_select alone (N / one selection)",
        "value": top["selected_sols_per_s"],
        "unit": "sols/s",
        "n_gpus": world,
        "steps": K,
        "warmup": 3,
        "ms_per_step": top["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "objectives saved from seeded softmax-simplex runs (generations 0, mid, last) and "
                "seeded adversarial sets",
        "config": {"workload": "select_m3_m5_m10", "value_of": "%s %s" % (top["workload"], top["objectives"]),
                   "l2": "flushed (256 MB write) before every timed selection",
                   "timing": "median of %d selections per matrix (CUDA events; the copy of the "
                             "objectives into the context, the graph and the copies of ranks and "
                             "indices out, all device to device)" % K,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "rows": rows,
        "gpu_launches": n_launch,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return line


def progress(msg):
    """One line of progress on stderr (stdout carries only the JSON line)."""
    print("[bench %.1fs] %s" % (time.perf_counter() - T_START, msg), file=sys.stderr, flush=True)


T_START = time.perf_counter()


def main(argv=None):
    import faulthandler
    faulthandler.enable()
    args = parse_args(argv)
    world, rank, local = dist_env()
    if args.steps is None:
        args.steps = {"headline": wl.LARGE.generations, "batched": 300, "served": 0, "sweep": 50,
                      "popsweep": 50, "select": 20, "shapes": 10}.get(args.workload)
        if args.steps is None:
            args.steps = WORKLOADS[args.workload].generations if args.workload in WORKLOADS else 20
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "headline":
        run_headline(args, world, rank, local)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "served":
        run_served(args, world, rank, local)
    elif args.workload in ("sweep", "popsweep"):
        run_sweep(args, world, rank, local)
    elif args.workload == "select":
        run_select(args, world, rank, local)
    elif args.workload == "shapes":
        run_shapes(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
