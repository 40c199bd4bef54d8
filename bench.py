#!/usr/bin/env python
"""EBIC population-evaluation benchmark on GB300.

One step = one EBIC generation's device work on one population: the population evaluator
(counts and row bitmaps of every candidate on every row) followed by the overlap-penalised
fitness against a device-resident elite archive, both through the C ABI with device buffers.
The workload is the methylation-shaped matrix (436,444 x 64 Beta(0.5,0.5), 10 planted trend
biclusters, 0.5% NaN, missing-value exclusion on) with populations of 1,600 candidates of 2-16
columns (the paper's converging population size, Methods, "Support for Big Data") and an archive
of 20 biclusters. The rank transform runs once per matrix and is reported separately.

Metric: candidate-row evals/s (one eval = one candidate checked against one row, any length).
Inputs are resident in HBM when the timed region starts; L2 is flushed (512 MB write) between
timed steps outside the timed events. ``e2e`` repeats the step through the same public calls
with the population in pinned host memory and the fitness read back to pinned host memory.

On one GPU the default run also measures the batched workload (8 matrices, 64 populations in
one graph replay, against 64 plain per-population launches) and the served workload (32 runs,
Poisson arrivals at 0.7 x the served capacity, against FIFO per-request calls), and reports them
as the line's ``batched`` and ``served`` objects, each with its own plain arm and clock record.

Under torchrun every rank runs the same workload on its own GPU (replicas, no collective on the
data path); the value is all ranks' evals divided by the slowest rank's time.

``--impl reference`` times the plain CPU oracle (test infrastructure) on the host cores, on a
bounded sample of the same workload: the comparison arm, not a target.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("methylation-shaped: float32 436,444 x 64, Beta(0.5,0.5) background, 10 planted trend "
            "biclusters (5,000-50,000 rows x 5-16 cols), 0.5% NaN, missing-value exclusion on; "
            "population 1,600 candidates of 2-16 cols; elite archive of 20 (the 10 planted "
            "biclusters + the 10 best-quality candidates of a separate 1,600-candidate pool)")
N_POPS = 4          # distinct seeded populations, cycled over the steps
SERVE_MAX_BATCH = 16  # served: requests per batch
SERVE_INFLIGHT = 3    # served: batches on the GPU at once
ARCHIVE = 20
FLUSH_BYTES = 512 << 20
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=50)
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="target wall time of the oracle's bounded sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-pairs", action="store_true",
                   help="score with the rank-code evaluator instead of the pair table")
    p.add_argument("--unfused", action="store_true",
                   help="time ebic_eval_population + ebic_fitness instead of ebic_eval_fitness")
    p.add_argument("--pair-budget", type=int, default=8 << 30,
                   help="largest pair table to build, bytes")
    p.add_argument("--workload", choices=["methylation", "batched", "served", "ga"],
                   default="methylation")
    p.add_argument("--ga-generations", type=int, default=30,
                   help="ga: generations of each ebic_run")
    p.add_argument("--ga-loop", choices=["both", "host", "device"], default="both",
                   help="ga: which generation loop(s) to time")
    p.add_argument("--load", type=float, default=0.7,
                   help="served: arrival rate as a fraction of the measured capacity")
    p.add_argument("--runs", type=int, default=32, help="served: concurrent EBIC runs")
    p.add_argument("--requests", type=int, default=1000, help="served: requests per trace")
    p.add_argument("--shard-rows", action="store_true",
                   help="methylation workload with its rows split over the ranks (one shard per "
                        "GPU, one all-reduce per generation) instead of one replica per rank")
    p.add_argument("--main-only", action="store_true",
                   help="default workload: skip the batched and served legs")
    p.add_argument("--leg-steps", type=int, default=20,
                   help="default workload: timed steps per arm of the batched leg")
    p.add_argument("--leg-requests", type=int, default=500,
                   help="default workload: requests per trace of the served leg")
    p.add_argument("--leg-repeats", type=int, default=3,
                   help="default workload: traces of the served leg at --load")
    p.add_argument("--leg-generations", type=int, default=20,
                   help="default workload: generations of each ebic_run of the ga leg")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def synth_planted(ds):
    from paper_1807_09932_gb300 import synth
    return synth.population_from_lists([list(p.cols) for p in ds.planted])


def make_workload():
    from paper_1807_09932_gb300 import synth
    ds, cols, offs = synth.config3()
    pops = [(cols, offs)]
    for i in range(1, N_POPS):
        pops.append(synth.make_population(synth.BASE_SEED + 3 + 1000 + 17 * i, 1600, 64, 2, 16))
    arch_pool = synth.make_population(synth.BASE_SEED + 3 + 5000, 1600, 64, 2, 16)
    return ds, pops, arch_pool


# ---- clocks during the timed region ----------------------------------------------------------

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                         if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None,
                "reasons": reasons}


# ---- the oracle arm / CPU baseline -------------------------------------------------------------

def oracle_sample(ds, pops, arch, target_s):
    """Time the oracle (eval + fitness) on a bounded sample of candidates over all rows."""
    import oracle
    X = ds.X
    R = X.shape[0]
    acols, aoffs, abm = arch
    threads = oracle.max_threads()

    def run(n, i=0):
        cols, offs = pops[i % len(pops)]   # the GPU arm's populations, cycled the same way
        sc = cols[: offs[n]]
        so = offs[: n + 1]
        t = time.perf_counter()
        c, b = oracle.eval_population(X, sc, so, exclude_missing=True, nthreads=threads)
        oracle.fitness(R, sc, so, c, b, acols, aoffs, abm, want_overlaps=False,
                       nthreads=threads)
        return time.perf_counter() - t

    probe = 32
    t = run(probe)
    n = int(min(1600, max(probe, probe * target_s / max(t, 1e-6))))
    return n, threads, run


def combine_over_ranks(my_seconds, units_per_rank, dist=None, device=None):
    """The job's time and throughput over all ranks: the time is the slowest rank's (max over
    ranks), the value is the units every rank processed together divided by it. Every rank gets
    both; without a process group this is the one rank's own."""
    ws, t = 1, float(my_seconds)
    if dist is not None:
        import torch
        ws = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, float(units_per_rank) * ws / t


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    ds, pops, arch_pool = make_workload()
    import oracle
    X = ds.X
    R = X.shape[0]
    # archive: the 20 best candidates of a separate population, by the oracle itself
    ac, ao = arch_pool
    cnt, bm = oracle.eval_population(X, ac, ao, exclude_missing=True)
    pc, po = synth_planted(ds)
    _, pbm = oracle.eval_population(X, pc, po, exclude_missing=True)
    arch = _archive_from(ds, ac, ao, cnt, bm, pbm)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    n, threads, run = oracle_sample(ds, pops, arch, min(per_step, args.cpu_seconds))
    for i in range(args.warmup):
        run(n, i)
    times = [run(n, i) for i in range(args.steps)]
    ms = 1000 * statistics.mean(times)
    value = n * R / (ms / 1000)
    line = {"impl": "reference", "metric": "candidate-row evals/s", "value": value,
            "unit": "candidate-row evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": R, "cols": X.shape[1],
                       "population": 1600, "archive": ARCHIVE, "populations_cycled": N_POPS,
                       "sample_candidates_per_step": n},
            "cpu_baseline": {"value": value, "unit": "candidate-row evals/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"the first {n} of the 1,600 candidates x all {R} rows "
                                       f"per step, the {N_POPS} populations cycled (evaluation "
                                       "+ fitness vs 20-member archive)"},
            "e2e": {"value": value, "unit": "candidate-row evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def _archive_from(ds, cols, offs, counts, bitmaps, planted_bitmaps, k=ARCHIVE):
    """A stand-in elite archive, as a converged EBIC run holds: the planted biclusters (their
    column orders) and the best remaining slots filled with the highest-quality candidates
    (rows << (min(L,33)-1), ties by index) of a separate random pool."""
    from paper_1807_09932_gb300 import synth
    planted = [list(p.cols) for p in ds.planted][:k]
    L = np.diff(offs).astype(np.int64)
    q = counts.astype(np.int64) << (np.minimum(L, 33) - 1)
    order = np.lexsort((np.arange(len(counts)), -q))[: k - len(planted)]
    acand = planted + [list(cols[offs[i]:offs[i + 1]]) for i in order]
    acols, aoffs = synth.population_from_lists(acand)
    abm = np.concatenate([planted_bitmaps[: len(planted)], bitmaps[order]], axis=0)
    return acols, aoffs, np.ascontiguousarray(abm)


# ---- our arm -------------------------------------------------------------------------------------

def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batched":
        batched_workload(args)
        return
    if args.workload == "served":
        served_workload(args)
        return
    if args.workload == "ga":
        ga_workload(args)
        return
    if args.shard_rows:
        sharded_workload(args)
        return
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1807_09932_gb300 import ebic

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)   # the library's work on a stream of its own
    torch.cuda.set_stream(stream)
    ds, pops, arch_pool = make_workload()
    X = ds.X
    R, C = X.shape

    def d(a):
        view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
        return torch.from_numpy(np.ascontiguousarray(a).view(view)).to(dev)

    # load: rank transform, timed by the library's own events; then the pair table, built by the
    # evaluator on the population of all column pairs (once per matrix, like the transform)
    Xd = torch.from_numpy(X).to(dev)
    # one transform of a small slice first, so that the timed one does not include the
    # kernel's first-launch module load
    ebic.Matrix(Xd[:4096].contiguous(), exclude_missing=True).close()
    torch.cuda.synchronize(dev)
    ebic.ebic_timing_enable(True)
    m = ebic.Matrix(Xd, exclude_missing=True)
    rank_ms, _ = ebic.ebic_timing_read(ebic.EBIC_TIMING_RANK_TRANSFORM)
    del Xd
    pair_bytes = 0
    pair_ms = None
    if not args.no_pairs:
        ebic.ebic_timing_enable(True)
        pair_bytes = m.build_pairs(max_bytes=args.pair_budget)
        pair_ms, _ = ebic.ebic_timing_read(ebic.EBIC_TIMING_EVALUATE)
    ebic.ebic_timing_enable(False)  # the headline pass runs without the library's events
    P = len(pops[0][1]) - 1
    W = m.words

    # elite archive: the 20 best of a separate population, evaluated on the GPU
    ac, ao = arch_pool
    acnt, abm = ebic.eval_population(m, ac, ao)
    pc, po = synth_planted(ds)
    _, pbm = ebic.eval_population(m, pc, po)
    acols, aoffs, abm = _archive_from(ds, ac, ao, acnt, abm, pbm)
    dacols, daoffs, dabm = d(acols), d(aoffs), d(abm)
    K = len(aoffs) - 1

    dpops = [(d(c), d(o), len(o) - 1) for c, o in pops]
    counts = torch.empty(P, dtype=torch.int32, device=dev)
    bitmaps = torch.empty((P, W), dtype=torch.int32, device=dev)
    fit = torch.empty(P, dtype=torch.int64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    h = m.handle
    sp = stream.cuda_stream

    def step(i):
        dc, do, n = dpops[i % N_POPS]
        if args.unfused:
            rc = ebic.ebic_eval_population(h, dc, do, n, 0, counts, bitmaps, sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_population")
            rc = ebic.ebic_fitness(h, dc, do, n, counts, bitmaps, dacols, daoffs, dabm, K, 0,
                                   fit, None, sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_fitness")
            return
        rc = ebic.ebic_eval_fitness(h, dc, do, n, 0, dacols, daoffs, dabm, K, counts, None, fit,
                                    None, sp)
        if rc:
            raise ebic.EbicError(rc, "ebic_eval_fitness")

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if m.status() != ebic.EBIC_OK:
        raise SystemExit("device status error after warm-up")

    # ---- timed region: K steps, L2 flushed between steps outside the events ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    # the timed regions run with the garbage collector paused: a full collection in the middle
    # of a step would hold back its launches after its start event
    gc.collect()
    gc.disable()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ebic.ebic_launch_count()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        step(i)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = ebic.ebic_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    step_dist = {"p50": float(np.percentile(step_ms, 50)), "p90": float(np.percentile(step_ms, 90)),
                 "p99": float(np.percentile(step_ms, 99)), "max": float(max(step_ms)),
                 "first": float(step_ms[0])}
    if m.status() != ebic.EBIC_OK:
        raise SystemExit("device status error in the timed region")

    # ---- per-kernel durations: a second timed pass over the same steps with the library's
    # CUDA events around each launch (on the launching stream). Kept out of the headline pass:
    # the events would separate kernels that the library otherwise chains with programmatic
    # dependent launch.
    kb_steps = min(args.steps, 200)
    ebic.ebic_timing_enable(True)
    for i in range(kb_steps):
        flush.fill_(i & 0xFF)
        step(i)
    torch.cuda.synchronize()
    clk = clocks.stop()
    eval_ms, eval_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_EVALUATE)
    pev_ms, pev_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_PAIR_EVALUATE)
    ov_ms, ov_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_OVERLAP)
    fin_ms, fin_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_FITNESS)
    prep_ms, prep_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_PREPARE)
    ebic.ebic_timing_enable(False)
    if m.status() != ebic.EBIC_OK:
        raise SystemExit("device status error in the kernel-timing pass")
    my_time, value = combine_over_ranks(tot_ms / 1000.0, float(P) * R * args.steps, dist, dev)
    ms_per_step = 1000.0 * my_time / args.steps

    # ---- e2e: the same step through the public calls with pinned host inputs/outputs ----
    e2e = None
    if args.e2e_steps > 0:
        hpops = []
        for c, o in pops:
            hc = torch.from_numpy(np.ascontiguousarray(c).view(np.int16)).pin_memory()
            ho = torch.from_numpy(np.ascontiguousarray(o).view(np.int32)).pin_memory()
            hpops.append((hc, ho, len(o) - 1))
        hfit = torch.empty(P, dtype=torch.int64).pin_memory()
        h2d = sum(hc.numel() * 2 + ho.numel() * 4 for hc, ho, _ in hpops) / N_POPS
        d2h = P * 8 + 4

        def e2e_step(i):
            hc, ho, n = hpops[i % N_POPS]
            if args.unfused:
                rc = ebic.ebic_eval_population(h, hc, ho, n, 0, counts, bitmaps, sp)
                if rc:
                    raise ebic.EbicError(rc, "ebic_eval_population")
                rc = ebic.ebic_fitness(h, hc, ho, n, counts, bitmaps, dacols, daoffs, dabm, K,
                                       0, hfit, None, sp)   # host output: synchronizes
                if rc:
                    raise ebic.EbicError(rc, "ebic_fitness")
                return
            rc = ebic.ebic_eval_fitness(h, hc, ho, n, 0, dacols, daoffs, dabm, K, counts, None,
                                        hfit, None, sp)   # host output: synchronizes
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_fitness")

        for i in range(3):
            e2e_step(i)
        ts = []
        for i in range(args.e2e_steps):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(i)
            ts.append(time.perf_counter() - t0)
        et, e2e_value = combine_over_ranks(sum(ts), float(P) * R * args.e2e_steps, dist, dev)
        e2e = {"value": e2e_value,
               "unit": "candidate-row evals/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1000 * et / args.e2e_steps,
               "path": ("ebic_eval_population + ebic_fitness" if args.unfused
                        else "ebic_eval_fitness") +
                       ", population in pinned host memory, fitness back in pinned host memory "
                       "(the fused route's kernels read and write them in place over the "
                       "host link)"}

    # ---- the rank-code route on the same matrix and populations (context for the other
    # kernels' roofs): the evaluator with counts and bitmaps, then the overlap kernel and the
    # fitness; the library's events around each launch, L2 flushed between steps ----
    rc_steps = 0 if args.no_pairs or args.unfused else min(args.steps, 20)
    rc_ms = None
    if rc_steps:
        def rc_step(i):
            dc, do, n = dpops[i % N_POPS]
            rc = ebic.ebic_eval_population(h, dc, do, n, ebic.EBIC_EVAL_DIRECT, counts, bitmaps,
                                           sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_population")
            rc = ebic.ebic_fitness(h, dc, do, n, counts, bitmaps, dacols, daoffs, dabm, K, 0,
                                   fit, None, sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_fitness")
        for i in range(3):
            rc_step(i)
        torch.cuda.synchronize()
        ebic.ebic_timing_enable(True)
        for kind in (ebic.EBIC_TIMING_EVALUATE, ebic.EBIC_TIMING_OVERLAP):
            ebic.ebic_timing_read(kind)
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        rc_tot = 0.0
        for i in range(rc_steps):
            flush.fill_(i & 0xFF)
            a_ev.record(stream)
            rc_step(i)
            b_ev.record(stream)
            torch.cuda.synchronize()
            rc_tot += a_ev.elapsed_time(b_ev)
        rc_eval_ms, rc_eval_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_EVALUATE)
        rc_ov_ms, rc_ov_n = ebic.ebic_timing_read(ebic.EBIC_TIMING_OVERLAP)
        ebic.ebic_timing_enable(False)
        rc_ms = rc_tot / rc_steps
        if m.status() != ebic.EBIC_OK:
            raise SystemExit("device status error in the rank-code pass")

    gc.enable()

    # ---- roofline of the dominant kernel (the evaluator) ----
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    eval_launch_ms = eval_ms / max(eval_n, 1)
    kernels = {}
    if ov_n:
        kernels["overlap"] = roofline_overlap(pops, K, m, ov_ms / ov_n, sms, clk)
    if pev_n:
        kernels["pair_evaluate"] = roofline_pairs(pops, R, m, pev_ms / pev_n, clk, peaks,
                                                  not args.unfused, K)
    if eval_n:
        kernels["evaluate"] = roofline_eval(pops, R, m, eval_launch_ms, sms, clk, peaks)
    # the step's kernel with the largest share is the dominant one; the rank-code route's
    # kernels (timed beside the step, not in it) are reported among the others
    dominant = max(kernels, key=lambda k: kernels[k]["launch_ms"])
    if rc_ms is not None:
        if rc_eval_n:
            kernels["evaluate (rank-code route)"] = roofline_eval(
                pops, R, m, rc_eval_ms / rc_eval_n, sms, clk, peaks)
        if rc_ov_n:
            kernels["overlap (rank-code route)"] = roofline_overlap(pops, K, m, rc_ov_ms / rc_ov_n,
                                                                    sms, clk)
    roof = dict(kernels[dominant])
    roof["kernel_role"] = dominant
    roof["other_kernels"] = {k: v for k, v in kernels.items() if k != dominant}

    line = {"metric": "candidate-row evals/s", "value": value, "unit": "candidate-row evals/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "step_ms_distribution": step_dist,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8" if m.rank_bits == 8 else "u16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": R, "cols": C, "population": P,
                       "archive": K, "populations_cycled": N_POPS,
                       "step": ("ebic_eval_population + ebic_fitness" if args.unfused
                                else "ebic_eval_fitness (evaluation and archive overlaps fused)"),
                       "l2": "flushed between timed steps (512 MB write, outside the events)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "rank_bits": m.rank_bits, "tile": list(m.tile)},
            "roofline": roof,
            "gpu_launches": int(launches),
            "clocks": clk,
            "pair_table": {"bytes": pair_bytes, "build_ms": pair_ms},
            "kernels_ms_per_step": {"evaluate": eval_ms / kb_steps,
                                    "pair_evaluate": pev_ms / kb_steps,
                                    "overlap": ov_ms / kb_steps,
                                    "fitness": fin_ms / kb_steps,
                                    "prepare": prep_ms / kb_steps},
            "kernel_timing": f"second timed pass of {kb_steps} steps, library CUDA events around "
                             "each launch on its stream, kernels not chained there",
            "rank_transform_ms": rank_ms,
            "wall_s": wall}
    if rc_ms is not None:
        line["rank_code_route"] = {
            "ms_per_step": rc_ms, "value": float(P) * R / (rc_ms / 1000.0),
            "steps": rc_steps,
            "path": "ebic_eval_population (EBIC_EVAL_DIRECT: the rank-code evaluator, counts and "
                    "bitmaps) + ebic_fitness (overlap kernel, fitness), device buffers, L2 flushed "
                    "between steps; kernel figures in roofline.other_kernels"}
    if e2e:
        line["e2e"] = e2e
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n, threads, run = oracle_sample(ds, pops, (acols, aoffs, abm),
                                        args.cpu_seconds / N_POPS)
        t = sum(run(n, i) for i in range(N_POPS))
        line["cpu_baseline"] = {"value": N_POPS * n * R / t, "unit": "candidate-row evals/s",
                                "cores": threads, "kind": "oracle",
                                "sample": f"the first {n} of the 1,600 candidates of each of the "
                                          f"{N_POPS} populations x all {R} rows (evaluation + "
                                          "fitness vs 20-member archive), once each"}
    m.close()
    if ws == 1 and not args.main_only:
        # the batched and served workloads, each against its plain per-population arm, with its
        # own clock record (one process on one GPU; under torchrun the replicas line alone)
        del counts, bitmaps, fit, flush, dpops
        torch.cuda.empty_cache()
        # a leg that fails records its error in its own key; the headline above stands
        legs = (("batched", lambda: batched_measure(args, args.leg_steps)),
                ("served", lambda: served_measure(args, [args.load], args.leg_requests,
                                                  args.leg_repeats)),
                ("ga", lambda: ga_measure(args, args.leg_generations)))
        for name, fn in legs:
            try:
                line[name] = fn()
            except Exception as e:  # noqa: BLE001 - reported in the line, not swallowed
                gc.enable()
                line[name] = {"error": f"{type(e).__name__}: {e}"}
                print(f"bench: the {name} leg failed: {e!r}", file=sys.stderr, flush=True)
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        line["legs"] = ("batched: batched_measure, the config of its line; served: "
                        f"served_measure, {args.leg_repeats} traces of {args.leg_requests} "
                        f"requests at {args.load:.2f} x the served capacity, latencies pooled")
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def sharded_workload(args):
    """The methylation workload with its rows spread over the ranks, as the paper spreads them
    over GPUs (Abstract; Methods, "Support for Big Data"): rank r loads row shard r (32-row
    aligned), builds its pair table, and every step is one generation's scoring -- the shard's
    partials (ebic_eval_partials), one all-reduce of P + P*K + K values (NCCL under torchrun),
    and the fitness from the sums (ebic_fitness_reduced). The total work is fixed as the ranks
    grow ("scaling": "strong"); the value counts the whole matrix's rows."""
    import torch
    from paper_1807_09932_gb300 import ebic, shard
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ds, pops, arch_pool = make_workload()
    X = ds.X
    R, C = X.shape
    o, r = shard.shard_ranges(R, ws)[rank]
    m = ebic.Matrix(torch.from_numpy(np.ascontiguousarray(X[o:o + r])).to(dev),
                    exclude_missing=True, row_offset=o, total_rows=R)
    m.build_pairs(max_bytes=args.pair_budget)
    allreduce = shard.reduce_sum(dist) if dist else (lambda b: None)

    def d(a):
        view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
        return torch.from_numpy(np.ascontiguousarray(a).view(view)).to(dev)

    # the archive, chosen from whole-matrix counts (the same choice on every rank); its bitmaps
    # are this shard's rows of the members' bitmaps
    ac, ao = arch_pool
    acnt, abm = ebic.eval_population(m, ac, ao)
    t = torch.from_numpy(acnt.astype(np.int32)).to(dev)
    allreduce(t)
    acnt = t.cpu().numpy().astype(np.uint32)
    pc, po = synth_planted(ds)
    _, pbm = ebic.eval_population(m, pc, po)
    acols, aoffs, abm = _archive_from(ds, ac, ao, acnt, abm, pbm)
    K = len(aoffs) - 1
    dacols, daoffs, dabm = d(acols), d(aoffs), d(abm)
    P = len(pops[0][1]) - 1
    dpops = [(d(c), d(o_), len(o_) - 1) for c, o_ in pops]
    stream = torch.cuda.current_stream(dev)
    scorer = shard.ShardedScorer(m, P, K, allreduce, dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(i):
        dc, do, n = dpops[i % N_POPS]
        return scorer.score(dc, do, n, dacols, daoffs, dabm, K)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    check = None
    if ws == 1:  # one shard is the whole matrix: the sharded fitness must be the fused call's
        fit, _ = step(0)
        ref = torch.empty(P, dtype=torch.int64, device=dev)
        cnt = torch.empty(P, dtype=torch.int32, device=dev)
        dc, do, n = dpops[0]
        rc = ebic.ebic_eval_fitness(m.handle, dc, do, n, 0, dacols, daoffs, dabm, K, cnt, None,
                                    ref, None, stream.cuda_stream)
        if rc:
            raise ebic.EbicError(rc, "ebic_eval_fitness")
        check = bool(torch.equal(fit, ref))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    gc.collect()
    gc.disable()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ebic.ebic_launch_count()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        step(i)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    launches = ebic.ebic_launch_count() - launches0
    clk = clocks.stop()
    gc.enable()
    if m.status() != ebic.EBIC_OK:
        raise SystemExit("device status error in the timed region")
    tot_ms = sum(a.elapsed_time(b) for a, b in evs)
    # strong scaling: every rank processed its shard of the same P x R evaluations, so the job's
    # units are P x R per step in all; combine_over_ranks multiplies a rank's units by N
    my_time, value = combine_over_ranks(tot_ms / 1000.0, float(P) * R * args.steps / ws, dist,
                                        dev)
    line = {"metric": "candidate-row evals/s", "value": value, "unit": "candidate-row evals/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * my_time / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "u8" if m.rank_bits == 8 else "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": R, "cols": C, "population": P,
                       "archive": K, "populations_cycled": N_POPS,
                       "parallelism": f"row shards x{ws} (32-row aligned), one all-reduce of "
                                      f"{shard.packed_size(P, K)} uint32 per generation",
                       "shard_rows": r, "step": "ebic_eval_partials + all-reduce + "
                                                "ebic_fitness_reduced",
                       "l2": "flushed between timed steps (512 MB write, outside the events)"},
            "gpu_launches": int(launches), "clocks": clk,
            "sharded_fitness_equals_fused_call": check}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()


def traffic_record(name):
    """DRAM bytes per launch of a kernel from a committed ncu capture
    (profiles/<name>_traffic.json), if the kernel's sources are still the ones that were captured
    (SHA-256 over the listed files, concatenated in order)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    try:
        rec = json.load(open(path))
        sources = rec.get("sources") or [rec["source"]]
        h = hashlib.sha256()
        for src in sources:
            h.update(open(os.path.join(ROOT, src), "rb").read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest() != rec.get("source_sha256"):
        return None
    return rec["dram_bytes_per_launch"]


def roofline_pairs(pops, R, m, launch_ms, clk, peaks, fused, K):
    """The pair-table evaluator: an HBM stream. Algorithmic bytes per launch: the table rows the
    population needs (distinct consecutive column pairs, rows of W rounded up to 512 words;
    each read once) and its counts, plus the bitmaps it writes (unfused) or the padded archive
    rows it reads (fused), against the measured HBM copy bandwidth."""
    W = m.words
    Wt = (W + 511) // 512 * 512
    per = []
    for c, o in pops:
        pairs = set()
        for i in range(len(o) - 1):
            seq = c[o[i]:o[i + 1]]
            if len(seq) == 1:
                pairs.add((int(seq[0]), int(seq[0])))
            for a, b in zip(seq[:-1], seq[1:]):
                pairs.add((int(a), int(b)))
        extra = K * Wt * 4 if fused else (len(o) - 1) * W * 4
        per.append(len(pairs) * Wt * 4 + (len(o) - 1) * 4 + extra)
    hbm_bytes = float(np.mean(per))
    t = launch_ms / 1000.0
    peak = peaks.get("hbm_gbs", 6800.0)
    traffic = traffic_record("pair_eval_fused") if fused else None
    return {"bound": "hbm", "achieved": hbm_bytes / t / 1e9, "peak": peak, "unit": "GB/s",
            "frac": (hbm_bytes / t / 1e9) / peak, "traffic": traffic,
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                            "(profiles/pair_eval_fused_traffic.json); null if the kernel source "
                            "changed since that capture",
            "kernel": "pair_eval_kernel" + (" (fused overlaps)" if fused else ""),
            "launch_ms": launch_ms,
            "algorithmic_bytes_per_launch": hbm_bytes,
            "peak_basis": "MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)"
                          if "hbm_gbs" in peaks else "fallback 6.8 TB/s"}


def roofline_overlap(pops, K, m, launch_ms, sms, clk):
    """The overlap kernel: P x K x W AND+popcount of 32-bit words. Its roof is the popcount
    pipe (16 per SM per clock) for the plain formulation; the carry-save tree trades half of
    the popcounts for ALU work, so the ALU pipe (64 lanes/clk/SM, ~26 ops per 8 words) is the
    roof of the kernel as written. Both are reported; the larger minimum time binds."""
    P = 1600
    W = m.words
    units = float(P) * K * W
    clock_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
    t = launch_ms / 1000.0
    popc_peak = 16 * sms * clock_hz
    alu_ops = units / 8 * 26
    alu_peak = 64 * sms * clock_hz
    return {"bound": "alu", "achieved": alu_ops / t / 1e9, "peak": alu_peak / 1e9,
            "unit": "Gop/s", "frac": (alu_ops / t) / alu_peak, "traffic": None,
            "kernel": "overlap_kernel", "launch_ms": launch_ms,
            "algorithmic_ops_per_launch": alu_ops,
            "peak_basis": "64 INT32 lanes/clk/SM x SMs x median SM clock; 26 ALU ops per 8 words",
            "popc": {"units": units, "frac_of_popc_roof": (units / t) / popc_peak}}


def roofline_eval(pops, R, m, launch_ms, sms, clk, peaks):
    """The evaluator against the roof that binds it.

    Algorithmic work per launch (one population): every candidate column must be read for every
    row, sum_c L_c * R ranks of rank_bits/8 bytes each, out of shared memory (the row tile is
    staged there by TMA); and each is one packed-field compare, 32/rank_bits rows per 32-bit
    lane-op. Peaks from the recipe's unit counts and the median SM clock sampled during the
    timed region: shared memory 128 B/clk/SM, INT32 ALU 64 lanes/clk/SM. The shared-memory time
    is the larger of the two minimum times, so it is the binding roof ("bound"); the ALU and HBM
    roofs are reported beside it. HBM: rank matrix + bitmaps against the measured copy
    bandwidth (MEASURED_PEAKS.json).
    """
    sum_l = float(np.mean([int(o[-1]) for _, o in pops]))
    bytes_per_rank = m.rank_bits / 8
    fields_per_word = 32 // m.rank_bits
    clock_hz = (clk.get("sm_mhz") or peaks.get("sm_max_mhz") or 2070.0) * 1e6
    t = launch_ms / 1000.0
    smem_bytes = sum_l * R * bytes_per_rank
    smem_peak = 128 * sms * clock_hz
    lane_ops = sum_l * R / fields_per_word
    alu_peak = 64 * sms * clock_hz
    hbm_bytes = m.cols * R * bytes_per_rank + 1600 * m.words * 4
    return {"bound": "smem", "achieved": smem_bytes / t / 1e9, "peak": smem_peak / 1e9,
            "unit": "GB/s", "frac": (smem_bytes / t) / smem_peak,
            "traffic": traffic_record("eval_population"),
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch "
                            "(profiles/eval_population_traffic.json); null if the kernel source "
                            "changed since that capture",
            "kernel": "eval_population_kernel", "launch_ms": launch_ms,
            "algorithmic_bytes_per_launch": smem_bytes,
            "peak_basis": "shared memory 128 B/clk/SM x SMs x median SM clock in the timed region",
            "alu": {"achieved_gops": lane_ops / t / 1e9, "peak_gops": alu_peak / 1e9,
                    "frac": (lane_ops / t) / alu_peak,
                    "basis": "one 32-bit compare per column per 32/rank_bits rows; 64 INT32 lanes/clk/SM"},
            "hbm": {"algorithmic_bytes": hbm_bytes, "achieved_gbs": hbm_bytes / t / 1e9,
                    "peak_gbs": peaks.get("hbm_gbs"),
                    "frac": (hbm_bytes / t / 1e9) / peaks["hbm_gbs"] if "hbm_gbs" in peaks
                    else None, "basis": "rank matrix + bitmaps vs MEASURED_PEAKS.json hbm_gbs"}}


# ---- config 4: batched vs plain per-population launches ----------------------------------------

def ga_workload(args):
    print(json.dumps(ga_measure(args, args.ga_generations)), flush=True)


def ga_measure(args, generations):
    """The whole method on the methylation-shaped matrix: ebic_run (P = 1,600, archive 20,
    candidates of up to 16 columns) with the generation loop on the host and on the device. A step
    is one generation; the line reports ms per generation of each loop and whether their archives
    are identical (they must be)."""
    import torch
    from paper_1807_09932_gb300 import ebic
    torch.cuda.set_device(0)
    ds, _, _ = make_workload()
    R = ds.X.shape[0]
    loops = {"host": 0, "device": ebic.EBIC_RUN_ON_DEVICE}
    if args.ga_loop != "both":
        loops = {args.ga_loop: loops[args.ga_loop]}
    out, archives = {}, {}
    with ebic.Matrix(torch.from_numpy(ds.X).cuda(), exclude_missing=True) as m:
        if not args.no_pairs:
            m.build_pairs(max_bytes=args.pair_budget)
        for name, flag in loops.items():
            ebic.ebic_run(m.handle, ebic.ebic_params_default(population=1600, generations=2,
                                                             flags=flag))  # warm-up
            params = ebic.ebic_params_default(population=1600, generations=generations,
                                              archive_size=20, max_len=16, flags=flag)
            launches0 = ebic.ebic_launch_count()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = ebic.ebic_run(m.handle, params)
            wall = time.perf_counter() - t0
            out[name] = {"ms_per_generation": 1000.0 * wall / res["generations_run"],
                         "generations": res["generations_run"],
                         "gpu_launches": ebic.ebic_launch_count() - launches0}
            archives[name] = res
    line = {"metric": "ms per EBIC generation", "workload": "ga", "unit": "ms",
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": WORKLOAD + "; ebic_run, population 1,600, archive 20, "
                                   "candidates of 2-16 columns",
                       "rows": R, "pair_table": not args.no_pairs},
            "loops": out}
    if len(archives) == 2:
        a, b = archives["host"], archives["device"]
        line["same_archive"] = bool(a["members"] == b["members"] and
                                    np.array_equal(a["bitmaps"], b["bitmaps"]))
    return line


def batched_workload(args):
    print(json.dumps(batched_measure(args, max(3, min(args.steps, 50)))), flush=True)


def batched_measure(args, steps):
    """8 datasets (5k-200k rows, 20-500 cols) and 64 populations (200-3,200 candidates of 2-64
    columns), round-robin over the datasets. One step = all 64 populations scored. Plain: one
    ebic_eval_population per population. Batched: one ebic_batch_run (CUDA-graph replay of the
    check, plan and persistent kernels), with tile shapes from the autotuner. `steps` timed steps
    per arm. Returns the result line."""
    import torch

    from paper_1807_09932_gb300 import autotune, ebic, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    dspecs, pspecs = synth.config4_specs()
    mats, rows = [], []
    for d in dspecs:
        ds = synth.dataset_from_spec(d)
        mats.append(ebic.Matrix(torch.from_numpy(ds.X).to(dev)))
        rows.append(d["rows"])
        del ds
    pops = []
    for ps in pspecs:
        m = mats[ps["dataset"]]
        c, o = synth.make_population(ps["seed"], ps["n_cand"], m.cols, ps["lmin"],
                                     min(ps["lmax"], m.cols))
        n = len(o) - 1
        pops.append(dict(m=m, n=n, R=m.rows, mean_len=float(np.diff(o).mean()),
                         dc=torch.from_numpy(c.view(np.int16)).to(dev),
                         do=torch.from_numpy(o.view(np.int32)).to(dev),
                         cnt=torch.empty(n, dtype=torch.int32, device=dev),
                         bm=torch.empty((n, m.words), dtype=torch.int32, device=dev)))
    cache = autotune.Cache()
    tuned = {}
    t_tune = time.perf_counter()
    for p in pops:  # one tuning per matrix, on its first population
        if id(p["m"]) in tuned:
            continue
        tuned[id(p["m"])] = autotune.tune_matrix(p["m"], p["dc"], p["do"], p["n"], p["mean_len"],
                                                 p["cnt"], p["bm"], cache=cache, iters=2)
    t_tune = time.perf_counter() - t_tune
    # pair tables (once per matrix; 3.8 GB for these eight): both arms then use them, the plain
    # one through ebic_eval_population and the batched one through its pair-table pass
    pair_bytes, t_pairs = 0, 0.0
    if not args.no_pairs:
        t0 = time.perf_counter()
        for m in mats:
            pair_bytes += m.build_pairs(max_bytes=args.pair_budget)
        t_pairs = time.perf_counter() - t0
    evals_per_step = float(sum(p["n"] * p["R"] for p in pops))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def plain_step():
        for p in pops:
            rc = ebic.ebic_eval_population(p["m"].handle, p["dc"], p["do"], p["n"], 0, p["cnt"],
                                           p["bm"], stream.cuda_stream)
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_population")

    batch = ebic.ebic_batch_create(len(pops))
    arr = ebic.make_requests([(p["m"].handle, p["dc"], p["do"], p["n"], 0, p["cnt"], p["bm"])
                              for p in pops])

    def batched_step():
        rc = ebic.ebic_batch_run(batch, arr, len(pops), stream.cuda_stream)
        if rc:
            raise ebic.EbicError(rc, "ebic_batch_run")

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()
        evs = []
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        gc.enable()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    clocks = ClockSampler(0)
    clocks.start()
    launches0 = ebic.ebic_launch_count()
    ms_plain = timed(plain_step, steps)
    ms_batched = timed(batched_step, steps)
    launches = ebic.ebic_launch_count() - launches0
    clk = clocks.stop()
    rc, st = ebic.ebic_batch_status(batch, len(pops))
    if rc or any(st):
        raise SystemExit("batched status error")
    rank_code = None
    if pair_bytes:  # context: the same batch on the rank-code pass (tables dropped)
        for m in mats:
            m.drop_pairs()
        ms_rank = timed(batched_step, steps)
        ms_rank_plain = timed(plain_step, steps)
        rank_code = {"batched_ms_per_step": ms_rank, "plain_ms_per_step": ms_rank_plain,
                     "batched_value": evals_per_step / (ms_rank / 1000)}
    ebic.ebic_batch_free(batch)
    line = {"metric": "candidate-row evals/s", "value": evals_per_step / (ms_batched / 1000),
            "unit": "candidate-row evals/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_batched, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16", "data": "synthetic",
            "config": {"workload": "batched: 8 datasets (5k-200k rows x 20-500 cols, N(0,1)/Beta "
                                   "alternating, planted, 0.5% NaN), 64 populations of 200-3,200 "
                                   "candidates of 2-64 cols, round-robin; one step = all 64",
                       "evals_per_step": evals_per_step,
                       "l2": "flushed between timed steps (512 MB write, outside the events)",
                       "tiles": {str(i): list(v[:2]) for i, v in enumerate(tuned.values())},
                       "autotune_s": t_tune,
                       "pair_tables": {"bytes": pair_bytes, "build_s": t_pairs}},
            "plain": {"value": evals_per_step / (ms_plain / 1000), "ms_per_step": ms_plain,
                      "path": "64 x ebic_eval_population, one launch set per population"
                              + (" (pair tables)" if pair_bytes else "")},
            "batched_over_plain": ms_plain / ms_batched,
            "rank_code_pass": rank_code,
            "gpu_launches": int(launches), "clocks": clk}
    for m in mats:
        m.close()
    return line


# ---- config 5: served (continuous batching) vs plain per-population launches -------------------

def served_workload(args):
    line = served_measure(args, sorted({0.25, 0.5, args.load, 1.0}), args.requests, 1)
    print(json.dumps(line), flush=True)


def served_measure(args, loads, requests, repeats):
    """32 concurrent EBIC runs on datasets of 10,000-436,444 rows x 20-200 cols, 1,600 candidates
    per request (2-16 columns), Poisson arrivals at each of `loads` x the measured served
    capacity (`repeats` traces of `requests` requests at `args.load`, one at each other load).
    Served: the continuous-batching server. Plain: the same arrivals, FIFO, one request at a time
    through ebic_eval_fitness. Latency = completion - arrival (host clock). Returns the line; its
    headline figures at `args.load` pool the latencies of all repeats."""
    import torch

    from paper_1807_09932_gb300 import serve, synth
    torch.cuda.set_device(0)
    runs = synth.config5_specs(n_runs=args.runs)
    specs, rows_of = [], {}
    for i, r in enumerate(runs):
        ds = synth.dataset_from_spec(r)
        pool_c, pool_o = synth.make_population(r["seed"] + 1, 40, r["cols"], 2, 6)
        arch = synth.population_from_lists(
            [list(pool_c[pool_o[j]:pool_o[j + 1]]) for j in range(20)])
        specs.append(serve.RunSpec(run_id=i, X=ds.X, max_cand=r["n_cand"], max_len=16,
                                   archive_cols=arch[0], archive_offsets=arch[1]))
        rows_of[i] = r["rows"]
    # batches of at most 16 requests, three in flight: a sweep of 4-32 x 2-4 gave the highest
    # saturated throughput there, and p99 within 0.02 ms of the best at a fixed arrival rate
    be = serve.GpuBackend(max_batch=SERVE_MAX_BATCH, max_inflight=SERVE_INFLIGHT,
                          pair_budget=0 if args.no_pairs else args.pair_budget)
    budget = sum(be.footprint(s) for s in specs) + (1 << 30)
    srv = serve.Server(be, hbm_budget=budget, max_batch=SERVE_MAX_BATCH,
                       max_inflight=SERVE_INFLIGHT)
    for s in specs:
        srv.add_run(s)
    for s in specs:
        s.X = None  # the rank matrices are resident; host copies are not needed any more
    rng = np.random.default_rng(synth.BASE_SEED + 55)
    pools = [[synth.make_population(runs[i]["seed"] + 10 + j, runs[i]["n_cand"],
                                    runs[i]["cols"], 2, 16) for j in range(4)]
             for i in range(len(specs))]

    def trace(n, rate):
        t, out = 0.0, []
        for k in range(n):
            t += rng.exponential(1.0 / rate) if rate else 0.0
            run = int(rng.integers(len(specs)))
            c, o = pools[run][k % 4]
            out.append(serve.Request(run_id=run, cols=c, offsets=o, t_arrival=t))
        return out

    mean_evals = float(np.mean([runs[i]["n_cand"] * runs[i]["rows"] for i in range(len(runs))]))
    plain_stream = torch.cuda.Stream()

    def copy_trace(tr):
        return [serve.Request(run_id=r.run_id, cols=r.cols, offsets=r.offsets,
                              t_arrival=r.t_arrival, flags=r.flags) for r in tr]

    def run_served(tr):
        srv.done.clear()
        srv.batches = 0
        return serve.drive(srv, tr, rows_of)

    # warm-up, then capacity: a saturated trace (everything arrives at once) through each path
    serve.drive(srv, trace(2 * len(specs), 0.0), rows_of)
    serve.plain_serve(be, trace(len(specs), 0.0), rows_of, plain_stream)
    sat_trace = trace(4 * len(specs), 0.0)
    gc.collect()
    gc.disable()
    sat_served = run_served(copy_trace(sat_trace))
    sat_plain = serve.plain_serve(be, copy_trace(sat_trace), rows_of, plain_stream)
    gc.enable()
    capacity_rps = sat_served["evals_per_s"] / mean_evals
    gc.collect()
    gc.disable()
    clocks = ClockSampler(0)
    clocks.start()
    sweep = []
    headline = None
    for load in loads:
        reps = []
        for _ in range(repeats if load == args.load else 1):
            tr = trace(requests, load * capacity_rps)
            a, b = copy_trace(tr), copy_trace(tr)
            sv = run_served(a)
            pl = serve.plain_serve(be, b, rows_of, plain_stream)
            reps.append((sv, pl, [r.latency for r in a], [r.latency for r in b]))
        entry = {"load": load, "rate_rps": load * capacity_rps,
                 "served": pooled(reps, 0, 2), "plain": pooled(reps, 1, 3)}
        if len(reps) > 1:
            entry["repeats"] = [{"served_p50_ms": r[0]["p50_ms"], "served_p99_ms": r[0]["p99_ms"],
                                 "plain_p50_ms": r[1]["p50_ms"], "plain_p99_ms": r[1]["p99_ms"]}
                                for r in reps]
        sweep.append(entry)
        if load == args.load:
            headline = entry
    clk = clocks.stop()
    gc.enable()
    be.close()
    served, plain = headline["served"], headline["plain"]
    line = {"metric": "candidate-row evals/s", "value": served["evals_per_s"],
            "unit": "candidate-row evals/s", "n_gpus": 1, "steps": served["requests"],
            "warmup": 3 * len(specs), "ms_per_step": served["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/u16", "data": "synthetic",
            "config": {"workload": f"served: {len(specs)} EBIC runs on 10,000-436,444 x 20-200 "
                                   "matrices (N(0,1)/Beta, planted, 0.5% NaN), 1,600 candidates "
                                   "of 2-16 cols per request, archive of 20 per run, Poisson "
                                   f"arrivals at {args.load:.2f} x the served capacity",
                       "arrival_rate_rps": headline["rate_rps"], "capacity_rps": capacity_rps,
                       "max_batch": SERVE_MAX_BATCH, "batches_in_flight": SERVE_INFLIGHT,
                       "requests_per_trace": requests, "traces_at_headline_load": repeats},
            "served": served, "plain": plain,
            "saturated": {"served": sat_served, "plain": sat_plain,
                          "served_over_plain": sat_served["evals_per_s"] / sat_plain["evals_per_s"]},
            "sweep": sweep, "clocks": clk,
            "gpu_launches": int(ebic_launches())}
    return line


def pooled(reps, k, lat_k):
    """One load's figures over its repeated traces: p50/p99 of all their latencies together,
    evals/s over their summed wall time."""
    from paper_1807_09932_gb300 import serve
    if len(reps) == 1:
        return reps[0][k]
    lat = [x for r in reps for x in r[lat_k]]
    wall = sum(r[k]["wall_s"] for r in reps)
    evals = sum(r[k]["evals_per_s"] * r[k]["wall_s"] for r in reps)
    return {"requests": len(lat), "p50_ms": 1000 * serve.percentile(lat, 50),
            "p99_ms": 1000 * serve.percentile(lat, 99), "mean_ms": 1000 * sum(lat) / len(lat),
            "evals_per_s": evals / wall, "wall_s": wall}


def ebic_launches():
    from paper_1807_09932_gb300 import ebic
    return ebic.ebic_launch_count()


if __name__ == "__main__":
    main()
