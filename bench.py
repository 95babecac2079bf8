#!/usr/bin/env python3
"""Throughput of the Sample-Align-D decomposition hot path on GB300.

One step = kmer_count -> kmer_rank -> partition of one synthetic sequence set
(default: the largest workload, N = 100000 protein sequences in 500 families,
k = 3, p = 64) with the inputs already in HBM. The metric is k-mer pair
comparisons per second: the N(N-1)/2 pairs whose shared k-mer count (Eq. 1)
enters the ranks, per step time.

Prints one JSON line. Extra objects:
  roofline      the plane-GEMM kernel: the work of Eq. 1 as written (2 x 8000
                ops per unordered pair) per launch over its CUDA-event time,
                against the 4-bit (e2m1) tensor peak derived from the measured
                bf16 peak; the MMA work actually issued beside it
  calls         each call of the step run alone (L2 flushed before each run):
                kmer_count with its algorithmic bytes and HBM fraction,
                kmer_rank and partition as times
  cpu_baseline  the CPU oracle on a bounded sample of the same workload
  e2e           the same metric through the public API with host buffers
                (H2D of codes + offsets and D2H of the buckets and keys timed)
  clocks        SM clocks and throttle reasons sampled during the timed region
  configs       the other two workloads (N = 200 and N = 20000), each with the
                same roofline, calls, e2e and oracle figures
  globalised    the globalised rank of Sec. 3.1.1 on the N = 20000 set (local
                ranks, p - 1 samples per block, rank against the samples), timed,
                and how its buckets compare with the centralised ones
  distance_form the rank of Eq. 2 / Eq. 3 as written (mean -ln(1/10 + F)), timed
  table1_synthetic  the statistics of Table 1 (centralised vs globalised ranks in
                the distance form) on a synthetic 500-sequence family set
  sparse_ablation  the same keys by sparse intersection on the CUDA cores (the
                per-pair cost of Table 2), against the plane-GEMM rank time
  batching      512 uneven sets in one captured CUDA graph against plain per-set calls
  serving       continuous batching of Poisson arrivals (and a saturated burst)
                against one-at-a-time service, latency percentiles and sets/s

--impl reference times the CPU oracle on the same workload instead (one bounded
sample per step). Under torchrun each rank runs an independent replica of the
workload (the path does not shard); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0905_1744_gb300 import datagen  # noqa: E402

WORKLOADS = {
    1: "N=200 iid protein sequences, L uniform 100-400, k=3 (8000 words), p=4",
    2: "N=20000 sequences in 50 families (ancestor L ~ N(300,100) clipped to 50-1000, "
       "20-40% substitutions, 2% indels of length 1-10), k=3, p=16",
    3: "N=100000 sequences in 500 families (ancestor L log-uniform 50-2000, 20-40% "
       "substitutions, 2% indels of length 1-10), k=3, p=64",
}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (all ranks call it), then a barrier: the
    timed region of a replica job ends when its slowest replica does."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each processing units_per_rank in
    the job's time (the slowest replica's)."""
    return world * units_per_rank / seconds


def time_calls(calls: dict, reps: int, flush, stream, event_cls) -> dict:
    """Median device milliseconds of each call run alone: L2 flushed before every
    repetition, events recorded on the launching stream around the call."""
    out = {}
    for name, fn in calls.items():
        times = []
        for _ in range(reps):
            flush()
            e0, e1 = event_cls(enable_timing=True), event_cls(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = statistics.median(times)
    return out


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sad", choices=["sad", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3],
                    help="the main line's workload (default: the largest, N = 100000)")
    ap.add_argument("--subset", type=int, default=0,
                    help="profiling: evenly spaced N sequences of the workload instead of all")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the c1/c2 lines (and the legs that run on the paper-scale set)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=256, choices=[128, 256],
                    help="GEMM tile rows with --depth (default: the autotuner's choice)")
    ap.add_argument("--budget", type=int, default=0,
                    help="remainder budget with --depth (0 = the library default)")
    ap.add_argument("--depth", type=int, default=None,
                    help="threshold-plane depth (default: the autotuner's choice)")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-global", action="store_true",
                    help="skip the globalised-rank, distance-form and Table 1 legs")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-warmup", type=int, default=100)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-pool", type=int, default=256)
    ap.add_argument("--serve-burst", type=int, default=400)
    ap.add_argument("--batch-sets", type=int, default=512)
    ap.add_argument("--batch-reps", type=int, default=10)
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle ---

def oracle_counts(s):
    import oracle
    oracle.build()
    return oracle.kmer_count(s.codes, s.offsets)


def oracle_sample(s, seconds: float, seed: int = 0, counts=None):
    """Time the oracle's rank on a row sample sized to ~`seconds` of CPU work.

    Returns (pairs_per_s, rows, elapsed, threads). The oracle computes each
    sampled row's shared counts with all N sequences, so R rows are R (N - 1)
    ordered comparisons, R (N - 1) / 2 unordered pair-equivalents; the rate is
    that over the sample's own time (the full set would take N / R times as long).
    """
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    if counts is None:
        counts = oracle.kmer_count(s.codes, s.offsets)
    rng = np.random.default_rng(seed)
    r0 = max(threads, 8)
    rows = rng.choice(s.n, size=min(r0, s.n), replace=False)
    t0 = time.perf_counter()
    oracle.kmer_rank(counts, s.lengths, rows=rows, threads=threads)
    t_cal = time.perf_counter() - t0
    r = int(min(s.n, max(r0, r0 * seconds / max(t_cal, 1e-6))))
    rows = rng.choice(s.n, size=r, replace=False)
    t0 = time.perf_counter()
    oracle.kmer_rank(counts, s.lengths, rows=rows, threads=threads)
    t = time.perf_counter() - t0
    return r * (s.n - 1) / 2 / t, r, t, threads


def bench_config(cfg: int, s, seed: int) -> dict:
    """The workload description both arms print (identical dicts)."""
    return {"workload": WORKLOADS[cfg], "N": s.n, "p": s.p, "k": 3, "alphabet": 20,
            "seed": seed,
            "l2": "inputs larger than L2 (int32 counts 4 x 8000 x N bytes) and a 256 MB "
                  "write between timed GPU steps"}


def run_reference(args):
    """The oracle on the host cores: each step ranks a bounded random row sample
    against all N sequences; ms_per_step is that sample's own time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s = datagen.config(args.config, args.seed)
    per_step = max(0.5, 120.0 / max(1, args.steps + args.warmup))
    counts = oracle_counts(s)
    vals, secs, rows_used, threads = [], [], 0, 1
    for i in range(args.warmup + args.steps):
        v, r, t, threads = oracle_sample(s, per_step, seed=args.seed + i, counts=counts)
        if i >= args.warmup:
            vals.append(v)
            secs.append(t)
            rows_used = r
    value = statistics.mean(vals)
    out = {
        "impl": "reference", "metric": "k-mer pair comparisons/s", "value": value,
        "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64/uint128 (CPU)", "data": "synthetic",
        "device": f"host CPU cores (the oracle, {threads} threads; no GPU work)",
        "config": bench_config(args.config, s, args.seed),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step: {rows_used} random rows against all {s.n} "
                                   f"sequences ({rows_used} x {s.n - 1} / 2 pair-equivalents), "
                                   "timed alone",
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# --------------------------------------------------------------------- GPU ---

def gemm_traffic_per_launch(n: int, tile: int, depth: int, budget: int):
    """DRAM bytes (read + write) of one GEMM launch from the committed ncu captures,
    or None for a workload or plan shape not captured, or when the kernel source
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", "pair_gemm_traffic.json")
    src = os.path.join(ROOT, "paper_0905_1744_gb300", "csrc", "gemm.cu")
    try:
        with open(path) as f:
            d = json.load(f)
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    if d.get("gemm_cu_sha256") != sha:
        return None
    for e in d.get("captures", []):
        if (e.get("N"), e.get("tile"), e.get("depth"), e.get("budget")) == (n, tile, depth,
                                                                              budget):
            return e["dram_bytes_read_per_launch"] + e["dram_bytes_write_per_launch"]
    return None


def run_batching(args, dev):
    """512 uneven sets in one block-diagonal launch. The tile shape and plane depth
    come from the batching autotuner (timed on plans from host-side bounds); then
    every timed batch is a NEW batch as a user sees it: its inputs go up from
    pinned memory, its plan comes from host-side bounds (no synchronisation), its
    launches are captured into the one library graph (updated in place, not
    re-instantiated) and launched, and its bucket lists come back to pinned host
    memory. Two different 512-set batches alternate, so each launch of the graph
    runs other buffers and sizes than the one before. Against the plain per-set
    path: each set's inputs up, partition_set with the same plan shape, its
    bucket lists back."""
    import torch

    from paper_0905_1744_gb300 import autotune, sad
    sets_a = datagen.config4(args.seed, n_sets=args.batch_sets)
    sets_b = datagen.config4(args.seed + 1, n_sets=args.batch_sets)
    st = torch.cuda.Stream(dev)
    ws = (sad.Workspace(dev, 256), sad.Workspace(dev), sad.Workspace(dev))
    ba = sad.Batch(sets_a, device=dev, workspaces=ws, stream=st)
    bb = sad.Batch(sets_b, device=dev, workspaces=ws, stream=st)
    shape, trials = autotune.choose_batch_shape(ba, use_cache=False, stream=st)
    g = sad.Graph()
    outs = {}
    for b in (ba, bb):
        outs[id(b)] = (torch.empty(b.members.shape, dtype=torch.int32).pin_memory(),
                       torch.empty(b.bucket_offsets.shape, dtype=torch.int32).pin_memory())

    def new_batch(b):
        b.upload(st)
        b.plan(depth=shape.depth, tile=shape.tile, budget=shape.budget, stream=st)
        b.capture(g, stream=st)
        g.launch(st)
        h_mem, h_boff = outs[id(b)]
        with torch.cuda.stream(st):
            h_mem.copy_(b.members, non_blocking=True)
            h_boff.copy_(b.bucket_offsets, non_blocking=True)

    for b in (ba, bb, ba, bb):
        new_batch(b)
        st.synchronize()
        b.check(st)
    torch.cuda.synchronize(dev)
    launches0 = sad.launch_count()
    dev_ms, wall_ms = [], []
    for r in range(args.batch_reps):
        b = ba if r % 2 == 0 else bb
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(st)
        new_batch(b)
        e1.record(st)
        st.synchronize()
        wall_ms.append(1e3 * (time.perf_counter() - t0))
        dev_ms.append(e0.elapsed_time(e1))
        b.check(st)
    launches = sad.launch_count() - launches0
    gstats = g.stats()
    ms = statistics.median(wall_ms)
    n_a = np.array([x.n for x in sets_a], dtype=np.int64)
    n_b = np.array([x.n for x in sets_b], dtype=np.int64)
    pairs = float(((n_a * (n_a - 1) // 2).sum() + (n_b * (n_b - 1) // 2).sum()) / 2)
    # plain per-set path on batch A: inputs up, the public per-set call, buckets back
    wsp = sad.Workspace(dev)
    h_sets = [(torch.from_numpy(x.codes).pin_memory(), torch.from_numpy(x.offsets).pin_memory(),
               x.p) for x in sets_a]

    def plain_one(c, o, p):
        res = sad.partition_set(c.to(dev, non_blocking=True), o.to(dev, non_blocking=True), p,
                                ws=wsp, depth=shape.depth, tile=shape.tile,
                                budget=shape.budget)
        return {k: res[k].cpu() for k in ("members", "bucket_offsets", "key_hi", "key_lo",
                                          "pivot_idx")}
    for c, o, p in h_sets[:4]:
        plain_one(c, o, p)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plain = [plain_one(c, o, p) for c, o, p in h_sets]
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    # batch A's results (its last run) against the plain per-set results
    new_batch(ba)
    st.synchronize()
    ba.check(st)
    exact = True
    for i in range(0, len(sets_a), max(1, len(sets_a) // 32)):
        got = ba.result(i)
        for key in ("key_hi", "key_lo", "bucket_offsets", "members", "pivot_idx"):
            exact &= bool(np.array_equal(got[key], plain[i][key].numpy()))
    h2d = (ba.h2d_bytes + bb.h2d_bytes) / 2
    d2h = sum(t.numel() * 4 for t in outs[id(ba)]) / 2 + sum(t.numel() * 4 for t in outs[id(bb)]) / 2
    return {
        "workload": f"{len(sets_a)} sets a batch, N log-uniform 50-5000, L log-uniform 50-2000, "
                    "5-100 families per set, p = ceil(N/500); two batches (seeds "
                    f"{args.seed}, {args.seed + 1}) alternate",
        "sets": len(sets_a), "sequences": int((n_a.sum() + n_b.sum()) // 2), "pairs": pairs,
        "ms_per_batch": ms, "device_ms_per_batch": statistics.median(dev_ms),
        "sets_per_s": len(sets_a) / (ms / 1e3), "pairs_per_s": pairs / (ms / 1e3),
        "plain_ms_per_batch": 1e3 * t_plain, "plain_sets_per_s": len(sets_a) / t_plain,
        "speedup_vs_plain": (t_plain * 1e3) / ms,
        "timing": "per new batch, host wall clock: pinned H2D of codes/offsets/sizes, bound "
                  "plan, graph capture + in-place update, graph launch, D2H of members and "
                  "bucket offsets, stream synchronize; plain: per set H2D, partition_set, D2H",
        "h2d_bytes_per_batch": int(h2d), "d2h_bytes_per_batch": int(d2h),
        "shape": shape._asdict(), "autotune_trial_ms": trials,
        "graph": gstats, "gpu_launches_per_batch": launches / max(args.batch_reps, 1),
        "rows": int(ba.plan_.rows_total), "tiles": int(ba.plan_.tiles_total),
        "exact_vs_plain": exact,
    }


def run_global(args, dev, counts, lengths, word_max, keys, p, reps: int = 10):
    """The globalised rank of Sec. 3.1.1 (Algorithm 2 steps 2-6) on the same set:
    local ranks of the p blocks, p - 1 regular samples per block, every sequence
    against the p (p - 1) samples; timed per run with CUDA events (L2 flushed
    between runs). Also how the buckets of the globalised partition compare with
    the centralised ones of the main step."""
    import torch

    from paper_0905_1744_gb300 import sad
    ks = max(p - 1, 1)
    g = sad.GlobalRank(counts, lengths, p, ks, word_max=word_max)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        g.run()
    g.check()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        g.run()
        e1.record(stream)
    torch.cuda.synchronize()
    g.check()
    ms = statistics.median([a.elapsed_time(b) for a, b in evs])
    n = counts.shape[0]
    offs_c, mem_c, _ = sad.partition(keys[0], keys[1], p)
    offs_g, mem_g, _ = sad.partition(g.key_hi, g.key_lo, p)
    bucket_c = torch.empty(n, dtype=torch.int64, device=dev)
    bucket_g = torch.empty(n, dtype=torch.int64, device=dev)
    for b in range(p):
        bucket_c[mem_c[int(offs_c[b]):int(offs_c[b + 1])].long()] = b
        bucket_g[mem_g[int(offs_g[b]):int(offs_g[b + 1])].long()] = b
    rc, rg = keys[2], g.rank
    return {"workload": f"same set, p = {p} blocks, {ks} samples per block "
                        f"({p * ks} references)",
            "ms_per_run": ms, "pairs": g.pairs(), "pairs_per_s": g.pairs() / (ms / 1e3),
            "rank_views": {"centralised": {"min": float(rc.min()), "max": float(rc.max()),
                                           "mean": float(rc.mean())},
                           "globalised": {"min": float(rg.min()), "max": float(rg.max()),
                                          "mean": float(rg.mean())},
                           "pearson": float(torch.corrcoef(torch.stack([rc, rg]))[0, 1])},
            "same_bucket_fraction": float((bucket_c == bucket_g).double().mean()),
            "max_bucket": int((offs_g[1:] - offs_g[:-1]).max())}


def run_distance(args, dev, counts, lengths, word_max, depth, reps: int = 5):
    """Eq. 2 / Eq. 3 as written (mean of -ln(1/b + F), b = 10) on the same set and
    plane depth: one plan, then timed kmer_rank_dist calls (CUDA events, L2
    flushed between runs)."""
    import torch

    from paper_0905_1744_gb300 import sad
    b = 10
    ws = sad.Workspace(dev)
    plan = sad.kmer_rank_plan(counts, depth=depth, ws=ws)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(2):
        out = sad.kmer_rank_dist(counts, lengths, b, plan=plan, word_max=word_max, ws=ws)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        out = sad.kmer_rank_dist(counts, lengths, b, plan=plan, word_max=word_max, ws=ws,
                                 check=False)
        e1.record(stream)
    torch.cuda.synchronize()
    ws.check("kmer_rank_dist")
    ms = statistics.median([a.elapsed_time(c) for a, c in evs])
    n = counts.shape[0]
    rank = out[3]
    return {"delta": f"1/{b}", "depth": depth, "ms_per_rank": ms,
            "pairs_per_s": n * (n - 1) / 2 / (ms / 1e3),
            "rank_nats": {"min": float(rank.min()), "max": float(rank.max()),
                          "mean": float(rank.mean())}}


def run_sparse(args, dev, counts, lengths, rank_ms, reps: int = 2):
    """The ablation of Table 2's per-pair cost: the same keys by sparse
    intersection on the CUDA cores (O(L) per pair, every ordered pair), timed
    with CUDA events on the same set, beside the plane-GEMM rank time."""
    import torch

    from paper_0905_1744_gb300 import sad
    ws = sad.Workspace(dev)
    entries = sad.sparse_entries(counts, lengths, ws=ws)
    sad.kmer_rank_sparse(counts, lengths, ws=ws, entries=entries)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for e0, e1 in evs:
        e0.record(stream)
        sad.kmer_rank_sparse(counts, lengths, ws=ws, entries=entries, check=False)
        e1.record(stream)
    torch.cuda.synchronize()
    ws.check("kmer_rank_sparse")
    ms = statistics.median([a.elapsed_time(b) for a, b in evs])
    n = counts.shape[0]
    return {"kind": "sparse intersection on CUDA cores (every ordered pair)",
            "list_entries": int(entries), "ms_per_rank": ms,
            "pairs_per_s": n * (n - 1) / 2 / (ms / 1e3),
            "plane_gemm_rank_ms": rank_ms,
            # the rank time comes from the depth trials (absent when --depth is given)
            "plane_gemm_speedup": ms / rank_ms if rank_ms else None}


def run_table1(args, dev, seed: int = 0):
    """A synthetic re-run of the comparison of Table 1 (Sec. 3.1.1): 500 sequences
    in 10 families, distance-form ranks (Delta = 1/10) against all sequences
    (centralised) and against 8 samples from each of 4 blocks (globalised)."""
    import torch

    from paper_0905_1744_gb300 import sad
    s = datagen.family_set(10, 50, lambda r: int(np.clip(r.normal(300, 100), 50, 1000)), p=4,
                           seed=seed, stream=41, name="table1")
    codes = torch.from_numpy(s.codes).to(dev)
    offsets = torch.from_numpy(s.offsets).to(dev)
    lengths = torch.from_numpy(s.lengths.astype(np.int32)).to(dev)
    word_max = torch.empty(8000, dtype=torch.int32, device=dev)
    counts = sad.kmer_count(codes, offsets, word_max=word_max)
    _, _, _, central = sad.kmer_rank_dist(counts, lengths, 10, word_max=word_max)
    g = sad.GlobalRank(counts, lengths, 4, 8, word_max=word_max, delta_den=10)
    g.run()
    g.check()
    c, gl = central.cpu().numpy(), g.rank.cpu().numpy()
    diff = gl - c
    return {"workload": "500 sequences in 10 families (ancestor L ~ N(300,100) clipped to "
                        "50-1000, 20-40% substitutions, 2% indels), k = 3, Delta = 1/10; "
                        "globalised: p = 4 blocks, 8 samples each",
            "central_max_min": [float(c.max()), float(c.min())],
            "central_mean": float(c.mean()),
            "global_max_min": [float(gl.max()), float(gl.min())],
            "global_mean": float(gl.mean()),
            "variance_wrt_central": float(np.mean(diff ** 2)),
            "std_wrt_central": float(np.sqrt(np.mean(diff ** 2))),
            "pearson": float(np.corrcoef(c, gl)[0, 1]),
            "spearman": float(np.corrcoef(np.argsort(np.argsort(c)),
                                          np.argsort(np.argsort(gl)))[0, 1])}


def run_serving(args, dev, shape=None):
    """Poisson arrivals of sets (N log-uniform 100-20000, p = 16) served with
    continuous batching under a 150 GB HBM budget (plan-free admission, one reusable
    graph per slot), and the same arrivals served one at a time with the plain
    per-set calls, both with the same plan shape (the batching autotuner's, on a
    batch of serving sets when none is given)."""
    import torch

    from paper_0905_1744_gb300 import autotune, sad, serve
    pool = datagen.many_sets("serve", range(args.serve_pool), args.seed)
    if shape is None:
        probe = sad.Batch(pool[:8], device=dev)
        shape, _ = autotune.choose_batch_shape(probe, use_cache=False)
        shape = tuple(shape)
        del probe
    total = args.serve_warmup + args.serve_requests
    arrivals = datagen.poisson_arrivals(total, args.serve_rate, args.seed)
    out = {"workload": f"Poisson arrivals at {args.serve_rate:g} sets/s, {args.serve_requests} "
                       f"timed after {args.serve_warmup} warm-up, request i is set i mod "
                       f"{len(pool)} of a pool of {len(pool)} distinct sets (N log-uniform "
                       "100-20000, L log-uniform 50-2000, p = 16)",
           "budget_gb": 150, "shape": dict(zip(("tile", "depth", "budget"), shape))}
    # the server warms its slots with the two largest sets of the pool (buffer pools,
    # workspaces and graphs sized before the clock starts)
    warm = sorted(pool, key=lambda x: int(x.offsets[-1] - x.offsets[0]))[-2:]
    out["warm"] = "each slot runs the pool's two largest sets (alone and together) first"
    st_mixed = {}
    mixed = serve.serve(serve.make_requests(pool, arrivals), shape=shape, device=dev,
                        stats=st_mixed, warm=warm)
    plain = serve.serve_plain(serve.make_requests(pool, arrivals), shape=shape, device=dev)
    out["continuous_batching"] = {**serve.latency_stats(mixed, args.serve_warmup), **st_mixed}
    out["plain_per_set"] = serve.latency_stats(plain, args.serve_warmup)
    pairs = np.array([r.seqset.n * (r.seqset.n - 1) / 2 for r in mixed[args.serve_warmup:]])
    out["offered_pairs_per_s"] = float(pairs.mean() * args.serve_rate)
    # capacity: a burst of requests all arriving at once (saturated server)
    burst = np.zeros(args.serve_burst)
    st_burst = {}
    mixed_b = serve.serve(serve.make_requests(pool, burst), shape=shape, device=dev,
                          stats=st_burst, warm=warm)
    plain_b = serve.serve_plain(serve.make_requests(pool, burst), shape=shape, device=dev)
    out["saturated"] = {
        "requests": int(args.serve_burst),
        "continuous_batching": {**serve.latency_stats(mixed_b), **st_burst},
        "plain_per_set": serve.latency_stats(plain_b),
    }
    out["saturated"]["sets_per_s_ratio"] = (out["saturated"]["continuous_batching"]["sets_per_s"]
                                            / out["saturated"]["plain_per_set"]["sets_per_s"])
    out["p50_ratio_vs_plain"] = (out["continuous_batching"]["p50_ms"]
                                 / out["plain_per_set"]["p50_ms"])
    out["exact_vs_plain"] = all(
        np.array_equal(a.result[k], b.result[k]) for a, b in zip(mixed + mixed_b, plain + plain_b)
        for k in ("bucket_offsets", "members", "key_hi", "key_lo"))
    torch.cuda.synchronize(dev)
    return out


def measure_config(cfg: int, args, dev, world: int, steps: int, warmup: int,
                   with_e2e: bool, with_cpu: bool, cpu_seconds: float) -> dict:
    """One config's step (kmer_count -> kmer_rank -> partition, inputs in HBM):
    autotuned plan, CUDA-event timing of `steps` steps after `warmup`, the plane
    GEMM's roofline, each call alone, the public API with host buffers (e2e) and
    the oracle on a bounded sample."""
    import torch
    import torch.distributed as dist

    from paper_0905_1744_gb300 import autotune, sad

    s = datagen.config(cfg, args.seed)
    if args.subset and args.subset < s.n:
        # every (n / subset)-th sequence: the same family and length mix, fewer members
        s = s.take(np.linspace(0, s.n - 1, args.subset).astype(np.int64))
    n, p = s.n, s.p
    pairs = n * (n - 1) / 2
    stream = torch.cuda.current_stream()

    codes = torch.from_numpy(s.codes).to(dev)
    offsets = torch.from_numpy(s.offsets).to(dev)
    lengths = torch.from_numpy(s.lengths.astype(np.int32)).to(dev)
    ws = sad.Workspace(dev)
    counts = torch.empty((n, 8000), dtype=torch.int32, device=dev)
    word_max = torch.empty(8000, dtype=torch.int32, device=dev)
    sad.kmer_count(codes, offsets, ws=ws, out=counts, word_max=word_max)
    # GEMM tile shape, plane depth and remainder budget chosen by the autotuner (timed
    # trials, outside the timed region)
    if args.depth is None:
        shape, trials = autotune.choose_shape(counts, lengths, ws, use_cache=False,
                                              word_max=word_max)
    else:
        shape, trials = autotune.Shape(args.tile, args.depth, args.budget), {}
    depth = shape.depth
    plan = autotune.plan_for(counts, shape, ws)
    keys = (torch.empty(n, dtype=torch.uint64, device=dev),
            torch.empty(n, dtype=torch.uint64, device=dev),
            torch.empty(n, dtype=torch.float64, device=dev))
    ws_part = sad.Workspace(dev, sad.workspace_bytes(sad.OP_PARTITION, n, p=p))
    part = (torch.empty(p + 1, dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.int32, device=dev),
            torch.empty(max(p - 1, 1), dtype=torch.int32, device=dev))

    def step():
        sad.kmer_count(codes, offsets, ws=ws, out=counts, check=False, word_max=word_max)
        sad.seq_lengths(offsets, out=lengths, ws=ws)
        sad.kmer_rank(counts, lengths, ws=ws, out=keys, check=False, plan=plan,
                      word_max=word_max)
        sad.partition(keys[0], keys[1], p, ws=ws_part, out=part, check=False)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 2x the 129 MB L2
    for _ in range(warmup):
        step()
    ws.check("warmup rank")
    ws_part.check("warmup partition")
    info = sad.rank_info(ws)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sad.launch_count()
    sad.profile(True)
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    sad.profile(False)
    launches = sad.launch_count() - launches0
    clocks = sampler.stop()
    gemm_ms, gemm_n = sad.profile_read()
    ws.check("timed rank")
    ws_part.check("timed partition")
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    ms_per_step = total_ms / steps
    value = job_value(pairs, world, ms_per_step / 1e3)

    # roofline of the plane GEMM (the dominant kernel)
    pk, pk_kind = peaks()
    # e2m1 dense = 6 x bf16 (nominal 13.5 / 2.25 PFLOP/s), applied to the measured bf16
    # peak. The burst figure: the timed loop is short and runs at the maximum SM clock
    # (see "clocks").
    f4_ratio = 13.5 / 2.25
    f4_peak = f4_ratio * pk["bf16_tflops"]
    gemm_launch_ms = gemm_ms / max(gemm_n, 1)
    useful_flops = 2.0 * 8000 * pairs                    # Eq. 1 as written: 2 eps per pair
    # MMA work actually issued: K chunks of 256 plane columns over tile x tile tiles
    exec_flops = 2.0 * shape.tile * shape.tile * 256 * info["k_chunks"]
    achieved = useful_flops / (gemm_launch_ms / 1e3) / 1e12
    kernel = ("pair_gemm_kernel (CTA pairs, tcgen05.mma.cta_group::2 kind::mxf4nvf4, 256 x 256 "
              "tiles" if shape.tile == 256 else
              "plane_gemm_kernel (tcgen05.mma kind::mxf4nvf4, 128 x 128 tiles")
    roofline = {
        "bound": "tensor",
        "kernel": kernel + ", e2m1 0/1 planes, unit scales)",
        "achieved": achieved, "peak": f4_peak, "unit": "TFLOP/s", "frac": achieved / f4_peak,
        "work": "Eq. 1 as written: 2 x 8000 ops (min and add over the 8000 words) per "
                "unordered pair, N(N-1)/2 pairs per launch",
        "peak_source": f"{pk_kind}: 6 x bf16_tflops burst (e2m1/bf16 nominal ratio "
                       f"13.5/2.25); sustained would be "
                       f"{f4_ratio * pk['bf16_tflops_sustained']:.1f}",
        "traffic": gemm_traffic_per_launch(n, shape.tile, shape.depth, shape.budget),
        "gemm_ms_per_launch": gemm_launch_ms, "gemm_share_of_step": gemm_launch_ms / ms_per_step,
        "executed_tflops": exec_flops / (gemm_launch_ms / 1e3) / 1e12,
        "executed_frac": exec_flops / (gemm_launch_ms / 1e3) / 1e12 / f4_peak,
        "plan": {k: info[k] for k in ("k_eff", "k_pad", "t_max", "tiles", "k_chunks", "depth",
                                      "rem_entries", "rem_blocks", "heavy_entries", "bm_cols")},
    }

    # each call of the step alone (a2 count: HBM-bound; a7-a10 partition: latency-bound)
    call_ms = time_calls(
        {"kmer_count": lambda: sad.kmer_count(codes, offsets, ws=ws, out=counts, check=False,
                                              word_max=word_max),
         "kmer_rank": lambda: sad.kmer_rank(counts, lengths, ws=ws, out=keys, check=False,
                                            plan=plan, word_max=word_max),
         "partition": lambda: sad.partition(keys[0], keys[1], p, ws=ws_part, out=part,
                                            check=False)},
        reps=max(3, min(steps, 10)), flush=flush.zero_, stream=stream,
        event_cls=torch.cuda.Event)
    ws.check("per-call timing")
    ws_part.check("per-call timing")
    # codes and offsets read, counts [N][8000] and the per-word maxima written
    count_bytes = int(s.codes.nbytes + s.offsets.nbytes + 4 * 8000 * n + 4 * 8000)
    count_gbs = count_bytes / (call_ms["kmer_count"] / 1e3) / 1e9
    calls = {
        "kmer_count": {"ms": call_ms["kmer_count"], "algorithmic_bytes": count_bytes,
                       "gbs": count_gbs, "hbm_peak_gbs": pk["hbm_gbs"],
                       "frac": count_gbs / pk["hbm_gbs"], "peak_source": pk_kind},
        "kmer_rank": {"ms": call_ms["kmer_rank"], "depth": info["depth"]},
        "partition": {"ms": call_ms["partition"], "p": p},
        "timing": "median of alone-runs, L2 flushed before each, CUDA events on the stream",
    }

    # end to end through the public API, host buffers, H2D/D2H inside the timed region
    e2e = None
    if with_e2e:
        h_codes = torch.from_numpy(s.codes).pin_memory()
        h_offs = torch.from_numpy(s.offsets).pin_memory()
        h_mem = torch.empty(n, dtype=torch.int32).pin_memory()
        h_boff = torch.empty(p + 1, dtype=torch.int32).pin_memory()
        h_hi = torch.empty(n, dtype=torch.uint64).pin_memory()
        h_lo = torch.empty(n, dtype=torch.uint64).pin_memory()
        ws_e = sad.Workspace(dev)

        def e2e_step():
            d_codes = h_codes.to(dev, non_blocking=True)
            d_offs = h_offs.to(dev, non_blocking=True)
            res = sad.partition_set(d_codes, d_offs, p, ws=ws_e, depth=shape.depth,
                                    tile=shape.tile, budget=shape.budget)
            h_mem.copy_(res["members"], non_blocking=True)
            h_boff.copy_(res["bucket_offsets"], non_blocking=True)
            h_hi.copy_(res["key_hi"], non_blocking=True)
            h_lo.copy_(res["key_lo"], non_blocking=True)
            torch.cuda.synchronize()

        for _ in range(2):
            e2e_step()
        reps = max(3, min(steps, 20))
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            e2e_step()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / reps, world, dev)
        e2e = {"value": job_value(pairs, world, t_e2e), "unit": "pairs/s",
               "h2d_bytes_per_step": int(s.codes.nbytes + s.offsets.nbytes),
               "d2h_bytes_per_step": int(4 * n + 4 * (p + 1) + 16 * n),
               "ms_per_step": 1e3 * t_e2e}

    cpu = None
    if with_cpu:
        v, r, t, threads = oracle_sample(s, cpu_seconds, seed=args.seed)
        cpu = {"value": v, "unit": "pairs/s", "cores": threads, "kind": "oracle",
               "sample": f"{r} random rows against all {n} sequences "
                         f"({r} x {n - 1} / 2 pair-equivalents) in {t:.1f} s",
               "cpu": cpu_model()}

    return {"s": s, "value": value, "ms_per_step": ms_per_step, "steps": steps,
            "warmup": warmup, "launches": int(launches), "clocks": clocks,
            "autotune": {"shape": shape._asdict(), "trial_ms": trials,
                         "searched": "tile {256, 128} x depth {0,1,2,3,4,6} at the default "
                                     "budget, then budgets {256, 1536} at the best, then the "
                                     "three fastest twice more in turn; trial_ms = medians"},
            "roofline": roofline, "calls": calls, "e2e": e2e, "cpu_baseline": cpu,
            "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
            "tensors": (counts, lengths, word_max, keys, shape, trials)}


def extra_line(m: dict) -> dict:
    """A secondary config's figures, in the main line's vocabulary."""
    return {"N": m["s"].n, "p": m["s"].p, "value": m["value"], "unit": "pairs/s",
            "ms_per_step": m["ms_per_step"], "steps": m["steps"], "warmup": m["warmup"],
            "autotune": m["autotune"], "roofline": m["roofline"], "calls": m["calls"],
            "e2e": m["e2e"], "cpu_baseline": m["cpu_baseline"], "clocks": m["clocks"]}


def run_sad(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    cpu_ok = rank == 0 and world == 1 and not args.no_cpu_baseline

    main = measure_config(args.config, args, dev, world, args.steps, args.warmup,
                          with_e2e=not args.no_e2e, with_cpu=cpu_ok,
                          cpu_seconds=args.cpu_seconds)
    extras = {}
    side = None
    if not args.no_extra_configs and world == 1:
        for c in (1, 2, 3):
            if c == args.config:
                continue
            m = measure_config(c, args, dev, world, min(args.steps, 20), 3, with_e2e=True,
                               with_cpu=cpu_ok, cpu_seconds=min(args.cpu_seconds, 8.0))
            extras[f"c{c}"] = {"workload": WORKLOADS[c], **extra_line(m)}
            if c == 2:
                side = m
    if side is None and args.config == 2:
        side = main

    globalised = distance = table1 = sparse = None
    if not args.no_global and world == 1 and side is not None:
        counts, lengths, word_max, keys, shape2, trials2 = side["tensors"]
        p2 = side["s"].p
        globalised = run_global(args, dev, counts, lengths, word_max, keys, p2)
        distance = run_distance(args, dev, counts, lengths, word_max, shape2.depth)
        sparse = run_sparse(args, dev, counts, lengths, trials2.get(shape2.key))
        table1 = run_table1(args, dev, args.seed)
        for leg in (globalised, distance, sparse):
            leg["on"] = "the paper-scale set: " + WORKLOADS[2]
    batching = None
    if not args.no_batching:
        batching = run_batching(args, dev)
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(args, dev)

    if rank == 0:
        s = main["s"]
        out = {
            "metric": "k-mer pair comparisons/s", "value": main["value"], "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e2m1 0/1 planes (fp4), f32 acc (exact), u128 keys",
            "data": "synthetic",
            "config": {**bench_config(args.config, s, args.seed),
                       **({"subset": args.subset} if args.subset else {})},
            "parallelism": "replicas" if world > 1 else "single GPU",
            "gpu_launches": main["launches"],
            "autotune": main["autotune"],
            "roofline": main["roofline"],
            "calls": main["calls"],
            "cpu_baseline": main["cpu_baseline"],
            "e2e": main["e2e"],
            "clocks": main["clocks"],
            "configs": extras,
            "globalised": globalised,
            "distance_form": distance,
            "table1_synthetic": table1,
            "sparse_ablation": sparse,
            "batching": batching,
            "serving": serving,
            "step_ms_min": main["step_ms_min"], "step_ms_median": main["step_ms_median"],
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_sad(args)


if __name__ == "__main__":
    main()
