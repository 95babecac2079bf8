"""Autotuner for kmer_rank: picks the threshold-plane depth by timing.

At depth D the tensor-core GEMM runs over the first D threshold sections only
(K = sum_{t<=D} #{words with T_word >= t}) and the counts above D are added back
exactly by the sparse residual step, whose cost grows with the number of pairs
of sequences that share a word more than D times. Which D is fastest depends on
the set (its size, its repeat structure), so each candidate is timed on the
device with CUDA events and the fastest kept. Results are cached per size class
(log2 N, t_max, log2 of the remainder bound at depth 1) in memory and, if a path
is given, in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

import torch

from . import sad

CANDIDATES = (0, 1, 2, 3, 4, 6)
_cache: dict[str, int] = {}
_lock = threading.Lock()


def _bucket(x: int) -> int:
    return 0 if x <= 0 else int(math.log2(x))


def signature(n: int, plan1: "sad.RankPlan") -> str:
    return f"n{_bucket(n)}_t{plan1.t_max}_r{_bucket(plan1.rem_bound)}"


def load_cache(path: str | None):
    if path and os.path.exists(path):
        with open(path) as f:
            with _lock:
                _cache.update(json.load(f))


def save_cache(path: str | None):
    if path:
        tmp = path + f".tmp{os.getpid()}"
        with _lock:
            data = dict(_cache)
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def time_rank(counts, lengths, plan, ws, k=3, alphabet=20, reps=3, stream=None,
              word_max=None) -> float:
    """Median milliseconds of kmer_rank with this plan (CUDA events)."""
    s = stream or torch.cuda.current_stream()
    n = counts.shape[0]
    out = (torch.empty(n, dtype=torch.uint64, device=counts.device),
           torch.empty(n, dtype=torch.uint64, device=counts.device), None)
    sad.kmer_rank(counts, lengths, k, alphabet, ws=ws, plan=plan, out=out, stream=s,
                  word_max=word_max)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sad.kmer_rank(counts, lengths, k, alphabet, ws=ws, plan=plan, out=out, stream=s,
                      check=False, word_max=word_max)
        e1.record(s)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ws.check("autotune kmer_rank", s)
    return statistics.median(times)


def choose_depth(counts, lengths, ws=None, k=3, alphabet=20, candidates=CANDIDATES, reps=3,
                 max_ws_bytes: int | None = None, use_cache=True, stream=None, word_max=None):
    """Fastest plane depth for this set: (depth, {depth: ms})."""
    n = counts.shape[0]
    ws = ws or sad.Workspace(counts.device)
    plan1 = sad.kmer_rank_plan(counts, k, alphabet, 1, ws, stream)
    key = signature(n, plan1)
    if use_cache:
        with _lock:
            if key in _cache:
                return _cache[key], {}
    trials = {}
    for d in candidates:
        plan = sad.kmer_rank_plan(counts, k, alphabet, d, ws, stream)
        if d > 0 and d >= plan.t_max:
            continue                                     # same as keeping every plane
        if max_ws_bytes is not None and plan.ws_bytes > max_ws_bytes:
            continue
        ws.ensure(plan.ws_bytes)
        trials[d] = time_rank(counts, lengths, plan, ws, k, alphabet, reps, stream, word_max)
    best = min(trials, key=trials.get)
    with _lock:
        _cache[key] = best
    return best, trials
