"""Autotuner for the rank's GEMM: tile shape, threshold-plane depth and remainder budget.

A rank plan has three knobs that change speed and never the keys:
  tile    GEMM tile rows: 128 (one CTA per 128 x 128 tile) or 256 (a CTA pair per
          256 x 256 tile, tcgen05 cta_group::2: half the operand bytes per MAC,
          twice the padding of a small set);
  depth   threshold planes kept as tensor-core K columns (0 = all of them); the
          thresholds above the depth of a column block are added back exactly as
          remainder chunks and heavy entries;
  budget  remainder entries per column block that the per-block depth rule aims at
          (0 = the library's default).
Which combination is fastest depends on the set (its size, its repeat structure,
the mix of set sizes in a batch), so candidates are timed on the device with CUDA
events: first every (tile, depth) at the default budget, then the other budgets at
the best (tile, depth), then the three fastest again, side by side; the shape with the
smallest median is kept. Results are cached per size class in memory and, if a path
is given, in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading
from typing import Callable, NamedTuple

import torch

from . import sad


class Shape(NamedTuple):
    tile: int
    depth: int
    budget: int

    @property
    def key(self) -> str:
        return f"t{self.tile}_d{self.depth}_b{self.budget}"

    @classmethod
    def parse(cls, key: str) -> "Shape":
        t, d, b = key.split("_")
        return cls(int(t[1:]), int(d[1:]), int(b[1:]))


TILES = (256, 128)
DEPTHS = (0, 1, 2, 3, 4, 6)
BUDGETS = (256, 1536)          # tried at the best (tile, depth) besides the default 0
_cache: dict[str, str] = {}
_lock = threading.Lock()


def _bucket(x: int) -> int:
    return 0 if x <= 0 else int(math.log2(x))


def first_round(t_max: int | None, tiles=TILES, depths=DEPTHS, min_depth: int = 0):
    """(tile, depth) candidates at the default budget. A depth at or above the
    largest count keeps every plane (the same plan as depth 0) and is skipped."""
    out = []
    for t in tiles:
        for d in depths:
            if d < min_depth:
                continue
            if d > 0 and t_max is not None and t_max > 0 and d >= t_max:
                continue
            out.append(Shape(t, d, 0))
    return out


def search(timer: Callable[[Shape], float | None], first: list[Shape],
           budgets=BUDGETS, confirm: int = 3, rounds: int = 2) -> tuple[Shape, dict[str, float]]:
    """Times every shape of ``first``, then the other budgets at the best one
    (when it cuts planes: depth >= 1), then the ``confirm`` fastest shapes again,
    ``rounds`` times in turn (single timings taken minutes apart in a long search
    can favour a shape that happened to run at a better moment; the re-timings
    compare the finalists side by side). ``timer`` returns milliseconds, or None for
    a shape that does not apply (too large a workspace). Returns the shape with the
    smallest median over its timings, and that median for every shape tried."""
    times: dict[str, list[float]] = {}

    def run(sh: Shape):
        ms = timer(sh)
        if ms is not None:
            times.setdefault(sh.key, []).append(ms)

    for sh in first:
        run(sh)
    if not times:
        raise RuntimeError("autotune: no candidate shape could run")
    best = Shape.parse(min(times, key=lambda k: times[k][0]))
    if best.depth >= 1:
        for b in budgets:
            sh = Shape(best.tile, best.depth, b)
            if sh.key not in times:
                run(sh)
    finalists = sorted(times, key=lambda k: times[k][0])[:confirm]
    if len(finalists) > 1:
        for _ in range(rounds):
            for k in finalists:
                run(Shape.parse(k))
    trials = {k: statistics.median(v) for k, v in times.items()}
    return Shape.parse(min(trials, key=trials.get)), trials


def load_cache(path: str | None):
    if path and os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
        with _lock:
            _cache.update({k: v for k, v in data.items() if isinstance(v, str)})


def save_cache(path: str | None):
    if path:
        tmp = path + f".tmp{os.getpid()}"
        with _lock:
            data = dict(_cache)
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _events_ms(fn, stream, reps: int) -> float:
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def signature(n: int, plan1: "sad.RankPlan") -> str:
    """Size class of one set: log2 N, the largest count, log2 of the remainder
    bound at depth 1."""
    return f"n{_bucket(n)}_t{plan1.t_max}_r{_bucket(plan1.rem_bound)}"


def plan_for(counts, shape: Shape, ws, k: int = 3, alphabet: int = 20, stream=None):
    plan = sad.kmer_rank_plan(counts, k, alphabet, shape.depth, ws, stream, budget=shape.budget,
                              tile=shape.tile)
    ws.ensure(plan.ws_bytes)
    return plan


def time_rank(counts, lengths, plan, ws, k=3, alphabet=20, reps=3, stream=None,
              word_max=None) -> float:
    """Median milliseconds of kmer_rank with this plan (CUDA events, after one
    untimed run)."""
    s = stream or torch.cuda.current_stream()
    n = counts.shape[0]
    out = (torch.empty(n, dtype=torch.uint64, device=counts.device),
           torch.empty(n, dtype=torch.uint64, device=counts.device), None)

    def once(check=False):
        sad.kmer_rank(counts, lengths, k, alphabet, ws=ws, plan=plan, out=out, stream=s,
                      check=check, word_max=word_max)
    once(check=True)
    ms = _events_ms(once, s, reps)
    ws.check("autotune kmer_rank", s)
    return ms


def choose_shape(counts, lengths, ws=None, k=3, alphabet=20, reps=3,
                 max_ws_bytes: int | None = None, use_cache=True, stream=None, word_max=None,
                 tiles=TILES, depths=DEPTHS):
    """Fastest (tile, depth, budget) for this set: (Shape, {shape key: ms})."""
    n = counts.shape[0]
    ws = ws or sad.Workspace(counts.device)
    plan1 = sad.kmer_rank_plan(counts, k, alphabet, 1, ws, stream)
    key = "set_" + signature(n, plan1)
    if use_cache:
        with _lock:
            if key in _cache:
                return Shape.parse(_cache[key]), {}

    def timer(sh: Shape):
        plan = sad.kmer_rank_plan(counts, k, alphabet, sh.depth, ws, stream, budget=sh.budget,
                                  tile=sh.tile)
        if max_ws_bytes is not None and plan.ws_bytes > max_ws_bytes:
            return None
        ws.ensure(plan.ws_bytes)
        return time_rank(counts, lengths, plan, ws, k, alphabet, reps, stream, word_max)

    best, trials = search(timer, first_round(plan1.t_max, tiles, depths))
    with _lock:
        _cache[key] = best.key
    return best, trials


def batch_signature(batch) -> str:
    """Size class of a batch: log2 of its sets, sequences and residues."""
    return (f"batch_s{_bucket(batch.n_sets)}_n{_bucket(int(batch.n.sum()))}"
            f"_l{_bucket(batch.total_len)}")


def choose_batch_shape(batch, reps=2, use_cache=True, stream=None, tiles=TILES,
                       depths=DEPTHS, max_ws_bytes: int | None = None):
    """Fastest (tile, depth, budget) for a batch on plans from host-side bounds
    (depth >= 1, the plan-free path a captured graph runs): each candidate times
    the whole batch (count, lengths, rank, partition). Returns (Shape, trials); the
    batch is left planned with the chosen shape."""
    key = batch_signature(batch)
    s = stream or torch.cuda.current_stream(batch.device)
    if use_cache:
        with _lock:
            hit = _cache.get(key)
        if hit is not None:
            best = Shape.parse(hit)
            batch.plan(depth=best.depth, tile=best.tile, budget=best.budget, stream=s)
            return best, {}

    def timer(sh: Shape):
        plan = batch.plan(depth=sh.depth, tile=sh.tile, budget=sh.budget, stream=s)
        if max_ws_bytes is not None and plan.rank.ws_bytes > max_ws_bytes:
            return None
        batch.run(stream=s)
        batch.check(s)
        ms = _events_ms(lambda: batch.run(stream=s), s, reps)
        batch.check(s)
        return ms

    best, trials = search(timer, first_round(None, tiles, depths, min_depth=1))
    batch.plan(depth=best.depth, tile=best.tile, budget=best.budget, stream=s)
    with _lock:
        _cache[key] = best.key
    return best, trials
