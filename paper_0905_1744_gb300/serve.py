"""Serving: continuous batching of sequence-set requests on one GPU.

Requests (one sequence set each, host memory) arrive over time. The server keeps
up to ``slots`` batches in flight, each on its own CUDA stream with its own
reusable CUDA graph. Whenever a slot is free, every request that has arrived and
fits the HBM budget is admitted and launched as one batch (count -> lengths ->
block-diagonal rank -> batched partition, see ``sad.Batch``) without any host
synchronisation: the inputs go up from pinned memory, the plan comes from
host-side bounds (``sad_batch_plan_bound``), the launches are captured into the
slot's graph (which is updated in place, not re-instantiated, from one batch to
the next) and the graph is launched; the bucket lists come back into pinned
memory on the same stream. A batch's device state (codes, counts, planes, keys,
buckets) lives until its results are on the host, and then its memory returns to
the budget. Requests that arrive while batches run wait for the next free slot,
and batches in flight on different streams overlap on the device. Latency = time
the results are on the host - arrival time.

The baseline (``serve_plain``) takes the same requests one at a time in arrival
order and runs the plain per-set calls for each.
"""
from __future__ import annotations

import dataclasses
import queue as _queue
import threading
import time

import numpy as np
import torch

from . import sad

GB = 1 << 30
DEFAULT_SHAPE = (256, 2, 0)     # (tile, depth >= 1, budget) when none is given


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    seqset: object          # datagen.SeqSet-like: codes, offsets, p
    done: float = -1.0
    result: dict | None = None
    nbytes: int = -1        # admission estimate (request_bytes), computed once


def request_bytes(s, depth: int, k: int = 3, alphabet: int = 20, tile: int = 256,
                  budget: int = 0) -> int:
    """HBM a request holds while it is in flight, for admission: codes, offsets,
    lengths, counts, the rank workspace of its plan from host-side bounds
    (kmer_rank_plan_bound: planes of ``depth`` sections, remainder and heavy lists
    sized by its k-mer windows; a batch's bound plan is at most the sum of its
    sets'), keys, ranks, partition buffers, and 64 MB of slack."""
    n = s.offsets.shape[0] - 1
    total_len = int(s.offsets[-1] - s.offsets[0])
    eps = alphabet ** k
    plan = sad.kmer_rank_plan_bound(n, total_len, k, alphabet, depth=max(depth, 1),
                                    budget=budget, tile=tile)
    part = sad.workspace_bytes(sad.OP_PARTITION, n, p=max(int(getattr(s, "p", 1)), 1))
    return int(total_len + 12 * (n + 1) + 4 * n * eps + plan.ws_bytes + part + 40 * n
               + (64 << 20))


def select_batch(queue, used: int, budget_bytes: int, max_batch: int, depth: int,
                 tile: int = 256, budget: int = 0):
    """The next batch to admit: the longest prefix of the arrival-ordered queue
    (at most max_batch requests) whose bytes fit beside the ``used`` bytes of the
    batches in flight. Returns (requests, bytes); empty when the head of the queue
    does not fit yet (it is never overtaken, so admission stays in arrival order)."""
    take, nbytes = [], 0
    for r in queue:
        if r.nbytes < 0:
            r.nbytes = request_bytes(r.seqset, depth, tile=tile, budget=budget)
        rb = r.nbytes
        if len(take) >= max_batch or used + nbytes + rb > budget_bytes:
            break
        take.append(r)
        nbytes += rb
    return take, nbytes


class _Slot:
    """One in-flight position: a stream, a reusable graph, (with ws_pool) a buffer
    pool its batches are built on, and (while busy) a batch."""

    def __init__(self, device, ws_pool: bool):
        self.stream = torch.cuda.Stream(device)
        self.graph = sad.Graph()
        self.pool = sad.BatchPool(device) if ws_pool else None
        self.reqs = self.batch = self.host = self.event = None
        self.ev0 = self.ev1 = None
        self.nbytes = 0


def _launch(slot: _Slot, reqs, shape, device, graph: bool = True):
    """Admit a batch on a free slot without synchronising the host: pinned H2D,
    plan from bounds, capture into the slot's graph (an update after the first
    batch), launch, D2H of the bucket lists, keys and status words into pinned
    memory."""
    tile, depth, budget = shape
    st = slot.stream
    pool = slot.pool

    def pinned(name, like, dtype):
        n = like.numel()
        if pool is not None:
            return pool.get(name, n, dtype, pinned=True)
        return torch.empty(n, dtype=dtype, pin_memory=True)
    with torch.cuda.stream(st):
        slot.ev0 = torch.cuda.Event(enable_timing=True)
        slot.ev0.record(st)
        if pool is not None:
            for ws in pool.workspaces:    # a pooled workspace starts each batch with no status
                ws.clear_status()         # (one not allocated yet is cleared when it is)
        if len(reqs) == 1 and pool is not None:
            # one request: the single-set calls, queued on the slot's stream at once
            b = _Single(reqs[0].seqset, pool, st, shape, device)
        else:
            # the count starts on the device as soon as the inputs are up, while the
            # host sets up the rest of the batch, plans it and builds the graph
            b = sad.Batch([r.seqset for r in reqs], device=device, stream=st, pool=pool,
                          count=True)
            b.plan(depth=depth, tile=tile, budget=budget, stream=st, bound=True)
            if graph:
                b.capture(slot.graph, stream=st, count=False)
                slot.graph.launch(st)
            else:
                b.run(stream=st, count=False)
        host = dict(bucket_offsets=pinned("r_boff", b.bucket_offsets, torch.int32),
                    members=pinned("r_members", b.members, torch.int32),
                    key_hi=pinned("r_key_hi", b.key_hi, torch.uint64),
                    key_lo=pinned("r_key_lo", b.key_lo, torch.uint64))
        for key, h in host.items():
            h.copy_(getattr(b, key), non_blocking=True)
        # the three workspaces' status words come back with the results: no
        # synchronous status read when the batch completes
        status = pinned("r_status", torch.empty(3), torch.int32)
        for i, ws in enumerate((b.ws_count, b.ws_rank, b.ws_part)):
            status[i:i + 1].copy_(ws.buf[:4].view(torch.int32), non_blocking=True)
        host["status"] = status
        slot.ev1 = torch.cuda.Event(enable_timing=True)
        slot.ev1.record(st)
    slot.reqs, slot.batch, slot.host, slot.event = reqs, b, host, slot.ev1


class _Single:
    """The device buffers and plan of a one-request batch on a slot (the single-set
    calls), shaped like a Batch for _finish."""

    def __init__(self, s, pool, st, shape, device, k: int = 3, alphabet: int = 20):
        import numpy as np
        tile, depth, budget = shape
        a, z = int(s.offsets[0]), int(s.offsets[-1])
        n, L, eps = s.offsets.shape[0] - 1, z - a, alphabet ** k
        self.seq_begin = np.array([0, n], dtype=np.int64)
        self.boff_begin = np.array([0, s.p + 1], dtype=np.int64)
        h_codes = pool.get("h_codes", max(L, 1), torch.uint8, pinned=True)
        h_offs = pool.get("h_offsets", n + 1, torch.int64, pinned=True)
        h_codes.numpy()[:L] = s.codes[a:z]
        np.subtract(s.offsets, a, out=h_offs.numpy())
        codes = pool.get("codes", max(L, 1), torch.uint8)
        offs = pool.get("offsets", n + 1, torch.int64)
        codes[:L].copy_(h_codes[:L], non_blocking=True)
        offs.copy_(h_offs, non_blocking=True)
        self.ws_count, self.ws_rank, self.ws_part = pool.workspaces
        counts = pool.get("counts", n * eps, torch.int32).view(n, eps)
        wm = pool.get("word_max", eps, torch.int32)
        sad.kmer_count(codes, offs, k, alphabet, ws=self.ws_count, out=counts, stream=st,
                       check=False, word_max=wm)
        lengths = sad.seq_lengths(offs, out=pool.get("lengths", n, torch.int32),
                                  ws=self.ws_count, stream=st)
        plan = sad.kmer_rank_plan_bound(n, L, k, alphabet, depth=depth, budget=budget, tile=tile)
        self.ws_rank.ensure(plan.ws_bytes)
        self.key_hi = pool.get("key_hi", n, torch.uint64)
        self.key_lo = pool.get("key_lo", n, torch.uint64)
        rank = pool.get("rank", n, torch.float64)
        sad.kmer_rank(counts, lengths, k, alphabet, ws=self.ws_rank, plan=plan,
                      out=(self.key_hi, self.key_lo, rank), stream=st, check=False, word_max=wm)
        self.bucket_offsets = pool.get("bucket_offsets", s.p + 1, torch.int32)
        self.members = pool.get("members", n, torch.int32)
        piv = pool.get("pivot_idx", max(s.p - 1, 1), torch.int32)
        sad.partition(self.key_hi, self.key_lo, s.p, ws=self.ws_part,
                      out=(self.bucket_offsets, self.members, piv), stream=st, check=False)

    def check(self, stream=None):
        self.ws_count.check("kmer_count", stream)
        self.ws_rank.check("kmer_rank", stream)
        self.ws_part.check("partition", stream)


def _finish(slot: _Slot, now: float):
    b = slot.batch
    for where, st in zip(("kmer_count (batch)", "sad_batch_rank", "sad_batch_partition"),
                         slot.host["status"].tolist()):
        if st != 0:
            b.check(slot.stream)       # raises with the status's message
            raise sad.SadError(st, where)
    for i, r in enumerate(slot.reqs):
        a, e = int(b.seq_begin[i]), int(b.seq_begin[i + 1])
        oa, ob = int(b.boff_begin[i]), int(b.boff_begin[i + 1])
        r.result = dict(bucket_offsets=slot.host["bucket_offsets"][oa:ob].numpy().copy(),
                        members=slot.host["members"][a:e].numpy().copy(),
                        key_hi=slot.host["key_hi"][a:e].numpy().copy(),
                        key_lo=slot.host["key_lo"][a:e].numpy().copy())
        r.done = now


def max_overlap(intervals) -> int:
    """Largest number of (start, end) intervals open at one time."""
    ev = sorted([(a, 1) for a, _ in intervals] + [(b, -1) for _, b in intervals],
                key=lambda x: (x[0], x[1]))
    best = cur = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def serve(requests, shape=DEFAULT_SHAPE, budget_bytes: int = 150 * GB, slots: int = 3,
          max_batch: int = 64, device=None, t0: float | None = None, stats: dict | None = None,
          ws_pool: bool = True, graph: bool = True, warm=None):
    """Continuous batching over ``requests`` (sorted by arrival). Returns them with
    ``done`` and ``result`` filled in. Arrival times are honoured in real time.
    ``shape``: (tile, depth >= 1, budget) of every batch's rank plan. ``stats``
    (a dict) receives the batches, the most batches in flight on the host and on
    the device at once (from each batch's start and end events on its stream),
    the most HBM bytes admitted at once, and the slots' graph updates and
    instantiations. ``ws_pool``: each slot keeps its three workspaces across
    batches (they grow to the largest batch the slot has run and stay allocated;
    the admission estimate of a request includes its workspace, so the bytes a
    slot keeps between batches are at most one earlier request's estimate and lie
    outside the budget). ``graph``: launch each batch through the slot's reusable
    graph (else the same calls are launched directly on the slot's stream).
    ``warm``: sequence sets that every slot runs once before the clock starts, alone
    and (two or more) together, so that its buffer pool, workspaces and graphs are
    sized and instantiated for them; a server warms with its largest expected
    requests so that no large allocation falls inside a request's latency."""
    tile, depth, budget = shape
    if slots < 1 or max_batch < 1:
        raise ValueError("serve: slots and max_batch must be at least 1")
    if depth < 1:
        raise ValueError("serve: the plan-free path needs depth >= 1")
    for r in requests:
        need = request_bytes(r.seqset, depth, tile=tile, budget=budget)
        if need > budget_bytes:
            # it could never be admitted, and the loop below would wait for it forever
            raise ValueError(f"serve: request {r.rid} needs {need} bytes, above the "
                             f"{budget_bytes}-byte budget")
    device = torch.device(device or "cuda")
    all_slots = [_Slot(device, ws_pool) for _ in range(slots)]
    free = list(all_slots)
    busy: list[_Slot] = []
    pending = list(requests)
    queue: list[Request] = []
    used = peak_used = peak_busy = 0
    done_ev = []
    base = torch.cuda.Event(enable_timing=True)
    base.record(torch.cuda.current_stream(device))
    n_batches = 0
    # One waiter thread per slot blocks on its batch's completion event, copies the
    # results out and wakes the admission loop, which otherwise sleeps until the
    # next arrival: completions are seen as they happen, not at a polling tick.
    cond = threading.Condition()
    completed: list[_Slot] = []

    def waiter(sl: _Slot):
        while True:
            ev = sl.jobs.get()
            if ev is None:
                return
            try:
                ev.synchronize()
                _finish(sl, time.perf_counter() - start)
            except BaseException as e:  # re-raised by the admission loop
                sl.error = e
            with cond:
                completed.append(sl)
                cond.notify()

    if warm:
        # each slot once with the largest warm set alone, once with all of them
        big = max(warm, key=lambda x: int(x.offsets[-1] - x.offsets[0]))
        for sl in all_slots:
            for group in ([big], list(warm)) if len(warm) > 1 else ([big],):
                _launch(sl, [Request(-1, 0.0, x) for x in group], shape, device, graph)
                sl.event.synchronize()
                _finish(sl, 0.0)
                sl.batch = sl.host = sl.reqs = None
        torch.cuda.synchronize(device)
    start = time.perf_counter() if t0 is None else t0
    for sl in all_slots:
        sl.jobs, sl.error = _queue.SimpleQueue(), None
        sl.thread = threading.Thread(target=waiter, args=(sl,), daemon=True)
        sl.thread.start()
    try:
        while pending or queue or busy:
            now = time.perf_counter() - start
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            # completions
            with cond:
                done, completed[:] = list(completed), []
            for sl in done:
                if sl.error is not None:
                    raise sl.error
                done_ev.append((sl.ev0, sl.ev1))
                busy.remove(sl)
                free.append(sl)
                used -= sl.nbytes
                sl.batch = sl.host = sl.reqs = None
            # admissions: everything queued that fits, one batch per free slot
            while queue and free:
                take, nbytes = select_batch(queue, used, budget_bytes, max_batch, depth, tile,
                                            budget)
                if not take:
                    break
                queue = queue[len(take):]
                sl = free.pop(0)
                _launch(sl, take, shape, device, graph)
                sl.nbytes = nbytes
                busy.append(sl)
                sl.jobs.put(sl.event)
                n_batches += 1
                used += nbytes
                peak_used = max(peak_used, used)
                peak_busy = max(peak_busy, len(busy))
            # wait for the next arrival or a completion
            with cond:
                if not completed:
                    if pending:
                        cond.wait(max(pending[0].arrival - (time.perf_counter() - start), 0.0))
                    elif busy:
                        cond.wait(0.05)
    finally:
        for sl in all_slots:
            sl.jobs.put(None)
        for sl in all_slots:
            sl.thread.join()
    if stats is not None:
        torch.cuda.synchronize(device)
        iv = [(base.elapsed_time(a), base.elapsed_time(b)) for a, b in done_ev]
        g = [sl.graph.stats() for sl in all_slots if sl.graph.h]
        stats.update(batches=n_batches, max_inflight_host=peak_busy,
                     max_inflight_device=max_overlap(iv), peak_admitted_bytes=peak_used,
                     graph_updates=sum(x["updates"] for x in g),
                     graph_instantiations=sum(x["instantiations"] for x in g))
    return requests


def serve_plain(requests, shape=DEFAULT_SHAPE, device=None, t0: float | None = None):
    """Baseline: one request at a time, arrival order, plain per-set calls with
    the same plan shape (tile, depth, budget)."""
    tile, depth, budget = shape
    device = torch.device(device or "cuda")
    ws = sad.Workspace(device)
    start = time.perf_counter() if t0 is None else t0
    for r in requests:
        now = time.perf_counter() - start
        if r.arrival > now:
            time.sleep(r.arrival - now)
        s = r.seqset
        codes = torch.from_numpy(s.codes).to(device, non_blocking=True)
        offsets = torch.from_numpy(s.offsets).to(device, non_blocking=True)
        res = sad.partition_set(codes, offsets, s.p, ws=ws, depth=depth, tile=tile,
                                budget=budget)
        r.result = dict(bucket_offsets=res["bucket_offsets"].cpu().numpy(),
                        members=res["members"].cpu().numpy(),
                        key_hi=res["key_hi"].cpu().numpy(), key_lo=res["key_lo"].cpu().numpy())
        r.done = time.perf_counter() - start
    return requests


def latency_stats(requests, skip: int = 0):
    lat = np.array([r.done - r.arrival for r in requests[skip:]])
    span = max(r.done for r in requests[skip:]) - min(r.arrival for r in requests[skip:])
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()),
            "sets_per_s": len(lat) / span}


def make_requests(pool, arrivals):
    return [Request(i, float(a), pool[i % len(pool)]) for i, a in enumerate(arrivals)]
