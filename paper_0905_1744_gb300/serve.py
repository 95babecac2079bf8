"""Serving: continuous batching of sequence-set requests on one GPU.

Requests (one sequence set each, host memory) arrive over time. The server keeps
up to ``slots`` batches in flight, each on its own CUDA stream. Whenever a slot
is free, every request that has arrived and fits the HBM budget is admitted and
launched as one batch (count -> block-diagonal rank -> batched partition, see
``sad.Batch``); its device state (codes, counts, planes, keys, buckets) lives
until the batch completes and its bucket lists have been copied back, and then
its memory returns to the budget. Requests that arrive while batches run wait
for the next free slot, and batches in flight on different streams overlap on
the device. Latency = time the results are on the host - arrival time.

The baseline (``serve_plain``) takes the same requests one at a time in arrival
order and runs the plain per-set calls for each.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import sad

GB = 1 << 30


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    seqset: object          # datagen.SeqSet-like: codes, offsets, p
    done: float = -1.0
    result: dict | None = None


def request_bytes(s, depth: int, k: int = 3, alphabet: int = 20) -> int:
    """HBM a request holds while it is in flight, estimated for admission: codes,
    offsets, counts, the rank workspace (4-bit planes of min(D, 4) full sections of
    the word columns, which covers protein sets, where few words repeat more than
    once in a sequence; padded rows; every 128 x 128 u16 residual block of the
    upper triangle), keys, partition buffers, 64 MB of slack."""
    n = s.offsets.shape[0] - 1
    eps = alphabet ** k
    rows = (n + 127) // 128 * 128
    d = depth if depth > 0 else 4
    planes = rows * (eps * min(d, 4) + 256) // 2
    blocks = (rows // 128) * (rows // 128 + 1) // 2
    residual = blocks * 2 * 128 * 128 if depth > 0 else 0
    return int(s.codes.nbytes + 8 * (n + 1) + 4 * n * eps + planes + residual + 96 * n
               + (64 << 20))


def select_batch(queue, used: int, budget_bytes: int, max_batch: int, depth: int):
    """The next batch to admit: the longest prefix of the arrival-ordered queue
    (at most max_batch requests) whose bytes fit beside the ``used`` bytes of the
    batches in flight. Returns (requests, bytes); empty when the head of the queue
    does not fit yet (it is never overtaken, so admission stays in arrival order)."""
    take, nbytes = [], 0
    for r in queue:
        rb = request_bytes(r.seqset, depth)
        if len(take) >= max_batch or used + nbytes + rb > budget_bytes:
            break
        take.append(r)
        nbytes += rb
    return take, nbytes


class _InFlight:
    def __init__(self, reqs, batch, stream, event, host, nbytes):
        self.reqs, self.batch, self.stream, self.event = reqs, batch, stream, event
        self.host, self.nbytes = host, nbytes


def _launch(reqs, depth, device, stream):
    """Admit a batch: H2D, plan (synchronises this stream only), run, D2H."""
    with torch.cuda.stream(stream):
        b = sad.Batch([r.seqset for r in reqs], device=device)
        b.plan(depth=depth, stream=stream)
        b.run(stream=stream, count=False)
        host = dict(bucket_offsets=torch.empty(b.bucket_offsets.shape, dtype=torch.int32,
                                               pin_memory=True),
                    members=torch.empty(b.members.shape, dtype=torch.int32, pin_memory=True),
                    key_hi=torch.empty(b.key_hi.shape, dtype=torch.uint64, pin_memory=True),
                    key_lo=torch.empty(b.key_lo.shape, dtype=torch.uint64, pin_memory=True))
        for key, h in host.items():
            h.copy_(getattr(b, key), non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(stream)
    return b, host, ev


def _finish(f: _InFlight, now: float):
    f.batch.check(f.stream)
    for i, r in enumerate(f.reqs):
        a, e = int(f.batch.seq_begin[i]), int(f.batch.seq_begin[i + 1])
        oa, ob = int(f.batch.boff_begin[i]), int(f.batch.boff_begin[i + 1])
        r.result = dict(bucket_offsets=f.host["bucket_offsets"][oa:ob].numpy().copy(),
                        members=f.host["members"][a:e].numpy().copy(),
                        key_hi=f.host["key_hi"][a:e].numpy().copy(),
                        key_lo=f.host["key_lo"][a:e].numpy().copy())
        r.done = now


def serve(requests, depth: int = 2, budget_bytes: int = 150 * GB, slots: int = 3,
          max_batch: int = 64, device=None, t0: float | None = None):
    """Continuous batching over ``requests`` (sorted by arrival). Returns them with
    ``done`` and ``result`` filled in. Arrival times are honoured in real time."""
    if slots < 1 or max_batch < 1:
        raise ValueError("serve: slots and max_batch must be at least 1")
    for r in requests:
        if request_bytes(r.seqset, depth) > budget_bytes:
            # it could never be admitted, and the loop below would wait for it forever
            raise ValueError(f"serve: request {r.rid} needs "
                             f"{request_bytes(r.seqset, depth)} bytes, above the "
                             f"{budget_bytes}-byte budget")
    device = torch.device(device or "cuda")
    streams = [torch.cuda.Stream(device) for _ in range(slots)]
    free_streams = list(streams)
    pending = list(requests)
    queue: list[Request] = []
    inflight: list[_InFlight] = []
    used = 0
    start = time.perf_counter() if t0 is None else t0
    while pending or queue or inflight:
        now = time.perf_counter() - start
        while pending and pending[0].arrival <= now:
            queue.append(pending.pop(0))
        # completions
        for f in list(inflight):
            if f.event.query():
                _finish(f, time.perf_counter() - start)
                inflight.remove(f)
                free_streams.append(f.stream)
                used -= f.nbytes
        # admissions: everything queued that fits, one batch per free slot
        while queue and free_streams:
            take, nbytes = select_batch(queue, used, budget_bytes, max_batch, depth)
            if not take:
                break
            queue = queue[len(take):]
            st = free_streams.pop(0)
            b, host, ev = _launch(take, depth, device, st)
            inflight.append(_InFlight(take, b, st, ev, host, nbytes))
            used += nbytes
        if not (queue and free_streams):
            # nothing to launch right now: wait a little for an arrival or a completion
            nxt = pending[0].arrival - (time.perf_counter() - start) if pending else 0.0
            time.sleep(min(max(nxt, 0.0), 2e-4))
    return requests


def serve_plain(requests, depth: int = 2, device=None, t0: float | None = None):
    """Baseline: one request at a time, arrival order, plain per-set calls."""
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
        res = sad.partition_set(codes, offsets, s.p, ws=ws, depth=depth)
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
