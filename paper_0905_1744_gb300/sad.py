"""Thin Python binding of libsad (include/sad.h).

Argument marshalling only: every step runs in the CUDA library. torch tensors
provide device memory and streams. The library is loaded on first use; if it is
missing or fails to load, the call raises -- there is no fallback.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

import torch

from . import build as _build

OK, ERR_INVALID_ARGUMENT, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, \
    ERR_BAD_INPUT = range(7)
OP_COUNT, OP_RANK, OP_PARTITION = 0, 1, 2

_lib = None
_lock = threading.Lock()
_DEVICE_TYPE = "cuda"       # where every tensor handed to the library must live


class RankPlan(ctypes.Structure):
    """sad_rank_plan: depth and budget in; sizes and capacities out (see include/sad.h)."""
    _fields_ = [("depth", ctypes.c_int32), ("budget", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("t_max", ctypes.c_int32),
                ("t_bits", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("k_eff", ctypes.c_int64), ("list_entries", ctypes.c_int64),
                ("rem_bound", ctypes.c_int64), ("heavy_entries", ctypes.c_int64),
                ("k_cap", ctypes.c_int64), ("list_cap", ctypes.c_int64),
                ("rem_cap", ctypes.c_int64), ("heavy_cap", ctypes.c_int64),
                ("bm_cols", ctypes.c_int64), ("ws_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class BatchPlan(ctypes.Structure):
    """sad_batch_plan (see include/sad.h)."""
    _fields_ = [("rank", RankPlan), ("n_sets", ctypes.c_int32), ("max_p", ctypes.c_int32),
                ("n_total", ctypes.c_int64), ("rows_total", ctypes.c_int64),
                ("tiles_total", ctypes.c_int64), ("tileof_total", ctypes.c_int64),
                ("sum_p", ctypes.c_int64), ("sum_p1", ctypes.c_int64),
                ("sum_pp1", ctypes.c_int64), ("sum_pp", ctypes.c_int64),
                ("part_ws_bytes", ctypes.c_size_t)]


class SadError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _load().sad_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsad.so not found at {path}: run __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU path)")
        lib = ctypes.CDLL(path)
        P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        lib.sad_status_string.argtypes = [ctypes.c_int]
        lib.sad_status_string.restype = ctypes.c_char_p
        lib.sad_abi_version.restype = ctypes.c_int
        lib.sad_launch_count.restype = ctypes.c_uint64
        lib.sad_workspace_bytes.argtypes = [i32, i32, i32, i32, i32, i32]
        lib.sad_workspace_bytes.restype = sz
        lib.kmer_count.argtypes = [P, P, i32, i32, i32, P, P, P, sz, P]
        lib.kmer_count.restype = ctypes.c_int
        lib.kmer_rank_plan.argtypes = [P, i32, i32, i32, ctypes.POINTER(RankPlan), P, sz, P]
        lib.kmer_rank_plan.restype = ctypes.c_int
        lib.kmer_rank_plan_bound.argtypes = [i32, i64, i32, i32, ctypes.POINTER(RankPlan)]
        lib.kmer_rank_plan_bound.restype = ctypes.c_int
        lib.kmer_rank.argtypes = [P, P, P, i32, i32, i32, ctypes.POINTER(RankPlan), P, P, P, P,
                                  sz, P]
        lib.kmer_rank.restype = ctypes.c_int
        lib.partition.argtypes = [P, P, i32, i32, P, P, P, P, sz, P]
        lib.partition.restype = ctypes.c_int
        lib.sad_status_read.argtypes = [P, i32, P]
        lib.sad_status_read.restype = ctypes.c_int
        lib.sad_batch_plan_make.argtypes = [P, P, P, P, i32, i32, i32, ctypes.POINTER(BatchPlan),
                                            P, sz, P]
        lib.sad_batch_plan_make.restype = ctypes.c_int
        lib.sad_batch_rank.argtypes = [P, P, P, P, i32, i32, ctypes.POINTER(BatchPlan), P, P, P,
                                       P, sz, P]
        lib.sad_batch_rank.restype = ctypes.c_int
        lib.sad_batch_partition.argtypes = [P, P, P, P, ctypes.POINTER(BatchPlan), P, P, P, P, sz,
                                            P]
        lib.sad_batch_partition.restype = ctypes.c_int
        lib.partition_noalloc.argtypes = [P, P, i32, i32, P, P, P, P]
        lib.partition_noalloc.restype = ctypes.c_int
        lib.sad_rank_info.argtypes = [P, ctypes.POINTER(i64), P]
        lib.sad_rank_info.restype = ctypes.c_int
        lib.sad_local_samples_workspace_bytes.argtypes = [i32, i32]
        lib.sad_local_samples_workspace_bytes.restype = sz
        lib.sad_local_samples.argtypes = [P, P, i32, i32, i32, P, P, sz, P]
        lib.sad_local_samples.restype = ctypes.c_int
        lib.kmer_rank_vs_workspace_bytes.argtypes = [ctypes.POINTER(RankPlan), i32, i32, i32, i32,
                                                     i32]
        lib.kmer_rank_vs_workspace_bytes.restype = sz
        lib.kmer_rank_vs.argtypes = [P, P, P, i32, i32, i32, P, i32, i32,
                                     ctypes.POINTER(RankPlan), P, P, P, P, P, sz, P]
        lib.kmer_rank_vs.restype = ctypes.c_int
        lib.kmer_rank_dist_workspace_bytes.argtypes = [ctypes.POINTER(RankPlan), i32, i32, i32,
                                                       i32]
        lib.kmer_rank_dist_workspace_bytes.restype = sz
        lib.kmer_rank_dist.argtypes = [P, P, P, i32, i32, i32, i32, ctypes.POINTER(RankPlan), P,
                                       P, P, P, P, sz, P]
        lib.kmer_rank_dist.restype = ctypes.c_int
        lib.sad_ln_q.argtypes = [P, i64, P, P]
        lib.sad_ln_q.restype = ctypes.c_int
        lib.kmer_rank_sparse_workspace_bytes.argtypes = [i32, i64]
        lib.kmer_rank_sparse_workspace_bytes.restype = sz
        lib.kmer_rank_sparse_entries.argtypes = [P, P, i32, i32, i32, ctypes.POINTER(i64), P, sz,
                                                 P]
        lib.kmer_rank_sparse_entries.restype = ctypes.c_int
        lib.kmer_rank_sparse.argtypes = [P, P, i32, i32, i32, i64, P, P, P, P, sz, P]
        lib.kmer_rank_sparse.restype = ctypes.c_int
        lib.sad_profile.argtypes = [i32]
        lib.sad_profile.restype = ctypes.c_int
        lib.sad_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        lib.sad_profile_read.restype = ctypes.c_int
        lib.sad_debug_wait_budget_ns.argtypes = [ctypes.c_uint64]
        lib.sad_debug_wait_budget_ns.restype = ctypes.c_int
        lib.sad_batch_plan_bound.argtypes = [P, P, i32, i64, i32, i32, ctypes.POINTER(BatchPlan)]
        lib.sad_batch_plan_bound.restype = ctypes.c_int
        lib.sad_seq_lengths.argtypes = [P, i32, P, P, P]
        lib.sad_seq_lengths.restype = ctypes.c_int
        lib.sad_graph_begin.argtypes = [P]
        lib.sad_graph_begin.restype = ctypes.c_int
        lib.sad_graph_end.argtypes = [P, ctypes.POINTER(P)]
        lib.sad_graph_end.restype = ctypes.c_int
        lib.sad_graph_launch.argtypes = [P, P]
        lib.sad_graph_launch.restype = ctypes.c_int
        lib.sad_graph_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                        ctypes.POINTER(i32)]
        lib.sad_graph_stats.restype = ctypes.c_int
        lib.sad_graph_destroy.argtypes = [P]
        lib.sad_graph_destroy.restype = ctypes.c_int
        _lib = lib
        return lib


def lib():
    return _load()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, elem_bytes: int, name: str, where: str):
    """A tensor whose data pointer goes to the library: on a CUDA device, dense,
    with the element size the C-ABI declares for it (None passes: optional)."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or t.device.type != _DEVICE_TYPE:
        raise TypeError(f"{where}: {name} must be a CUDA tensor")
    if t.element_size() != elem_bytes:
        raise TypeError(f"{where}: {name} must have {elem_bytes}-byte elements, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{where}: {name} must be contiguous")


def _need_counts(counts, k: int, alphabet: int, where: str, word_max=None):
    """int32 [N][alphabet^k] count vectors (and the optional per-word maxima)."""
    _need(counts, 4, "counts", where)
    if counts.dim() != 2 or counts.shape[1] != alphabet ** k:
        raise ValueError(f"{where}: counts must be [N, {alphabet ** k}], not "
                         f"{list(counts.shape)}")
    _need(word_max, 4, "word_max", where)
    if word_max is not None and word_max.numel() < alphabet ** k:
        raise ValueError(f"{where}: word_max needs {alphabet ** k} entries")


def _need_keys(key_hi, key_lo, where: str):
    _need(key_hi, 8, "key_hi", where)
    _need(key_lo, 8, "key_lo", where)
    if key_hi.numel() != key_lo.numel():
        raise ValueError(f"{where}: key_hi and key_lo differ in length")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc: int, where: str):
    if rc != OK:
        raise SadError(rc, where)


def launch_count() -> int:
    return int(_load().sad_launch_count())


def workspace_bytes(op: int, n: int, k: int = 3, alphabet: int = 20, p: int = 1,
                    depth: int = 1) -> int:
    return int(_load().sad_workspace_bytes(op, n, k, alphabet, p, depth))


class Workspace:
    """A reusable device workspace (uint8 tensor, grown on demand)."""

    def __init__(self, device=None, nbytes: int = 0):
        self.device = torch.device(device or "cuda")
        self.buf = None
        if nbytes:
            self.ensure(nbytes)

    def ensure(self, nbytes: int):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.clear_status()
        return self.buf

    @property
    def nbytes(self) -> int:
        return 0 if self.buf is None else self.buf.numel()

    def clear_status(self):
        if self.buf is not None:
            self.buf[:8].zero_()

    def status(self, clear: bool = True, stream=None) -> int:
        return int(_load().sad_status_read(_ptr(self.buf), 1 if clear else 0, _stream(stream)))

    def check(self, where: str, stream=None):
        _check(self.status(True, stream), where)


def kmer_count(codes: torch.Tensor, offsets: torch.Tensor, k: int = 3, alphabet: int = 20,
               ws: Workspace | None = None, out: torch.Tensor | None = None, stream=None,
               check: bool = True, word_max: torch.Tensor | None = None) -> torch.Tensor:
    """int32 [N, alphabet**k] count vectors (Sec. 3, "k-mer Rank"). If ``word_max``
    (int32 [alphabet**k]) is given it receives the largest count of every word."""
    _need(codes, 1, "codes", "kmer_count")
    _need(offsets, 8, "offsets", "kmer_count")
    _need(word_max, 4, "word_max", "kmer_count")
    n = offsets.numel() - 1
    if out is not None:
        _need(out, 4, "out", "kmer_count")
        if out.dim() != 2 or tuple(out.shape) != (n, alphabet ** k):
            raise ValueError(f"kmer_count: out must be [{n}, {alphabet ** k}]")
    if word_max is not None and word_max.numel() < alphabet ** k:
        raise ValueError(f"kmer_count: word_max needs {alphabet ** k} entries")
    ws = ws or Workspace(codes.device)
    ws.ensure(workspace_bytes(OP_COUNT, n, k, alphabet))
    if out is None:
        out = torch.empty((n, alphabet ** k), dtype=torch.int32, device=codes.device)
    _check(_load().kmer_count(_ptr(codes), _ptr(offsets), n, k, alphabet, _ptr(out),
                              _ptr(word_max), _ptr(ws.buf), ws.nbytes, _stream(stream)),
           "kmer_count")
    if check:
        ws.check("kmer_count", stream)
    return out


def seq_lengths(offsets: torch.Tensor, out: torch.Tensor | None = None, ws: Workspace | None = None,
                stream=None) -> torch.Tensor:
    """int32 lengths off[i + 1] - off[i] of an int64 offsets array, on the device
    (sad_seq_lengths; no synchronisation). ``ws``: a workspace whose status
    records a negative or oversized length."""
    _need(offsets, 8, "offsets", "sad_seq_lengths")
    n = offsets.numel() - 1
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
    _need(out, 4, "lengths", "sad_seq_lengths")
    if out.numel() < n:
        raise ValueError(f"sad_seq_lengths: out must hold {n} entries")
    _check(_load().sad_seq_lengths(_ptr(offsets), n, _ptr(out), _ptr(ws.buf) if ws else None,
                                   _stream(stream)), "sad_seq_lengths")
    return out


class Graph:
    """A reusable CUDA graph of library calls (sad_graph_*). ``capture(fn, stream)``
    records fn(stream) (which must only make asynchronous library calls on that
    stream: no torch operation, no synchronisation); the first capture is
    instantiated and every later one updates the instantiated graph in place when
    its launch sequence has the same topology. ``launch(stream)`` runs it."""

    def __init__(self):
        self.h = ctypes.c_void_p()

    def capture(self, fn, stream):
        lib, st = _load(), _stream(stream)
        _check(lib.sad_graph_begin(st), "sad_graph_begin")
        try:
            fn(stream)
        except BaseException:
            # end the broken capture (its graph is dropped; the handle keeps its last one)
            lib.sad_graph_end(st, ctypes.byref(self.h))
            raise
        _check(lib.sad_graph_end(st, ctypes.byref(self.h)), "sad_graph_end")

    def launch(self, stream=None):
        _check(_load().sad_graph_launch(self.h, _stream(stream)), "sad_graph_launch")

    def stats(self) -> dict:
        u, i, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_load().sad_graph_stats(self.h, ctypes.byref(u), ctypes.byref(i), ctypes.byref(k)),
               "sad_graph_stats")
        return dict(updates=u.value, instantiations=i.value, kernels=k.value)

    def close(self):
        if self.h:
            _load().sad_graph_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kmer_rank_plan(counts: torch.Tensor, k: int = 3, alphabet: int = 20, depth: int = 0,
                   ws: Workspace | None = None, stream=None, budget: int = 0,
                   tile: int = 0) -> RankPlan:
    """Sizes and capacities for kmer_rank at plane depth ``depth`` (0 = all
    planes) with ``budget`` remainder entries per column block (0 = default) and
    GEMM tiles of ``tile`` rows (0/128: one CTA a tile; 256: CTA pairs).
    Synchronous."""
    _need_counts(counts, k, alphabet, "kmer_rank_plan")
    n = counts.shape[0]
    ws = ws or Workspace(counts.device)
    ws.ensure(workspace_bytes(OP_RANK, n, k, alphabet, depth=0))
    plan = RankPlan(depth=int(depth), budget=int(budget), tile=int(tile))
    rc = _load().kmer_rank_plan(_ptr(counts), n, k, alphabet, ctypes.byref(plan), _ptr(ws.buf),
                                ws.nbytes, _stream(stream))
    if rc == ERR_WORKSPACE and plan.ws_bytes > ws.nbytes:
        # the fixed part of a layout with other padding (tile = 256): the size it needs
        ws.ensure(plan.ws_bytes)
        plan = RankPlan(depth=int(depth), budget=int(budget), tile=int(tile))
        rc = _load().kmer_rank_plan(_ptr(counts), n, k, alphabet, ctypes.byref(plan),
                                    _ptr(ws.buf), ws.nbytes, _stream(stream))
    _check(rc, "kmer_rank_plan")
    return plan


def kmer_rank_plan_bound(n: int, total_len: int, k: int = 3, alphabet: int = 20,
                         depth: int = 1, budget: int = 0, tile: int = 0) -> RankPlan:
    """Capacities for kmer_rank at plane depth ``depth`` >= 1 that hold for any
    counts of ``n`` sequences of ``total_len`` residues in all: no device work and
    no synchronisation (bounds from the number of windows; see include/sad.h)."""
    plan = RankPlan(depth=int(depth), budget=int(budget), tile=int(tile))
    _check(_load().kmer_rank_plan_bound(int(n), int(total_len), k, alphabet, ctypes.byref(plan)),
           "kmer_rank_plan_bound")
    return plan


def kmer_rank(counts: torch.Tensor, lengths: torch.Tensor, k: int = 3, alphabet: int = 20,
              ws: Workspace | None = None, with_rank: bool = True, stream=None,
              out=None, check: bool = True, plan: RankPlan | None = None, depth: int = 0,
              word_max: torch.Tensor | None = None, tile: int = 0, budget: int = 0):
    """(key_hi uint64, key_lo uint64, rank float64 | None), Eq. 1 and Eq. 3.

    ``plan``: a RankPlan from kmer_rank_plan (reused as is); if None, one is made
    here for ``depth`` (0 = all planes), ``tile`` and ``budget``, which
    synchronises the stream.
    """
    _need_counts(counts, k, alphabet, "kmer_rank", word_max)
    n = counts.shape[0]
    dev = counts.device
    if out is not None:
        hi, lo, rank = out
        _need_keys(hi, lo, "kmer_rank")
        _need(rank, 8, "rank", "kmer_rank")
        if hi.numel() != n or (rank is not None and rank.numel() != n):
            raise ValueError(f"kmer_rank: outputs must hold {n} entries")
    ws = ws or Workspace(dev)
    if plan is None:
        plan = kmer_rank_plan(counts, k, alphabet, depth, ws, stream, budget=budget, tile=tile)
    ws.ensure(plan.ws_bytes)
    if out is None:
        hi = torch.empty(n, dtype=torch.uint64, device=dev)
        lo = torch.empty(n, dtype=torch.uint64, device=dev)
        rank = torch.empty(n, dtype=torch.float64, device=dev) if with_rank else None
    lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
    _check(_load().kmer_rank(_ptr(counts), _ptr(lengths), _ptr(word_max), n, k, alphabet,
                             ctypes.byref(plan),
                             _ptr(hi), _ptr(lo), _ptr(rank), _ptr(ws.buf), ws.nbytes,
                             _stream(stream)), "kmer_rank")
    if check:
        ws.check("kmer_rank", stream)
    return hi, lo, rank


def _need_partition_out(offs, mem, piv, n: int, p: int, where: str):
    _need(offs, 4, "bucket_offsets", where)
    _need(mem, 4, "members", where)
    _need(piv, 4, "pivot_idx", where)
    if offs.numel() < p + 1 or mem.numel() < n or (p > 1 and piv.numel() < p - 1):
        raise ValueError(f"{where}: outputs need p + 1, N and p - 1 entries")


def partition(key_hi: torch.Tensor, key_lo: torch.Tensor, p: int, ws: Workspace | None = None,
              stream=None, out=None, check: bool = True):
    """(bucket_offsets int32 [p+1], members int32 [N], pivot_idx int32 [p-1])."""
    _need_keys(key_hi, key_lo, "partition")
    n = key_hi.numel()
    dev = key_hi.device
    if out is not None:
        _need_partition_out(*out, n, p, "partition")
    ws = ws or Workspace(dev)
    ws.ensure(workspace_bytes(OP_PARTITION, n, p=p))
    if out is None:
        offs = torch.empty(p + 1, dtype=torch.int32, device=dev)
        mem = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        piv = torch.empty(max(p - 1, 1), dtype=torch.int32, device=dev)
    else:
        offs, mem, piv = out
    _check(_load().partition(_ptr(key_hi), _ptr(key_lo), n, p, _ptr(offs), _ptr(mem),
                             _ptr(piv) if p > 1 else None, _ptr(ws.buf), ws.nbytes,
                             _stream(stream)), "partition")
    if check:
        ws.check("partition", stream)
    return offs, mem[:n], piv[:max(p - 1, 0)]


def partition_set(codes: torch.Tensor, offsets: torch.Tensor, p: int, k: int = 3,
                  alphabet: int = 20, ws: Workspace | None = None, stream=None,
                  depth: int = 0, tile: int = 0, budget: int = 0):
    """count -> lengths -> rank -> partition of one sequence set on the device,
    with a rank plan of ``depth``, ``tile`` and ``budget`` (see kmer_rank_plan).
    With ``depth`` >= 1 the rank runs on the host-side capacity bounds
    (kmer_rank_plan_bound), so the calls queue without a synchronisation; the
    workspace status (the first error any of them recorded) is read once at the
    end."""
    ws = ws or Workspace(codes.device)
    n = offsets.numel() - 1
    plan = (kmer_rank_plan_bound(n, codes.numel(), k, alphabet, depth, budget=budget, tile=tile)
            if depth >= 1 else None)
    if plan is not None:
        # one size for the three calls: a later growth would drop an earlier status
        ws.ensure(max(plan.ws_bytes, workspace_bytes(OP_COUNT, n, k, alphabet),
                      workspace_bytes(OP_PARTITION, n, p=p)))
    word_max = torch.empty(alphabet ** k, dtype=torch.int32, device=codes.device)
    counts = kmer_count(codes, offsets, k, alphabet, ws=ws, stream=stream, word_max=word_max,
                        check=plan is None)
    lengths = seq_lengths(offsets, ws=ws, stream=stream)
    hi, lo, rank = kmer_rank(counts, lengths, k, alphabet, ws=ws, stream=stream, depth=depth,
                             word_max=word_max, plan=plan, check=plan is None, tile=tile,
                             budget=budget)
    offs, mem, piv = partition(hi, lo, p, ws=ws, stream=stream, check=False)
    ws.check("partition_set", stream)
    return dict(counts=counts, key_hi=hi, key_lo=lo, rank=rank, bucket_offsets=offs,
                members=mem, pivot_idx=piv)


def rank_info(ws: Workspace, stream=None) -> dict:
    """Plan the device chose in the last kmer_rank on this workspace (synchronous)."""
    info = (ctypes.c_int64 * 16)()
    _check(_load().sad_rank_info(_ptr(ws.buf), info, _stream(stream)), "sad_rank_info")
    keys = ("status", "k_eff", "k_pad", "t_max", "tiles", "k_chunks", "depth",
            "rem_entries", "rem_blocks", "heavy_entries", "bm_cols")
    return {k: int(info[i]) for i, k in enumerate(keys)}


def profile(enable: bool):
    _check(_load().sad_profile(1 if enable else 0), "sad_profile")


def profile_read():
    """(summed plane-GEMM milliseconds, launches) since the last read (synchronous)."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(_load().sad_profile_read(ctypes.byref(ms), ctypes.byref(n)), "sad_profile_read")
    return float(ms.value), int(n.value)


def debug_wait_budget_ns(ns: int):
    """Budget of the plane GEMM's main-loop waits for later launches (0 = the
    default 2 s). A test hook: a few nanoseconds drives the timeout path."""
    _check(_load().sad_debug_wait_budget_ns(int(ns)), "sad_debug_wait_budget_ns")


NOALLOC_MAX_N, NOALLOC_MAX_P = 32768, 64


def partition_noalloc(key_hi: torch.Tensor, key_lo: torch.Tensor, p: int, stream=None,
                      out=None):
    """partition() without a workspace, for callers that cannot allocate device
    memory: the library keeps a fixed scratch array per device (about 2.1 MiB,
    sized for the largest accepted call), so the call allocates nothing beyond
    the outputs (which the caller may pass in ``out``). Limits: N <= 32768 and
    p <= 64 in any combination. Calls sharing a device must not overlap."""
    _need_keys(key_hi, key_lo, "partition_noalloc")
    n = key_hi.numel()
    dev = key_hi.device
    if out is None:
        offs = torch.empty(p + 1, dtype=torch.int32, device=dev)
        mem = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        piv = torch.empty(max(p - 1, 1), dtype=torch.int32, device=dev)
    else:
        offs, mem, piv = out
        _need_partition_out(offs, mem, piv, n, p, "partition_noalloc")
    _check(_load().partition_noalloc(_ptr(key_hi), _ptr(key_lo), n, p, _ptr(offs), _ptr(mem),
                                     _ptr(piv) if p > 1 else None, _stream(stream)),
           "partition_noalloc")
    return offs, mem[:n], piv[:max(p - 1, 0)]


def block_bounds(n: int, p: int):
    """Starts of the p contiguous blocks, floor(b N / p), and N (Algorithm 2 step 1)."""
    return [b * n // p for b in range(p + 1)]


def local_ranks(counts: torch.Tensor, lengths: torch.Tensor, p: int, k: int = 3,
                alphabet: int = 20, depth: int = 0, word_max: torch.Tensor | None = None,
                ws: Workspace | None = None, stream=None):
    """Algorithm 2 step 2: every block of sequences ranked against its own block,
    as one block-diagonal batched rank (blocks as sets). Synchronous (plans).
    Returns (key_hi, key_lo, rank) in input order; rank = key / (w_b 2^64)."""
    import numpy as np
    _need_counts(counts, k, alphabet, "local_ranks", word_max)
    n = counts.shape[0]
    dev = counts.device
    if not 1 <= p <= n:
        raise ValueError("need 1 <= p <= N")
    h_n = np.ascontiguousarray(np.diff(block_bounds(n, p)), dtype=np.int32)
    h_p = np.ones(p, dtype=np.int32)
    d_n = torch.from_numpy(h_n).to(dev)
    ws = ws or Workspace(dev)
    ws.ensure(256)
    plan = BatchPlan()
    plan.rank.depth = int(depth)
    args = (_ptr(counts), h_n.ctypes.data_as(ctypes.c_void_p), h_p.ctypes.data_as(ctypes.c_void_p),
            _ptr(d_n), p, k, alphabet, ctypes.byref(plan))
    rc = _load().sad_batch_plan_make(*args, _ptr(ws.buf), ws.nbytes, _stream(stream))
    if rc == ERR_WORKSPACE:
        ws.ensure(plan.rank.ws_bytes)
        plan.rank.depth = int(depth)
        rc = _load().sad_batch_plan_make(*args, _ptr(ws.buf), ws.nbytes, _stream(stream))
    _check(rc, "sad_batch_plan_make (local ranks)")
    ws.ensure(plan.rank.ws_bytes)
    hi = torch.empty(n, dtype=torch.uint64, device=dev)
    lo = torch.empty(n, dtype=torch.uint64, device=dev)
    rank = torch.empty(n, dtype=torch.float64, device=dev)
    lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
    _check(_load().sad_batch_rank(_ptr(counts), _ptr(lengths), _ptr(word_max), _ptr(d_n), k,
                                  alphabet, ctypes.byref(plan), _ptr(hi), _ptr(lo), _ptr(rank),
                                  _ptr(ws.buf), ws.nbytes, _stream(stream)), "sad_batch_rank")
    ws.check("local ranks", stream)
    return hi, lo, rank


def local_samples(key_hi: torch.Tensor, key_lo: torch.Tensor, p: int, ks: int,
                  ws: Workspace | None = None, stream=None, out=None, check: bool = True):
    """Algorithm 2 steps 3-5: ks evenly spaced samples of every block's sorted
    order; int32 [p * ks] input indices, block-major."""
    _need_keys(key_hi, key_lo, "local_samples")
    n = key_hi.numel()
    dev = key_hi.device
    if out is not None:
        _need(out, 4, "out", "local_samples")
        if out.numel() < p * ks:
            raise ValueError(f"local_samples: out needs {p * ks} entries")
    ws = ws or Workspace(dev)
    ws.ensure(int(_load().sad_local_samples_workspace_bytes(n, p)))
    out = out if out is not None else torch.empty(p * ks, dtype=torch.int32, device=dev)
    _check(_load().sad_local_samples(_ptr(key_hi), _ptr(key_lo), n, p, ks, _ptr(out),
                                     _ptr(ws.buf), ws.nbytes, _stream(stream)),
           "sad_local_samples")
    if check:
        ws.check("sad_local_samples", stream)
    return out


def kmer_rank_vs(counts: torch.Tensor, lengths: torch.Tensor, ref: torch.Tensor, k: int = 3,
                 alphabet: int = 20, plan: RankPlan | None = None,
                 word_max: torch.Tensor | None = None, ws: Workspace | None = None,
                 stream=None, check: bool = True, delta_den: int = 0):
    """Algorithm 2 step 6: every sequence ranked against the reference multiset
    ``ref`` (input indices). ``plan``: a depth-0 RankPlan (made here if None,
    synchronous). Returns (key_hi, key_lo, rank), rank = key / (len(ref) 2^64);
    with ``delta_den`` = b > 0 the distance form (Eq. 2, Delta = 1/b): returns
    (key int64, key_hi, key_lo, rank), rank = key 2^-32 / len(ref)."""
    _need_counts(counts, k, alphabet, "kmer_rank_vs", word_max)
    n = counts.shape[0]
    dev = counts.device
    ws = ws or Workspace(dev)
    if plan is None:
        plan = kmer_rank_plan(counts, k, alphabet, 0, ws, stream)
    ref = ref.to(device=dev, dtype=torch.int32).contiguous()
    n_ref = ref.numel()
    ws.ensure(int(_load().kmer_rank_vs_workspace_bytes(ctypes.byref(plan), n, k, alphabet,
                                                       n_ref, delta_den)))
    key = torch.empty(n, dtype=torch.int64, device=dev) if delta_den else None
    hi = torch.empty(n, dtype=torch.uint64, device=dev)
    lo = torch.empty(n, dtype=torch.uint64, device=dev)
    rank = torch.empty(n, dtype=torch.float64, device=dev)
    lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
    _check(_load().kmer_rank_vs(_ptr(counts), _ptr(lengths), _ptr(word_max), n, k, alphabet,
                                _ptr(ref), n_ref, delta_den, ctypes.byref(plan), _ptr(key),
                                _ptr(hi), _ptr(lo), _ptr(rank), _ptr(ws.buf), ws.nbytes,
                                _stream(stream)), "kmer_rank_vs")
    if check:
        ws.check("kmer_rank_vs", stream)
    return (key, hi, lo, rank) if delta_den else (hi, lo, rank)


def ln_q(x: torch.Tensor, stream=None) -> torch.Tensor:
    """ln(x) * 2^32 as the deterministic fixed-point value of the distance-form rank."""
    if not isinstance(x, torch.Tensor) or x.device.type != _DEVICE_TYPE:
        raise TypeError("ln_q: x must be a CUDA tensor")
    x = x.to(dtype=torch.uint64).contiguous()
    out = torch.empty(x.shape, dtype=torch.int64, device=x.device)
    _check(_load().sad_ln_q(_ptr(x), x.numel(), _ptr(out), _stream(stream)), "sad_ln_q")
    return out


def kmer_rank_dist(counts: torch.Tensor, lengths: torch.Tensor, delta_den: int = 10, k: int = 3,
                   alphabet: int = 20, plan: RankPlan | None = None, depth: int = 0,
                   word_max: torch.Tensor | None = None, ws: Workspace | None = None,
                   stream=None, check: bool = True):
    """Eq. 2 / Eq. 3 literally: the mean of d = -ln(1/delta_den + F) over the set.
    Returns (key int64, key_hi, key_lo, rank float64); (key_hi, key_lo) order as
    the signed key, for partition."""
    _need_counts(counts, k, alphabet, "kmer_rank_dist", word_max)
    n = counts.shape[0]
    dev = counts.device
    ws = ws or Workspace(dev)
    if plan is None:
        plan = kmer_rank_plan(counts, k, alphabet, depth, ws, stream)
    ws.ensure(int(_load().kmer_rank_dist_workspace_bytes(ctypes.byref(plan), n, k, alphabet,
                                                         delta_den)))
    key = torch.empty(n, dtype=torch.int64, device=dev)
    hi = torch.empty(n, dtype=torch.uint64, device=dev)
    lo = torch.empty(n, dtype=torch.uint64, device=dev)
    rank = torch.empty(n, dtype=torch.float64, device=dev)
    lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
    _check(_load().kmer_rank_dist(_ptr(counts), _ptr(lengths), _ptr(word_max), n, k, alphabet,
                                  delta_den, ctypes.byref(plan), _ptr(key), _ptr(hi), _ptr(lo),
                                  _ptr(rank), _ptr(ws.buf), ws.nbytes, _stream(stream)),
           "kmer_rank_dist")
    if check:
        ws.check("kmer_rank_dist", stream)
    return key, hi, lo, rank


def sparse_entries(counts: torch.Tensor, lengths: torch.Tensor, k: int = 3, alphabet: int = 20,
                   ws: Workspace | None = None, stream=None) -> int:
    """(sequence, word) entries with a nonzero count: the list capacity of
    kmer_rank_sparse. Synchronous."""
    _need_counts(counts, k, alphabet, "sparse_entries")
    n = counts.shape[0]
    ws = ws or Workspace(counts.device)
    ws.ensure(int(_load().kmer_rank_sparse_workspace_bytes(n, 0)))
    lengths = lengths.to(device=counts.device, dtype=torch.int32).contiguous()
    e = ctypes.c_int64()
    _check(_load().kmer_rank_sparse_entries(_ptr(counts), _ptr(lengths), n, k, alphabet,
                                            ctypes.byref(e), _ptr(ws.buf), ws.nbytes,
                                            _stream(stream)), "kmer_rank_sparse_entries")
    return int(e.value)


def kmer_rank_sparse(counts: torch.Tensor, lengths: torch.Tensor, k: int = 3,
                     alphabet: int = 20, ws: Workspace | None = None, stream=None,
                     entries: int | None = None, check: bool = True):
    """The kmer_rank keys by sparse intersection on the CUDA cores (the O(L)-per-pair
    comparison point of Table 2). ``entries``: the list capacity (sized here,
    synchronously, if None). Returns (key_hi, key_lo, rank)."""
    _need_counts(counts, k, alphabet, "kmer_rank_sparse")
    n = counts.shape[0]
    dev = counts.device
    ws = ws or Workspace(dev)
    lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
    if entries is None:
        entries = sparse_entries(counts, lengths, k, alphabet, ws, stream)
    ws.ensure(int(_load().kmer_rank_sparse_workspace_bytes(n, entries)))
    hi = torch.empty(n, dtype=torch.uint64, device=dev)
    lo = torch.empty(n, dtype=torch.uint64, device=dev)
    rank = torch.empty(n, dtype=torch.float64, device=dev)
    _check(_load().kmer_rank_sparse(_ptr(counts), _ptr(lengths), n, k, alphabet, entries,
                                    _ptr(hi), _ptr(lo), _ptr(rank), _ptr(ws.buf), ws.nbytes,
                                    _stream(stream)), "kmer_rank_sparse")
    if check:
        ws.check("kmer_rank_sparse", stream)
    return hi, lo, rank


class GlobalRank:
    """Algorithm 2 steps 2-6 (Sec. 3.1.1) for one set of counts: local ranks per
    block, ks samples per block, every sequence re-ranked against the ks x p
    samples. The constructor plans (synchronous); ``run()`` then launches the
    three steps with no host synchronisation."""

    def __init__(self, counts: torch.Tensor, lengths: torch.Tensor, p: int, ks: int,
                 k: int = 3, alphabet: int = 20, word_max: torch.Tensor | None = None,
                 local_depth: int = 0, stream=None, delta_den: int = 0):
        import numpy as np
        _need_counts(counts, k, alphabet, "GlobalRank", word_max)
        n = counts.shape[0]
        dev = counts.device
        if not 1 <= p <= n or ks < 1:
            raise ValueError("need 1 <= p <= N and ks >= 1")
        self.counts, self.word_max, self.p, self.ks = counts, word_max, p, ks
        self.delta_den = int(delta_den)
        self.k, self.alphabet, self.n = k, alphabet, n
        self.lengths = lengths.to(device=dev, dtype=torch.int32).contiguous()
        self.h_n = np.ascontiguousarray(np.diff(block_bounds(n, p)), dtype=np.int32)
        h_p = np.ones(p, dtype=np.int32)
        self.d_n = torch.from_numpy(self.h_n).to(dev)
        self.ws_local = Workspace(dev, 256)
        plan = BatchPlan()
        plan.rank.depth = int(local_depth)
        args = (_ptr(counts), self.h_n.ctypes.data_as(ctypes.c_void_p),
                h_p.ctypes.data_as(ctypes.c_void_p), _ptr(self.d_n), p, k, alphabet,
                ctypes.byref(plan))
        rc = _load().sad_batch_plan_make(*args, _ptr(self.ws_local.buf), self.ws_local.nbytes,
                                         _stream(stream))
        if rc == ERR_WORKSPACE:
            self.ws_local.ensure(plan.rank.ws_bytes)
            plan.rank.depth = int(local_depth)
            rc = _load().sad_batch_plan_make(*args, _ptr(self.ws_local.buf),
                                             self.ws_local.nbytes, _stream(stream))
        _check(rc, "sad_batch_plan_make (local ranks)")
        self.ws_local.ensure(plan.rank.ws_bytes)
        self.local_plan = plan
        self.ws_vs = Workspace(dev)
        self.vs_plan = kmer_rank_plan(counts, k, alphabet, 0, self.ws_vs, stream)
        self.ws_vs.ensure(int(_load().kmer_rank_vs_workspace_bytes(
            ctypes.byref(self.vs_plan), n, k, alphabet, p * ks, self.delta_den)))
        self.key = torch.empty(n, dtype=torch.int64, device=dev) if self.delta_den else None
        self.ws_samp = Workspace(dev, int(_load().sad_local_samples_workspace_bytes(n, p)))
        self.local_hi = torch.empty(n, dtype=torch.uint64, device=dev)
        self.local_lo = torch.empty(n, dtype=torch.uint64, device=dev)
        self.local_rank = torch.empty(n, dtype=torch.float64, device=dev)
        self.samples = torch.empty(p * ks, dtype=torch.int32, device=dev)
        self.key_hi = torch.empty(n, dtype=torch.uint64, device=dev)
        self.key_lo = torch.empty(n, dtype=torch.uint64, device=dev)
        self.rank = torch.empty(n, dtype=torch.float64, device=dev)

    def run(self, stream=None):
        lib, st = _load(), _stream(stream)
        _check(lib.sad_batch_rank(_ptr(self.counts), _ptr(self.lengths), _ptr(self.word_max),
                                  _ptr(self.d_n), self.k, self.alphabet,
                                  ctypes.byref(self.local_plan), _ptr(self.local_hi),
                                  _ptr(self.local_lo), _ptr(self.local_rank),
                                  _ptr(self.ws_local.buf), self.ws_local.nbytes, st),
               "sad_batch_rank (local ranks)")
        _check(lib.sad_local_samples(_ptr(self.local_hi), _ptr(self.local_lo), self.n, self.p,
                                     self.ks, _ptr(self.samples), _ptr(self.ws_samp.buf),
                                     self.ws_samp.nbytes, st), "sad_local_samples")
        _check(lib.kmer_rank_vs(_ptr(self.counts), _ptr(self.lengths), _ptr(self.word_max),
                                self.n, self.k, self.alphabet, _ptr(self.samples),
                                self.p * self.ks, self.delta_den, ctypes.byref(self.vs_plan),
                                _ptr(self.key), _ptr(self.key_hi), _ptr(self.key_lo),
                                _ptr(self.rank), _ptr(self.ws_vs.buf), self.ws_vs.nbytes, st),
               "kmer_rank_vs")

    def check(self, stream=None):
        self.ws_local.check("local ranks", stream)
        self.ws_samp.check("sad_local_samples", stream)
        self.ws_vs.check("kmer_rank_vs", stream)

    def pairs(self) -> int:
        """Pairs whose shared counts enter: each block's pairs plus N x (ks p)."""
        return int(sum(int(w) * (int(w) + 1) // 2 for w in self.h_n)) + self.n * self.p * self.ks


def global_rank(counts: torch.Tensor, lengths: torch.Tensor, p: int, ks: int, k: int = 3,
                alphabet: int = 20, word_max: torch.Tensor | None = None, local_depth: int = 0,
                stream=None):
    """Algorithm 2 steps 2-6 (Sec. 3.1.1): local ranks per block, ks samples per
    block, every sequence re-ranked against the ks x p samples.
    Returns (key_hi, key_lo, rank, samples)."""
    g = GlobalRank(counts, lengths, p, ks, k, alphabet, word_max, local_depth, stream)
    g.run(stream)
    g.check(stream)
    return g.key_hi, g.key_lo, g.rank, g.samples


def global_partition_set(codes: torch.Tensor, offsets: torch.Tensor, p: int, ks: int,
                         k: int = 3, alphabet: int = 20, stream=None):
    """count -> globalised rank -> partition (Algorithm 2 steps 1-11 without the
    alignment) of one sequence set on the device."""
    ws = Workspace(codes.device)
    word_max = torch.empty(alphabet ** k, dtype=torch.int32, device=codes.device)
    counts = kmer_count(codes, offsets, k, alphabet, ws=ws, stream=stream, word_max=word_max)
    lengths = seq_lengths(offsets, ws=ws, stream=stream)
    hi, lo, rank, samples = global_rank(counts, lengths, p, ks, k, alphabet, word_max,
                                        stream=stream)
    offs, mem, piv = partition(hi, lo, p, ws=ws, stream=stream)
    return dict(counts=counts, key_hi=hi, key_lo=lo, rank=rank, samples=samples,
                bucket_offsets=offs, members=mem, pivot_idx=piv)


class BatchPool:
    """Buffers that the successive batches of one stream reuse (a serving slot, a
    loop over batches): pinned host staging, the device arrays of a Batch and its
    three workspaces. Each buffer grows (at least doubling) when a batch needs more and
    is otherwise handed out as a view, so building a new batch on the pool
    allocates nothing once the pool has warmed up. A batch built on a pool must
    have finished on the device, and its results been read, before the next batch
    is built on the same pool."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.bufs: dict = {}
        self.workspaces = (Workspace(self.device, 256), Workspace(self.device),
                           Workspace(self.device))

    def get(self, name: str, n: int, dtype, pinned: bool = False) -> torch.Tensor:
        t = self.bufs.get(name)
        if t is None or t.numel() < n or t.dtype != dtype:
            cap = max(int(n), 1)
            if t is not None and t.dtype == dtype:
                cap = max(cap, 2 * t.numel())
            t = (torch.empty(cap, dtype=dtype, pin_memory=True) if pinned else
                 torch.empty(cap, dtype=dtype, device=self.device))
            self.bufs[name] = t
        return t[:n]


class Batch:
    """Many independent sequence sets ranked and partitioned together.

    ``sets``: objects with ``codes`` (uint8), ``offsets`` (int64, N+1) and ``p``.
    All sets share one count launch, one block-diagonal rank (one persistent
    GEMM launch over every set's tiles) and one batched partition.

    The host arrays are staged in pinned memory and copied with ``upload()``
    (asynchronous, on the given stream). ``plan(depth, tile, budget)`` sizes the
    work: with ``bound=True`` (depth >= 1) from host-side bounds alone
    (sad_batch_plan_bound: no device work, no synchronisation), otherwise from the
    counts (sad_batch_plan_make: counts the batch and synchronises). ``run()``
    then launches count -> lengths -> rank -> partition without any host
    synchronisation, so ``capture(graph)`` records it into a library Graph:
    the first batch instantiates it and each later batch captured into the same
    Graph only updates its parameters. ``workspaces`` (count, rank, partition)
    may be shared by batches that never run at the same time; ``pool`` (a
    BatchPool) supplies them and every other buffer. ``count=True`` launches the
    count on ``stream`` as soon as the inputs are uploaded (then run or capture
    with count=False).
    """

    def __init__(self, sets, device=None, k: int = 3, alphabet: int = 20, workspaces=None,
                 stream=None, pin: bool = True, pool: "BatchPool | None" = None,
                 count: bool = False):
        import numpy as np
        self.device = torch.device(device or "cuda")
        self.k, self.alphabet = k, alphabet
        self.n = np.array([s.offsets.shape[0] - 1 for s in sets], dtype=np.int32)
        self.p = np.array([s.p for s in sets], dtype=np.int32)
        nt = int(self.n.sum())
        self.seq_begin = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.boff_begin = np.concatenate([[0], np.cumsum(self.p + 1)]).astype(np.int64)
        self.piv_begin = np.concatenate([[0], np.cumsum(self.p - 1)]).astype(np.int64)
        spans = [(int(s.offsets[0]), int(s.offsets[-1])) for s in sets]
        self.total_len = sum(b - a for a, b in spans)
        dev = self.device
        on_gpu = dev.type == "cuda"
        pin = pin and on_gpu
        if pool is not None:
            def dbuf(name, n, dtype):
                return pool.get(name, n, dtype)

            def hbuf(name, n, dtype):
                return pool.get(name, n, dtype, pinned=pin)
            workspaces = pool.workspaces
        else:
            def dbuf(name, n, dtype):
                return torch.empty(n, dtype=dtype, device=dev)

            def hbuf(name, n, dtype):
                return torch.empty(n, dtype=dtype, pin_memory=pin)
        # host staging, written in place: codes set after set, offsets rebased
        h_codes = hbuf("h_codes", max(self.total_len, 1), torch.uint8)
        h_offsets = hbuf("h_offsets", nt + 1, torch.int64)
        hc, ho = h_codes.numpy(), h_offsets.numpy()
        at, row = 0, 0
        ho[0] = 0
        for s, (a, b) in zip(sets, spans):
            hc[at:at + b - a] = s.codes[a:b]
            m = s.offsets.shape[0] - 1
            ho[row + 1:row + m + 1] = s.offsets[1:] - a + at
            at += b - a
            row += m
        h_n = hbuf("h_n", self.n_sets, torch.int32)
        h_p = hbuf("h_p", self.n_sets, torch.int32)
        h_n.numpy()[:] = self.n
        h_p.numpy()[:] = self.p
        self.h_codes, self.h_offsets = hc[:self.total_len], ho
        self.h_in = dict(codes=h_codes[:self.total_len], offsets=h_offsets, n=h_n, p=h_p)
        self.codes = dbuf("codes", max(self.total_len, 1), torch.uint8)
        self.offsets = dbuf("offsets", nt + 1, torch.int64)
        self.d_n = dbuf("d_n", self.n_sets, torch.int32)
        self.d_p = dbuf("d_p", self.n_sets, torch.int32)
        eps = alphabet ** k
        self.counts = dbuf("counts", nt * eps, torch.int32).view(nt, eps)
        self.word_max = dbuf("word_max", eps, torch.int32)
        if workspaces is None:
            workspaces = (Workspace(dev, 256), Workspace(dev), Workspace(dev))
        self.ws_count, self.ws_rank, self.ws_part = workspaces
        self.upload(stream)
        if count:
            # the device counts while the host sets up the rest
            self.count(stream)
        # lengths: derived on the device by the library in run(); host-built off the GPU
        self.lengths = (dbuf("lengths", nt, torch.int32) if on_gpu else
                        torch.from_numpy(np.diff(ho).astype(np.int32)))
        self.key_hi = dbuf("key_hi", nt, torch.uint64)
        self.key_lo = dbuf("key_lo", nt, torch.uint64)
        self.rank = dbuf("rank", nt, torch.float64)
        self.bucket_offsets = dbuf("bucket_offsets", int(self.boff_begin[-1]), torch.int32)
        self.members = dbuf("members", nt, torch.int32)
        self.pivot_idx = dbuf("pivot_idx", max(int(self.piv_begin[-1]), 1), torch.int32)
        self.plan_ = None
        self.graph = None

    @property
    def n_sets(self) -> int:
        return int(self.n.shape[0])

    @property
    def h2d_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in self.h_in.values())

    def upload(self, stream=None):
        """Host -> device copies of the batch's inputs (asynchronous from pinned memory)."""
        nb = self.device.type == "cuda"
        ctx = torch.cuda.stream(stream) if (nb and stream is not None) else contextlib.nullcontext()
        with ctx:
            self.codes[:self.h_in["codes"].numel()].copy_(self.h_in["codes"], non_blocking=nb)
            self.offsets.copy_(self.h_in["offsets"], non_blocking=nb)
            self.d_n.copy_(self.h_in["n"], non_blocking=nb)
            self.d_p.copy_(self.h_in["p"], non_blocking=nb)

    def count(self, stream=None):
        kmer_count(self.codes, self.offsets, self.k, self.alphabet, ws=self.ws_count,
                   out=self.counts, stream=stream, check=False, word_max=self.word_max)

    def plan(self, depth: int = 1, stream=None, tile: int = 0, budget: int = 0,
             bound: bool | None = None) -> BatchPlan:
        """Sizes the rank and partition workspaces. ``bound`` (default: depth >= 1):
        from host-side bounds, asynchronous; otherwise counts the batch and reads
        the exact sizes back (synchronous)."""
        import numpy as np
        if bound is None:
            bound = depth >= 1
        plan = BatchPlan()
        plan.rank.depth, plan.rank.budget, plan.rank.tile = int(depth), int(budget), int(tile)
        h_n = np.ascontiguousarray(self.n)
        h_p = np.ascontiguousarray(self.p)
        n_ptr = h_n.ctypes.data_as(ctypes.c_void_p)
        p_ptr = h_p.ctypes.data_as(ctypes.c_void_p)
        if bound:
            _check(_load().sad_batch_plan_bound(n_ptr, p_ptr, self.n_sets, self.total_len, self.k,
                                                self.alphabet, ctypes.byref(plan)),
                   "sad_batch_plan_bound")
        else:
            self.count(stream)
            self.ws_count.check("kmer_count (batch)", stream)
            args = (_ptr(self.counts), n_ptr, p_ptr, _ptr(self.d_n), self.n_sets, self.k,
                    self.alphabet, ctypes.byref(plan))
            self.ws_rank.ensure(256)
            rc = _load().sad_batch_plan_make(*args, _ptr(self.ws_rank.buf), self.ws_rank.nbytes,
                                             _stream(stream))
            if rc == ERR_WORKSPACE:
                self.ws_rank.ensure(plan.rank.ws_bytes)
                plan.rank.depth, plan.rank.budget = int(depth), int(budget)
                plan.rank.tile = int(tile)
                rc = _load().sad_batch_plan_make(*args, _ptr(self.ws_rank.buf),
                                                 self.ws_rank.nbytes, _stream(stream))
            _check(rc, "sad_batch_plan_make")
        # every workspace at its size before run() (which a capture records: no
        # allocation may happen inside it)
        self.ws_count.ensure(workspace_bytes(OP_COUNT, int(self.n.sum()), self.k, self.alphabet))
        self.ws_rank.ensure(plan.rank.ws_bytes)
        self.ws_part.ensure(plan.part_ws_bytes)
        self.plan_ = plan
        return plan

    def run(self, stream=None, count: bool = True):
        """count -> lengths -> rank -> partition of every set; no host synchronisation."""
        if self.plan_ is None:
            raise RuntimeError("Batch.plan() first")
        lib, st = _load(), _stream(stream)
        if count:
            self.count(stream)
        _check(lib.sad_seq_lengths(_ptr(self.offsets), int(self.offsets.numel() - 1),
                                   _ptr(self.lengths), _ptr(self.ws_count.buf), st),
               "sad_seq_lengths")
        _check(lib.sad_batch_rank(_ptr(self.counts), _ptr(self.lengths), _ptr(self.word_max),
                                  _ptr(self.d_n),
                                  self.k, self.alphabet, ctypes.byref(self.plan_),
                                  _ptr(self.key_hi), _ptr(self.key_lo), _ptr(self.rank),
                                  _ptr(self.ws_rank.buf), self.ws_rank.nbytes, st),
               "sad_batch_rank")
        _check(lib.sad_batch_partition(_ptr(self.key_hi), _ptr(self.key_lo), _ptr(self.d_n),
                                       _ptr(self.d_p), ctypes.byref(self.plan_),
                                       _ptr(self.bucket_offsets), _ptr(self.members),
                                       _ptr(self.pivot_idx), _ptr(self.ws_part.buf),
                                       self.ws_part.nbytes, st), "sad_batch_partition")

    def capture(self, graph: Graph | None = None, stream=None, count: bool = True) -> Graph:
        """Records run() into ``graph`` (a new Graph if None): instantiated on its
        first capture, updated in place on later ones. Capture needs a stream other
        than the legacy default one: a side stream is used when none is given.
        ``count=False`` leaves the count out of the graph (the caller launched it
        already, e.g. to start the device while the host builds the graph)."""
        g = graph or Graph()
        s = stream or torch.cuda.Stream(self.device)
        if stream is None:
            s.wait_stream(torch.cuda.current_stream(self.device))
        g.capture(lambda st: self.run(stream=st, count=count), s)
        self.graph = g
        return g

    def replay(self, stream=None):
        """Runs the batch's captured graph on ``stream`` (default: the current stream)."""
        self.graph.launch(stream if stream is not None else torch.cuda.current_stream(self.device))

    def check(self, stream=None):
        self.ws_count.check("kmer_count (batch)", stream)
        self.ws_rank.check("sad_batch_rank", stream)
        self.ws_part.check("sad_batch_partition", stream)

    def result(self, s: int) -> dict:
        """Host copies of set s's outputs."""
        a, b = int(self.seq_begin[s]), int(self.seq_begin[s + 1])
        oa, ob = int(self.boff_begin[s]), int(self.boff_begin[s + 1])
        pa, pb = int(self.piv_begin[s]), int(self.piv_begin[s + 1])
        return dict(counts=self.counts[a:b].cpu().numpy(), key_hi=self.key_hi[a:b].cpu().numpy(),
                    key_lo=self.key_lo[a:b].cpu().numpy(), rank=self.rank[a:b].cpu().numpy(),
                    bucket_offsets=self.bucket_offsets[oa:ob].cpu().numpy(),
                    members=self.members[a:b].cpu().numpy(),
                    pivot_idx=self.pivot_idx[pa:pb].cpu().numpy())
