"""CPU oracle for the k-mer count, k-mer rank and regular-sampling partition.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this package to check the CUDA library; the product path
never imports it. The arithmetic lives in ``sad_oracle.c`` (plain C, built here
with gcc); this module only builds, loads and marshals numpy arrays. It shares no
code with the CUDA path.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  kmer_count   brute-force substring enumeration; sum of counts = L - k + 1;
               homopolymer closed form.
  shared/term  threshold identity, self-similarity F(x,x)=1, symmetry,
               0 <= F <= 1, hand-derived examples from Eq. 1, exact big-integer
               floor for every (S, D) on a grid.
  kmer_rank    exact rational sum with fractions on small sets:
               0 <= 2^64 * sum_j F - key < N; hand-derived example; FP64 view
               within 1e-12 of the compensated FP64 mean.
  partition    hand-derived regular-sampling example (N=16, p=4; N=8, p=2),
               concatenated buckets equal the sorted order, bucket intervals
               (y_{i-1}, y_i], the 2N/p load bound when p | N and N >= p^3.
  rank_vs      exact big-integer sum over a reference multiset with shared counts
               from substring enumeration; duplicates count twice; reference =
               every sequence gives the centralised key.
  local_samples  hand-derived positions (keys = index and reversed keys), block
               bounds floor(bN/p).
  ln_q         within 2^-30 of ln x (decimal arithmetic) over a sweep of x,
               including powers of two and values near them.
  rank_dist    closed forms (F = 0 gives ln b, F = 1 gives -ln(1 + 1/b)), exact
               sums from string multisets, the FP64 mean within the
               quantisation bound.
  global_rank  p = 1 with ks = N samples every sequence once (positions
               floor(j N / (N + 1)), j = 1..N, are 0..N-1), so the globalised key
               equals the centralised one; the whole pipeline against exact
               big-integer sums built from the sampled indices.
  local_ranks  each block's keys equal the centralised keys of that block taken
               as a set of its own (nothing outside the block enters).
  rank_vs_dist every sequence as the reference set gives rank_dist.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sad_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no fast-math, no FP contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC",
                           "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.sad_oracle_kmer_count.argtypes = [P, P, i32, i32, i32, P]
        lib.sad_oracle_kmer_count.restype = ctypes.c_int
        lib.sad_oracle_shared_count.argtypes = [P, P, i64]
        lib.sad_oracle_shared_count.restype = i64
        lib.sad_oracle_term.argtypes = [u64, u64, P, P]
        lib.sad_oracle_term.restype = None
        lib.sad_oracle_kmer_rank.argtypes = [P, P, i32, i32, i32, P, i32, P, P, P, P, i32]
        lib.sad_oracle_kmer_rank.restype = ctypes.c_int
        lib.sad_oracle_partition.argtypes = [P, P, i32, i32, P, P, P]
        lib.sad_oracle_partition.restype = ctypes.c_int
        lib.sad_oracle_rank_vs.argtypes = [P, P, i32, i32, i32, P, i32, P, P, P, i32]
        lib.sad_oracle_rank_vs.restype = ctypes.c_int
        lib.sad_oracle_local_samples.argtypes = [P, P, i32, i32, i32, P]
        lib.sad_oracle_local_samples.restype = ctypes.c_int
        lib.sad_oracle_ln_q.argtypes = [u64]
        lib.sad_oracle_ln_q.restype = ctypes.c_int64
        lib.sad_oracle_rank_dist.argtypes = [P, P, i32, i32, i32, i32, P, P, P, i32]
        lib.sad_oracle_rank_dist.restype = ctypes.c_int
        lib.sad_oracle_rank_vs_dist.argtypes = [P, P, i32, i32, i32, i32, P, i32, P, P, i32]
        lib.sad_oracle_rank_vs_dist.restype = ctypes.c_int
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what}: status {rc}")


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
               else (os.cpu_count() or 1))


def kmer_count(codes: np.ndarray, offsets: np.ndarray, k: int = 3,
               alphabet: int = 20) -> np.ndarray:
    """int32 [N, alphabet**k] count vectors (Sec. 3, "k-mer Rank")."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.shape[0] - 1
    out = np.zeros((n, alphabet ** k), dtype=np.int32)
    _check(_load().sad_oracle_kmer_count(_ptr(codes), _ptr(offsets), n, k, alphabet,
                                         _ptr(out)), "kmer_count")
    return out


def shared_count(cx: np.ndarray, cy: np.ndarray) -> int:
    """Eq. 1 numerator: sum over words of min(c^X, c^Y)."""
    cx = np.ascontiguousarray(cx, dtype=np.int32)
    cy = np.ascontiguousarray(cy, dtype=np.int32)
    return int(_load().sad_oracle_shared_count(_ptr(cx), _ptr(cy), cx.shape[0]))


def term(s: int, d: int) -> int:
    """floor(S * 2^64 / D) as a Python int."""
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    _load().sad_oracle_term(s, d, ctypes.byref(hi), ctypes.byref(lo))
    return (hi.value << 64) | lo.value


def kmer_rank(counts: np.ndarray, lengths: np.ndarray, k: int = 3, alphabet: int = 20,
              rows=None, threads: int | None = None, with_fp64: bool = False):
    """Keys (hi, lo) and rank views for all rows, or for ``rows`` only (Eq. 3).

    Returns (key_hi uint64, key_lo uint64, rank float64[, rank_fp64 float64]).
    """
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    n = counts.shape[0]
    if rows is None:
        rows_arr, n_rows, rows_p = None, n, None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int32)
        n_rows, rows_p = rows_arr.shape[0], _ptr(rows_arr)
    hi = np.zeros(n_rows, np.uint64)
    lo = np.zeros(n_rows, np.uint64)
    rank = np.zeros(n_rows, np.float64)
    fp = np.zeros(n_rows, np.float64) if with_fp64 else None
    _check(_load().sad_oracle_kmer_rank(
        _ptr(counts), _ptr(lengths), n, k, alphabet, rows_p, n_rows, _ptr(hi), _ptr(lo),
        _ptr(rank), _ptr(fp) if fp is not None else None,
        threads or default_threads()), "kmer_rank")
    return (hi, lo, rank, fp) if with_fp64 else (hi, lo, rank)


def partition(key_hi: np.ndarray, key_lo: np.ndarray, p: int):
    """Regular-sampling partition (Sec. 3.1.2, Algorithm 2 steps 7-11).

    Returns (bucket_offsets int32[p+1], members int32[N], pivot_idx int32[p-1]).
    """
    key_hi = np.ascontiguousarray(key_hi, dtype=np.uint64)
    key_lo = np.ascontiguousarray(key_lo, dtype=np.uint64)
    n = key_hi.shape[0]
    offs = np.zeros(p + 1, np.int32)
    mem = np.zeros(max(n, 1), np.int32)
    piv = np.zeros(max(p - 1, 1), np.int32)
    _check(_load().sad_oracle_partition(_ptr(key_hi), _ptr(key_lo), n, p, _ptr(offs),
                                        _ptr(mem), _ptr(piv)), "partition")
    return offs, mem[:n], piv[:max(p - 1, 0)]


def run_set(codes, offsets, p: int, k: int = 3, alphabet: int = 20, threads=None):
    """count -> rank -> partition for one set; returns a dict of numpy arrays."""
    counts = kmer_count(codes, offsets, k, alphabet)
    lengths = np.diff(np.asarray(offsets, dtype=np.int64))
    hi, lo, rank = kmer_rank(counts, lengths, k, alphabet, threads=threads)
    offs, mem, piv = partition(hi, lo, p)
    return dict(counts=counts, key_hi=hi, key_lo=lo, rank=rank,
                bucket_offsets=offs, members=mem, pivot_idx=piv)


def rank_vs(counts: np.ndarray, lengths: np.ndarray, ref, k: int = 3, alphabet: int = 20,
            threads: int | None = None):
    """Globalised rank (Sec. 3.1.1, Algorithm 2 step 6): every sequence against the
    reference multiset ``ref`` (input indices). Returns (key_hi, key_lo, rank) with
    rank = key / (len(ref) 2^64)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    n = counts.shape[0]
    hi = np.zeros(n, np.uint64)
    lo = np.zeros(n, np.uint64)
    rank = np.zeros(n, np.float64)
    _check(_load().sad_oracle_rank_vs(_ptr(counts), _ptr(lengths), n, k, alphabet, _ptr(ref),
                                      ref.shape[0], _ptr(hi), _ptr(lo), _ptr(rank),
                                      threads or default_threads()), "rank_vs")
    return hi, lo, rank


def block_bounds(n: int, p: int) -> np.ndarray:
    """Start of each of the p contiguous blocks, floor(b N / p), and N at the end."""
    return np.array([b * n // p for b in range(p + 1)], dtype=np.int64)


def local_ranks(counts: np.ndarray, lengths: np.ndarray, p: int, k: int = 3,
                alphabet: int = 20, threads: int | None = None):
    """Algorithm 2 step 2: each block's sequences ranked against their own block
    only (Eq. 3 over the block). Returns (key_hi, key_lo) in input order."""
    n = counts.shape[0]
    bnd = block_bounds(n, p)
    hi = np.zeros(n, np.uint64)
    lo = np.zeros(n, np.uint64)
    for b in range(p):
        a, e = int(bnd[b]), int(bnd[b + 1])
        if e > a:
            h, l, _ = kmer_rank(counts[a:e], np.asarray(lengths)[a:e], k, alphabet,
                                threads=threads)
            hi[a:e], lo[a:e] = h, l
    return hi, lo


def local_samples(key_hi: np.ndarray, key_lo: np.ndarray, p: int, ks: int) -> np.ndarray:
    """Algorithm 2 steps 3-4: ks regular samples per block of the locally sorted
    order (positions floor(j w_b / (ks + 1)), j = 1..ks); input indices, block-major."""
    key_hi = np.ascontiguousarray(key_hi, dtype=np.uint64)
    key_lo = np.ascontiguousarray(key_lo, dtype=np.uint64)
    out = np.zeros(p * ks, np.int32)
    _check(_load().sad_oracle_local_samples(_ptr(key_hi), _ptr(key_lo), key_hi.shape[0], p, ks,
                                            _ptr(out)), "local_samples")
    return out


def global_rank(counts: np.ndarray, lengths: np.ndarray, p: int, ks: int, k: int = 3,
                alphabet: int = 20, threads: int | None = None):
    """Algorithm 2 steps 2-6: local ranks per block, ks samples per block of the
    locally sorted order, every sequence re-ranked against the ks x p samples.
    Returns (key_hi, key_lo, rank, samples)."""
    lh, ll = local_ranks(counts, lengths, p, k, alphabet, threads)
    samples = local_samples(lh, ll, p, ks)
    hi, lo, rank = rank_vs(counts, lengths, samples, k, alphabet, threads)
    return hi, lo, rank, samples


def ln_q(x: int) -> int:
    """ln(x) * 2^32 as the fixed-point value of the distance-form rank (x >= 1)."""
    return int(_load().sad_oracle_ln_q(int(x)))


def rank_dist(counts: np.ndarray, lengths: np.ndarray, delta_den: int, k: int = 3,
              alphabet: int = 20, threads: int | None = None, with_fp64: bool = False):
    """Eq. 2 / Eq. 3 literally, with Delta = 1 / delta_den: key_i = sum_j
    (ln_q(b D) - ln_q(D + b S)) (ln times 2^32), rank_i = key_i 2^-32 / N.
    Returns (key int64, rank float64[, rank_fp64])."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    n = counts.shape[0]
    key = np.zeros(n, np.int64)
    rank = np.zeros(n, np.float64)
    fp = np.zeros(n, np.float64) if with_fp64 else None
    _check(_load().sad_oracle_rank_dist(_ptr(counts), _ptr(lengths), n, k, alphabet, delta_den,
                                        _ptr(key), _ptr(rank),
                                        _ptr(fp) if fp is not None else None,
                                        threads or default_threads()), "rank_dist")
    return (key, rank, fp) if with_fp64 else (key, rank)


def dist_sort_key(key: np.ndarray):
    """The signed distance keys as unsigned (hi, lo) keys with the same order
    (offset binary), for the partition."""
    lo = (np.asarray(key, np.int64).view(np.uint64) ^ np.uint64(1 << 63))
    return np.zeros_like(lo), lo


def rank_vs_dist(counts: np.ndarray, lengths: np.ndarray, delta_den: int, ref, k: int = 3,
                 alphabet: int = 20, threads: int | None = None):
    """The distance form against a reference multiset (input indices):
    key_i = sum_r (ln_q(b D) - ln_q(D + b S)), rank_i = key_i 2^-32 / len(ref).
    Returns (key int64, rank float64)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    lengths = np.ascontiguousarray(lengths, dtype=np.int64)
    ref = np.ascontiguousarray(ref, dtype=np.int32)
    n = counts.shape[0]
    key = np.zeros(n, np.int64)
    rank = np.zeros(n, np.float64)
    _check(_load().sad_oracle_rank_vs_dist(_ptr(counts), _ptr(lengths), n, k, alphabet, delta_den,
                                           _ptr(ref), ref.shape[0], _ptr(key), _ptr(rank),
                                           threads or default_threads()), "rank_vs_dist")
    return key, rank
