"""Seeded synthetic protein sequence sets shaped like the paper's workloads.

This module only draws random inputs. It holds none of the method's arithmetic
(no k-mer counting, no similarity, no ranks, no sorting of keys), so both the CPU
oracle's tests and the CUDA path can take their inputs from it.

The paper evaluates on Rose-generated protein families with lengths 100-2000,
set sizes 100-20000 and a range of phylogenetic distances (Sec. 4, "Rose"
experiments), and on PF00500 (1048 sequences, maximal length 523). Neither the
Rose generator nor those datasets are available, so the sets here follow a
simple star-phylogeny family model instead:

* residues are drawn from a 20-letter amino-acid background distribution
  (Robinson & Robinson 1991 frequencies, the table BLAST uses as its default
  composition), alphabet order ``ACDEFGHIKLMNPQRSTVWY`` and codes 0..19;
* a family is a random ancestor; every member is derived from it
  independently: each position is substituted with probability r ~ U[0.20, 0.40]
  by a background residue different from the original, then each position
  starts an indel with probability 0.02 (insertion or deletion with equal odds,
  length uniform in 1..10, inserted residues from the background; overlapping
  deletions merge, and a member that would drop below ``MIN_LEN`` residues
  keeps none of its deletions). All members of a family are drawn at once.

A sequence set is returned in the layout the C-ABI consumes: ``codes`` (uint8,
all sequences concatenated) and ``offsets`` (int64, N+1 entries, CSR).

Every generator takes ``seed`` and builds its stream from
``numpy.random.Generator(PCG64(SeedSequence([seed, config_id, ...])))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ALPHABET = "ACDEFGHIKLMNPQRSTVWY"

# Robinson & Robinson (1991) amino-acid background frequencies, in ALPHABET order.
BACKGROUND = np.array([
    0.07805, 0.01925, 0.05364, 0.06295, 0.03856, 0.07377, 0.02199, 0.05142,
    0.05744, 0.09019, 0.02243, 0.04487, 0.05203, 0.04264, 0.05129, 0.07120,
    0.05841, 0.06441, 0.01330, 0.03216,
], dtype=np.float64)
BACKGROUND = BACKGROUND / BACKGROUND.sum()
_CDF = np.cumsum(BACKGROUND)
_CDF[-1] = 1.0

MIN_LEN = 3            # no sequence shorter than the default k-mer length
SUB_RATE = (0.20, 0.40)
INDEL_RATE = 0.02
INDEL_LEN = (1, 10)


@dataclasses.dataclass
class SeqSet:
    """One sequence set: CSR layout plus the partition parameter p."""
    codes: np.ndarray      # uint8 [sum L]
    offsets: np.ndarray    # int64 [N + 1]
    p: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def seq(self, i: int) -> np.ndarray:
        return self.codes[self.offsets[i]:self.offsets[i + 1]]

    def take(self, idx, p: int | None = None) -> "SeqSet":
        """The sequences idx (in that order) as a set of their own."""
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx]
        offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        codes = np.concatenate([self.seq(i) for i in idx]) if idx.size else self.codes[:0]
        return SeqSet(codes=codes, offsets=offs, p=self.p if p is None else p,
                      name=f"{self.name}[{idx.size}]")


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


# residue of each 16-bit uniform value: the background CDF quantised to 1/65536
_TABLE = np.searchsorted(_CDF, (np.arange(65536) + 0.5) / 65536.0, side="right").clip(0, 19) \
    .astype(np.uint8)


def background(rng: np.random.Generator, n: int) -> np.ndarray:
    """n residues iid from the background distribution (codes 0..19)."""
    return _TABLE[rng.integers(0, 65536, size=n, dtype=np.uint16)]


def mutate_family(rng, ancestor: np.ndarray, m: int):
    """m members of one family, all derived from ``ancestor`` at once.

    Member j gets its own substitution rate r_j ~ U[0.20, 0.40]: each position is
    replaced with probability r_j by a background residue different from the
    original. Then each position starts an indel with probability 0.02:
    insertion or deletion with equal odds, length uniform in 1..10. A deletion at
    i removes positions [i, i + len) (overlapping deletions merge); an insertion
    at i puts len background residues before position i. A member that would end
    up shorter than MIN_LEN keeps its insertions but none of its deletions.
    Returns (codes uint8 [total], lengths int64 [m]).
    """
    L = ancestor.shape[0]
    rate = rng.uniform(SUB_RATE[0], SUB_RATE[1], size=m).astype(np.float32)
    seq = np.broadcast_to(ancestor, (m, L)).copy()
    idx = np.nonzero(rng.random((m, L), dtype=np.float32) < rate[:, None])
    new = background(rng, idx[0].size)
    same = new == seq[idx]
    while same.any():                                   # redraw until different
        new[same] = background(rng, int(same.sum()))
        same = new == seq[idx]
    seq[idx] = new
    ev = np.flatnonzero(rng.random(m * L, dtype=np.float32) < INDEL_RATE)
    is_ins = rng.random(ev.size, dtype=np.float32) < 0.5
    ln = rng.integers(INDEL_LEN[0], INDEL_LEN[1] + 1, size=ev.size)
    # deleted positions: difference array of the deletion ranges
    d, dl = ev[~is_ins], ln[~is_ins]
    dr, dc = d // L, d % L
    diff = np.zeros((m, L + 1), dtype=np.int8)
    np.add.at(diff, (dr, dc), 1)
    np.add.at(diff, (dr, np.minimum(dc + dl, L)), -1)
    keep = np.cumsum(diff[:, :L], axis=1, dtype=np.int8) == 0
    ins = np.zeros(m * L, dtype=np.int32)
    ins[ev[is_ins]] = ln[is_ins]
    ins = ins.reshape(m, L)
    short = keep.sum(axis=1) + ins.sum(axis=1) < MIN_LEN
    if short.any():
        keep[short] = True
    piece = (ins + keep).ravel()                         # output slots per position
    lengths = (ins.sum(axis=1) + keep.sum(axis=1)).astype(np.int64)
    total = int(lengths.sum())
    out = np.empty(total, dtype=np.uint8)
    kept = keep.ravel()
    res_slot = (np.cumsum(piece) - piece + ins.ravel())[kept]  # slot of each kept residue
    is_res = np.zeros(total, dtype=bool)
    is_res[res_slot] = True
    out[res_slot] = seq.ravel()[kept]
    out[~is_res] = background(rng, total - res_slot.size)
    return out, lengths


def _pack(seqs, p: int, name: str) -> SeqSet:
    lens = np.fromiter((s.shape[0] for s in seqs), dtype=np.int64, count=len(seqs))
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    codes = np.concatenate(seqs).astype(np.uint8) if seqs else np.zeros(0, np.uint8)
    return SeqSet(codes=codes, offsets=offsets, p=p, name=name)


def iid_set(n: int, len_lo: int, len_hi: int, p: int, seed: int = 0,
            stream: int = 1, name: str = "") -> SeqSet:
    """n sequences of iid background residues, lengths uniform in [len_lo, len_hi]."""
    rng = rng_for(seed, stream)
    lens = rng.integers(len_lo, len_hi + 1, size=n)
    return _pack([background(rng, int(L)) for L in lens], p, name)


def loguniform_int(rng, lo: float, hi: float, size=None):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def family_set(n_families: int, per_family, ancestor_len, p: int, seed: int,
               stream, name: str = "") -> SeqSet:
    """Families under the star model above.

    ``per_family``: int or array of member counts. ``ancestor_len(rng)`` draws one
    ancestor length.
    """
    rng = rng_for(seed, *np.atleast_1d(stream).tolist())
    sizes = np.full(n_families, per_family) if np.isscalar(per_family) else np.asarray(per_family)
    chunks, lens = [], []
    for f in range(n_families):
        anc = background(rng, max(MIN_LEN, int(ancestor_len(rng))))
        if int(sizes[f]) == 0:
            continue
        codes, ln = mutate_family(rng, anc, int(sizes[f]))
        chunks.append(codes)
        lens.append(ln)
    lens = np.concatenate(lens) if lens else np.zeros(0, np.int64)
    offsets = np.zeros(lens.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    codes = np.concatenate(chunks) if chunks else np.zeros(0, np.uint8)
    return SeqSet(codes=codes, offsets=offsets, p=p, name=name)


def _split_even(n: int, parts: int) -> np.ndarray:
    base = np.full(parts, n // parts, dtype=np.int64)
    base[: n % parts] += 1
    return base


# ---- the five workload configurations --------------------------------------

def config1(seed: int = 0) -> SeqSet:
    """N=200 iid sequences, lengths uniform 100-400, p=4."""
    return iid_set(200, 100, 400, p=4, seed=seed, stream=1, name="c1_n200_iid")


def config2(seed: int = 0) -> SeqSet:
    """N=20000 in 50 families of 400; ancestor length N(300,100) clipped to [50,1000]; p=16."""
    def alen(rng):
        return int(np.clip(round(rng.normal(300.0, 100.0)), 50, 1000))
    return family_set(50, 400, alen, p=16, seed=seed, stream=2, name="c2_n20000_fam50")


def config3(seed: int = 0) -> SeqSet:
    """N=100000 in 500 families of 200; ancestor length log-uniform [50,2000]; p=64."""
    def alen(rng):
        return int(loguniform_int(rng, 50, 2000))
    return family_set(500, 200, alen, p=64, seed=seed, stream=3, name="c3_n100000_fam500")


def batch_set(index: int, seed: int = 0, n_lo=50, n_hi=5000, stream_id=4,
              p_rule=lambda n: max(1, math.ceil(n / 500))) -> SeqSet:
    """One set of the batching workload: N log-uniform [50,5000], lengths
    log-uniform [50,2000], 5-100 families, p = ceil(N/500)."""
    rng = rng_for(seed, stream_id, index, 0)
    n = int(loguniform_int(rng, n_lo, n_hi))
    fams = int(min(rng.integers(5, 101), n))
    sizes = _split_even(n, fams)

    def alen(r):
        return int(loguniform_int(r, 50, 2000))
    s = family_set(fams, sizes, alen, p=p_rule(n), seed=seed, stream=[stream_id, index, 1],
                   name=f"c{stream_id}_set{index}")
    return s


def _batch_set_job(args):
    kind, index, seed = args
    return serving_set(index, seed) if kind == "serve" else batch_set(index, seed)


def many_sets(kind: str, indices, seed: int = 0, workers: int | None = None):
    """Sets ``indices`` of the batching ("batch") or serving ("serve") workload.
    Independent sets are drawn in a pool of ``workers`` spawned processes (each
    set has its own seed stream, so the result does not depend on the pool)."""
    import os
    indices = list(indices)
    if workers is None:
        workers = min(len(indices), max(1, (os.cpu_count() or 1) - 1), 32)
    jobs = [(kind, i, seed) for i in indices]
    if workers <= 1 or len(indices) < 8:
        return [_batch_set_job(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_batch_set_job, jobs, chunksize=max(1, len(jobs) // (4 * workers)))


def config4(seed: int = 0, n_sets: int = 512, workers: int | None = None):
    """512 independent sets for the batched launch."""
    return many_sets("batch", range(n_sets), seed, workers)


def serving_set(index: int, seed: int = 0) -> SeqSet:
    """One request of the serving workload: N log-uniform [100,20000], lengths
    log-uniform [50,2000], 5-100 families, p=16."""
    return batch_set(index, seed, n_lo=100, n_hi=20000, stream_id=5, p_rule=lambda n: 16)


def poisson_arrivals(n_requests: int, rate_per_s: float = 200.0, seed: int = 0) -> np.ndarray:
    """Arrival times (seconds from start) of a Poisson process."""
    rng = rng_for(seed, 5, 999_999)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))


CONFIGS = {1: config1, 2: config2, 3: config3}


def config(i: int, seed: int = 0):
    if i in CONFIGS:
        return CONFIGS[i](seed)
    if i == 4:
        return config4(seed)
    raise ValueError(f"no single-set generator for config {i}")


# ---- small helpers used by tests -------------------------------------------

def from_strings(seqs, p: int = 1, name: str = "") -> SeqSet:
    """Pack amino-acid strings (letters of ALPHABET) into a SeqSet."""
    idx = {c: i for i, c in enumerate(ALPHABET)}
    arrs = [np.array([idx[c] for c in s], dtype=np.uint8) for s in seqs]
    return _pack(arrs, p, name)


def random_small(n: int, len_lo: int, len_hi: int, seed: int, alphabet: int = 20,
                 p: int = 1) -> SeqSet:
    """n uniform-random sequences over ``alphabet`` letters (for tiny cases)."""
    rng = rng_for(seed, 77)
    lens = rng.integers(len_lo, len_hi + 1, size=n)
    return _pack([rng.integers(0, alphabet, size=int(L)).astype(np.uint8) for L in lens],
                 p, f"rand{n}")


def random_keys(n: int, seed: int, distinct: int | None = None):
    """Seeded 128-bit keys (hi, lo) for partition-only cases. ``distinct`` limits
    the number of distinct values so ties occur."""
    rng = rng_for(seed, 88)
    if distinct is None:
        hi = rng.integers(0, 1 << 20, size=n, dtype=np.uint64)
        lo = rng.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)
    else:
        pool_hi = rng.integers(0, 1 << 20, size=distinct, dtype=np.uint64)
        pool_lo = rng.integers(0, np.iinfo(np.uint64).max, size=distinct, dtype=np.uint64,
                               endpoint=True)
        pick = rng.integers(0, distinct, size=n)
        hi, lo = pool_hi[pick], pool_lo[pick]
    return hi.astype(np.uint64), lo.astype(np.uint64)
