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
  length uniform in 1..10, inserted residues from the background; a deletion
  that would leave fewer than ``MIN_LEN`` residues is skipped).

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


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def background(rng: np.random.Generator, n: int) -> np.ndarray:
    """n residues iid from the background distribution (codes 0..19)."""
    u = rng.random(n)
    return np.searchsorted(_CDF, u, side="right").astype(np.uint8).clip(0, 19)


def _substitute(rng, seq: np.ndarray, rate: float) -> np.ndarray:
    out = seq.copy()
    pos = np.nonzero(rng.random(seq.shape[0]) < rate)[0]
    if pos.size:
        new = background(rng, pos.size)
        same = new == out[pos]
        while same.any():                      # redraw until different
            new[same] = background(rng, int(same.sum()))
            same = new == out[pos]
        out[pos] = new
    return out


def _indels(rng, seq: np.ndarray) -> np.ndarray:
    starts = np.nonzero(rng.random(seq.shape[0]) < INDEL_RATE)[0]
    if starts.size == 0:
        return seq
    kinds = rng.random(starts.size) < 0.5           # True = insertion
    lens = rng.integers(INDEL_LEN[0], INDEL_LEN[1] + 1, size=starts.size)
    pieces = []
    cur = 0
    length = seq.shape[0]
    for s, ins, ln in zip(starts.tolist(), kinds.tolist(), lens.tolist()):
        if s < cur:                                  # inside an earlier deletion
            continue
        if ins:
            pieces.append(seq[cur:s])
            pieces.append(background(rng, ln))
            length += ln
            cur = s
        else:
            ln = min(ln, seq.shape[0] - s)
            if length - ln < MIN_LEN:
                continue
            pieces.append(seq[cur:s])
            length -= ln
            cur = s + ln
    pieces.append(seq[cur:])
    return np.concatenate(pieces)


def mutate(rng, ancestor: np.ndarray) -> np.ndarray:
    rate = rng.uniform(*SUB_RATE)
    return _indels(rng, _substitute(rng, ancestor, rate))


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
    seqs = []
    for f in range(n_families):
        anc = background(rng, max(MIN_LEN, int(ancestor_len(rng))))
        for _ in range(int(sizes[f])):
            seqs.append(mutate(rng, anc))
    return _pack(seqs, p, name)


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


def config4(seed: int = 0, n_sets: int = 512):
    """512 independent sets for the batched launch."""
    return [batch_set(i, seed) for i in range(n_sets)]


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
