"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here retypes the oracle's formulas: counts are checked against string
enumeration, similarities against multiset intersection of the k-mer lists,
keys against exact rational sums, partitions against hand-derived runs and
against properties every regular-sampling partition must have. A plausible slip
in the oracle (a dropped self term, max for min in the denominator, a wrong
word index, an off-by-one pivot) fails at least one test below.
"""
import collections
import fractions
import itertools

import numpy as np
import pytest

from conftest import golden_lines
from paper_0905_1744_gb300 import datagen

ALPHA = datagen.ALPHABET


def kmer_multiset(codes, k):
    """Multiset of k-letter words of one sequence, straight from the string."""
    return collections.Counter(tuple(int(c) for c in codes[i:i + k])
                               for i in range(len(codes) - k + 1))


# ------------------------------------------------------------------ counts ---

@pytest.mark.parametrize("k,alphabet", [(1, 20), (2, 20), (3, 20), (4, 5), (3, 4)])
def test_count_matches_string_enumeration(oracle_mod, k, alphabet):
    s = datagen.random_small(17, k, 30, seed=k * 100 + alphabet, alphabet=alphabet)
    counts = oracle_mod.kmer_count(s.codes, s.offsets, k, alphabet)
    assert counts.shape == (s.n, alphabet ** k)
    for x in range(s.n):
        expect = np.zeros(alphabet ** k, np.int64)
        for word, c in kmer_multiset(s.seq(x), k).items():
            expect[np.ravel_multi_index(word, (alphabet,) * k)] = c
        np.testing.assert_array_equal(counts[x], expect)


def test_count_totals_and_homopolymer(oracle_mod):
    s = datagen.from_strings(["A" * 50, "AC" * 10, "ACD", "W" * 3, ALPHA])
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    np.testing.assert_array_equal(c.sum(axis=1), s.lengths - 2)   # L - k + 1 windows
    assert c[0, 0] == 48 and c[0].sum() == 48                      # AAA x (L - 2)
    aca = np.ravel_multi_index((0, 1, 0), (20,) * 3)
    cac = np.ravel_multi_index((1, 0, 1), (20,) * 3)
    assert c[1, aca] == 9 and c[1, cac] == 9                        # ACAC..AC: 18 windows
    w = ALPHA.index("W")
    www = np.ravel_multi_index((w, w, w), (20,) * 3)
    assert c[3, www] == 1
    assert (c[4] <= 1).all() and c[4].sum() == 18                  # all words distinct


def test_count_rejects_bad_input(oracle_mod):
    s = datagen.from_strings(["ACDE", "AC"])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.kmer_count(s.codes, s.offsets)                  # L < k
    s = datagen.from_strings(["ACDE"])
    codes = s.codes.copy()
    codes[1] = 20
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.kmer_count(codes, s.offsets)                    # code >= alphabet


# ---------------------------------------------------- similarity, Eq. 1 ---

def test_threshold_identity_exhaustive():
    """min(a, b) = sum_t [a >= t][b >= t] for all a, b <= 64 (the identity the
    tensor-core path relies on)."""
    t = np.arange(1, 65)
    a = np.arange(0, 65)
    planes = (a[:, None] >= t[None, :]).astype(np.int64)          # [a, t]
    np.testing.assert_array_equal(planes @ planes.T, np.minimum.outer(a, a))


def test_eq1_hand_examples(oracle_mod):
    rows = list(golden_lines("eq1_similarity.txt"))
    assert len(rows) >= 5
    for x, y, S, D in rows:
        s = datagen.from_strings([x, y])
        c = oracle_mod.kmer_count(s.codes, s.offsets)
        assert oracle_mod.shared_count(c[0], c[1]) == int(S), (x, y)
        assert min(len(x), len(y)) - 3 + 1 == int(D)


def test_shared_count_is_multiset_intersection(oracle_mod):
    s = datagen.random_small(24, 3, 60, seed=5, alphabet=4)          # small alphabet: repeats
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, 4)
    ms = [kmer_multiset(s.seq(x), 3) for x in range(s.n)]
    for x, y in itertools.product(range(s.n), repeat=2):
        expect = sum((ms[x] & ms[y]).values())
        assert oracle_mod.shared_count(c[x], c[y]) == expect


def test_similarity_invariants(oracle_mod):
    s = datagen.random_small(30, 3, 80, seed=6, alphabet=3)
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, 3)
    m = s.lengths - 2
    for x in range(s.n):
        assert oracle_mod.shared_count(c[x], c[x]) == m[x]          # F(x, x) = 1
        for y in range(s.n):
            sxy = oracle_mod.shared_count(c[x], c[y])
            assert sxy == oracle_mod.shared_count(c[y], c[x])       # symmetric
            assert 0 <= sxy <= min(m[x], m[y])                      # 0 <= F <= 1


def test_term_is_exact_floor(oracle_mod):
    rng = np.random.default_rng(3)
    cases = [(s, d) for d in range(1, 70) for s in range(0, d + 1)]
    cases += [(int(d), int(d)) for d in rng.integers(1, 70000, 50)]
    cases += [(int(s), int(d)) for d, s in zip(rng.integers(1, 70000, 200),
                                               rng.integers(0, 70000, 200)) if s <= d]
    for s, d in cases:
        assert oracle_mod.term(s, d) == (s << 64) // d


# -------------------------------------------------------- rank, Eq. 3 -----

def exact_rank_sums(s, k=3):
    ms = [kmer_multiset(s.seq(x), k) for x in range(s.n)]
    L = s.lengths
    out = []
    for x in range(s.n):
        tot = fractions.Fraction(0)
        for y in range(s.n):
            tot += fractions.Fraction(int(sum((ms[x] & ms[y]).values())),
                                      int(min(L[x], L[y])) - k + 1)
        out.append(tot)
    return out


@pytest.mark.parametrize("seed,alphabet", [(1, 20), (2, 4), (3, 2)])
def test_keys_against_exact_rationals(oracle_mod, seed, alphabet):
    s = datagen.random_small(11, 3, 40, seed=seed, alphabet=alphabet)
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, alphabet)
    hi, lo, rank, fp = oracle_mod.kmer_rank(c, s.lengths, 3, alphabet, with_fp64=True)
    exact = exact_rank_sums(s)
    for x in range(s.n):
        key = (int(hi[x]) << 64) | int(lo[x])
        scaled = exact[x] * (1 << 64)
        assert 0 <= scaled - key < s.n                              # N floors, each < 1 short
        r = float(exact[x] / s.n)
        assert abs(rank[x] - r) <= 1e-12 * r
        assert abs(fp[x] - r) <= 1e-12 * r


def test_eq3_hand_example(oracle_mod):
    rows = list(golden_lines("eq3_rank.txt"))
    seqs = [r[0] for r in rows if r[0] != "order"]
    order = [int(v) for v in next(r for r in rows if r[0] == "order")[1:]]
    s = datagen.from_strings(seqs)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank = oracle_mod.kmer_rank(c, s.lengths)
    for x, (_, h, l, num, den) in enumerate(r for r in rows if r[0] != "order"):
        assert (int(hi[x]), int(lo[x])) == (int(h), int(l))
        assert rank[x] == float(fractions.Fraction(int(num), int(den)))
    assert list(np.lexsort((np.arange(s.n), lo, hi))) == order


def test_identical_sequences_have_identical_keys(oracle_mod):
    s = datagen.from_strings(["ACDEFGHIKLM", "MLKIHGFEDCA", "ACDEFGHIKLM", "AAAAAAAC",
                              "ACDEFGHIKLM"])
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, _ = oracle_mod.kmer_rank(c, s.lengths)
    assert hi[0] == hi[2] == hi[4] and lo[0] == lo[2] == lo[4]


def test_rank_row_subset_matches_full(oracle_mod):
    s = datagen.random_small(40, 3, 50, seed=9)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank = oracle_mod.kmer_rank(c, s.lengths, threads=3)
    rows = [39, 0, 17, 17]
    h2, l2, r2 = oracle_mod.kmer_rank(c, s.lengths, rows=rows, threads=2)
    np.testing.assert_array_equal(h2, hi[rows])
    np.testing.assert_array_equal(l2, lo[rows])
    np.testing.assert_array_equal(r2, rank[rows])


# ---------------------------------------------- partition, Sec. 3.1.2 -----

def golden_partition_cases():
    cases, cur = [], None
    for tok in golden_lines("regular_sampling.txt"):
        if tok[0] == "case":
            cur = dict(name=tok[1], n=int(tok[2]), p=int(tok[3]))
            cases.append(cur)
        else:
            cur[tok[0]] = [int(v) for v in tok[1:]]
    return cases


@pytest.mark.parametrize("case", golden_partition_cases(), ids=lambda c: c["name"])
def test_partition_hand_examples(oracle_mod, case):
    lo = np.array(case["keys"], np.uint64)
    hi = np.zeros_like(lo)
    offs, mem, piv = oracle_mod.partition(hi, lo, case["p"])
    assert list(offs) == case["offsets"]
    assert list(mem) == case["members"]
    assert list(piv) == case["pivots"]


def check_partition_properties(hi, lo, p, offs, mem, piv):
    n = hi.shape[0]
    order = np.lexsort((np.arange(n), lo, hi))                       # (key, index) order
    np.testing.assert_array_equal(mem, order)                       # buckets tile the order
    assert offs[0] == 0 and offs[-1] == n and (np.diff(offs) >= 0).all()
    rank_of = np.empty(n, np.int64)
    rank_of[order] = np.arange(n)
    for i in range(p - 1):                                           # bucket i ends at y_i
        assert offs[i + 1] == rank_of[piv[i]] + 1


@pytest.mark.parametrize("n,p,distinct", [(64, 4, None), (1000, 8, None), (1000, 8, 7),
                                          (513, 16, None), (4096, 16, 100), (77, 77, None),
                                          (50, 1, None)])
def test_partition_properties(oracle_mod, n, p, distinct):
    hi, lo = datagen.random_keys(n, seed=n + p, distinct=distinct)
    offs, mem, piv = oracle_mod.partition(hi, lo, p)
    check_partition_properties(hi, lo, p, offs, mem, piv)


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_partition_load_bound(oracle_mod, p):
    """Sec. 3.3.2: no bucket exceeds 2N/p when N >= p^3 (regular sampling)."""
    for trial in range(5):
        n = p ** 3 * (1 + trial)
        for distinct in (None, n // 3 + 1):
            hi, lo = datagen.random_keys(n, seed=1000 * p + trial, distinct=distinct)
            offs, _, _ = oracle_mod.partition(hi, lo, p)
            assert np.diff(offs).max() <= 2 * n // p


def test_partition_load_bound_on_ranked_workloads(oracle_mod):
    """Sec. 3.3.2 on real keys: the 200-sequence set (p = 4) and set 7 of the
    batching workload (N = 1631, p = 4), both with N >= p^3, rank then partition; no
    bucket exceeds 2N/p and the buckets tile the (key, index) order."""
    for s in (datagen.config1(), datagen.batch_set(7)):
        assert s.p >= 4
        assert s.n >= s.p ** 3
        r = oracle_mod.run_set(s.codes, s.offsets, s.p)
        assert np.diff(r["bucket_offsets"]).max() <= 2 * s.n // s.p
        check_partition_properties(r["key_hi"], r["key_lo"], s.p, r["bucket_offsets"],
                                   r["members"], r["pivot_idx"])


def test_partition_rejects_bad_p(oracle_mod):
    hi, lo = datagen.random_keys(5, seed=1)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.partition(hi, lo, 6)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.partition(hi, lo, 0)
    offs, mem, piv = oracle_mod.partition(hi[:0], lo[:0], 3)
    assert list(offs) == [0, 0, 0, 0] and mem.size == 0


# ----------------------------------------- globalised rank, Sec. 3.1.1 ------

def exact_term(sx, sy, lx, ly, k=3):
    """floor(|multiset intersection| 2^64 / (min(L_x, L_y) - k + 1)), from the strings."""
    s = sum((sx & sy).values())
    return (s << 64) // (min(lx, ly) - k + 1)


def test_rank_vs_against_exact_floors(oracle_mod):
    s = datagen.random_small(13, 3, 60, seed=21, alphabet=5)
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, 5)
    ref = np.array([4, 0, 4, 12, 7], np.int32)            # a multiset: 4 counts twice
    hi, lo, rank = oracle_mod.rank_vs(c, s.lengths, ref, 3, 5)
    ms = [kmer_multiset(s.seq(x), 3) for x in range(s.n)]
    for x in range(s.n):
        want = sum(exact_term(ms[x], ms[r], int(s.lengths[x]), int(s.lengths[r])) for r in ref)
        assert ((int(hi[x]) << 64) | int(lo[x])) == want
        assert abs(rank[x] - want / 2.0 ** 64 / len(ref)) <= 1e-12 * max(rank[x], 1e-300)


def test_rank_vs_every_sequence_is_the_centralised_key(oracle_mod):
    s = datagen.random_small(40, 3, 200, seed=22)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    h0, l0, r0 = oracle_mod.kmer_rank(c, s.lengths)
    h1, l1, r1 = oracle_mod.rank_vs(c, s.lengths, np.arange(s.n)[::-1])
    np.testing.assert_array_equal(h0, h1)
    np.testing.assert_array_equal(l0, l1)
    np.testing.assert_array_equal(r0, r1)


def golden_sample_cases():
    cases, cur = [], None
    for tok in golden_lines("local_samples.txt"):
        if tok[0] == "case":
            cur = dict(name=tok[1], n=int(tok[2]), p=int(tok[3]), ks=int(tok[4]))
            cases.append(cur)
        else:
            cur[tok[0]] = [int(v) for v in tok[1:]]
    return cases


@pytest.mark.parametrize("case", golden_sample_cases(), ids=lambda c: c["name"])
def test_local_samples_hand_examples(oracle_mod, case):
    lo = np.array(case["keys"], np.uint64)
    got = oracle_mod.local_samples(np.zeros_like(lo), lo, case["p"], case["ks"])
    assert list(got) == case["samples"]


def test_local_ranks_see_only_their_block(oracle_mod):
    s = datagen.random_small(30, 3, 150, seed=23)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    h, l = oracle_mod.local_ranks(c, s.lengths, 3)
    # blocks [0,10) [10,20) [20,30): shuffling the rows of other blocks changes nothing
    perm = np.concatenate([np.arange(10), 10 + np.random.default_rng(0).permutation(10),
                           20 + np.random.default_rng(1).permutation(10)])
    h2, l2 = oracle_mod.local_ranks(c[perm], s.lengths[perm], 3)
    np.testing.assert_array_equal(h[:10], h2[:10])
    np.testing.assert_array_equal(l[:10], l2[:10])
    # and a block's keys are the centralised keys of the block alone
    hb, lb, _ = oracle_mod.kmer_rank(c[10:20], s.lengths[10:20])
    np.testing.assert_array_equal(h[10:20], hb)
    np.testing.assert_array_equal(l[10:20], lb)


def test_global_rank_with_every_sequence_sampled_is_centralised(oracle_mod):
    s = datagen.random_small(25, 3, 120, seed=24)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank, samples = oracle_mod.global_rank(c, s.lengths, 1, s.n)
    assert sorted(samples.tolist()) == list(range(s.n))     # floor(j N/(N+1)) = 0..N-1
    h0, l0, r0 = oracle_mod.kmer_rank(c, s.lengths)
    np.testing.assert_array_equal(hi, h0)
    np.testing.assert_array_equal(lo, l0)


def test_global_rank_against_exact_pipeline(oracle_mod):
    """Steps 2-6 redone from the strings with Python integers: local keys, local
    order, regular samples, keys against the samples."""
    s = datagen.random_small(14, 3, 50, seed=25, alphabet=4)
    p, ks = 3, 2
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, 4)
    hi, lo, _, samples = oracle_mod.global_rank(c, s.lengths, p, ks, 3, 4)
    ms = [kmer_multiset(s.seq(x), 3) for x in range(s.n)]
    L = [int(v) for v in s.lengths]
    want_samples = []
    for b in range(p):
        blk = list(range(b * s.n // p, (b + 1) * s.n // p))
        key = {x: sum(exact_term(ms[x], ms[y], L[x], L[y]) for y in blk) for x in blk}
        order = sorted(blk, key=lambda x: (key[x], x))
        want_samples += [order[j * len(blk) // (ks + 1)] for j in range(1, ks + 1)]
    assert list(samples) == want_samples
    for x in range(s.n):
        want = sum(exact_term(ms[x], ms[r], L[x], L[r]) for r in want_samples)
        assert ((int(hi[x]) << 64) | int(lo[x])) == want


# ------------------------------------- distance-form rank, Eq. 2 / Eq. 3 -----

def test_ln_q_against_decimal_logarithm(oracle_mod):
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    xs = list(range(1, 300)) + [2 ** e + d for e in range(1, 40) for d in (-1, 0, 1)]
    xs += [65535, 65536, 720885, 11 * 65535, 129 * 65535, 1025 * 65535]
    prev = -1
    for x in sorted(set(xs)):
        got = oracle_mod.ln_q(x)
        exact = Decimal(x).ln() * (Decimal(2) ** 32)
        assert 0 <= exact - got < 2, x              # truncation below 2^-32 (plus < 1 ulp)
        assert got >= prev
        prev = got


def test_rank_dist_closed_forms(oracle_mod):
    # x = ACDE, y = CDEF (Eq. 1 example: S = 1, D = 2, F = 1/2); z shares nothing
    s = datagen.from_strings(["ACDE", "CDEF", "WWWWW"])
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    b = 10
    key, rank = oracle_mod.rank_dist(c, s.lengths, b)
    q = oracle_mod.ln_q
    self_xy = q(b * 2) - q(2 + b * 2)          # F = 1: -ln(1 + 1/b)
    half = q(b * 2) - q(2 + b * 1)             # F = 1/2: -ln(1/b + 1/2)
    zero = lambda d: q(b * d) - q(d)           # F = 0: ln b
    assert key[0] == self_xy + half + zero(2)
    assert key[1] == half + self_xy + zero(2)
    assert key[2] == zero(2) + zero(2) + (q(b * 3) - q(3 + b * 3))
    assert abs(zero(2) / 2 ** 32 - np.log(b)) < 1e-9


def test_rank_dist_against_exact_sums(oracle_mod):
    s = datagen.random_small(12, 3, 45, seed=31, alphabet=4)
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, 4)
    for b in (1, 10, 100):
        key, rank, fp = oracle_mod.rank_dist(c, s.lengths, b, 3, 4, with_fp64=True)
        ms = [kmer_multiset(s.seq(x), 3) for x in range(s.n)]
        for x in range(s.n):
            want = 0
            for y in range(s.n):
                S = sum((ms[x] & ms[y]).values())
                D = min(int(s.lengths[x]), int(s.lengths[y])) - 2
                want += oracle_mod.ln_q(b * D) - oracle_mod.ln_q(D + b * S)
            assert key[x] == want
            # each term within 2^-31 of -ln(1/b + S/D): the mean too
            assert abs(rank[x] - fp[x]) <= 2.0 ** -31 + 1e-13 * abs(fp[x])


def test_rank_dist_orders_against_similarity(oracle_mod):
    """d decreases in F, so for equal denominators a larger shared count gives a
    smaller distance sum term by term: identical rows get identical keys and the
    distance rank orders opposite to a strictly larger similarity everywhere."""
    s = datagen.from_strings(["ACDEFGHIKLMN", "ACDEFGHIKLMN", "ACDEFGHIKLMW", "WYWYWYWYWYWY"])
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    key, _ = oracle_mod.rank_dist(c, s.lengths, 10)
    assert key[0] == key[1]
    assert key[0] < key[2] < key[3]


def test_rank_vs_dist_every_sequence_is_rank_dist(oracle_mod):
    s = datagen.random_small(30, 3, 150, seed=32)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    k0, r0 = oracle_mod.rank_dist(c, s.lengths, 10)
    k1, r1 = oracle_mod.rank_vs_dist(c, s.lengths, 10, np.arange(s.n)[::-1])
    np.testing.assert_array_equal(k0, k1)
    np.testing.assert_array_equal(r0, r1)
    # a reference listed twice counts twice
    k2, _ = oracle_mod.rank_vs_dist(c, s.lengths, 10, [4, 4])
    k3, _ = oracle_mod.rank_vs_dist(c, s.lengths, 10, [4])
    np.testing.assert_array_equal(k2, 2 * k3)
