"""Distance-form rank (Eq. 2 / Eq. 3 as written) through the C-ABI against the CPU
oracle: the fixed-point natural log, the signed keys bit for bit, the float64 view
exactly (same rounding), and within the quantisation bound of the FP64 mean.
"""
import numpy as np
import pytest

from paper_0905_1744_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sad():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0905_1744_gb300 import build, sad as sadmod
    build.build()
    return sadmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def test_ln_q_matches_oracle(sad, oracle_mod):
    rng = np.random.default_rng(5)
    xs = np.concatenate([np.arange(0, 5000), rng.integers(1, 1 << 40, 20000),
                         [(1 << e) + d for e in range(1, 62) for d in (-1, 0, 1)]]).astype(np.uint64)
    got = host(sad.ln_q(dev(xs)))
    want = np.array([oracle_mod.ln_q(int(x)) if x else 0 for x in xs], np.int64)
    np.testing.assert_array_equal(got, want)


def family(n, seed):
    nf = max(2, n // 60)
    return datagen.family_set(nf, max(1, n // nf), lambda r: int(r.integers(40, 700)), p=4,
                              seed=seed, stream=6)


@pytest.mark.parametrize("n,b,depth", [(1, 10, 0), (2, 1, 0), (129, 10, 0), (257, 100, 0),
                                       (700, 10, 1), (900, 50, 2), (1300, 10, 0)])
def test_rank_dist_matches_oracle(sad, oracle_mod, n, b, depth):
    s = datagen.random_small(n, 3, 400, seed=n) if n < 300 else family(n, n + 4)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    key, hi, lo, rank = sad.kmer_rank_dist(counts, dev(s.lengths.astype(np.int32)), b,
                                           depth=depth)
    okey, orank, ofp = oracle_mod.rank_dist(c, s.lengths, b, with_fp64=True)
    np.testing.assert_array_equal(host(key), okey)
    np.testing.assert_array_equal(host(rank), orank)
    ohi, olo = oracle_mod.dist_sort_key(okey)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)
    # each term within 2^-31 of -ln(1/b + S/D), so the mean too
    assert np.all(np.abs(host(rank) - ofp) <= 2.0 ** -31 + 1e-13 * np.abs(ofp))


def test_rank_dist_homopolymers_and_residual(sad, oracle_mod):
    seqs = ["A" * 3000, "A" * 2000, "AC" * 700, "A" * 5, "C" * 900, "A" * 1200 + "C" * 800]
    s = datagen.from_strings(seqs)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    for depth in (0, 1, 3):
        key, _, _, _ = sad.kmer_rank_dist(counts, dev(s.lengths.astype(np.int32)), 10,
                                          depth=depth)
        okey, _ = oracle_mod.rank_dist(c, s.lengths, 10)
        np.testing.assert_array_equal(host(key), okey)


def test_partition_of_distance_keys(sad, oracle_mod):
    s = family(800, 9)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    _, hi, lo, _ = sad.kmer_rank_dist(counts, dev(s.lengths.astype(np.int32)), 10)
    offs, mem, piv = sad.partition(hi, lo, 8)
    okey, _ = oracle_mod.rank_dist(c, s.lengths, 10)
    ohi, olo = oracle_mod.dist_sort_key(okey)
    o_offs, o_mem, o_piv = oracle_mod.partition(ohi, olo, 8)
    np.testing.assert_array_equal(host(offs), o_offs)
    np.testing.assert_array_equal(host(mem), o_mem)
    np.testing.assert_array_equal(host(piv), o_piv)


@pytest.mark.parametrize("n,n_ref,b", [(1, 1, 10), (300, 64, 10), (700, 129, 50)])
def test_rank_vs_distance_matches_oracle(sad, oracle_mod, n, n_ref, b):
    s = datagen.random_small(n, 3, 400, seed=n + 3) if n < 300 else family(n, n + 5)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    ref = np.random.default_rng(n_ref + 1).integers(0, s.n, n_ref).astype(np.int32)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    key, hi, lo, rank = sad.kmer_rank_vs(counts, dev(s.lengths.astype(np.int32)), dev(ref),
                                         delta_den=b)
    okey, orank = oracle_mod.rank_vs_dist(c, s.lengths, b, ref)
    np.testing.assert_array_equal(host(key), okey)
    np.testing.assert_array_equal(host(rank), orank)
    ohi, olo = oracle_mod.dist_sort_key(okey)
    np.testing.assert_array_equal(host(lo), olo)


def test_rank_vs_distance_every_sequence_is_rank_dist(sad):
    s = family(600, 12)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    lengths = dev(s.lengths.astype(np.int32))
    k0, _, _, r0 = sad.kmer_rank_dist(counts, lengths, 10)
    k1, _, _, r1 = sad.kmer_rank_vs(counts, lengths, dev(np.arange(s.n, dtype=np.int32)),
                                    delta_den=10)
    np.testing.assert_array_equal(host(k0), host(k1))
    np.testing.assert_array_equal(host(r0), host(r1))


def test_global_rank_distance_form_matches_oracle(sad, oracle_mod):
    """Steps 2-6 with the re-rank in the distance form: local ranks (similarity
    form) pick the samples, then every sequence against them in Eq. 2's form."""
    s = family(500, 14)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    g = sad.GlobalRank(counts, dev(s.lengths.astype(np.int32)), 4, 8, delta_den=10)
    g.run()
    g.check()
    lh, ll = oracle_mod.local_ranks(c, s.lengths, 4)
    samples = oracle_mod.local_samples(lh, ll, 4, 8)
    np.testing.assert_array_equal(host(g.samples), samples)
    okey, orank = oracle_mod.rank_vs_dist(c, s.lengths, 10, samples)
    np.testing.assert_array_equal(host(g.key), okey)
    np.testing.assert_array_equal(host(g.rank), orank)
