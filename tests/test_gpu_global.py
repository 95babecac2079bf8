"""Globalised rank (Sec. 3.1.1, Algorithm 2 steps 2-6) through the C-ABI against
the CPU oracle: local ranks per block, regular samples of the local order, every
sequence against the samples, and the partition of the result. Keys, sample
indices and buckets bit for bit; the float64 rank view exactly (same rounding).
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


@pytest.mark.parametrize("n,p,ks,distinct", [(16, 4, 3, True), (10, 3, 2, True), (3, 1, 5, True),
                                             (1000, 7, 6, False), (1000, 16, 15, True),
                                             (4097, 3, 40, False), (9000, 64, 63, True),
                                             (5, 5, 2, False)])
def test_local_samples_match_oracle(sad, oracle_mod, n, p, ks, distinct):
    hi, lo = datagen.random_keys(n, seed=n + p + ks, distinct=None if distinct else 5)
    got = host(sad.local_samples(dev(hi), dev(lo), p, ks))
    np.testing.assert_array_equal(got, oracle_mod.local_samples(hi, lo, p, ks))


def test_local_samples_rejects_bad_arguments(sad):
    hi, lo = datagen.random_keys(10, seed=1)
    for p, ks in ((0, 1), (11, 1), (2, 0)):
        with pytest.raises(sad.SadError) as e:
            sad.local_samples(dev(hi), dev(lo), p, ks)
        assert e.value.status == sad.ERR_INVALID_ARGUMENT


def family(n, seed):
    return datagen.family_set(max(2, n // 60), max(1, n // max(2, n // 60)),
                              lambda r: int(r.integers(40, 700)), p=4, seed=seed, stream=5)


@pytest.mark.parametrize("n,n_ref", [(1, 1), (130, 7), (300, 64), (700, 129), (1200, 300)])
def test_rank_vs_matches_oracle(sad, oracle_mod, n, n_ref):
    s = datagen.random_small(n, 3, 500, seed=n + 7) if n < 300 else family(n, n)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    ref = np.random.default_rng(n_ref).integers(0, s.n, n_ref).astype(np.int32)  # repeats
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    hi, lo, rank = sad.kmer_rank_vs(counts, dev(s.lengths.astype(np.int32)), dev(ref))
    ohi, olo, orank = oracle_mod.rank_vs(c, s.lengths, ref)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)
    np.testing.assert_array_equal(host(rank), orank)


def test_rank_vs_every_sequence_is_kmer_rank(sad):
    s = family(900, 3)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    lengths = dev(s.lengths.astype(np.int32))
    h0, l0, r0 = sad.kmer_rank(counts, lengths)
    h1, l1, r1 = sad.kmer_rank_vs(counts, lengths, dev(np.arange(s.n, dtype=np.int32)))
    np.testing.assert_array_equal(host(h0), host(h1))
    np.testing.assert_array_equal(host(l0), host(l1))
    np.testing.assert_array_equal(host(r0), host(r1))


def test_rank_vs_rejects_out_of_range_reference(sad):
    s = datagen.random_small(50, 3, 100, seed=9)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank_vs(counts, dev(s.lengths.astype(np.int32)),
                         dev(np.array([3, 50], np.int32)))
    assert e.value.status == sad.ERR_INVALID_ARGUMENT


@pytest.mark.parametrize("n,p", [(7, 7), (300, 4), (1000, 16)])
def test_local_ranks_match_oracle(sad, oracle_mod, n, p):
    s = family(n, n + 1) if n >= 300 else datagen.random_small(n, 3, 300, seed=n)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    hi, lo, _ = sad.local_ranks(counts, dev(s.lengths.astype(np.int32)), p)
    ohi, olo = oracle_mod.local_ranks(c, s.lengths, p)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)


@pytest.mark.parametrize("n,p,ks", [(240, 4, 3), (1000, 8, 7), (1500, 16, 15), (600, 3, 1)])
def test_global_partition_matches_oracle(sad, oracle_mod, n, p, ks):
    s = family(n, n + 2)
    res = sad.global_partition_set(dev(s.codes), dev(s.offsets), p, ks)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank, samples = oracle_mod.global_rank(c, s.lengths, p, ks)
    np.testing.assert_array_equal(host(res["samples"]), samples)
    np.testing.assert_array_equal(host(res["key_hi"]), hi)
    np.testing.assert_array_equal(host(res["key_lo"]), lo)
    np.testing.assert_array_equal(host(res["rank"]), rank)
    offs, mem, piv = oracle_mod.partition(hi, lo, p)
    np.testing.assert_array_equal(host(res["bucket_offsets"]), offs)
    np.testing.assert_array_equal(host(res["members"]), mem)
    np.testing.assert_array_equal(host(res["pivot_idx"]), piv)


@pytest.mark.slow
def test_rank_vs_paper_scale_sample(sad, oracle_mod):
    """N = 5000 in 20 families against 240 references (16 blocks x 15 samples of
    the paper-scale partition), references drawn independently of the device."""
    s = datagen.family_set(20, 250, lambda r: int(np.clip(r.normal(300, 100), 50, 1000)),
                           p=16, seed=11, stream=3)
    ref = np.random.default_rng(240).integers(0, s.n, 240).astype(np.int32)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    hi, lo, rank = sad.kmer_rank_vs(counts, dev(s.lengths.astype(np.int32)), dev(ref))
    ohi, olo, orank = oracle_mod.rank_vs(c, s.lengths, ref)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)
