"""The sparse-intersection rank on the CUDA cores (the O(L)-per-pair comparison
point of Table 2) through the C-ABI: the same keys as the oracle and as the
tensor-core kmer_rank, bit for bit."""
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


@pytest.mark.parametrize("n,alphabet", [(1, 20), (2, 20), (33, 20), (257, 20), (300, 4),
                                        (900, 20)])
def test_sparse_rank_matches_oracle(sad, oracle_mod, n, alphabet):
    s = datagen.random_small(n, 3, 600, seed=n + alphabet, alphabet=alphabet)
    c = oracle_mod.kmer_count(s.codes, s.offsets, 3, alphabet)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets), 3, alphabet)
    hi, lo, rank = sad.kmer_rank_sparse(counts, dev(s.lengths.astype(np.int32)), 3, alphabet)
    ohi, olo, orank = oracle_mod.kmer_rank(c, s.lengths, 3, alphabet)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)
    np.testing.assert_array_equal(host(rank), orank)


def test_sparse_rank_equals_tensor_rank(sad):
    s = datagen.family_set(20, 60, lambda r: int(r.integers(50, 2000)), p=4, seed=5, stream=8)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    lengths = dev(s.lengths.astype(np.int32))
    h0, l0, _ = sad.kmer_rank(counts, lengths)
    h1, l1, _ = sad.kmer_rank_sparse(counts, lengths)
    np.testing.assert_array_equal(host(h0), host(h1))
    np.testing.assert_array_equal(host(l0), host(l1))


def test_sparse_rank_homopolymers(sad, oracle_mod):
    s = datagen.from_strings(["A" * 20000, "A" * 15000, "AC" * 6000, "A" * 3, "C" * 9000])
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    hi, lo, _ = sad.kmer_rank_sparse(counts, dev(s.lengths.astype(np.int32)))
    ohi, olo, _ = oracle_mod.kmer_rank(c, s.lengths)
    np.testing.assert_array_equal(host(hi), ohi)
    np.testing.assert_array_equal(host(lo), olo)


def test_sparse_rank_reports_small_capacity(sad):
    s = datagen.random_small(50, 3, 200, seed=3)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank_sparse(counts, dev(s.lengths.astype(np.int32)), entries=10)
    assert e.value.status == sad.ERR_WORKSPACE
