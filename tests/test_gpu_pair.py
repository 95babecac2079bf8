"""The rank on CTA pairs (plans with tile = 256: 256 x 256 tiles, tcgen05
cta_group::2) against the oracle.

Same Eq. 1 / Eq. 3 keys as the one-CTA tiles, on sizes that leave ragged 256-row
blocks (1, 2, 255, 256, 257, 511, 700), a family set at several plane depths (the
remainder of the cut planes through the pair's chunk buffers), deep counts on a
small alphabet (entries above the remainder bitmap: heavy entries), identical
sequences (ties), and the paper-scale set's first rows.
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


def check_pair(sad, oracle_mod, s, depth, k=3, alphabet=20, budget=0):
    codes, offsets = dev(s.codes), dev(s.offsets)
    wm = torch.empty(alphabet ** k, dtype=torch.int32, device="cuda")
    counts = sad.kmer_count(codes, offsets, k, alphabet, word_max=wm)
    ws = sad.Workspace(codes.device)
    plan = sad.kmer_rank_plan(counts, k, alphabet, depth=depth, ws=ws, tile=256, budget=budget)
    hi, lo, rank = sad.kmer_rank(counts, dev(s.lengths.astype(np.int32)), k, alphabet, ws=ws,
                                 plan=plan, word_max=wm)
    c = oracle_mod.kmer_count(s.codes, s.offsets, k, alphabet)
    ohi, olo, orank = oracle_mod.kmer_rank(c, s.lengths, k, alphabet)
    np.testing.assert_array_equal(hi.cpu().numpy(), ohi)
    np.testing.assert_array_equal(lo.cpu().numpy(), olo)
    np.testing.assert_array_equal(rank.cpu().numpy(), orank)
    return sad.rank_info(ws)


@pytest.mark.parametrize("n", [1, 2, 255, 256, 257, 511, 700])
def test_pair_sizes_and_ragged_blocks(sad, oracle_mod, n):
    s = datagen.random_small(n, 3, 420, seed=100 + n, alphabet=20)
    check_pair(sad, oracle_mod, s, depth=0)


@pytest.mark.parametrize("depth,budget", [(0, 0), (1, 0), (2, 0), (3, 0), (2, 64), (6, 256)])
def test_pair_family_set_depths(sad, oracle_mod, depth, budget):
    s = datagen.family_set(6, 230, lambda r: int(r.integers(40, 900)), p=4, seed=3, stream=9)
    info = check_pair(sad, oracle_mod, s, depth=depth, budget=budget)
    if depth >= 1:
        assert info["tiles"] == (1380 + 255) // 256 * ((1380 + 255) // 256 + 1) // 2


@pytest.mark.parametrize("depth", [1, 2])
def test_pair_deep_counts_heavy_entries(sad, oracle_mod, depth):
    # 4 letters: counts in the hundreds, far above the bitmap's thresholds
    s = datagen.random_small(300, 3, 2500, seed=11, alphabet=4)
    info = check_pair(sad, oracle_mod, s, depth=depth, alphabet=4)
    assert info["heavy_entries"] > 0


def test_pair_identical_sequences(sad, oracle_mod):
    s = datagen.from_strings(["ACDEFGHIKLMNPQ"] * 300 + ["WYWYWYWY"] * 10)
    check_pair(sad, oracle_mod, s, depth=1)


@pytest.mark.slow
def test_pair_paper_scale_rows(sad, oracle_mod):
    s = datagen.config2()
    s = s.take(np.arange(3000))
    check_pair(sad, oracle_mod, s, depth=2)
