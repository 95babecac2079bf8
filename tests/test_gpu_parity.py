"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Integers are compared bit for bit: counts, 128-bit keys, bucket offsets,
members and pivots. The float64 rank view is compared exactly too (both sides
round the same three IEEE operations), and against the compensated FP64 mean
within 1e-12 relative.
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


def gpu_counts(sad, s, k=3, alphabet=20):
    return host(sad.kmer_count(dev(s.codes), dev(s.offsets), k, alphabet))


# ------------------------------------------------------------------ count ---

@pytest.mark.parametrize("k,alphabet,n,lo,hi", [(3, 20, 200, 3, 400), (1, 20, 50, 1, 70),
                                                (2, 20, 64, 2, 600), (4, 5, 33, 4, 1000),
                                                (8, 4, 20, 8, 3000), (5, 7, 40, 5, 37)])
def test_count_matches_oracle(sad, oracle_mod, k, alphabet, n, lo, hi):
    s = datagen.random_small(n, lo, hi, seed=k * 31 + alphabet, alphabet=alphabet)
    np.testing.assert_array_equal(gpu_counts(sad, s, k, alphabet),
                                  oracle_mod.kmer_count(s.codes, s.offsets, k, alphabet))


def test_count_unaligned_offsets_and_homopolymers(sad, oracle_mod):
    seqs = ["A" * 3, "A" * 5000, "C" * 17, "ACDEFGHIKLMNPQRSTVWY" * 40, "W" * 511, "Y" * 513,
            "AC" * 300, "M" * 4]
    s = datagen.from_strings(seqs)
    np.testing.assert_array_equal(gpu_counts(sad, s), oracle_mod.kmer_count(s.codes, s.offsets))


def test_count_reports_bad_input(sad):
    s = datagen.from_strings(["ACDEF", "ACD"])
    codes = s.codes.copy()
    codes[2] = 25
    with pytest.raises(sad.SadError) as e:
        sad.kmer_count(dev(codes), dev(s.offsets))
    assert e.value.status == sad.ERR_BAD_INPUT
    s = datagen.from_strings(["ACDEF", "AC"])
    with pytest.raises(sad.SadError) as e:
        sad.kmer_count(dev(s.codes), dev(s.offsets))
    assert e.value.status == sad.ERR_BAD_INPUT


# ------------------------------------------------------------------- rank ---

def check_rank(sad, oracle_mod, s, rows=None, k=3, alphabet=20, depth=0, word_max=False):
    wm = torch.empty(alphabet ** k, dtype=torch.int32, device="cuda") if word_max else None
    counts_g = sad.kmer_count(dev(s.codes), dev(s.offsets), k, alphabet, word_max=wm)
    if wm is not None:
        np.testing.assert_array_equal(host(wm), host(counts_g).max(axis=0))
    lengths = dev(s.lengths.astype(np.int32))
    hi, lo, rank = sad.kmer_rank(counts_g, lengths, k, alphabet, depth=depth, word_max=wm)
    hi, lo, rank = host(hi), host(lo), host(rank)
    counts = oracle_mod.kmer_count(s.codes, s.offsets, k, alphabet)
    if rows is None:
        ohi, olo, orank, ofp = oracle_mod.kmer_rank(counts, s.lengths, k, alphabet, with_fp64=True)
        rows = np.arange(s.n)
    else:
        rows = np.asarray(rows)
        ohi, olo, orank, ofp = oracle_mod.kmer_rank(counts, s.lengths, k, alphabet, rows=rows,
                                                    with_fp64=True)
    np.testing.assert_array_equal(hi[rows], ohi)
    np.testing.assert_array_equal(lo[rows], olo)
    np.testing.assert_array_equal(rank[rows], orank)
    assert np.all(np.abs(rank[rows] - ofp) <= 1e-12 * ofp)
    return hi, lo, rank


@pytest.mark.parametrize("n", [1, 2, 3, 127, 128, 129, 255, 256, 257, 383, 700])
def test_rank_sizes_and_ragged_tails(sad, oracle_mod, n):
    s = datagen.random_small(n, 3, 420, seed=n, alphabet=20)
    check_rank(sad, oracle_mod, s)


@pytest.mark.parametrize("depth,word_max", [(0, False), (1, False), (2, False), (3, False),
                                            (0, True), (1, True), (2, True)])
def test_rank_family_set_several_tiles(sad, oracle_mod, depth, word_max):
    sets = datagen.family_set(6, 230, lambda r: int(r.integers(40, 900)), p=4, seed=3, stream=9)
    check_rank(sad, oracle_mod, sets, depth=depth, word_max=word_max)


@pytest.mark.parametrize("depth,word_max", [(0, False), (1, False), (5, False), (40, False),
                                            (1, True), (40, True)])
def test_rank_small_alphabet_deep_planes(sad, oracle_mod, depth, word_max):
    # 4 letters, k = 3: 64 words, counts up to hundreds -> many threshold sections,
    # and, when the planes are cut, remainder chunks plus heavy entries (counts above
    # the remainder bitmap) added in the epilogue
    s = datagen.random_small(300, 3, 2500, seed=11, alphabet=4)
    check_rank(sad, oracle_mod, s, k=3, alphabet=4, depth=depth, word_max=word_max)


@pytest.mark.parametrize("depth", [0, 1, 7])
def test_rank_long_homopolymers_exact_accumulation(sad, oracle_mod, depth):
    """Shared counts close to the longest supported m (S = min(m_i, m_j) up to
    19998): the f32 tensor-core accumulation, the remainder chunks and the heavy
    entries must stay exact."""
    seqs = ["A" * 20000, "A" * 15000, "A" * 19999, "AC" * 6000, "A" * 3, "C" * 9000,
            "A" * 12000 + "C" * 8000]
    s = datagen.from_strings(seqs)
    check_rank(sad, oracle_mod, s, depth=depth)


@pytest.mark.parametrize("n,depth", [(129, 1), (257, 2), (700, 1)])
def test_rank_depth_cap_ragged(sad, oracle_mod, n, depth):
    s = datagen.random_small(n, 3, 900, seed=n + 17, alphabet=8)
    check_rank(sad, oracle_mod, s, k=3, alphabet=8, depth=depth)


def test_rank_identical_sequences_tie(sad, oracle_mod):
    s = datagen.from_strings(["ACDEFGHIKLMNPQ"] * 300 + ["WYWYWYWY"] * 10)
    hi, lo, _ = check_rank(sad, oracle_mod, s)
    assert len(set(zip(hi[:300].tolist(), lo[:300].tolist()))) == 1


def test_rank_reports_workspace_too_small(sad):
    s = datagen.random_small(300, 3, 400, seed=2)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    ws = sad.Workspace()
    ws.ensure(sad.workspace_bytes(sad.OP_RANK, s.n, depth=0) + 600 * 520)  # K_cap = 512
    plan = sad.kmer_rank_plan(counts, ws=ws)
    plan.k_cap = 512                                  # too few plane columns for the data
    ws.ensure(ws.nbytes + (4 << 20))                  # room for that layout: the device finds out
    plan.ws_bytes = ws.nbytes
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank(counts, dev(s.lengths.astype(np.int32)), ws=ws, plan=plan)
    assert e.value.status == sad.ERR_WORKSPACE


def test_rank_rejects_inconsistent_lengths(sad):
    s = datagen.random_small(50, 3, 100, seed=4)
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    bad = s.lengths.astype(np.int32).copy()
    bad[7] += 1
    with pytest.raises(sad.SadError) as e:
        sad.kmer_rank(counts, dev(bad))
    assert e.value.status == sad.ERR_BAD_INPUT


# -------------------------------------------------------------- partition ---

@pytest.mark.parametrize("n,p,distinct", [(16, 4, None), (1000, 4, None), (1000, 16, 5),
                                          (20000, 16, None), (100000, 64, None),
                                          (100000, 64, 50), (4097 * 3, 3, None),
                                          (30000, 2, 1000), (57, 57, None), (77, 1, None),
                                          (5000, 100, None), (1, 1, None),
                                          # the bounds of the chunk-merge route (p <= 64,
                                          # blocks of at most 64 x 256 items)
                                          (6500, 65, None), (6400, 64, 3), (16384, 1, None),
                                          (16385, 1, None), (40000, 2, 7), (300, 64, None),
                                          # pivots by ranking p (p - 1) <= 1024 samples,
                                          # blocks shorter than p (samples taken twice)
                                          (40, 16, None), (20, 8, 2), (33, 32, None),
                                          (992, 32, 4), (3, 2, None)])
def test_partition_matches_oracle(sad, oracle_mod, n, p, distinct):
    hi, lo = datagen.random_keys(n, seed=n * 7 + p, distinct=distinct)
    offs, mem, piv = sad.partition(dev(hi), dev(lo), p)
    ooffs, omem, opiv = oracle_mod.partition(hi, lo, p)
    np.testing.assert_array_equal(host(offs), ooffs)
    np.testing.assert_array_equal(host(mem), omem)
    np.testing.assert_array_equal(host(piv), opiv)


def test_partition_empty_set(sad):
    z = torch.zeros(0, dtype=torch.uint64, device="cuda")
    offs, mem, piv = sad.partition(z, z, 4)
    assert host(offs).tolist() == [0, 0, 0, 0, 0] and mem.numel() == 0


# ---------------------------------------------------------- whole configs ---

def test_config1_end_to_end(sad, oracle_mod):
    s = datagen.config1()
    res = sad.partition_set(dev(s.codes), dev(s.offsets), s.p)
    ref = oracle_mod.run_set(s.codes, s.offsets, s.p)
    for key in ("counts", "key_hi", "key_lo", "rank", "bucket_offsets", "members", "pivot_idx"):
        np.testing.assert_array_equal(host(res[key]), ref[key], err_msg=key)


@pytest.mark.parametrize("depth", [1, 2])
def test_config1_end_to_end_on_bound_plan(sad, oracle_mod, depth):
    """partition_set with depth >= 1 queues count -> rank -> partition on the
    host-side capacity bounds, without a synchronisation in between."""
    s = datagen.config1()
    res = sad.partition_set(dev(s.codes), dev(s.offsets), s.p, depth=depth)
    ref = oracle_mod.run_set(s.codes, s.offsets, s.p)
    for key in ("counts", "key_hi", "key_lo", "rank", "bucket_offsets", "members", "pivot_idx"):
        np.testing.assert_array_equal(host(res[key]), ref[key], err_msg=key)


@pytest.mark.parametrize("depth", [1, 2, 5])
def test_rank_on_bound_plan(sad, oracle_mod, depth):
    """kmer_rank_plan_bound's capacities hold for long repeats (a large residual)
    and for a family set; the keys are the oracle's."""
    sets = [datagen.from_strings(["A" * 3000, "A" * 2000, "AC" * 900, "ACD" * 400, "W" * 5,
                                  "ACDEFGHIKLMNPQRSTVWY" * 30]),
            datagen.family_set(6, 230, lambda r: int(r.integers(40, 900)), p=4, seed=3,
                               stream=9)]
    for s in sets:
        wm = torch.empty(8000, dtype=torch.int32, device="cuda")
        counts = sad.kmer_count(dev(s.codes), dev(s.offsets), word_max=wm)
        plan = sad.kmer_rank_plan_bound(s.n, s.codes.size, depth=depth)
        hi, lo, rank = sad.kmer_rank(counts, dev(s.lengths.astype(np.int32)), plan=plan,
                                     word_max=wm)
        c = oracle_mod.kmer_count(s.codes, s.offsets)
        ohi, olo, orank, _ = oracle_mod.kmer_rank(c, s.lengths, 3, 20, with_fp64=True)
        np.testing.assert_array_equal(host(hi), ohi)
        np.testing.assert_array_equal(host(lo), olo)
        np.testing.assert_array_equal(host(rank), orank)


def csr_invariants(hi, lo, p, offs, mem, piv):
    n = hi.shape[0]
    order = np.lexsort((np.arange(n), lo, hi))
    np.testing.assert_array_equal(mem, order)
    rank_of = np.empty(n, np.int64)
    rank_of[order] = np.arange(n)
    assert offs[0] == 0 and offs[-1] == n
    for i in range(p - 1):
        assert offs[i + 1] == rank_of[piv[i]] + 1


@pytest.mark.slow
def test_config2_paper_scale(sad, oracle_mod):
    """N = 20000 in 50 families, p = 16: counts in full, keys on 256 sampled rows
    (first, last, random), buckets against the sorted order of the keys."""
    s = datagen.config2()
    res = sad.partition_set(dev(s.codes), dev(s.offsets), s.p)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([[0, 1, s.n - 1], rng.integers(0, s.n, 253)]))
    counts_g = host(res["counts"])
    counts = oracle_mod.kmer_count(s.codes, s.offsets)
    np.testing.assert_array_equal(counts_g, counts)
    ohi, olo, orank = oracle_mod.kmer_rank(counts, s.lengths, rows=rows)
    hi, lo = host(res["key_hi"]), host(res["key_lo"])
    np.testing.assert_array_equal(hi[rows], ohi)
    np.testing.assert_array_equal(lo[rows], olo)
    np.testing.assert_array_equal(host(res["rank"])[rows], orank)
    offs, mem, piv = host(res["bucket_offsets"]), host(res["members"]), host(res["pivot_idx"])
    csr_invariants(hi, lo, s.p, offs, mem, piv)
    assert np.diff(offs).max() <= 2 * s.n // s.p
