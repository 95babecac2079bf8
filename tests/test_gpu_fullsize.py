"""Parity at full size, through the calls and plans the benchmark times.

bench.py runs kmer_count (with the per-word maxima) -> sad_seq_lengths ->
kmer_rank_plan at the autotuner's shape (GEMM tile 128 or 256 rows, plane depth,
remainder budget) -> kmer_rank on that plan -> partition. These tests run the same
sequence on the paper-scale set (N = 20000, 50 families, p = 16) at every shape the
autotuner may choose (tile x depth x budget) and on the large set (N = 100000, 500
families, p = 64) at every tile and depth and some of the other budgets, plus the
public partition_set path:

  N = 20000   every key and rank against the oracle's full rank (Eq. 1, Eq. 3; all
              N(N-1)/2 pairs on the host cores, computed once for the module), and
              the bucket offsets, members and pivots element by element against
              the oracle's regular-sampling partition (Sec. 3.1.2, Algorithm 2
              steps 7-11) of the same keys.
  N = 100000  keys and ranks of 128 rows (first, last, longest, shortest and
              random ones; each row against all N sequences in the oracle), and the
              partition element by element against the oracle's partition of the
              GPU's full key set (the oracle's partition is the reference for any
              keys; the sampled rows tie those keys to the oracle's rank).
"""
import numpy as np
import pytest

from paper_0905_1744_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEPTHS = (0, 1, 2, 3, 4, 6)     # the autotuner's candidates
TILES = (128, 256)
SHAPES = [(t, d, 0) for t in TILES for d in DEPTHS] + [(256, 2, 256), (256, 6, 1536),
                                                       (128, 4, 1536)]
# every shape the autotuner can pick: both tiles, every depth, and at depths >= 1 the
# budgets it tries (the default, 256, 1536)
ALL_SHAPES = [(t, d, b) for t in TILES for d in DEPTHS for b in ((0,) if d == 0 else (0, 256, 1536))]


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


def bench_path(sad, s, depth, tile=128, budget=0):
    """The benchmark's step at this plan shape (its plan made once, as there)."""
    codes, offsets = dev(s.codes), dev(s.offsets)
    ws = sad.Workspace(codes.device)
    word_max = torch.empty(8000, dtype=torch.int32, device="cuda")
    counts = sad.kmer_count(codes, offsets, ws=ws, word_max=word_max)
    lengths = sad.seq_lengths(offsets, ws=ws)
    plan = sad.kmer_rank_plan(counts, depth=depth, ws=ws, tile=tile, budget=budget)
    hi, lo, rank = sad.kmer_rank(counts, lengths, ws=ws, plan=plan, word_max=word_max)
    offs, mem, piv = sad.partition(hi, lo, s.p)
    torch.cuda.synchronize()
    return dict(counts=counts, key_hi=host(hi), key_lo=host(lo), rank=host(rank),
                bucket_offsets=host(offs), members=host(mem), pivot_idx=host(piv),
                depth=plan.depth, t_max=plan.t_max)


def assert_partition(res, oracle_mod, p):
    offs, mem, piv = oracle_mod.partition(res["key_hi"], res["key_lo"], p)
    np.testing.assert_array_equal(res["bucket_offsets"], offs)
    np.testing.assert_array_equal(res["members"], mem)
    np.testing.assert_array_equal(res["pivot_idx"], piv)


@pytest.fixture(scope="module")
def c2_oracle(oracle_mod):
    s = datagen.config2()
    counts = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank = oracle_mod.kmer_rank(counts, s.lengths)
    offs, mem, piv = oracle_mod.partition(hi, lo, s.p)
    return s, counts, dict(key_hi=hi, key_lo=lo, rank=rank, bucket_offsets=offs, members=mem,
                           pivot_idx=piv)


def assert_c2(res, ref, what):
    for key in ("key_hi", "key_lo", "rank", "bucket_offsets", "members", "pivot_idx"):
        np.testing.assert_array_equal(res[key], ref[key], err_msg=f"{what}: {key}")


def test_c2_counts_in_full(sad, c2_oracle):
    s, counts, _ = c2_oracle
    res = bench_path(sad, s, 1)
    np.testing.assert_array_equal(host(res["counts"]), counts)


@pytest.mark.parametrize("tile,depth,budget", ALL_SHAPES)
def test_c2_bench_path_every_key_and_bucket(sad, c2_oracle, tile, depth, budget):
    s, _, ref = c2_oracle
    res = bench_path(sad, s, depth, tile, budget)
    assert res["depth"] == depth
    assert_c2(res, ref, f"tile {tile} depth {depth} budget {budget}")


@pytest.mark.parametrize("tile,depth", [(128, 1), (256, 2), (256, 6)])
def test_c2_partition_set_on_host_bounds(sad, c2_oracle, tile, depth):
    """The public call the end-to-end figure times (capacity bounds, no sync)."""
    s, _, ref = c2_oracle
    out = sad.partition_set(dev(s.codes), dev(s.offsets), s.p, depth=depth, tile=tile)
    res = {k: host(out[k]) for k in ("key_hi", "key_lo", "rank", "bucket_offsets", "members",
                                     "pivot_idx")}
    assert_c2(res, ref, f"partition_set tile {tile} depth {depth}")


def test_c2_autotuned_shape(sad, c2_oracle):
    from paper_0905_1744_gb300 import autotune
    s, _, ref = c2_oracle
    counts = sad.kmer_count(dev(s.codes), dev(s.offsets))
    shape, trials = autotune.choose_shape(counts, dev(s.lengths.astype(np.int32)),
                                          use_cache=False)
    assert shape.key in trials and len(trials) >= 8
    assert {autotune.Shape.parse(k).tile for k in trials} == {128, 256}
    assert_c2(bench_path(sad, s, shape.depth, shape.tile, shape.budget), ref,
              f"autotuned {shape.key}")


@pytest.fixture(scope="module")
def c3_oracle(oracle_mod):
    s = datagen.config3()
    rng = np.random.default_rng(33)
    fixed = [0, 1, s.n - 1, int(np.argmax(s.lengths)), int(np.argmin(s.lengths))]
    rest = rng.choice(np.setdiff1d(np.arange(s.n), fixed), size=128 - len(set(fixed)),
                      replace=False)
    rows = np.unique(np.concatenate([fixed, rest]))
    assert rows.size == 128
    counts = oracle_mod.kmer_count(s.codes, s.offsets)
    hi, lo, rank = oracle_mod.kmer_rank(counts, s.lengths, rows=rows)
    sample_counts = counts[rows].copy()
    del counts
    return s, rows, sample_counts, dict(key_hi=hi, key_lo=lo, rank=rank)


@pytest.mark.parametrize("tile,depth,budget", SHAPES)
def test_c3_bench_path_sampled_keys_and_buckets(sad, oracle_mod, c3_oracle, tile, depth, budget):
    s, rows, sample_counts, ref = c3_oracle
    res = bench_path(sad, s, depth, tile, budget)
    np.testing.assert_array_equal(host(res["counts"][dev(rows)]), sample_counts)
    for key in ("key_hi", "key_lo", "rank"):
        np.testing.assert_array_equal(res[key][rows], ref[key], err_msg=f"depth {depth}: {key}")
    assert_partition(res, oracle_mod, s.p)


def test_c3_partition_set_on_host_bounds(sad, oracle_mod, c3_oracle):
    s, rows, _, ref = c3_oracle
    out = sad.partition_set(dev(s.codes), dev(s.offsets), s.p, depth=6, tile=256)
    res = {k: host(out[k]) for k in ("key_hi", "key_lo", "rank", "bucket_offsets", "members",
                                     "pivot_idx")}
    for key in ("key_hi", "key_lo", "rank"):
        np.testing.assert_array_equal(res[key][rows], ref[key], err_msg=key)
    assert_partition(res, oracle_mod, s.p)
