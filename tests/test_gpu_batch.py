"""Batched rank and partition (many independent sets in one block-diagonal GEMM
launch and one batched partition) against the oracle run on every set alone."""
import numpy as np
import pytest

from paper_0905_1744_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("counts", "key_hi", "key_lo", "rank", "bucket_offsets", "members", "pivot_idx")


@pytest.fixture(scope="module")
def sad():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0905_1744_gb300 import build, sad as sadmod
    build.build()
    return sadmod


def mixed_sets():
    sets = [datagen.random_small(1, 3, 50, seed=1, p=1),
            datagen.random_small(2, 3, 60, seed=2, p=2),
            datagen.random_small(300, 3, 400, seed=3, p=5),
            datagen.family_set(4, 60, lambda r: int(r.integers(40, 700)), p=3, seed=4, stream=41),
            datagen.random_small(129, 50, 2000, seed=5, alphabet=20, p=16),
            datagen.batch_set(7), datagen.batch_set(11)]
    for s in sets:
        s.p = min(s.p, s.n)
    return sets


def check_sets(b, sets, oracle_mod, which=None):
    for i in (range(len(sets)) if which is None else which):
        s = sets[i]
        ref = oracle_mod.run_set(s.codes[s.offsets[0]:s.offsets[-1]],
                                 s.offsets - s.offsets[0], s.p)
        got = b.result(i)
        for key in KEYS:
            np.testing.assert_array_equal(got[key], ref[key], err_msg=f"set {i} {key}")


@pytest.mark.parametrize("tile", [128, 256])
@pytest.mark.parametrize("depth,bound", [(0, False), (1, True), (2, True), (2, False),
                                         (3, True), (4, True), (6, True)])
def test_batch_matches_oracle_per_set(sad, oracle_mod, tile, depth, bound):
    """Every (tile, depth) the autotuner can pick for a batch, on bound plans (the
    plan-free path) and on exact plans."""
    sets = mixed_sets()
    b = sad.Batch(sets)
    plan = b.plan(depth=depth, tile=tile, bound=bound)
    b.run()
    torch.cuda.synchronize()
    b.check()
    check_sets(b, sets, oracle_mod)
    # every set's rows are padded to the tile
    pad = ((b.n + tile - 1) // tile * tile).sum()
    assert plan.rows_total == pad


def test_batch_budgets(sad, oracle_mod):
    sets = mixed_sets()
    b = sad.Batch(sets)
    for budget in (64, 1536):
        b.plan(depth=2, tile=256, budget=budget)
        b.key_hi.zero_()
        b.run()
        torch.cuda.synchronize()
        b.check()
        check_sets(b, sets, oracle_mod)


def test_one_graph_serves_different_batches(sad, oracle_mod):
    """One library graph captured for a batch, then updated in place for a second
    batch of other sizes (new buffers, new bound plan) and for the first again:
    each replay equals the oracle per set, with no re-instantiation."""
    sets_a = [datagen.batch_set(i) for i in range(12)]
    sets_b = [datagen.batch_set(i, seed=7) for i in range(9)] + [datagen.random_small(3, 3, 90,
                                                                                     seed=4, p=2)]
    ws = (sad.Workspace(torch.device("cuda"), 256), sad.Workspace(torch.device("cuda")),
          sad.Workspace(torch.device("cuda")))
    s = torch.cuda.Stream()
    ba = sad.Batch(sets_a, workspaces=ws, stream=s)
    bb = sad.Batch(sets_b, workspaces=ws, stream=s)
    g = sad.Graph()
    for b, sets in ((ba, sets_a), (bb, sets_b), (ba, sets_a)):
        b.key_hi.zero_()
        b.members.fill_(-1)
        torch.cuda.synchronize()
        b.plan(depth=2, tile=256, stream=s)
        b.capture(g, stream=s)
        g.launch(s)
        s.synchronize()
        b.check(s)
        check_sets(b, sets, oracle_mod, which=(0, len(sets) // 2, len(sets) - 1))
    st = g.stats()
    assert st["instantiations"] == 1 and st["updates"] == 2 and st["kernels"] >= 10


def test_batch_graph_replay_is_identical(sad, oracle_mod):
    sets = [datagen.batch_set(i) for i in range(12)]
    b = sad.Batch(sets)
    b.plan(depth=1)
    b.capture()
    for _ in range(2):
        b.key_hi.zero_()
        b.members.fill_(-1)
        b.replay()
        torch.cuda.synchronize()
        b.check()
        check_sets(b, sets, oracle_mod, which=(0, 5, 11))


def test_seq_lengths_from_offsets(sad):
    off = torch.tensor([3, 3, 10, 400, 401], dtype=torch.int64, device="cuda")
    np.testing.assert_array_equal(sad.seq_lengths(off).cpu().numpy(), [0, 7, 390, 1])
    ws = sad.Workspace(torch.device("cuda"), 256)
    bad = torch.tensor([5, 2, 9], dtype=torch.int64, device="cuda")
    out = sad.seq_lengths(bad, ws=ws)
    assert ws.status() == sad.ERR_BAD_INPUT
    assert out.cpu().tolist() == [0, 7]


def test_graph_keeps_single_and_multi_set_captures_apart(sad, oracle_mod):
    """A single-set batch and a multi-set batch launch different preparation
    kernels in as many graph nodes; the handle instantiates each launch sequence
    once and updates only a graph of the same sequence, so every batch through it
    equals the oracle."""
    pool = [datagen.batch_set(i, seed=3, n_lo=40, n_hi=900) for i in range(8)]
    groups = [[0], [1, 2, 3, 4], [5, 6, 7], [0, 1], [3], [2, 3, 4, 5, 6, 7]]
    s = torch.cuda.Stream()
    g = sad.Graph()
    for grp in groups:
        sets = [pool[i] for i in grp]
        b = sad.Batch(sets, stream=s)
        b.plan(depth=1, tile=256, stream=s)
        b.capture(g, stream=s)
        g.launch(s)
        s.synchronize()
        b.check(s)
        check_sets(b, sets, oracle_mod)
    st = g.stats()
    assert st["instantiations"] == 2 and st["updates"] == 4


def test_batches_on_one_pool(sad, oracle_mod):
    """Batches built one after another on one BatchPool (staging, device arrays and
    workspaces reused) each equal the oracle; once the pool holds the largest batch,
    building another allocates nothing new."""
    pool_sets = [datagen.batch_set(i, seed=5, n_lo=40, n_hi=700) for i in range(10)]
    groups = [[0, 1, 2], [3, 4, 5, 6, 7, 8, 9], [2], [0, 1, 2]]
    pool = sad.BatchPool()
    s = torch.cuda.Stream()
    ptrs = None
    for gi, grp in enumerate(groups):
        sets = [pool_sets[i] for i in grp]
        b = sad.Batch(sets, stream=s, pool=pool)
        b.plan(depth=2, tile=256, stream=s)
        for ws in pool.workspaces:
            ws.buf[:8].zero_()
        b.run(stream=s)
        s.synchronize()
        b.check(s)
        check_sets(b, sets, oracle_mod)
        if gi == 1:
            ptrs = {k: t.data_ptr() for k, t in pool.bufs.items()}
    assert {k: t.data_ptr() for k, t in pool.bufs.items()} == ptrs
