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


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_batch_matches_oracle_per_set(sad, oracle_mod, depth):
    sets = mixed_sets()
    b = sad.Batch(sets)
    b.plan(depth=depth)
    b.run()
    torch.cuda.synchronize()
    b.check()
    for i, s in enumerate(sets):
        ref = oracle_mod.run_set(s.codes[s.offsets[0]:s.offsets[-1]],
                                 s.offsets - s.offsets[0], s.p)
        got = b.result(i)
        for key in KEYS:
            np.testing.assert_array_equal(got[key], ref[key], err_msg=f"set {i} {key}")


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
        for i in (0, 5, 11):
            s = sets[i]
            ref = oracle_mod.run_set(s.codes, s.offsets, s.p)
            got = b.result(i)
            for key in KEYS:
                np.testing.assert_array_equal(got[key], ref[key], err_msg=f"set {i} {key}")
