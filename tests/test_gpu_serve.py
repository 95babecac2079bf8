"""Serving with continuous batching: every request's buckets and keys are the same
when it is served in a mix (batched with whatever else arrived) as when it is
computed alone, and both equal the oracle."""
import numpy as np
import pytest

from paper_0905_1744_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0905_1744_gb300 import build, sad, serve
    build.build()
    return sad, serve


def test_served_results_equal_alone_and_oracle(mods, oracle_mod):
    sad, serve = mods
    pool = [datagen.batch_set(i, seed=3, n_lo=40, n_hi=900) for i in range(8)]
    arrivals = np.cumsum(np.full(24, 1.0 / 3000.0))        # arrivals faster than service
    stats = {}
    mixed = serve.serve(serve.make_requests(pool, arrivals), shape=(256, 1, 0), slots=2,
                        stats=stats, max_batch=4)
    alone = serve.serve_plain(serve.make_requests(pool, arrivals), shape=(128, 2, 0))
    for rm, ra in zip(mixed, alone):
        for key in ("bucket_offsets", "members", "key_hi", "key_lo"):
            np.testing.assert_array_equal(rm.result[key], ra.result[key], err_msg=f"{rm.rid} {key}")
    for i, s in enumerate(pool):
        ref = oracle_mod.run_set(s.codes, s.offsets, s.p)
        for key in ("bucket_offsets", "members", "key_hi", "key_lo"):
            np.testing.assert_array_equal(mixed[i].result[key], ref[key], err_msg=f"{i} {key}")
    assert all(r.done >= r.arrival for r in mixed)
    # several batches, two of them in flight together (host) and overlapping on the
    # device (start and end events on their streams); the slots' graphs were
    # updated for later batches, not re-instantiated
    assert stats["batches"] >= 3
    assert stats["max_inflight_host"] >= 2 and stats["max_inflight_device"] >= 2
    assert stats["graph_updates"] >= 1


def test_admission_respects_budget(mods):
    sad, serve = mods
    pool = [datagen.batch_set(i, seed=4, n_lo=40, n_hi=300) for i in range(6)]
    one = max(serve.request_bytes(s, 1, tile=128) for s in pool)
    arrivals = np.zeros(12)
    stats = {}
    reqs = serve.serve(serve.make_requests(pool, arrivals), shape=(128, 1, 0), slots=3,
                       budget_bytes=int(1.5 * one), stats=stats)   # one request at a time
    assert all(r.result is not None for r in reqs)
    assert stats["max_inflight_host"] == 1 and stats["peak_admitted_bytes"] <= 1.5 * one
