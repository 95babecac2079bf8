"""Failure detection by a bounded device wait (no hang, no fault).

Every wait of the plane GEMM is a spin on %globaltimer with a budget. These tests
shorten the budget of the main-loop waits to a few nanoseconds through the
library's test hook, so the first wait that does not succeed at once gives up:
the kernel must record SAD_ERR_TIMEOUT in the workspace status, drain its own
copies and MMAs, free its tensor memory and return. The status is read on the
host; the context stays usable, and the next call with the normal budget on a
fresh workspace gives the oracle's keys bit for bit.
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


@pytest.mark.parametrize("depth", (0, 1))
def test_short_wait_budget_returns_timeout_then_recovers(sad, oracle_mod, depth):
    # long sequences: each tile's MMAs take microseconds, longer than the budget
    s = datagen.family_set(6, 150, lambda r: int(r.integers(600, 1800)), p=4, seed=11,
                           stream=21)
    codes, offsets = dev(s.codes), dev(s.offsets)
    lengths = dev(s.lengths.astype(np.int32))
    counts = sad.kmer_count(codes, offsets)
    ws = sad.Workspace(codes.device)
    plan = sad.kmer_rank_plan(counts, depth=depth, ws=ws)
    try:
        sad.debug_wait_budget_ns(4)
        sad.kmer_rank(counts, lengths, ws=ws, plan=plan, check=False)
        torch.cuda.synchronize()
        assert ws.status() == sad.ERR_TIMEOUT
    finally:
        sad.debug_wait_budget_ns(0)
    # the context is usable and a normal call on a fresh workspace is exact
    ws2 = sad.Workspace(codes.device)
    hi, lo, rank = sad.kmer_rank(counts, lengths, ws=ws2, depth=depth)
    c = oracle_mod.kmer_count(s.codes, s.offsets)
    ohi, olo, orank = oracle_mod.kmer_rank(c, s.lengths)
    np.testing.assert_array_equal(hi.cpu().numpy(), ohi)
    np.testing.assert_array_equal(lo.cpu().numpy(), olo)
    np.testing.assert_array_equal(rank.cpu().numpy(), orank)
    # the workspace that saw the timeout also works again once its status is cleared
    ws.clear_status()
    hi2, lo2, _ = sad.kmer_rank(counts, lengths, ws=ws, plan=plan)
    np.testing.assert_array_equal(hi2.cpu().numpy(), ohi)
    np.testing.assert_array_equal(lo2.cpu().numpy(), olo)
