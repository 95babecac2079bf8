"""partition_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (a pool or arena that owns every device byte, an embedding that
forbids allocation after start-up) get the partition with its scratch in a fixed
array inside the library. This file is collected last on purpose: if it fails, a
run that stops at the first failure has already run everything else. The test
calls the entry point through the C-ABI twice in a row (the second call sees the
first call's leftovers in the shared array) and compares it with partition().
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


def test_noalloc_matches_partition_twice(sad):
    # second call: smaller N, more buckets, ties; then the documented maximum with
    # few and with the most buckets (the scratch is sized for the largest accepted call)
    cases = [(20000, 16, None), (5000, 64, 40), (sad.NOALLOC_MAX_N, 16, None),
             (sad.NOALLOC_MAX_N, sad.NOALLOC_MAX_P, None), (sad.NOALLOC_MAX_N, 1, 100)]
    for n, p, distinct in cases:
        hi, lo = datagen.random_keys(n, seed=1000 + n, distinct=distinct)
        d_hi, d_lo = torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda()
        ref = sad.partition(d_hi, d_lo, p)
        got = sad.partition_noalloc(d_hi, d_lo, p)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):                    # integer outputs: bit for bit
            np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_scratch(sad):
    hi, lo = datagen.random_keys(sad.NOALLOC_MAX_N + 1, seed=5)
    d_hi, d_lo = torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda()
    with pytest.raises(sad.SadError) as e:
        sad.partition_noalloc(d_hi, d_lo, 16)
    assert e.value.status == sad.ERR_UNSUPPORTED
    with pytest.raises(sad.SadError) as e:
        sad.partition_noalloc(d_hi[:1000], d_lo[:1000], sad.NOALLOC_MAX_P + 1)
    assert e.value.status == sad.ERR_UNSUPPORTED
