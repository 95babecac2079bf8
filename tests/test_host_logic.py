"""Host-side logic that needs no GPU: serving admission, the depth autotuner's
choice and cache, and the bench's per-call timing helper (the device calls and
events they use are replaced by fakes here; the same paths run on the GPU in
test_gpu_serve.py, test_gpu_configs.py and bench.py)."""
import json
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_0905_1744_gb300 import autotune, datagen, serve  # noqa: E402


def _set(n, length=50, seed=0):
    return datagen.random_small(n, 3, length, seed=seed)


# ------------------------------------------------------------------ serving ---

def test_request_bytes_grows_with_set_size_and_depth():
    small, big = _set(10), _set(300)
    for d in (1, 2, 4):
        assert serve.request_bytes(small, d) < serve.request_bytes(big, d)
    b = [serve.request_bytes(big, d) for d in (1, 2, 3, 4)]
    assert b == sorted(b) and len(set(b)) == 4
    # the counts alone (4 bytes x 8000 words a sequence) are inside the estimate
    assert serve.request_bytes(big, 1) > 4 * 300 * 8000
    # CTA-pair tiles pad rows to 256: never less than 128-row tiles
    assert serve.request_bytes(big, 2, tile=256) >= serve.request_bytes(big, 2, tile=128)
    # the rank workspace is the library's bound plan for the set
    from paper_0905_1744_gb300 import sad
    plan = sad.kmer_rank_plan_bound(300, int(big.offsets[-1]), 3, 20, depth=2, tile=256)
    assert serve.request_bytes(big, 2) > plan.ws_bytes


def test_select_batch_takes_the_fitting_prefix_in_arrival_order():
    sets = [_set(20 + 10 * i, seed=i) for i in range(5)]
    reqs = serve.make_requests(sets, np.zeros(5))
    rb = [serve.request_bytes(s, 1) for s in sets]
    # everything fits
    take, nb = serve.select_batch(reqs, 0, sum(rb), 64, 1)
    assert [r.rid for r in take] == [0, 1, 2, 3, 4] and nb == sum(rb)
    # max_batch caps the batch
    take, nb = serve.select_batch(reqs, 0, sum(rb), 2, 1)
    assert [r.rid for r in take] == [0, 1] and nb == rb[0] + rb[1]
    # the bytes in flight count against the budget
    take, _ = serve.select_batch(reqs, sum(rb) - rb[0] - rb[1], sum(rb), 64, 1)
    assert [r.rid for r in take] == [0, 1]
    # a later, smaller request never overtakes a head that does not fit
    take, nb = serve.select_batch(reqs[1:], 0, rb[1] - 1, 64, 1)
    assert take == [] and nb == 0
    take, _ = serve.select_batch(reqs, 0, rb[0], 64, 1)
    assert [r.rid for r in take] == [0]


def test_serve_rejects_a_request_above_the_budget_before_any_device_call():
    reqs = serve.make_requests([_set(50)], [0.0])
    need = serve.request_bytes(reqs[0].seqset, 2)
    with pytest.raises(ValueError, match="budget"):
        serve.serve(reqs, shape=(256, 2, 0), budget_bytes=need - 1, device="cpu")
    with pytest.raises(ValueError):
        serve.serve(reqs, shape=(256, 2, 0), slots=0, device="cpu")
    # the plan-free path needs cut planes (depth >= 1)
    with pytest.raises(ValueError, match="depth"):
        serve.serve(reqs, shape=(256, 0, 0), device="cpu")


def test_max_overlap_counts_open_intervals():
    assert serve.max_overlap([]) == 0
    assert serve.max_overlap([(0, 1), (1, 2)]) == 1          # touching ends do not overlap
    assert serve.max_overlap([(0, 3), (1, 2), (2.5, 4)]) == 2
    assert serve.max_overlap([(0, 5), (1, 4), (2, 3)]) == 3


def test_latency_stats():
    reqs = serve.make_requests([_set(5)], [0.0, 0.5, 1.0, 1.5])
    for r, d in zip(reqs, (0.1, 0.7, 1.3, 2.0)):
        r.done = d
    st = serve.latency_stats(reqs)
    lat = np.array([0.1, 0.2, 0.3, 0.5])
    assert st["mean_ms"] == pytest.approx(1e3 * lat.mean())
    assert st["p50_ms"] == pytest.approx(1e3 * np.percentile(lat, 50))
    assert st["sets_per_s"] == pytest.approx(4 / 2.0)
    assert serve.latency_stats(reqs, skip=2)["sets_per_s"] == pytest.approx(2 / 1.0)


# ---------------------------------------------------------------- autotuner ---

def _fake_plans(monkeypatch, t_max, ws_bytes, rem_bound=1000):
    calls = []

    def plan(counts, k=3, alphabet=20, depth=0, ws=None, stream=None, budget=0, tile=0):
        calls.append((tile, depth, budget))
        return types.SimpleNamespace(depth=depth, tile=tile, budget=budget, t_max=t_max,
                                     rem_bound=rem_bound, ws_bytes=ws_bytes(tile, depth))
    monkeypatch.setattr(autotune.sad, "kmer_rank_plan", plan)
    return calls


class _FakeWs:
    def __init__(self):
        self.ensured = []

    def ensure(self, nbytes):
        self.ensured.append(nbytes)


S = autotune.Shape


def test_search_picks_among_tile_shapes_then_budgets():
    """Faked timings: the fastest (tile, depth) of the first round, then the other
    budgets at that (tile, depth) only."""
    ms = {S(256, 0, 0): 3.0, S(256, 2, 0): 1.4, S(128, 0, 0): 2.5, S(128, 2, 0): 1.6,
          S(256, 2, 256): 1.5, S(256, 2, 1536): 1.3}
    timed = []

    def timer(sh):
        timed.append(sh)
        return ms[sh]
    first = autotune.first_round(None, tiles=(256, 128), depths=(0, 2))
    assert first == [S(256, 0, 0), S(256, 2, 0), S(128, 0, 0), S(128, 2, 0)]
    best, trials = autotune.search(timer, first)
    assert best == S(256, 2, 1536)
    # first round, the budgets at the best, then the three fastest twice more in turn
    finalists = [S(256, 2, 1536), S(256, 2, 0), S(256, 2, 256)]
    assert timed == first + [S(256, 2, 256), S(256, 2, 1536)] + finalists + finalists
    assert trials == {k.key: v for k, v in ms.items()}
    # the other tile shape wins when it is faster; depth 0 cuts nothing: no budget round
    ms2 = {S(256, 0, 0): 2.0, S(128, 0, 0): 1.0}
    best, trials = autotune.search(lambda sh: ms2[sh],
                                   autotune.first_round(None, tiles=(256, 128), depths=(0,)))
    assert best == S(128, 0, 0) and len(trials) == 2
    # shapes that do not apply (None) are skipped; nothing at all is an error
    best, _ = autotune.search(lambda sh: None if sh.tile == 256 else 1.0,
                              autotune.first_round(None, tiles=(256, 128), depths=(0,)))
    assert best == S(128, 0, 0)
    with pytest.raises(RuntimeError):
        autotune.search(lambda sh: None, [S(128, 0, 0)])
    assert S.parse(S(256, 6, 768).key) == S(256, 6, 768)


def test_search_confirms_the_finalists():
    """A shape whose first timing was lucky loses to one that is steadily faster when
    the finalists are timed again side by side (medians decide)."""
    seq = {S(256, 4, 0): iter([1.0, 2.0, 2.1]), S(256, 6, 0): iter([1.2, 1.2, 1.2]),
           S(128, 4, 0): iter([3.0, 3.0, 3.0])}
    best, trials = autotune.search(lambda sh: next(seq[sh]), list(seq), budgets=())
    assert best == S(256, 6, 0)
    assert trials[S(256, 4, 0).key] == 2.0 and trials[S(256, 6, 0).key] == 1.2


def test_first_round_skips_depths_that_keep_every_plane():
    assert autotune.first_round(3, tiles=(128,), depths=(0, 1, 2, 3, 4)) == \
        [S(128, 0, 0), S(128, 1, 0), S(128, 2, 0)]
    assert autotune.first_round(None, tiles=(256,), depths=(0, 1, 2), min_depth=1) == \
        [S(256, 1, 0), S(256, 2, 0)]


def test_choose_shape_times_candidates_and_keeps_the_fastest(monkeypatch):
    autotune._cache.clear()
    _fake_plans(monkeypatch, t_max=4, ws_bytes=lambda t, d: 100 * (d + 1) + t)
    ms = {(256, 0): 3.0, (256, 1): 1.5, (256, 2): 1.1, (256, 3): 2.0,
          (128, 0): 3.5, (128, 1): 1.9, (128, 2): 1.2, (128, 3): 2.2}
    bud = {256: 1.3, 1536: 1.0}
    timed = []

    def time_rank(counts, lengths, plan, ws, *a, **kw):
        timed.append((plan.tile, plan.depth, plan.budget))
        return ms[(plan.tile, plan.depth)] if plan.budget == 0 else bud[plan.budget]
    monkeypatch.setattr(autotune, "time_rank", time_rank)
    ws = _FakeWs()
    counts = torch.zeros(300, 8000, dtype=torch.int32)
    best, trials = autotune.choose_shape(counts, None, ws, use_cache=False,
                                         depths=(0, 1, 2, 3, 4))
    # depth 4 >= t_max keeps every plane (the work of depth 0): not timed
    assert timed[:8] == [(t, d, 0) for t in (256, 128) for d in range(4)]
    assert timed[8:10] == [(256, 2, 256), (256, 2, 1536)]
    # the three fastest again, twice, in turn
    assert timed[10:] == [(256, 2, 1536), (256, 2, 0), (128, 2, 0)] * 2
    assert best == S(256, 2, 1536) and len(trials) == 10
    # a workspace limit drops the shapes that need more
    timed.clear()
    best, trials = autotune.choose_shape(counts, None, ws, use_cache=False, max_ws_bytes=330,
                                         depths=(0, 1, 2, 3, 4))
    assert best == S(128, 1, 1536)
    assert all(100 * (d + 1) + t <= 330 for t, d, b in timed)


def test_choose_shape_cache_by_size_class(monkeypatch, tmp_path):
    autotune._cache.clear()
    _fake_plans(monkeypatch, t_max=3, ws_bytes=lambda t, d: 1)
    monkeypatch.setattr(autotune, "time_rank",
                        lambda counts, lengths, plan, ws, *a, **kw:
                        {0: 2.0, 1: 1.0, 2: 3.0}[plan.depth] + (0.5 if plan.tile == 128 else 0))
    counts = torch.zeros(1000, 1, dtype=torch.int32)
    best, trials = autotune.choose_shape(counts, None, _FakeWs())
    assert best == S(256, 1, 0) and trials
    # same size class (log2 N, t_max, log2 remainder bound): answered from the cache
    best2, trials2 = autotune.choose_shape(torch.zeros(1023, 1, dtype=torch.int32), None,
                                           _FakeWs())
    assert best2 == best and trials2 == {}
    path = str(tmp_path / "tune.json")
    autotune.save_cache(path)
    with open(path) as f:
        saved = json.load(f)
    plan1 = types.SimpleNamespace(t_max=3, rem_bound=1000)
    assert saved == {"set_" + autotune.signature(1000, plan1): best.key}
    autotune._cache.clear()
    autotune.load_cache(path)
    assert autotune._cache == saved
    autotune._cache.clear()


def test_signature_buckets():
    p = types.SimpleNamespace(t_max=5, rem_bound=0)
    assert autotune.signature(1024, p) == autotune.signature(2047, p) == "n10_t5_r0"
    assert autotune.signature(2048, p) == "n11_t5_r0"
    assert autotune.signature(0, types.SimpleNamespace(t_max=1, rem_bound=3)) == "n0_t1_r1"


# ------------------------------------------------------------ bench helpers ---

def test_time_calls_brackets_each_call_after_a_flush():
    import bench
    log = []
    clock = [0.0]

    class Ev:
        def __init__(self, enable_timing=False):
            assert enable_timing
            self.t = None

        def record(self, stream):
            assert stream == "s"
            self.t = clock[0]
            log.append("record")

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    def work(ms):
        def fn():
            log.append("call")
            clock[0] += ms
        return fn

    out = bench.time_calls({"a": work(2.0), "b": work(5.0)}, reps=3,
                           flush=lambda: log.append("flush"), stream="s", event_cls=Ev)
    assert out == {"a": 2.0, "b": 5.0}
    assert log == ["flush", "record", "call", "record"] * 6


# ------------------------------------------------- binding argument checks ---

@pytest.fixture
def sad_no_lib(monkeypatch):
    """The binding with its library replaced by a tripwire: every check below must
    raise before any library call."""
    from paper_0905_1744_gb300 import sad

    def tripwire():
        raise AssertionError("the library was reached")
    monkeypatch.setattr(sad, "_load", tripwire)
    return sad


def test_binding_refuses_host_tensors(sad_no_lib):
    sad = sad_no_lib
    u8, i64 = torch.zeros(10, dtype=torch.uint8), torch.tensor([0, 5, 10])
    counts = torch.zeros((2, 8000), dtype=torch.int32)
    keys = torch.zeros(4, dtype=torch.uint64)
    lengths = torch.tensor([5, 5], dtype=torch.int32)
    calls = [lambda: sad.kmer_count(u8, i64),
             lambda: sad.kmer_rank_plan(counts),
             lambda: sad.kmer_rank(counts, lengths),
             lambda: sad.partition(keys, keys, 2),
             lambda: sad.partition_noalloc(keys, keys, 2),
             lambda: sad.local_samples(keys, keys, 2, 1),
             lambda: sad.local_ranks(counts, lengths, 1),
             lambda: sad.kmer_rank_vs(counts, lengths, torch.tensor([0, 1])),
             lambda: sad.kmer_rank_dist(counts, lengths),
             lambda: sad.sparse_entries(counts, lengths),
             lambda: sad.kmer_rank_sparse(counts, lengths),
             lambda: sad.ln_q(keys),
             lambda: sad.GlobalRank(counts, lengths, 1, 1)]
    for f in calls:
        with pytest.raises(TypeError, match="CUDA tensor"):
            f()


def test_binding_checks_element_size_layout_and_shape(sad_no_lib, monkeypatch):
    sad = sad_no_lib
    monkeypatch.setattr(sad, "_DEVICE_TYPE", "cpu")   # host tensors stand in for device ones
    u8, i64 = torch.zeros(10, dtype=torch.uint8), torch.tensor([0, 5, 10])
    with pytest.raises(TypeError, match="8-byte"):
        sad.kmer_count(u8, i64.to(torch.int32))      # offsets are int64 in the C-ABI
    with pytest.raises(TypeError, match="1-byte"):
        sad.kmer_count(u8.to(torch.int32), i64)
    with pytest.raises(ValueError, match="out must be"):
        sad.kmer_count(u8, i64, out=torch.zeros((3, 8000), dtype=torch.int32))
    with pytest.raises(ValueError, match="word_max"):
        sad.kmer_count(u8, i64, word_max=torch.zeros(10, dtype=torch.int32))
    counts = torch.zeros((2, 8000), dtype=torch.int32)
    lengths = torch.tensor([5, 5], dtype=torch.int32)
    with pytest.raises(ValueError, match="contiguous"):
        sad.kmer_rank(torch.zeros((8000, 2), dtype=torch.int32).t(), lengths)
    with pytest.raises(ValueError, match=r"\[N, 64\]"):
        sad.kmer_rank(counts, lengths, 3, 4)          # counts of another alphabet
    with pytest.raises(TypeError, match="4-byte"):
        sad.kmer_rank(counts.to(torch.int64), lengths)
    with pytest.raises(ValueError, match="outputs"):
        sad.kmer_rank(counts, lengths,
                      out=(torch.zeros(3, dtype=torch.uint64), torch.zeros(3, dtype=torch.uint64),
                           None))
    keys = torch.zeros(4, dtype=torch.uint64)
    with pytest.raises(ValueError, match="differ"):
        sad.partition(keys, keys[:3], 2)
    with pytest.raises(TypeError, match="8-byte"):
        sad.partition(keys.to(torch.int32), keys, 2)
    with pytest.raises(ValueError, match="outputs need"):
        sad.partition(keys, keys, 2, out=(torch.zeros(3, dtype=torch.int32),
                                          torch.zeros(2, dtype=torch.int32),
                                          torch.zeros(1, dtype=torch.int32)))
    with pytest.raises(ValueError, match="out needs"):
        sad.local_samples(keys, keys, 2, 3, out=torch.zeros(5, dtype=torch.int32))


# ------------------------------------------------------------ batch layout ---

def test_batch_layout_and_per_set_results_on_the_host():
    """The batch concatenates every set's sequences (offsets rebased), and its
    per-set views cut the shared outputs at the right places: sequences, p + 1
    bucket offsets and p - 1 pivots per set."""
    from paper_0905_1744_gb300 import sad
    sets = [datagen.random_small(n, 3, 40, seed=n) for n in (5, 1, 12)]
    sets[0].p, sets[1].p, sets[2].p = 2, 1, 4
    # a set whose offsets start past 0 (a view into a larger code buffer)
    big = datagen.random_small(9, 3, 30, seed=99)
    view = types.SimpleNamespace(codes=big.codes, offsets=big.offsets[3:], p=3)
    sets.append(view)
    b = sad.Batch(sets, device="cpu")
    n = [5, 1, 12, 6]
    assert b.n.tolist() == n and b.p.tolist() == [2, 1, 4, 3] and b.n_sets == 4
    assert b.seq_begin.tolist() == [0, 5, 6, 18, 24]
    assert b.boff_begin.tolist() == [0, 3, 5, 10, 14]
    assert b.piv_begin.tolist() == [0, 1, 1, 4, 6]
    codes = np.concatenate([s.codes[s.offsets[0]:s.offsets[-1]] for s in sets])
    np.testing.assert_array_equal(b.codes.numpy(), codes)
    lens = np.concatenate([np.diff(s.offsets) for s in sets])
    np.testing.assert_array_equal(np.diff(b.offsets.numpy()), lens)
    assert b.offsets[0] == 0 and b.lengths.dtype == torch.int32
    np.testing.assert_array_equal(b.lengths.numpy(), lens)
    assert tuple(b.counts.shape) == (24, 8000)
    # per-set results are slices of the shared outputs
    b.key_hi.copy_(torch.arange(24, dtype=torch.int64).to(torch.uint64))
    b.members.copy_(torch.arange(24, dtype=torch.int32))
    b.bucket_offsets.copy_(torch.arange(14, dtype=torch.int32))
    b.pivot_idx.copy_(torch.arange(6, dtype=torch.int32))
    r = b.result(2)
    assert r["key_hi"].tolist() == list(range(6, 18))
    assert r["members"].tolist() == list(range(6, 18))
    assert r["bucket_offsets"].tolist() == [5, 6, 7, 8, 9]
    assert r["pivot_idx"].tolist() == [1, 2, 3]
    assert b.result(1)["pivot_idx"].tolist() == []
    with pytest.raises(RuntimeError, match="plan"):
        b.run()


def test_gemm_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    """The DRAM traffic in the roofline comes from a committed ncu capture and is
    reported only while the GEMM source is byte-identical to the captured one and
    the set size and plan shape (tile, depth, budget) match; otherwise it is null."""
    import hashlib

    import bench
    src = tmp_path / "paper_0905_1744_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "gemm.cu").write_bytes(b"// kernel v1\n")
    (tmp_path / "profiles").mkdir()
    sha = hashlib.sha256(b"// kernel v1\n").hexdigest()
    (tmp_path / "profiles" / "pair_gemm_traffic.json").write_text(json.dumps(
        {"gemm_cu_sha256": sha, "captures": [
            {"N": 20000, "tile": 256, "depth": 6, "budget": 0,
             "dram_bytes_read_per_launch": 100, "dram_bytes_write_per_launch": 23},
            {"N": 20000, "tile": 256, "depth": 6, "budget": 1536,
             "dram_bytes_read_per_launch": 200, "dram_bytes_write_per_launch": 1}]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.gemm_traffic_per_launch(20000, 256, 6, 0) == 123
    assert bench.gemm_traffic_per_launch(20000, 256, 6, 1536) == 201
    assert bench.gemm_traffic_per_launch(200, 256, 6, 0) is None
    assert bench.gemm_traffic_per_launch(20000, 128, 6, 0) is None
    assert bench.gemm_traffic_per_launch(20000, 256, 4, 0) is None
    (src / "gemm.cu").write_bytes(b"// kernel v2\n")
    assert bench.gemm_traffic_per_launch(20000, 256, 6, 0) is None


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """One JSON line with the main line's keys plus impl, cpu_baseline and e2e (the
    oracle's timing replaced by a stub here; its real run takes minutes)."""
    import bench
    monkeypatch.setattr(bench, "oracle_counts", lambda s: None)
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda s, sec, seed=0, counts=None: (2.0e6, 40, sec, 4))
    for var in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(var, raising=False)
    bench.run_reference(bench.parse(["--impl", "reference", "--config", "1", "--steps", "4",
                                     "--warmup", "3"]))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 4 and d["warmup"] == 3
    assert d["value"] == 2.0e6 and d["higher_is_better"] is True
    # a step is the timed sample itself (here the stub's 120 s / 7 samples), not an
    # extrapolation to the full set, so K steps fit in the run's wall time
    assert d["ms_per_step"] == pytest.approx(1e3 * 120.0 / 7)
    assert d["config"]["workload"] == bench.WORKLOADS[1] and d["config"]["N"] == 200
    # the GPU arm prints the same config dict for the same workload
    from paper_0905_1744_gb300 import datagen
    assert d["config"] == bench.bench_config(1, datagen.config(1, 0), 0)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 4 and cb["value"] == d["value"]
    assert "sample" in cb
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


# ------------------------------------------------------------- buffer pool ---

def test_batch_pool_hands_out_views_and_grows_by_doubling():
    from paper_0905_1744_gb300 import sad
    pool = sad.BatchPool("cpu")
    a = pool.get("x", 10, torch.int32)
    assert a.numel() == 10 and a.dtype == torch.int32
    base = pool.bufs["x"]
    # a smaller request is a view of the same buffer
    b = pool.get("x", 7, torch.int32)
    assert b.data_ptr() == base.data_ptr() and b.numel() == 7
    # a larger one at least doubles the buffer
    c = pool.get("x", 11, torch.int32)
    assert pool.bufs["x"].numel() >= 20 and c.numel() == 11
    # another dtype under the same name replaces the buffer
    d = pool.get("x", 5, torch.float64)
    assert d.dtype == torch.float64 and pool.bufs["x"].dtype == torch.float64
    # the three workspaces come with the pool
    assert len(pool.workspaces) == 3


# --------------------------------------------------------- batch autotuner ---

class _FakeBatch:
    """The parts of sad.Batch that choose_batch_shape touches."""

    def __init__(self):
        import numpy as np
        self.n_sets, self.n, self.total_len = 4, np.array([100, 200, 300, 400]), 500000
        self.device = torch.device("cpu")
        self.planned = []

    def plan(self, depth, tile, budget, stream=None):
        self.planned.append((tile, depth, budget))
        return types.SimpleNamespace(rank=types.SimpleNamespace(ws_bytes=depth * 10 + tile))

    def run(self, stream=None):
        pass

    def check(self, stream=None):
        pass


def test_choose_batch_shape_times_bound_plans_and_leaves_the_best_planned(monkeypatch):
    autotune._cache.clear()
    b = _FakeBatch()
    ms = {(256, 1): 5.0, (256, 2): 3.0, (256, 3): 4.0, (256, 4): 4.5, (256, 6): 6.0,
          (128, 1): 5.5, (128, 2): 2.5, (128, 3): 3.5, (128, 4): 4.0, (128, 6): 5.0}

    def events_ms(fn, stream, reps):
        tile, depth, budget = b.planned[-1]
        return ms[(tile, depth)] - (0.2 if budget == 1536 else 0.0)
    monkeypatch.setattr(autotune, "_events_ms", events_ms)
    monkeypatch.setattr(autotune.torch.cuda, "current_stream", lambda device=None: None)
    best, trials = autotune.choose_batch_shape(b, use_cache=False)
    # bound plans need cut planes: depth 0 is never tried
    assert all(autotune.Shape.parse(k).depth >= 1 for k in trials)
    assert best == autotune.Shape(128, 2, 1536)
    assert b.planned[-1] == (128, 2, 1536)          # left planned with the choice
    # the size class is cached: a second call answers without timing
    best2, trials2 = autotune.choose_batch_shape(b)
    assert best2 == best and trials2 == {} and b.planned[-1] == (128, 2, 1536)
    # a workspace limit drops the shapes that need more
    autotune._cache.clear()
    best3, trials3 = autotune.choose_batch_shape(b, use_cache=False, max_ws_bytes=160)
    assert all(10 * autotune.Shape.parse(k).depth + autotune.Shape.parse(k).tile <= 160
               for k in trials3)
    autotune._cache.clear()
