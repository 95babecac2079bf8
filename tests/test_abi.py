"""The C-ABI library builds, loads, and exports every symbol include/sad.h declares.

CPU only: no compute call is made here (there may be no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sad.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0905_1744_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_three_calls():
    names = declared_functions()
    for f in ("kmer_count", "kmer_rank", "partition", "kmer_rank_plan", "kmer_rank_plan_bound",
              "sad_workspace_bytes",
              "sad_status_read", "sad_status_string", "sad_abi_version", "sad_launch_count"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_queries(lib):
    lib.sad_abi_version.restype = ctypes.c_int
    assert lib.sad_abi_version() == 7
    lib.sad_status_string.restype = ctypes.c_char_p
    lib.sad_status_string.argtypes = [ctypes.c_int]
    assert lib.sad_status_string(0) == b"ok"
    assert b"workspace" in lib.sad_status_string(2)
    ws = lib.sad_workspace_bytes
    ws.restype = ctypes.c_size_t
    ws.argtypes = [ctypes.c_int32] * 6
    assert ws(0, 100, 3, 20, 1, 1) == 256
    rank_fixed = ws(1, 20000, 3, 20, 1, 0)
    rank_d2 = ws(1, 20000, 3, 20, 1, 2)
    # planes at depth 2: 20096 stored rows x 16000 columns, two 4-bit values a byte
    assert rank_fixed > 0 and rank_d2 >= rank_fixed + 20096 * 16000 // 2
    assert ws(2, 1000, 3, 20, 16, 1) > 1000 * 48
    assert ws(2, 1000, 3, 20, 0, 1) == 0          # p < 1
    assert ws(1, 10, 9, 20, 1, 1) == 0            # k > 8 unsupported
    assert ws(1, 10, 4, 20, 1, 1) == 0            # eps = 160000 > 65536


def test_argument_errors_need_no_gpu(lib):
    """Host-side argument checks return before any CUDA call."""
    P = ctypes.c_void_p
    lib.partition.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, ctypes.c_size_t, P]
    assert lib.partition(None, None, 10, 0, None, None, None, None, 0, None) == 1
    assert lib.partition(None, None, 10, 11, None, None, None, None, 0, None) == 1
    lib.kmer_rank.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P,
                              P, P, ctypes.c_size_t, P]
    assert lib.kmer_rank(None, None, None, 10, 9, 20, None, None, None, None, None, 0, None) == 5
    assert lib.kmer_rank(None, None, None, -1, 3, 20, None, None, None, None, None, 0, None) == 1


class _Plan(ctypes.Structure):
    """sad_rank_plan as include/sad.h declares it (written out here, independently
    of the binding's copy)."""
    _fields_ = [("depth", ctypes.c_int32), ("budget", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("t_max", ctypes.c_int32),
                ("t_bits", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("k_eff", ctypes.c_int64), ("list_entries", ctypes.c_int64),
                ("rem_bound", ctypes.c_int64), ("heavy_entries", ctypes.c_int64),
                ("k_cap", ctypes.c_int64), ("list_cap", ctypes.c_int64),
                ("rem_cap", ctypes.c_int64), ("heavy_cap", ctypes.c_int64),
                ("bm_cols", ctypes.c_int64), ("ws_bytes", ctypes.c_size_t)]


def _bound(lib, n, total_len, depth, k=3, alphabet=20):
    f = lib.kmer_rank_plan_bound
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(_Plan)]
    f.restype = ctypes.c_int
    plan = _Plan(depth=depth)
    return f(n, total_len, k, alphabet, ctypes.byref(plan)), plan


def test_rank_plan_bound_is_host_only(lib):
    rc, plan = _bound(lib, 20000, 6_000_000, 1)
    w = 6_000_000 - 2 * 20000                            # windows
    assert rc == 0
    assert plan.k_cap == 8192                            # eps * 1 rounded up to 256
    assert plan.list_cap == w // 2
    assert plan.rem_cap == w - 20000
    assert plan.heavy_cap == w // 6                      # T_b = 1 + 4
    assert plan.bm_cols == 4 * 8000                      # sections 2..5, eps words each
    assert plan.ws_bytes > 20096 * 8192 // 2 + plan.bm_cols * 20096 // 8
    assert plan.k_eff == -1 and plan.t_max == -1 and plan.t_bits == -1
    assert _bound(lib, 20000, 6_000_000, 2)[1].k_cap == 16128       # 16000 rounded up
    assert _bound(lib, 20000, 6_000_000, 12)[1].k_cap == 64000      # at most 8 sections
    small = _bound(lib, 10, 1000, 1)[1]                  # few windows bound the bitmap
    assert small.bm_cols == sum(min(8000, 980 // t) for t in range(2, 6))
    assert _bound(lib, 10, 100, 0)[0] == 1               # all planes need the word maxima
    assert _bound(lib, -1, 100, 1)[0] == 1
    assert _bound(lib, 10, 100, 1, k=9)[0] == 5
    # the tile list packs row-block ids in 15 bits: at most 32767 blocks of 128 rows
    assert _bound(lib, 32767 * 128, 300 * 32767 * 128, 1)[0] == 0
    assert _bound(lib, 32767 * 128 + 1, 300 * (32767 * 128 + 1), 1)[0] == 5


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_rank_plan_bound_holds_for_the_data(lib, oracle_mod, depth):
    """The capacities bound what the data need (counted here from the oracle's
    counts): K_eff = sum_tau min(T_tau, D), the entries counted twice or more, the
    remainder entries sum of min(c, T_b) - 1 over them, the counts above T_b and
    the bitmap columns sum_{t=2..T_b} #{tau : T_tau >= t}; on sets with long
    repeats and on a family set."""
    import numpy as np
    from paper_0905_1744_gb300 import datagen
    sets = [datagen.from_strings(["A" * 3000, "AC" * 900, "ACD" * 400, "W" * 5, "ACDEFGHIK"]),
            datagen.random_small(300, 3, 2500, seed=11, alphabet=4),
            datagen.family_set(6, 40, lambda r: int(r.integers(40, 900)), p=4, seed=3,
                               stream=9)]
    for s in sets:
        alphabet = int(s.codes.max()) + 1 if s.codes.size else 20
        alphabet = 4 if alphabet <= 4 else 20
        c = oracle_mod.kmer_count(s.codes, s.offsets, 3, alphabet)
        rc, plan = _bound(lib, s.n, int(s.codes.size), depth, 3, alphabet)
        assert rc == 0
        tb = min(depth + 4, 16)
        assert np.minimum(c.max(axis=0), depth).sum() <= plan.k_cap
        assert int((c >= 2).sum()) <= plan.list_cap
        assert int((np.minimum(c, tb) - 1)[c >= 2].sum()) <= plan.rem_cap
        assert int((c > tb).sum()) <= plan.heavy_cap
        T = c.max(axis=0)
        assert sum(int((T >= t).sum()) for t in range(2, tb + 1)) <= plan.bm_cols


def test_every_kernel_waits_for_its_predecessor_first():
    """Kernels are launched with programmatic stream serialization: each must wait
    (pdl_enter, griddepcontrol.wait) before it touches memory, so its first
    statement is pdl_enter()."""
    src_dir = os.path.join(ROOT, "paper_0905_1744_gb300", "csrc")
    found = 0
    for name in sorted(os.listdir(src_dir)):
        if not name.endswith(".cu"):
            continue
        text = open(os.path.join(src_dir, name)).read()
        for m in re.finditer(r"__global__", text):
            # the kernel's parameter list, then its body
            i = text.index("(", text.index("(", m.end()) + 1) if "__launch_bounds__" in \
                text[m.end():text.index("(", m.end()) + 1] else text.index("(", m.end())
            depth, j = 0, i
            while True:
                if text[j] == "(":
                    depth += 1
                elif text[j] == ")":
                    depth -= 1
                    if depth == 0:
                        break
                j += 1
            k = text.index("{", j)
            if ";" in text[j:k]:
                continue  # a declaration
            body = text[k + 1:k + 400].lstrip()
            assert body.startswith("pdl_enter();"), (name, text[m.start():k][:120])
            found += 1
    assert found >= 40


def test_every_entry_point_checks_its_arguments_on_the_host():
    """Each compute entry point rejects bad sizes, missing buffers, unsupported
    k/alphabet and undersized workspaces before it touches the device (through the
    binding's own prototypes). A fake, 256-aligned, never-dereferenced address
    stands in for device buffers where a call needs one to reach its next check."""
    from paper_0905_1744_gb300 import sad
    L = sad.lib()
    OK, INV, WS, UNS = sad.OK, sad.ERR_INVALID_ARGUMENT, sad.ERR_WORKSPACE, sad.ERR_UNSUPPORTED
    d = 1 << 20                              # fake device address, aligned, never used
    byref = ctypes.byref
    # kmer_count
    assert L.kmer_count(None, None, -1, 3, 20, None, None, d, 4096, None) == INV
    assert L.kmer_count(None, None, 5, 9, 20, None, None, d, 4096, None) == UNS
    assert L.kmer_count(None, None, 5, 3, 20, None, None, None, 4096, None) == INV
    assert L.kmer_count(None, None, 5, 3, 20, None, None, d + 8, 4096, None) == INV  # unaligned
    assert L.kmer_count(None, None, 5, 3, 20, None, None, d, 0, None) == INV
    assert L.kmer_count(None, None, 5, 3, 20, None, None, d, 4096, None) == INV      # no codes
    assert L.kmer_count(d, d + 4, 5, 3, 20, d, None, d, 4096, None) == INV           # offsets
    assert L.kmer_count(None, None, 0, 3, 20, None, None, d, 4096, None) == OK       # empty set
    # kmer_rank_plan: the fixed part of the workspace is reported when it is too small
    plan = sad.RankPlan(depth=1)
    assert L.kmer_rank_plan(None, 10, 9, 20, byref(plan), d, 0, None) == UNS
    assert L.kmer_rank_plan(None, 10, 3, 20, None, d, 0, None) == INV
    assert L.kmer_rank_plan(None, -1, 3, 20, byref(plan), d, 0, None) == INV
    assert L.kmer_rank_plan(None, 10, 3, 20, byref(sad.RankPlan(depth=-1)), d, 0, None) == INV
    assert L.kmer_rank_plan(None, 10, 3, 20, byref(plan), d, 0, None) == WS
    assert plan.ws_bytes > 0
    # kmer_rank: a plan's capacities are checked, then the workspace against them
    good = sad.RankPlan(depth=1, k_cap=8192, list_cap=0, rem_cap=0)
    args = (d, d, None, 300, 3, 20)
    outs = (d, d, None)
    assert L.kmer_rank(*args, byref(good), *outs, d, 0, None) == WS
    assert L.kmer_rank(*args, None, *outs, d, 0, None) == WS
    assert L.kmer_rank(*args, byref(sad.RankPlan(depth=1, k_cap=100)), *outs, d, 1 << 30,
                       None) == INV
    assert L.kmer_rank(*args, byref(sad.RankPlan(depth=1, k_cap=8192, list_cap=-1)), *outs, d,
                       1 << 30, None) == INV
    assert L.kmer_rank(None, d, None, 300, 3, 20, byref(good), *outs, d, 1 << 30, None) == INV
    assert L.kmer_rank(d, d, None, 300, 3, 20, byref(good), None, d, None, d, 1 << 30,
                       None) == INV
    assert L.kmer_rank(None, None, None, 0, 3, 20, None, None, None, None, d, 0, None) == OK
    # partition and the allocation-free partition
    assert L.partition(d, d, 10, 65, d, d, None, d, 1 << 20, None) == INV   # p above 64
    assert L.partition(d, d, 10, 4, None, d, None, d, 1 << 20, None) == INV
    assert L.partition(d, d, 10, 4, d, d, None, d, 0, None) == WS
    assert L.partition_noalloc(d, d, 10, 0, d, d, None, None) == INV
    assert L.partition_noalloc(d, d, 10, 11, d, d, None, None) == INV
    assert L.partition_noalloc(d, d, 40000, 4, d, d, None, None) == UNS
    assert L.partition_noalloc(d, d, 10, 4, None, d, None, None) == INV
    # globalised rank: local samples, then every sequence against the references
    assert L.sad_local_samples_workspace_bytes(10, 11) == 0
    assert L.sad_local_samples(d, d, 10, 11, 2, d, d, 1 << 20, None) == INV
    assert L.sad_local_samples(d, d, 10, 2, 0, d, d, 1 << 20, None) == INV
    assert L.sad_local_samples(d, d, 10, 2, 2, None, d, 1 << 20, None) == INV
    full = sad.RankPlan(depth=0, k_cap=8192)
    assert L.kmer_rank_vs_workspace_bytes(byref(sad.RankPlan(depth=0, k_cap=0)), 10, 3, 20, 4,
                                          0) == 0
    assert L.kmer_rank_vs_workspace_bytes(byref(full), 10, 3, 20, 4, 0) > 0
    vs = lambda plan, n_ref=4, delta=0: L.kmer_rank_vs(  # noqa: E731
        d, d, None, 10, 3, 20, d, n_ref, delta, plan, None, d, d, None, d, 1 << 30, None)
    assert vs(byref(sad.RankPlan(depth=1, k_cap=8192))) == INV      # needs every plane
    assert vs(byref(sad.RankPlan(depth=0, k_cap=8000))) == INV      # k_cap not 256-aligned
    assert vs(byref(full), n_ref=0) == INV
    assert vs(byref(full), delta=1025) == INV
    assert vs(None) == INV
    # distance form
    assert L.kmer_rank_dist_workspace_bytes(byref(good), 10, 3, 20, 0) == 0
    assert L.kmer_rank_dist_workspace_bytes(byref(good), 10, 3, 20, 10) > 0
    dist = lambda plan, delta=10, ws=1 << 30: L.kmer_rank_dist(  # noqa: E731
        d, d, None, 10, 3, 20, delta, plan, None, d, d, None, d, ws, None)
    assert dist(byref(good), delta=0) == INV
    assert dist(byref(sad.RankPlan(depth=1, k_cap=8192, rem_cap=-1))) == INV
    assert dist(byref(sad.RankPlan(depth=1, k_cap=8192, budget=-1))) == INV
    assert dist(byref(good), ws=0) == WS
    assert L.sad_ln_q(None, -1, None, None) == INV
    assert L.sad_ln_q(None, 5, None, None) == INV
    # sparse ablation
    n_entries = ctypes.c_int64(0)
    assert L.kmer_rank_sparse_workspace_bytes(0, 5) == 0
    assert L.kmer_rank_sparse_workspace_bytes(10, -1) == 0
    assert L.kmer_rank_sparse_entries(d, d, 0, 3, 20, byref(n_entries), d, 1 << 20, None) == INV
    assert L.kmer_rank_sparse_entries(d, d, 10, 3, 20, None, d, 1 << 20, None) == INV
    assert L.kmer_rank_sparse_entries(d, d, 10, 9, 20, byref(n_entries), d, 1 << 20,
                                      None) == UNS
    assert L.kmer_rank_sparse(d, d, 10, 3, 20, -1, d, d, None, d, 1 << 20, None) == INV
    assert L.kmer_rank_sparse(d, d, 10, 3, 20, 5, d, None, None, d, 1 << 20, None) == INV
    # batched forms
    bp = sad.BatchPlan()
    n_arr = (ctypes.c_int32 * 2)(10, 20)
    p_arr = (ctypes.c_int32 * 2)(2, 25)                  # the second set has p > N
    assert L.sad_batch_plan_make(d, n_arr, p_arr, d, 0, 3, 20, byref(bp), d, 1 << 20,
                                 None) == INV
    assert L.sad_batch_plan_make(d, n_arr, p_arr, d, 2, 3, 20, byref(bp), d, 1 << 20,
                                 None) == INV
    assert L.sad_batch_plan_make(d, n_arr, p_arr, d, 2, 3, 20, None, d, 1 << 20, None) == INV
    assert L.sad_batch_rank(d, d, None, d, 3, 20, byref(bp), d, d, None, d, 1 << 20,
                            None) == INV                   # n_sets = 0
    bp.n_sets, bp.part_ws_bytes = 2, 1 << 20
    assert L.sad_batch_partition(d, d, d, d, byref(bp), d, d, None, d, 1024, None) == WS
    assert L.sad_batch_partition(d, d, d, None, byref(bp), d, d, None, d, 1 << 20, None) == INV
    # status and info reads
    info = (ctypes.c_int64 * 9)()
    assert L.sad_rank_info(None, info, None) == INV
    assert L.sad_status_read(None, 0, None) == INV
