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
    for f in ("kmer_count", "kmer_rank", "partition", "kmer_rank_plan", "sad_workspace_bytes",
              "sad_status_read", "sad_status_string", "sad_abi_version", "sad_launch_count"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_queries(lib):
    lib.sad_abi_version.restype = ctypes.c_int
    assert lib.sad_abi_version() == 3
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
