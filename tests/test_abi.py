"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/pdq.h
declares; host-side argument checks answer without a GPU (no compute calls here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdq.h")


@pytest.fixture(scope="module")
def L():
    from paper_2106_05123_gb300 import _build
    _build.build()
    import paper_2106_05123_gb300 as pdq
    return pdq.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdq_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("pdq_sort_keys", "pdq_sort_pairs", "pdq_sort_segmented", "pdq_workspace_bytes",
                 "pdq_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_workspace_bytes_is_host_logic(L):
    import paper_2106_05123_gb300 as pdq
    small = pdq.pdq_workspace_bytes(1000, pdq.PDQ_I32, 0)
    big = pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_I32, 0)
    pairs = pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_I32, 4)
    wide = pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_U64, 0)
    assert 0 < small < big < pairs and big < wide
    seg = pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_I32, 0, num_segments=20000)
    assert seg >= big                     # the segmented layout also covers the plain one
    assert big >= 4 * (1 << 20)          # at least the temp key buffer
    assert pdq.pdq_workspace_bytes(10, 7, 0) == 0       # unknown dtype
    # composite keys (two 4-byte fields) take the 8-byte layout
    for code in (pdq.PDQ_I32I32, pdq.PDQ_F32U32):
        for vb in (0, 4, 8):
            assert pdq.pdq_workspace_bytes(1 << 20, code, vb) == pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_U64, vb)
        assert (pdq.pdq_workspace_bytes(1 << 20, code, 0, num_segments=300)
                == pdq.pdq_workspace_bytes(1 << 20, pdq.PDQ_U64, 0, num_segments=300))
    assert pdq.pdq_workspace_bytes(10, pdq.PDQ_I32, 3) == 0
    # the temp key buffer plus every key's 2-byte bin slot of the current level
    assert big >= (4 + 2) * (1 << 20) and wide >= (8 + 2) * (1 << 20)


def test_noalloc_limit_fits_its_fixed_array(L):
    """pdq_sort_keys_noalloc promises every key type up to 2^20 keys inside its fixed 64 MiB
    device array: the keys-only workspace at that size must fit for every type."""
    import paper_2106_05123_gb300 as pdq
    for code in (pdq.PDQ_I32, pdq.PDQ_U32, pdq.PDQ_F32, pdq.PDQ_I64, pdq.PDQ_U64, pdq.PDQ_I32I32, pdq.PDQ_F32U32):
        assert 0 < pdq.pdq_workspace_bytes(1 << 20, code, 0) <= 64 << 20, code


def test_argument_errors_need_no_device(L):
    import paper_2106_05123_gb300 as pdq
    st = pdq.Stats()
    # unknown dtype, bad value width, n out of range, null pointers: rejected before any CUDA call
    assert L.pdq_sort_keys(None, 10, 9, None, 0, None, None, ctypes.byref(st)) == -2
    assert L.pdq_sort_pairs(None, None, 3, 10, 0, None, 0, None, None, ctypes.byref(st)) == -1
    assert L.pdq_sort_keys(None, 1 << 33, 0, None, 0, None, None, ctypes.byref(st)) == -1
    assert L.pdq_sort_keys(None, 10, 0, None, 0, None, None, ctypes.byref(st)) == -1
    assert b"keys" in L.pdq_last_error()
    # n = 0 / 1 are no-ops
    assert L.pdq_sort_keys(None, 0, 0, None, 0, None, None, ctypes.byref(st)) == 0
    assert L.pdq_sort_keys(None, 1, 0, None, 0, None, None, ctypes.byref(st)) == 0
    # misaligned workspace
    assert L.pdq_sort_keys(ctypes.c_void_p(4096), 10, 0, ctypes.c_void_p(4100), 1 << 20, None, None,
                           ctypes.byref(st)) == -3
    # bad tuning values
    bad = pdq.Tuning(log2_buckets=10)
    assert L.pdq_sort_keys(ctypes.c_void_p(4096), 10, 0, ctypes.c_void_p(4096), 1 << 20, None,
                           ctypes.byref(bad), ctypes.byref(st)) in (-1, -3)


def test_autotune_host_logic(L):
    # scratch = keys copy + values copy + sort workspace, each 256-byte aligned
    ws = L.pdq_workspace_bytes(1000, 0, 0, 4)
    sc = L.pdq_autotune_scratch_bytes(1000, 0, 0, 4)
    assert sc == 4096 + 4096 + ws
    assert L.pdq_autotune_scratch_bytes(1000, 0, 9, 0) == 0       # unknown dtype
    assert L.pdq_autotune_scratch_bytes(1000, 0, 0, 3) == 0       # bad value width
    assert L.pdq_autotune_scratch_bytes(1000, 7, 2, 0) >= 1000 * 8  # segmented
    L.pdq_autotune_reset()
    assert L.pdq_autotune_lookup(1000, 0, 0, 0, None) == 0
    # argument errors answer on the host, before any device work
    assert L.pdq_autotune(None, None, 0, None, 0, 1000, 0, None, 0, None, None, None) == -1
    assert L.pdq_autotune(None, None, 0, None, 0, 1000, 9, None, 0, None, None, None) == -2
    assert L.pdq_autotune(ctypes.c_void_p(256), None, 0, None, 0, 1000, 0, None, 0, None, None, None) == -3
    assert L.pdq_autotune(ctypes.c_void_p(256), None, 0, None, 5, 1000, 0, ctypes.c_void_p(256), 1 << 30,
                          None, None, None) == -1  # segmented without offsets
