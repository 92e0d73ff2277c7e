"""The allocation-free entry point pdq_sort_keys_noalloc, through the C ABI.

It exists for callers that cannot call cudaMalloc (frameworks that own all device memory,
fixed-budget plug-ins, loops where an allocation would synchronise the device): it takes only
the keys and keeps its scratch in the library's fixed 64 MiB device array.  Its output must
equal the oracle's and pdq_sort_keys' (which uses a fresh caller workspace) on calls in a row,
since the array keeps the previous call's contents.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, oracle_sorted, to_device, to_host

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20


def _noalloc(dk, code):
    L = pdq.lib()
    st = pdq.Stats()
    rc = L.pdq_sort_keys_noalloc(ctypes.c_void_p(dk.data_ptr()), dk.numel(), code,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                 ctypes.byref(st))
    return rc, st.as_dict()


def _with_workspace(dk, code):
    L = pdq.lib()
    n = dk.numel()
    ws = torch.empty(max(256, pdq.pdq_workspace_bytes(n, code, 0)), dtype=torch.uint8, device="cuda")
    st = pdq.Stats()
    rc = L.pdq_sort_keys(ctypes.c_void_p(dk.data_ptr()), n, code, ctypes.c_void_p(ws.data_ptr()),
                         ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), None,
                         ctypes.byref(st))
    return rc


def _check_one(a: np.ndarray):
    """One no-alloc call on `a`: bit-identical to the oracle and to pdq_sort_keys."""
    code = CODE[a.dtype]
    d_ref = to_device(a)
    assert _with_workspace(d_ref, code) == 0
    d_new = to_device(a)
    rc, st = _noalloc(d_new, code)
    assert rc == 0, pdq.lib().pdq_last_error()
    torch.cuda.synchronize()
    got = bits(to_host(d_new, a.dtype))
    assert np.array_equal(got, bits(oracle_sorted(a)))
    assert np.array_equal(got, bits(to_host(d_ref, a.dtype)))
    return st


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64])
def test_noalloc_matches_oracle_and_workspace_entry_point_twice(dtype):
    for call, n in enumerate([MAX_KEYS, 300007]):  # two calls in a row share the scratch array
        if dtype == np.float32:
            a, _ = workloads.normal_f32_specials(n, 40 + call, frac=0.01)
        else:
            a = workloads.uniform_bits(n, dtype, 40 + call)
        _check_one(a)


def test_noalloc_back_to_back_through_every_scratch_region():
    """Calls in a row whose inputs reach the regions most likely to be read stale: the
    nearly-sorted fix-up (marks, tile counts, the peeled keys' own workspace), the reverse exit,
    equality buckets and the fallback lists."""
    n = 1 << 18
    nearly = workloads.pattern("asc_swaps", n, workloads.config_seed(120), dtype=np.int32)
    st = _check_one(nearly)
    assert st["fixup_peeled"] > 0
    desc = np.arange(n, dtype=np.int32)[::-1].copy()
    st = _check_one(desc)
    assert st["reversed"] == 1
    few = workloads.pattern("mod16", n, workloads.config_seed(121), dtype=np.int32)
    st = _check_one(few)
    assert st["equal_buckets"] >= 16
    st = _check_one(nearly)  # the fix-up once more, after the regions held other data
    assert st["fixup_peeled"] > 0
    _check_one(workloads.uniform_bits(n, np.int32, workloads.config_seed(122)))


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
def test_noalloc_limit_is_exact(dtype):
    # 2^20 keys of any type fit the array; one more key is rejected with the limit in the message
    a = workloads.uniform_bits(MAX_KEYS, dtype, 45)
    _check_one(a)
    d = torch.zeros(MAX_KEYS + 1, dtype=torch.int32 if np.dtype(dtype).itemsize == 4 else torch.int64,
                    device="cuda")
    rc, _ = _noalloc(d, CODE[np.dtype(dtype)])
    assert rc == -1
    assert b"2^20" in pdq.lib().pdq_last_error()
