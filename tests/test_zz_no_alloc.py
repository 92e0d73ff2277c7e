"""The allocation-free entry point pdq_sort_keys_noalloc, through the C ABI.

It exists for callers that cannot call cudaMalloc (frameworks that own all device memory,
fixed-budget plug-ins, loops where an allocation would synchronise the device): it takes only
the keys and keeps its scratch in the library's fixed 64 MiB device array.  Its output must be
bit-identical to pdq_sort_keys (which uses a caller workspace) on two calls in a row, since the
array keeps the previous call's contents.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, to_device, to_host

pytestmark = pytest.mark.gpu


def _noalloc(dk, code):
    L = pdq.lib()
    st = pdq.Stats()
    rc = L.pdq_sort_keys_noalloc(ctypes.c_void_p(dk.data_ptr()), dk.numel(), code,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                 ctypes.byref(st))
    return rc, st


def _with_workspace(dk, code):
    L = pdq.lib()
    n = dk.numel()
    ws = torch.empty(max(256, pdq.pdq_workspace_bytes(n, code, 0)), dtype=torch.uint8, device="cuda")
    st = pdq.Stats()
    rc = L.pdq_sort_keys(ctypes.c_void_p(dk.data_ptr()), n, code, ctypes.c_void_p(ws.data_ptr()),
                         ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), None,
                         ctypes.byref(st))
    return rc


@pytest.mark.parametrize("dtype", [np.int32, np.float32, np.uint64])
def test_noalloc_matches_workspace_entry_point_twice(dtype):
    code = CODE[np.dtype(dtype)]
    for call, n in enumerate([(1 << 20), 300007]):  # two calls in a row share the scratch array
        if dtype == np.float32:
            a, _ = workloads.normal_f32_specials(n, 40 + call, frac=0.01)
        else:
            a = workloads.uniform_bits(n, dtype, 40 + call)
        d_ref = to_device(a)
        assert _with_workspace(d_ref, code) == 0
        d_new = to_device(a)
        rc, _ = _noalloc(d_new, code)
        assert rc == 0, pdq.lib().pdq_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(bits(to_host(d_new, dtype)), bits(to_host(d_ref, dtype)))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # up to 2^20 keys of any type are guaranteed to fit; 2^24 four-byte keys cannot (their
    # temporary key buffer alone is 64 MiB)
    n = 1 << 24
    d = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc, _ = _noalloc(d, pdq.PDQ_I32)
    assert rc == -1
    assert b"2^20" in pdq.lib().pdq_last_error()
