"""The remaining C-ABI calls on the GPU: the host-buffer sort, in-place reversal, sorting on a
caller stream, workspace errors, and the library's own launch counting and per-kernel timing."""

import numpy as np
import pytest
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, oracle_sorted, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
def test_sort_host_matches_oracle(dtype):
    n = 777_777
    a = workloads.uniform_bits(n, dtype, workloads.config_seed(90)) if dtype != np.float32 else \
        workloads.normal_f32_specials(n, workloads.config_seed(90))[0]
    h = torch.from_numpy(a.copy() if dtype == np.float32 else
                         a.view({4: np.int32, 8: np.int64}[a.dtype.itemsize]).copy()).pin_memory()
    d = torch.empty(n, dtype=h.dtype, device="cuda")
    ws = pdq.workspace_for(n, CODE[a.dtype])
    # the binding infers the code from the tensor dtype; unsigned keys need the explicit code
    st = pdq.Stats()
    rc = pdq.lib().pdq_sort_host(h.data_ptr(), None, 0, n, CODE[a.dtype], d.data_ptr(), None, ws.data_ptr(),
                                 ws.numel(), None, None, pdq.ctypes.byref(st))
    assert rc == 0, pdq.lib().pdq_last_error()
    got = h.numpy().view(a.dtype)
    want = a.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(got), bits(want))


def test_sort_host_pairs():
    n = 300_001
    k = workloads.uniform_bits(n, np.int32, workloads.config_seed(91)) % 5000
    hk = torch.from_numpy(k.copy()).pin_memory()
    hv = torch.arange(n, dtype=torch.int32).pin_memory()
    dk = torch.empty_like(hk, device="cuda")
    dv = torch.empty_like(hv, device="cuda")
    ws = pdq.workspace_for(n, torch.int32, 4)
    pdq.pdq_sort_host(hk, dk, ws, h_vals=hv, d_vals=dv)
    ko, vo = hk.numpy(), hv.numpy().astype(np.int64)
    ok, ov = k.copy(), np.arange(n, dtype=np.int32)
    oracle.pdqsort_pairs(ok, ov)
    assert np.array_equal(ko, ok)
    assert np.array_equal(k[vo], ko)


@pytest.mark.parametrize("elem", [np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 1000, 100_003])
def test_reverse(elem, n):
    a = (np.arange(n) * 7 + 3).astype(elem)
    t = torch.from_numpy(a.copy()).cuda()
    pdq.pdq_reverse(t)
    assert np.array_equal(t.cpu().numpy(), a[::-1])


def test_reverse_rejects_other_element_widths():
    t = torch.arange(100, dtype=torch.int16, device="cuda")
    with pytest.raises(pdq.PdqError) as ei:
        pdq.pdq_reverse(t)
    assert ei.value.status == -1


def test_sort_on_a_caller_stream():
    n = 1 << 20
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(92))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = torch.from_numpy(a.copy()).cuda(non_blocking=False)
        ws = pdq.workspace_for(n, torch.int32)
        pdq.pdq_sort_keys(d, ws, stream=s)
    s.synchronize()
    assert np.array_equal(d.cpu().numpy(), oracle_sorted(a))


def test_workspace_too_small_is_an_error():
    n = 1 << 20
    d = to_device(workloads.uniform_bits(n, np.int32, workloads.config_seed(93)))
    small = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pdq.PdqError) as ei:
        pdq.pdq_sort_keys(d, small)
    assert ei.value.status == -3


def test_launch_count_and_kernel_profile():
    n = 1 << 22
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(94))
    d = to_device(a)
    ws = pdq.workspace_for(n, torch.int32)
    l0 = pdq.launch_count()
    pdq.profile_reset()
    pdq.profile_enable(True)
    st = pdq.pdq_sort_keys(d, ws)
    torch.cuda.synchronize()
    prof = pdq.profile_read()
    pdq.profile_enable(False)
    assert pdq.launch_count() - l0 == st["kernel_launches"] > 0
    for k in ("count", "scatter", "base_sort"):
        assert k in prof and prof[k][0] > 0 and prof[k][1] >= 1
    # algorithmic bytes of the base pass: every key outside the equality buckets (a few splitter
    # values) read and written once
    assert prof["base_sort"][2] == pytest.approx(2 * 4 * n, rel=1e-2)
    assert np.array_equal(to_host(d, np.int32), oracle_sorted(a))


@pytest.mark.parametrize("with_vals", [False, True])
def test_sort_host_streams_ranges_of_a_two_level_sort(with_vals):
    """Large enough for a second distribution level and for position-grouped base lists (2^26
    keys and up): the host-buffer call copies each group's range out as soon as its base sorts
    are done, while later groups sort; the result equals the oracle."""
    n = (1 << 26) + 5
    k = workloads.uniform_bits(n, np.int32, workloads.config_seed(95))
    hk = torch.from_numpy(k.copy()).pin_memory()
    dk = torch.empty_like(hk, device="cuda")
    hv = dv = None
    if with_vals:
        hv = torch.arange(n, dtype=torch.int32).pin_memory()
        dv = torch.empty_like(hv, device="cuda")
    ws = pdq.workspace_for(n, torch.int32, 4 if with_vals else 0)
    st = pdq.pdq_sort_host(hk, dk, ws, h_vals=hv, d_vals=dv)
    assert st["passes"] >= 2
    assert np.array_equal(hk.numpy(), oracle_sorted(k))
    if with_vals:
        assert np.array_equal(k[hv.numpy().astype(np.int64)], hk.numpy())


@pytest.mark.parametrize("case", ["u64_pairs", "descending", "nearly_sorted"])
def test_sort_host_large_other_paths(case):
    """Host-buffer sorts of 2^26 + 3 elements through the other paths: 8-byte keys with 8-byte
    values (position-grouped streaming), the reversal exit and the nearly-sorted fix-up (whose
    result goes back in one piece at the end) — against the oracle."""
    n = (1 << 26) + 3
    if case == "u64_pairs":
        k = workloads.uniform_bits(n, np.uint64, workloads.config_seed(96))
        v = np.arange(n, dtype=np.uint64)
        hk = torch.from_numpy(k.view(np.int64).copy()).pin_memory()
        hv = torch.from_numpy(v.view(np.int64).copy()).pin_memory()
        dk, dv = torch.empty_like(hk, device="cuda"), torch.empty_like(hv, device="cuda")
        ws = pdq.workspace_for(n, torch.int64, 8)
        st = pdq.lib().pdq_sort_host(hk.data_ptr(), hv.data_ptr(), 8, n, pdq.PDQ_U64, dk.data_ptr(),
                                     dv.data_ptr(), ws.data_ptr(), ws.numel(), None, None, None)
        assert st == 0, pdq.lib().pdq_last_error()
        ok, ov = k.copy(), v.copy()
        oracle.pdqsort_pairs(ok, ov)
        got = hk.numpy().view(np.uint64)
        assert np.array_equal(got, ok)
        assert np.array_equal(k[hv.numpy().astype(np.int64)], got)
        return
    if case == "descending":
        k = (n - 1 - np.arange(n)).astype(np.int32)
    else:
        k = workloads.pattern("asc_swaps", n, workloads.config_seed(97), dtype=np.int32)
    hk = torch.from_numpy(k.copy()).pin_memory()
    dk = torch.empty_like(hk, device="cuda")
    st = pdq.pdq_sort_host(hk, dk, pdq.workspace_for(n, torch.int32))
    assert np.array_equal(hk.numpy(), oracle_sorted(k))
    if case == "descending":
        assert st["reversed"] == 1
    else:
        assert st["fixup_peeled"] > 0
