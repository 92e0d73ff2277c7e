"""Guard zones: every entry point writes only inside the arrays and the workspace it was given.
The key, value and workspace buffers are carved out of larger allocations whose margins hold a
known byte pattern; after each call the margins must be unchanged and the result exact."""

import numpy as np
import pytest
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, oracle_sorted

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes of margin on each side
PATTERN = 0xA5


def _guarded(nbytes: int):
    """(whole buffer, inner view start) with the margins filled; the inner region is 256-aligned."""
    whole = torch.full((nbytes + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
    return whole


def _margins_intact(whole: torch.Tensor, nbytes: int) -> bool:
    head = whole[:GUARD]
    tail = whole[GUARD + nbytes:]
    return bool((head == PATTERN).all().item()) and bool((tail == PATTERN).all().item())


def _put(whole: torch.Tensor, a: np.ndarray) -> torch.Tensor:
    """Copy a's bytes into the inner region and return a typed view of it."""
    raw = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8)).cuda()
    whole[GUARD:GUARD + raw.numel()].copy_(raw)
    return whole[GUARD:GUARD + raw.numel()]


@pytest.mark.parametrize("dtype,vdtype,n", [
    (np.int32, None, 1_000_003), (np.uint64, None, 777_777), (np.float32, np.uint32, 500_001),
    (np.int64, np.uint64, 300_007), (np.int32, None, 5_000)])
def test_plain_sort_stays_inside_its_buffers(dtype, vdtype, n):
    a = workloads.uniform_bits(n, dtype, workloads.config_seed(100)) if dtype != np.float32 else \
        workloads.normal_f32_specials(n, workloads.config_seed(100))[0]
    code = CODE[np.dtype(dtype)]
    kw = _guarded(a.nbytes)
    kin = _put(kw, a)
    vb = np.dtype(vdtype).itemsize if vdtype else 0
    if vdtype:
        v = np.arange(n).astype(vdtype)
        vw = _guarded(v.nbytes)
        vin = _put(vw, v)
    wsb = pdq.pdq_workspace_bytes(n, code, vb)
    ww = _guarded(wsb)
    ws = ww[GUARD:GUARD + wsb]
    st = pdq.Stats()
    L = pdq.lib()
    if vdtype:
        rc = L.pdq_sort_pairs(kin.data_ptr(), vin.data_ptr(), vb, n, code, ws.data_ptr(), wsb, None, None,
                              pdq.ctypes.byref(st))
    else:
        rc = L.pdq_sort_keys(kin.data_ptr(), n, code, ws.data_ptr(), wsb, None, None, pdq.ctypes.byref(st))
    torch.cuda.synchronize()
    assert rc == 0, L.pdq_last_error()
    assert _margins_intact(kw, a.nbytes) and _margins_intact(ww, wsb)
    got = kin.cpu().numpy().view(dtype)
    want = a.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(got), bits(want))
    if vdtype:
        assert _margins_intact(vw, v.nbytes)
        idx = vin.cpu().numpy().view(vdtype).astype(np.int64)
        assert np.array_equal(bits(a[idx]), bits(got))


@pytest.mark.parametrize("name", ["asc_swaps", "desc", "ones", "sawtooth"])
def test_exits_and_fixup_stay_inside_their_buffers(name):
    n = (1 << 20) + 5
    a = workloads.pattern(name, n, workloads.config_seed(101), dtype=np.int32)
    kw = _guarded(a.nbytes)
    kin = _put(kw, a)
    wsb = pdq.pdq_workspace_bytes(n, pdq.PDQ_I32, 0)
    ww = _guarded(wsb)
    ws = ww[GUARD:GUARD + wsb]
    rc = pdq.lib().pdq_sort_keys(kin.data_ptr(), n, pdq.PDQ_I32, ws.data_ptr(), wsb, None, None, None)
    torch.cuda.synchronize()
    assert rc == 0
    assert _margins_intact(kw, a.nbytes) and _margins_intact(ww, wsb)
    assert np.array_equal(kin.cpu().numpy().view(np.int32), oracle_sorted(a))


def test_segmented_sort_stays_inside_its_buffers():
    offs = workloads.segment_offsets(3000, workloads.config_seed(102), max_log2=15)
    n = int(offs[-1])
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(103))
    kw = _guarded(a.nbytes)
    kin = _put(kw, a)
    doff = torch.from_numpy(offs.astype(np.int64)).cuda()
    wsb = pdq.pdq_workspace_bytes(n, pdq.PDQ_I32, 0, offs.size - 1)
    ww = _guarded(wsb)
    ws = ww[GUARD:GUARD + wsb]
    rc = pdq.lib().pdq_sort_segmented(kin.data_ptr(), None, 0, doff.data_ptr(), offs.size - 1, n, pdq.PDQ_I32,
                                      ws.data_ptr(), wsb, None, None, None)
    torch.cuda.synchronize()
    assert rc == 0, pdq.lib().pdq_last_error()
    assert _margins_intact(kw, a.nbytes) and _margins_intact(ww, wsb)
    want = a.copy()
    oracle.pdqsort_segmented(want, offs)
    assert np.array_equal(kin.cpu().numpy().view(np.int32), want)


def test_learned_sort_stays_inside_its_buffers():
    n = 2_000_003
    a, _ = workloads.mixture_f32(n, workloads.config_seed(104))
    kw = _guarded(a.nbytes)
    kin = _put(kw, a)
    wsb = pdq.pdq_workspace_bytes_learned(n)
    ww = _guarded(wsb)
    ws = ww[GUARD:GUARD + wsb]
    rc = pdq.lib().pdq_sort_keys_learned(kin.data_ptr(), n, pdq.PDQ_F32, ws.data_ptr(), wsb, None, None, None)
    torch.cuda.synchronize()
    assert rc == 0, pdq.lib().pdq_last_error()
    assert _margins_intact(kw, a.nbytes) and _margins_intact(ww, wsb)
    want = a.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(kin.cpu().numpy().view(np.float32)), bits(want))
