"""Composite keys on the CUDA path (records of two 4-byte fields ordered lexicographically, the
"small tuples" of Sec. 5.3), bit for bit against the CPU oracle: keys only, key/value pairs (values
inside a run of equal records are unordered: each value must sit with its own record, once) and
the segmented call."""

import numpy as np
import pytest
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import gpu_sort, gpu_sort_segmented

pytestmark = pytest.mark.gpu

KINDS = ["i32i32", "f32u32"]


def oracle_sorted(a):
    b = a.copy()
    oracle.pdqsort(b)
    return b


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [0, 1, 2, 33, 8193, 65537, 300001, (1 << 20) + 17])
@pytest.mark.parametrize("distinct", [0, 6, 5000])
def test_composite_keys(kind, n, distinct):
    a = workloads.composite_keys(kind, n, workloads.substream(51, n), distinct)
    got, _, _ = gpu_sort(a)
    assert got.tobytes() == oracle_sorted(a).tobytes()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name", ["asc", "desc", "asc_swaps", "organ"])
def test_composite_presorted_patterns(kind, name):
    # records already (nearly) in order: the probe's exits and the fix-up on composite codes
    n = 1 << 18
    a = oracle_sorted(workloads.composite_keys(kind, n, 61, first_distinct=300))
    order = workloads.pattern(name, n, 3, dtype=np.int64)  # indices in 0..n-1 (organ repeats some)
    a = a[order]
    got, _, _ = gpu_sort(a)
    assert got.tobytes() == oracle_sorted(a).tobytes()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("n", [5, 8193, 200001])
def test_composite_pairs(kind, vdtype, n):
    keys = workloads.composite_keys(kind, n, 71, first_distinct=40)
    keys["second"] = keys["second"] % 5  # many equal records
    vals = np.arange(n, dtype=vdtype)
    gk, gv, _ = gpu_sort(keys, vals)
    assert gk.tobytes() == oracle_sorted(keys).tobytes()
    idx = gv.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))
    assert keys[idx].tobytes() == gk.tobytes()


@pytest.mark.parametrize("kind", KINDS)
def test_composite_segmented(kind):
    offs = workloads.segment_offsets(300, 13, max_log2=14)
    n = int(offs[-1])
    a = workloads.composite_keys(kind, n, 81, first_distinct=100)
    got, _, _, _ = gpu_sort_segmented(a, offs)
    want = a.copy()
    oracle.pdqsort_segmented(want, offs)
    assert got.tobytes() == want.tobytes()


def test_composite_view_and_width_check():
    f = torch.tensor([[3, 1], [1, 9], [3, 0], [-2, 5]], dtype=torch.int32, device="cuda")
    k = pdq.composite_keys(f)
    assert k.dtype == torch.int64 and k.shape == (4,)
    pdq.pdq_sort_keys(k, key_dtype=pdq.PDQ_I32I32)
    assert f.cpu().tolist() == [[-2, 5], [1, 9], [3, 0], [3, 1]]
    with pytest.raises(pdq.PdqError):
        pdq.pdq_sort_keys(torch.zeros(8, dtype=torch.int32, device="cuda"), key_dtype=pdq.PDQ_I32I32)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [1000, 4097, 100003])
def test_composite_records_holding_the_sentinel_value(kind, n):
    # the largest record of each order (both fields at their maximum) is the base sort's sentinel
    a = workloads.composite_keys(kind, n, 91, first_distinct=50)
    pos = (workloads.splitmix64(5, n // 20 + 1) % np.uint64(n)).astype(np.int64)
    if kind == "i32i32":
        a["first"][pos] = np.iinfo(np.int32).max
        a["second"][pos] = np.iinfo(np.int32).max
    else:
        a["first"].view(np.uint32)[pos] = np.uint32(0x7FFFFFFF)
        a["second"][pos] = np.iinfo(np.uint32).max
    got, _, _ = gpu_sort(a)
    assert got.tobytes() == oracle_sorted(a).tobytes()
    vals = np.arange(n, dtype=np.uint32)
    gk, gv, _ = gpu_sort(a, vals)
    assert gk.tobytes() == oracle_sorted(a).tobytes()
    idx = gv.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))
    assert a[idx].tobytes() == gk.tobytes()
