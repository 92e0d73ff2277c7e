"""Parity at the full sizes of the measured configurations, in the launch configuration the
bench times (same inputs from bench.make_inputs, same entry points, autotuned where the bench
autotunes): every output is compared with the CPU oracle's element by element.  The oracle
sorts 2^28 keys in about 15 s on one host core, so these tests take a few minutes in total."""

import numpy as np
import pytest
import torch

import bench
import oracle
import paper_2106_05123_gb300 as pdq
from gpu_helpers import CODE, bits, to_device, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def fresh_tuning_table():
    pdq.pdq_autotune_reset()
    yield
    pdq.pdq_autotune_reset()
    torch.cuda.empty_cache()


def _oracle_sorted(a: np.ndarray) -> np.ndarray:
    b = a.copy()
    oracle.pdqsort(b)
    return b


@pytest.mark.parametrize("workload", ["uniform_i32_2p28", "uniform_i32_2p20", "sweep_i32_2p24"])
def test_fullsize_keys(workload):
    for keys, _ in bench.make_inputs(workload, 0):
        code = CODE[keys.dtype]
        d = to_device(keys)
        pdq.pdq_autotune(d, key_dtype=code)  # the bench's call shape: record, then sort untuned
        ws = torch.empty(pdq.pdq_workspace_bytes(keys.size, code, 0), dtype=torch.uint8, device="cuda")
        pdq.pdq_sort_keys(d, ws, key_dtype=code)
        torch.cuda.synchronize()
        got = to_host(d, keys.dtype)
        assert np.array_equal(bits(got), bits(_oracle_sorted(keys)))
        del d, ws


@pytest.mark.parametrize("workload", ["pairs_u64_zipf_2p27", "pairs_f32_normal_2p27"])
def test_fullsize_pairs(workload):
    (keys, vals), = bench.make_inputs(workload, 0)
    code = CODE[keys.dtype]
    dk, dv = to_device(keys), to_device(vals)
    pdq.pdq_autotune(dk, vals=dv, key_dtype=code)
    ws = torch.empty(pdq.pdq_workspace_bytes(keys.size, code, vals.dtype.itemsize), dtype=torch.uint8,
                     device="cuda")
    pdq.pdq_sort_pairs(dk, dv, ws, key_dtype=code)
    torch.cuda.synchronize()
    ko, vo = to_host(dk, keys.dtype), to_host(dv, vals.dtype)
    assert np.array_equal(bits(ko), bits(_oracle_sorted(keys)))
    # the payload is the original index: every pair of the input appears exactly once
    idx = vo.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(keys.size))
    assert np.array_equal(bits(keys[idx]), bits(ko))


@pytest.mark.parametrize("workload", ["segmented_i32_20k", "segmented_i64_20k"])
def test_fullsize_segmented(workload):
    offsets, n = bench.segment_layout()
    (keys, _), = bench.make_inputs(workload, 0)
    code = CODE[keys.dtype]
    dk = to_device(keys)
    doff = torch.from_numpy(offsets).cuda()
    pdq.pdq_autotune(dk, offsets=doff, key_dtype=code)
    ws = torch.empty(pdq.pdq_workspace_bytes(n, code, 0, offsets.size - 1), dtype=torch.uint8, device="cuda")
    pdq.pdq_sort_segmented(dk, doff, workspace=ws, key_dtype=code)
    torch.cuda.synchronize()
    got = to_host(dk, keys.dtype)
    want = keys.copy()
    oracle.pdqsort_segmented(want, offsets)
    assert np.array_equal(bits(got), bits(want))


def test_fullsize_learned_mixture():
    (keys, _), = bench.make_inputs("learned_f32_mixture_2p28", 0)
    d = to_device(keys)
    ws = torch.empty(pdq.pdq_workspace_bytes_learned(keys.size), dtype=torch.uint8, device="cuda")
    st = pdq.pdq_sort_keys_learned(d, ws)
    torch.cuda.synchronize()
    got = to_host(d, keys.dtype)
    assert np.array_equal(bits(got), bits(_oracle_sorted(keys)))
    assert st["learned_overflow"] >= 0
