"""Autotuner: picks a tuning per call shape on the GPU, records it, and later untuned calls of
that shape use it; results stay bit-exact against the oracle."""

import numpy as np
import pytest
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, gpu_sort, gpu_sort_segmented, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def fresh_table():
    pdq.pdq_autotune_reset()
    yield
    pdq.pdq_autotune_reset()


def test_plain_autotune_records_and_applies():
    n = 300_001
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(70))
    d = to_device(a)
    before = d.clone()
    best, ms = pdq.pdq_autotune(d, key_dtype=CODE[a.dtype])
    assert ms > 0
    assert torch.equal(d, before), "autotune must not modify its input"
    assert best["log2_buckets"] in (6, 7, 8, 9) and best["base_capacity"] in (4096, 8192, 16384)
    assert pdq.pdq_autotune_lookup(n, CODE[a.dtype]) == best
    # same shape class (ceil log2 n), different n: uses the record, still exact
    b = workloads.uniform_bits(280_000, np.int32, workloads.config_seed(71))
    k, _, _ = gpu_sort(b)
    exp = b.copy()
    oracle.pdqsort(exp)
    assert np.array_equal(bits(k), bits(exp))


def test_pairs_autotune_exact():
    n = 200_003
    k = workloads.uniform_bits(n, np.uint64, workloads.config_seed(72)) % np.uint64(1000)
    v = np.arange(n, dtype=np.uint32)
    dk, dv = to_device(k), to_device(v)
    best, _ = pdq.pdq_autotune(dk, vals=dv, key_dtype=CODE[k.dtype])
    assert pdq.pdq_autotune_lookup(n, CODE[k.dtype], 4) == best
    ko, vo, _ = gpu_sort(k, v)
    ok, ov = k.copy(), v.copy()
    oracle.pdqsort_pairs(ok, ov)
    assert np.array_equal(ko, ok)
    assert np.array_equal(k[vo.astype(np.int64)], ko)


def test_segmented_autotune_records_and_applies():
    nseg = 600
    offs = workloads.segment_offsets(nseg, workloads.config_seed(73), max_log2=14)
    n = int(offs[-1])
    keys = workloads.uniform_bits(n, np.int32, workloads.config_seed(74))
    dk = to_device(keys)
    doff = torch.from_numpy(offs.astype(np.int64)).cuda()
    best, ms = pdq.pdq_autotune(dk, offsets=doff, key_dtype=CODE[keys.dtype])
    assert best["seg_block"] in (256, 512) and 4 <= best["log2_buckets"] <= 8
    assert pdq.pdq_autotune_lookup(n, CODE[keys.dtype], 0, nseg) == best
    out, _, _, rc = gpu_sort_segmented(keys, offs)
    assert rc == 0
    exp = keys.copy()
    oracle.pdqsort_segmented(exp, offs)
    assert np.array_equal(bits(out), bits(exp))
