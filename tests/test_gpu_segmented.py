"""The batched segmented sort (one persistent launch over size-binned device queues, replayed
from a CUDA graph) against the oracle, segment by segment, bit for bit."""

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import bits, gpu_sort_segmented

pytestmark = pytest.mark.gpu


def oracle_segmented(keys, offsets):
    k = keys.copy()
    oracle.pdqsort_segmented(k, offsets)
    return k


def lengths_to_offsets(lens):
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lens, dtype=np.int64), out=off[1:])
    return off


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.int64, np.uint64, np.float32])
def test_log_uniform_segments(dtype):
    offsets = workloads.segment_offsets(600, 21, max_log2=16)
    n = int(offsets[-1])
    if dtype == np.float32:
        keys, _ = workloads.normal_f32_specials(n, 5, frac=0.01)
    else:
        keys = workloads.uniform_bits(n, dtype, 5)
    got, _, st, _ = gpu_sort_segmented(keys, offsets)
    assert np.array_equal(bits(got), bits(oracle_segmented(keys, offsets)))


@pytest.mark.parametrize("lens", [
    [0], [1], [0, 0, 0], [1, 0, 1, 2], [5, 0, 70000, 1, 0, 3],   # empty and one-key segments
    [8192, 8193, 16384, 16385],                                  # around the base capacity
    [1 << 20], [(1 << 20) + 3, 10],                              # one large segment, above the limit
    [7] * 3000,                                                  # many tiny segments
])
def test_edge_case_segments(lens):
    offsets = lengths_to_offsets(lens)
    n = int(offsets[-1])
    keys = workloads.uniform_bits(n, np.int32, 8)
    got, _, _, _ = gpu_sort_segmented(keys, offsets)
    assert np.array_equal(got, oracle_segmented(keys, offsets))


@pytest.mark.parametrize("pattern", ["mod8", "ones", "desc", "dupsq", "sawtooth"])
def test_patterns_in_segments(pattern):
    offsets = workloads.segment_offsets(300, 3, max_log2=16)
    n = int(offsets[-1])
    keys = workloads.pattern(pattern, n, 4, dtype=np.int32)
    got, _, st, _ = gpu_sort_segmented(keys, offsets)
    assert np.array_equal(got, oracle_segmented(keys, offsets))


@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
def test_segmented_pairs(vdtype):
    offsets = workloads.segment_offsets(400, 9, max_log2=16)
    n = int(offsets[-1])
    keys = (workloads.splitmix64(2, n) % np.uint64(5000)).astype(np.int64)
    vals = np.arange(n, dtype=vdtype)
    gk, gv, _, _ = gpu_sort_segmented(keys, offsets, vals)
    assert np.array_equal(gk, oracle_segmented(keys, offsets))
    idx = gv.astype(np.int64)
    assert np.array_equal(keys[idx], gk)
    # every value stays inside its own segment
    seg_of = np.repeat(np.arange(offsets.size - 1), np.diff(offsets))
    assert np.array_equal(seg_of[idx], seg_of)
    assert np.array_equal(np.sort(idx), np.arange(n))


@pytest.mark.parametrize("tuning", [dict(seg_block=256), dict(log2_buckets=2, oversample=2),
                                    dict(bad_allowed=-1), dict(bad_allowed=1, log2_buckets=1, oversample=1)])
def test_segmented_knobs(tuning):
    offsets = workloads.segment_offsets(200, 13, max_log2=17)
    n = int(offsets[-1])
    keys = workloads.pattern("dupsq", n, 6, dtype=np.int32)
    got, _, st, _ = gpu_sort_segmented(keys, offsets, tuning=tuning)
    assert np.array_equal(got, oracle_segmented(keys, offsets))
    if tuning.get("bad_allowed") == -1:
        assert st["fallback_buckets"] >= 1


def test_graph_replay_is_repeatable():
    """The same call shape replays the cached graph: identical results twice in a row."""
    import torch
    import paper_2106_05123_gb300 as pdq
    offsets = workloads.segment_offsets(500, 17, max_log2=16)
    n = int(offsets[-1])
    keys = workloads.uniform_bits(n, np.int32, 17)
    dk = torch.from_numpy(keys.copy()).cuda()
    doff = torch.from_numpy(offsets).cuda()
    ws = pdq.workspace_for(n, torch.int32, 0, offsets.size - 1)
    want = oracle_segmented(keys, offsets)
    for _ in range(3):
        dk.copy_(torch.from_numpy(keys))
        st = pdq.pdq_sort_segmented(dk, doff, workspace=ws)
        torch.cuda.synchronize()
        assert np.array_equal(dk.cpu().numpy(), want)
        assert st["kernel_launches"] >= 1


def test_bad_offsets_are_rejected():
    keys = workloads.uniform_bits(100, np.int32, 1)
    offsets = np.array([0, 60, 40, 100], dtype=np.int64)  # decreasing
    _, _, _, rc = gpu_sort_segmented(keys, offsets, raise_on_error=False)
    assert rc == -1


def test_bounded_wait_times_out_and_keeps_a_permutation():
    """Fault injection without a GPU fault: one CTA waits on a flag nothing sets, with a 1 ms
    bound; the call reports PDQ_ERR_TIMEOUT, the context stays usable, and the arrays still
    hold a permutation of each segment's input (salvage mode moves data home)."""
    offsets = workloads.segment_offsets(300, 23, max_log2=16)
    n = int(offsets[-1])
    keys = workloads.uniform_bits(n, np.int32, 23)
    got, _, _, rc = gpu_sort_segmented(keys, offsets, tuning=dict(inject_wait=1, wait_limit_us=1000),
                                       raise_on_error=False)
    assert rc == -5
    for s in range(offsets.size - 1):
        a, b = offsets[s], offsets[s + 1]
        assert np.array_equal(np.sort(got[a:b]), np.sort(keys[a:b]))
    # the context is still usable: a normal call afterwards succeeds
    got2, _, _, rc2 = gpu_sort_segmented(keys, offsets)
    assert rc2 == 0 and np.array_equal(got2, oracle_segmented(keys, offsets))
