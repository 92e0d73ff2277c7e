"""The speculative first level of small arrays, through the C ABI, against the oracle.

For arrays of 2^17 .. 2^22 keys the sampled sortedness probe (Sec. 5.2) and the whole first
distribution level are queued back to back and one read-back serves both.  The level is kept
when the probe asks for the ordinary sort, and dropped when it asks for the sorted exit, the
reversal or the nearly-sorted fix-up; either way the result must equal the oracle's.  These
tests check both outcomes (by the stats each exit leaves), the size limits on either side, the
hand-over of a kept level's further work (second-level tasks, fallback buckets), and calls in a
row that reuse the pinned upload staging.
"""

import numpy as np
import pytest
import torch

import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import CODE, bits, gpu_sort, oracle_sorted

pytestmark = pytest.mark.gpu

SPEC_MIN, SPEC_MAX = 1 << 17, 1 << 22


@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
def test_kept_level_matches_oracle(dtype):
    n = (1 << 21) + 5
    if dtype == np.float32:
        a, _ = workloads.normal_f32_specials(n, workloads.config_seed(130), frac=0.01)
    else:
        a = workloads.uniform_bits(n, dtype, workloads.config_seed(130))
    got, _, st = gpu_sort(a)
    assert np.array_equal(bits(got), bits(oracle_sorted(a)))
    assert st["sorted_exit"] == 0 and st["reversed"] == 0 and st["fixup_peeled"] == 0
    assert st["passes"] >= 1


def test_kept_level_pairs():
    n = (1 << 20) + 3
    k = workloads.uniform_bits(n, np.uint64, workloads.config_seed(131))
    v = np.arange(n, dtype=np.uint32)
    gk, gv, _ = gpu_sort(k, v)
    want = oracle_sorted(k)
    assert np.array_equal(gk, want)
    assert np.array_equal(k[gv], gk)                     # every value sits with its own key
    assert np.array_equal(np.sort(gv), v)                # each exactly once


@pytest.mark.parametrize("name,stat", [("asc", "sorted_exit"), ("desc", "reversed"), ("asc_swaps", "fixup_peeled")])
def test_dropped_level_takes_the_probe_exit(name, stat):
    n = 1 << 21
    a = workloads.pattern(name, n, workloads.config_seed(132), dtype=np.int32)
    got, _, st = gpu_sort(a)
    assert np.array_equal(got, oracle_sorted(a))
    assert st[stat] > 0
    if name != "asc_swaps":
        assert st["passes"] == 0


@pytest.mark.parametrize("n", [SPEC_MIN - 1, SPEC_MIN, SPEC_MIN + 1, SPEC_MAX - 1, SPEC_MAX, SPEC_MAX + 1])
def test_size_limits(n):
    a = workloads.uniform_bits(n, np.int32, workloads.substream(133, n))
    got, _, st = gpu_sort(a)
    assert np.array_equal(got, oracle_sorted(a))
    assert st["passes"] >= 1


def test_kept_level_hands_over_a_second_level():
    """A base capacity of 4096 keys: every first-level bucket of 2^22 keys (at most 512 of
    them) is above it, so the kept level must pass all of them on to a second level."""
    n = SPEC_MAX
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(134))
    got, _, st = gpu_sort(a, tuning=dict(base_capacity=4096))
    assert np.array_equal(got, oracle_sorted(a))
    assert st["passes"] >= 2


def test_kept_level_with_two_way_splits_and_an_early_fallback():
    """Two buckets a level, one-key samples and a budget of one bad split: the kept level hands
    over next-level tasks (and whatever fallback buckets the samples cause) to the loop."""
    n = (1 << 20) + 11
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(136))
    got, _, st = gpu_sort(a, tuning=dict(bad_allowed=1, log2_buckets=1, oversample=1, base_capacity=256))
    assert np.array_equal(got, oracle_sorted(a))
    assert st["passes"] > 1


def test_calls_in_a_row_reuse_the_staging():
    cases = [((1 << 21) + 1, np.int32), ((1 << 18) + 7, np.uint64), (SPEC_MAX, np.float32),
             (SPEC_MIN + 3, np.int32), ((1 << 23) + 9, np.int32), ((1 << 20) - 1, np.uint64)]
    for i, (n, dt) in enumerate(cases):
        if dt == np.float32:
            a, _ = workloads.normal_f32_specials(n, workloads.config_seed(140 + i), frac=0.01)
        else:
            a = workloads.uniform_bits(n, dt, workloads.config_seed(140 + i))
        got, _, _ = gpu_sort(a)
        assert np.array_equal(bits(got), bits(oracle_sorted(a))), (n, dt)


def test_host_buffer_call_with_a_kept_level():
    n = (1 << 21) + 13
    a = workloads.uniform_bits(n, np.int32, workloads.config_seed(137))
    h = torch.from_numpy(a.copy()).pin_memory()
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = pdq.workspace_for(n, CODE[a.dtype])
    st = pdq.Stats()
    rc = pdq.lib().pdq_sort_host(h.data_ptr(), None, 0, n, CODE[a.dtype], d.data_ptr(), None, ws.data_ptr(),
                                 ws.numel(), None, None, pdq.ctypes.byref(st))
    assert rc == 0, pdq.lib().pdq_last_error()
    assert np.array_equal(h.numpy(), oracle_sorted(a))
    assert st.as_dict()["passes"] >= 1
