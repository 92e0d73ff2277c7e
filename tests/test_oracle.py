"""Pins for the CPU oracle (Peters, arXiv 2106.05123) against facts fixed outside the oracle.

* exact results: exhaustive permutations (n <= 8) and exhaustive multisets (n <= 6) at the
  default and at tiny thresholds, random arrays against numpy's sort and against an
  independent merge sort, multiset histograms, key/value attachment;
* float32 order: a golden list written from IEEE 754-2008 totalOrder (clause 5.10);
* behaviour the paper proves or claims, through comparison counts: linear time on ascending,
  descending and ascending-plus-one-appended inputs (Sec. 5.2), O(nk) for k distinct values
  (Theorem 1), about 2n comparisons on all-equal input (Sec. 3), n log n on random input,
  and O(n log n) with the heapsort fallback under McIlroy's adversary (Sec. 4.1, Theorem 2);
* the constants: the bad-partition cut p = 1/8 computed by a shift (Sec. 4.1) and the counter
  start floor(log2 n); the closed form 1/H(p) the paper uses to justify p (Sec. 4.1).
"""

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY = dict(insertion_threshold=2, ninther_threshold=5, partial_limit=1)
DTYPES = [np.int32, np.uint32, np.int64, np.uint64, np.float32]


def _segmented_sort_all(rows: np.ndarray, params) -> np.ndarray:
    """Sort every row of a 2-D array with the oracle in one call (rows are segments)."""
    flat = np.ascontiguousarray(rows).reshape(-1).copy()
    m, n = rows.shape
    offsets = np.arange(0, (m + 1) * n, n, dtype=np.int64)
    oracle.pdqsort_segmented(flat, offsets, params)
    return flat.reshape(m, n)


@pytest.mark.parametrize("n", range(1, 9))
@pytest.mark.parametrize("knobs", [None, TINY], ids=["default", "tiny"])
def test_exhaustive_permutations(n, knobs):
    params = oracle.make_params(**knobs) if knobs else oracle.default_params()
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int32).reshape(-1, n)
    out = _segmented_sort_all(perms, params)
    assert (out == np.arange(n, dtype=np.int32)).all()


@pytest.mark.parametrize("n", range(1, 7))
@pytest.mark.parametrize("knobs", [None, TINY, dict(insertion_threshold=3, ninther_threshold=3,
                                                     partial_limit=0)], ids=["default", "tiny", "tiny2"])
def test_exhaustive_multisets(n, knobs):
    """Every sequence over {0..n-1}^n: duplicates exercise partition_left and equal pivots."""
    params = oracle.make_params(**knobs) if knobs else oracle.default_params()
    seqs = np.array(list(itertools.product(range(n), repeat=n)), dtype=np.int64).reshape(-1, n)
    out = _segmented_sort_all(seqs, params)
    assert (out == np.sort(seqs, axis=1)).all()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [0, 1, 2, 23, 24, 25, 128, 129, 1000, 65537])
def test_random_vs_numpy_and_mergesort(dtype, n):
    rng_seed = workloads.substream(12345, n)
    a = workloads.uniform_bits(n, dtype, rng_seed)
    if dtype == np.float32:
        # numeric-only floats: totalOrder coincides with numeric order here (no NaN, no -0)
        a = workloads.uniform01(rng_seed, n).astype(np.float32) * 2 - 1
        a[a == 0] = 0.5
    b = a.copy()
    oracle.pdqsort(b)
    assert np.array_equal(b, np.sort(a, kind="stable"))
    c = a.copy()
    oracle.mergesort_check(c)
    assert np.array_equal(b.view(np.uint8), c.view(np.uint8))


@pytest.mark.parametrize("dtype", DTYPES)
def test_few_distinct_multiset(dtype):
    n = 50000
    a = (workloads.splitmix64(7, n) % np.uint64(37)).astype(dtype)
    b = a.copy()
    oracle.pdqsort(b, oracle.make_params(**TINY))
    assert (np.diff(b.astype(np.float64)) >= 0).all()
    ua, ca = np.unique(a, return_counts=True)
    ub, cb = np.unique(b, return_counts=True)
    assert np.array_equal(ua, ub) and np.array_equal(ca, cb)


def _golden_f32() -> np.ndarray:
    words = []
    with open(os.path.join(GOLDEN, "float32_total_order.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                words.append(int(line, 16))
    return np.array(words, dtype=np.uint32)


@pytest.mark.parametrize("seed", range(5))
def test_float_total_order_golden(seed):
    want = _golden_f32()
    a = want[workloads.permutation(want.size, seed)].view(np.float32).copy()
    oracle.pdqsort(a)
    assert np.array_equal(a.view(np.uint32), want)
    b = want[workloads.permutation(want.size, seed)].view(np.float32).copy()
    oracle.mergesort_check(b)
    assert np.array_equal(b.view(np.uint32), want)


def test_float_specials_large_agree_with_mergesort():
    keys, _ = workloads.normal_f32_specials(200000, 99, frac=0.01)
    a = keys.copy()
    oracle.pdqsort(a)
    b = keys.copy()
    oracle.mergesort_check(b)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # the golden order's class boundaries hold in the big array too
    bits = a.view(np.uint32)
    neg_nan = (bits & 0x7FFFFFFF) > 0x7F800000
    pos = bits >> 31 == 0
    assert not (neg_nan & ~pos)[np.argmax(pos):].any()  # no negative datum after a positive one


@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("kdtype", DTYPES)
def test_pairs_values_stay_attached(kdtype, vdtype):
    n = 30000
    keys = (workloads.splitmix64(5, n) % np.uint64(1000)).astype(kdtype)  # many ties
    vals = np.arange(n, dtype=vdtype)
    k, v = keys.copy(), vals.copy()
    oracle.pdqsort_pairs(k, v)
    assert np.array_equal(k, np.sort(keys))
    assert np.array_equal(np.sort(v), vals)           # values are a permutation
    assert np.array_equal(keys[v.astype(np.int64)], k)  # each value still sits with its key


# ----------------------------------------------------------------------------- complexity pins
def _comps_per_n(name, sizes, dtype=np.int64):
    out = []
    for n in sizes:
        if name == "asc_append":  # ascending with one arbitrary element appended (Sec. 5.2)
            a = np.concatenate([np.arange(n - 1), [n // 3]]).astype(dtype)
        else:
            a = workloads.pattern(name, n, 3, dtype=dtype)
        st = oracle.pdqsort(a)
        assert (np.diff(a) >= 0).all()
        out.append(st["comparisons"] / n)
    return np.array(out)


SIZES = [1 << 10, 1 << 13, 1 << 16, 1 << 19]


@pytest.mark.parametrize("name", ["asc", "desc", "asc_append"])
def test_linear_on_sorted_patterns(name):
    """Sec. 5.2: ascending, descending and ascending-plus-one-appended sort in linear time."""
    c = _comps_per_n(name, SIZES)
    assert c.max() < 6.0
    assert c.max() / c.min() < 1.2


def test_all_equal_two_passes():
    """Sec. 3: all-equal input costs one partition_right then one partition_left (~2n)."""
    for n in SIZES:
        a = np.ones(n, dtype=np.int64)
        st = oracle.pdqsort(a)
        assert st["comparisons"] <= 2 * n + 64
        assert st["partition_left_calls"] == 1 and st["heapsort_calls"] == 0


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_theorem1_few_distinct_linear(k):
    """Theorem 1: O(nk) for k distinct values: comparisons per element stay bounded as n grows
    512-fold (an n log n sort would grow by 19/10 over these sizes)."""
    c = _comps_per_n(f"mod{k}", SIZES)
    assert c.max() / c.min() < 1.5
    assert c.max() < 2.0 * k + 4


def test_random_is_n_log_n():
    vals = []
    for n in SIZES:
        a = workloads.pattern("uniform", n, 11, dtype=np.int64)
        st = oracle.pdqsort(a)
        vals.append(st["comparisons"] / (n * math.log2(n)))
    vals = np.array(vals)
    assert 0.8 < vals.min() and vals.max() < 1.5
    assert vals.max() / vals.min() < 1.2


@pytest.mark.parametrize("lg", [10, 12, 14])
def test_theorem2_killer_adversary(lg):
    """Theorem 2 / Sec. 4.1: against McIlroy's adversary the oracle stays O(n log n): exactly
    floor(log2 n) bad partitions along the degenerate path, then the heapsort fallback."""
    n = 1 << lg
    values, st = oracle.killer_adversary(n)
    assert st["heapsort_calls"] >= 1
    assert st["bad_partitions"] >= lg
    assert st["comparisons"] < 4.0 * n * lg
    # the concrete input replays the same run (the sort is deterministic)
    a = values.copy()
    st2 = oracle.pdqsort(a)
    assert st2 == st
    assert np.array_equal(a, np.arange(n))


def test_bad_partition_counter_prevents_quadratic():
    """Without the counter (a huge start value) the same adversary forces Theta(n^2) comparisons:
    quadrupling n multiplies them by about 16, against about 4.8 with the counter."""
    counts = []
    for n in (1 << 10, 1 << 12):
        _, st = oracle.killer_adversary(n, oracle.make_params(bad_allowed_override=10 * n))
        assert st["heapsort_calls"] == 0
        assert st["comparisons"] > n * n / 16
        counts.append(st["comparisons"])
    assert counts[1] / counts[0] > 12


@pytest.mark.parametrize("rank,bad", [(124, True), (125, False), (874, False), (875, True)])
def test_bad_partition_cut_is_one_eighth(rank, bad):
    """Sec. 4.1: a partition is bad when a side is smaller than size/8 (a shift: 1000 >> 3 = 125).
    Median of 3 over (first, middle, last) = (0, rank, 999) puts exactly `rank` elements left;
    a large insertion threshold stops the sort after that single partition."""
    n = 1000
    rest = [v for v in range(n) if v not in (0, rank, n - 1)]
    a = np.empty(n, dtype=np.int64)
    a[0], a[n // 2], a[n - 1] = 0, rank, n - 1
    a[[i for i in range(n) if i not in (0, n // 2, n - 1)]] = rest
    st = oracle.pdqsort(a, oracle.make_params(insertion_threshold=900, ninther_threshold=10 ** 9))
    assert np.array_equal(a, np.arange(n))
    assert st["partition_right_calls"] == 1
    assert st["bad_partitions"] == (1 if bad else 0)


def test_counter_starts_at_floor_log2():
    """Sec. 4.1: the counter starts at log n; with the start forced to 0 the sort is heapsort."""
    a = workloads.pattern("uniform", 5000, 1, dtype=np.int64)
    st = oracle.pdqsort(a, oracle.make_params(bad_allowed_override=0))
    assert st["heapsort_calls"] == 1 and st["partition_right_calls"] == 0
    assert np.array_equal(a, np.arange(5000))
    n = 3000  # floor(log2 3000) = 11: the adversary sees 11 bad partitions on the degenerate path
    _, st = oracle.killer_adversary(n)
    assert st["bad_partitions"] == 11 and st["heapsort_calls"] >= 1


def _inv_entropy(p):
    return 1.0 / (-p * math.log2(p) - (1 - p) * math.log2(1 - p))


def test_entropy_closed_form_constants():
    """Sec. 4.1: the slowdown of an always-p split is 1/H(p); an 80/20 split is ~40% slower and
    p = 1/8 is close to the 2x that makes a bad partition about as slow as heapsort."""
    assert abs(_inv_entropy(0.2) - 1.3852) < 1e-4
    assert abs(_inv_entropy(0.125) - 1.8397) < 1e-4
    assert abs(_inv_entropy(0.5) - 1.0) < 1e-12


def test_partial_insertion_sort_gives_up():
    """Sec. 5.2: a swapless partition whose parts are far from sorted (a misdiagnosed best
    case) costs at most about n extra work, because the partial insertion sort gives up after a
    few corrections.  Two descending halves partition without swaps around the middle."""
    n = 1 << 14
    h = n // 2
    a = np.concatenate([np.arange(h)[::-1], np.arange(h, n)[::-1]]).astype(np.int64)
    st = oracle.pdqsort(a)
    assert np.array_equal(a, np.arange(n))
    assert st["comparisons"] < 1.5 * n * 14


@pytest.mark.parametrize("name", ["organ", "merge", "interleave", "two_desc"])
def test_fresh_candidates_defeat_patterns(name):
    """Sec. 4.2 / Sec. 6.2: after a bad partition fresh pivot candidates break self-similar
    patterns, so organ pipe, merge-of-two-runs and similar inputs stay close to random-input
    cost and never reach the heapsort fallback."""
    for lg in (14, 16):
        n = 1 << lg
        h = n // 2
        if name == "interleave":
            a = np.concatenate([np.arange(0, n, 2), np.arange(1, n, 2)])
        elif name == "two_desc":
            a = np.concatenate([np.arange(h)[::-1], np.arange(h, n)[::-1]])
        else:
            a = workloads.pattern(name, n, 1, dtype=np.int64)
        a = a.astype(np.int64)
        st = oracle.pdqsort(a)
        assert (np.diff(a) >= 0).all()
        assert st["heapsort_calls"] == 0
        assert st["comparisons"] < 1.6 * n * lg
