"""Pins for the oracle's composite keys (records of two 4-byte fields, ordered lexicographically:
the "small tuples" that a branchless comparison sort handles, Sec. 5.3).

What fixes the result: lexicographic order over two strict weak orders is the first field's order,
with ties (equivalent first fields) broken by the second field's order.  The first field of
TUPLE_F32U32 is a float32 under IEEE 754-2008 totalOrder, pinned by the golden list of bit patterns
in tests/golden/float32_total_order.txt.  Checks: brute force against Python's own sort on tuples,
the golden float order combined with second-field ties, the independent merge sort, and values
riding with their records.
"""

import itertools
import os

import numpy as np
import pytest

import oracle
import workloads

I32I32 = oracle.TUPLE_I32I32
F32U32 = oracle.TUPLE_F32U32


def golden_float_words():
    words = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "float32_total_order.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                words.append(int(line, 16))
    return words


def records(dt, pairs):
    a = np.zeros(len(pairs), dtype=dt)
    for i, (x, y) in enumerate(pairs):
        a[i] = (x, y)
    return a


def test_generator_dtypes_are_the_oracle_records():
    assert workloads.COMPOSITE_DTYPES["i32i32"] == I32I32
    assert workloads.COMPOSITE_DTYPES["f32u32"] == F32U32


@pytest.mark.parametrize("n", range(1, 7))
def test_exhaustive_small_i32i32(n):
    # every arrangement of a multiset with equal first fields and equal records
    base = [(1, 5), (0, 7), (1, -3), (0, 7), (-2, 0), (1, 5)][:n]
    want = sorted(base)
    for perm in set(itertools.permutations(base)):
        a = records(I32I32, perm)
        oracle.pdqsort(a)
        assert [tuple(int(v) for v in r) for r in a] == want


@pytest.mark.parametrize("n", [0, 1, 2, 24, 25, 1000, 20011])
@pytest.mark.parametrize("distinct", [0, 3, 50])
def test_random_i32i32_vs_python_sort(n, distinct):
    a = workloads.composite_keys("i32i32", n, workloads.substream(31, n), distinct)
    want = sorted((int(x), int(y)) for x, y in zip(a["first"], a["second"]))
    oracle.pdqsort(a)
    assert [(int(x), int(y)) for x, y in zip(a["first"], a["second"])] == want


def test_f32u32_golden_total_order_with_ties():
    # each golden float (ascending totalOrder) paired with seconds 2, 0, 1, 0: the sorted result
    # lists the floats in golden order, each with its seconds ascending
    words = golden_float_words()
    seconds = [2, 0, 1, 0]
    recs = [(w, s) for w in words for s in seconds]
    perm = workloads.permutation(len(recs), 5)
    a = np.zeros(len(recs), dtype=F32U32)
    a["first"] = np.array([recs[i][0] for i in perm], dtype=np.uint32).view(np.float32)
    a["second"] = np.array([recs[i][1] for i in perm], dtype=np.uint32)
    oracle.pdqsort(a)
    got = list(zip(a["first"].view(np.uint32).tolist(), a["second"].tolist()))
    assert got == [(w, s) for w in words for s in sorted(seconds)]


@pytest.mark.parametrize("kind", ["i32i32", "f32u32"])
@pytest.mark.parametrize("n", [1, 2, 3, 100, 65537])
@pytest.mark.parametrize("distinct", [0, 4])
def test_composite_agrees_with_independent_mergesort(kind, n, distinct):
    a = workloads.composite_keys(kind, n, workloads.substream(41, n), distinct)
    b = a.copy()
    oracle.pdqsort(a)
    oracle.mergesort_check(b)
    assert a.tobytes() == b.tobytes()


@pytest.mark.parametrize("kind", ["i32i32", "f32u32"])
def test_composite_pairs_values_ride_along(kind):
    n = 30011
    keys = workloads.composite_keys(kind, n, 8, first_distinct=20)
    keys["second"] = keys["second"] % 7  # many equal records
    vals = np.arange(n, dtype=np.uint32)
    k, v = keys.copy(), vals.copy()
    oracle.pdqsort_pairs(k, v)
    s = keys.copy()
    oracle.pdqsort(s)
    assert k.tobytes() == s.tobytes()
    assert np.array_equal(np.sort(v), vals)
    assert keys[v.astype(np.int64)].tobytes() == k.tobytes()


@pytest.mark.parametrize("kind", ["i32i32", "f32u32"])
def test_composite_segmented_is_per_segment(kind):
    a = workloads.composite_keys(kind, 5000, 12, first_distinct=9)
    offs = np.array([0, 0, 1, 17, 1000, 1000, 4999, 5000], dtype=np.int64)
    got = a.copy()
    oracle.pdqsort_segmented(got, offs)
    for s in range(offs.size - 1):
        seg = a[offs[s]:offs[s + 1]].copy()
        oracle.mergesort_check(seg)
        assert got[offs[s]:offs[s + 1]].tobytes() == seg.tobytes()
