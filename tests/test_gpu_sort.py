"""Parity of the CUDA path (through the C ABI) with the CPU oracle, bit for bit.

Keys must equal the oracle's output exactly (the sorted arrangement is unique under numeric
order and IEEE totalOrder).  For pairs, several outputs are correct (values inside a run of
equal keys are unordered, Sec. 1): keys must match exactly and every value must sit with its
own key, each exactly once.
"""

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import bits, gpu_sort, oracle_sorted

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.int64, np.uint64, np.float32]
SIZES = [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 8191, 8192, 8193, 8194, 65537, 300001]




def keys_for(dtype, n, seed):
    if dtype == np.float32:
        k, _ = workloads.normal_f32_specials(n, seed, frac=0.01)
        return k
    return workloads.uniform_bits(n, dtype, seed)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", SIZES)
def test_keys_random(dtype, n):
    a = keys_for(dtype, n, workloads.substream(1, n))
    got, _, _ = gpu_sort(a)
    assert np.array_equal(bits(got), bits(oracle_sorted(a)))


@pytest.mark.parametrize("name", workloads.SWEEP_PATTERNS + ["dupsq", "dup8", "mod8", "sort50",
                                                             "sort90", "sort99", "merge", "random"])
@pytest.mark.parametrize("n", [1 << 14, 100003, 1 << 20])
def test_patterns_int32(name, n):
    a = workloads.pattern(name, n, 7, dtype=np.int32)
    got, _, st = gpu_sort(a)
    assert np.array_equal(got, oracle_sorted(a))


TUNINGS = [
    dict(log2_buckets=1, base_capacity=256),                # two-way splits: many levels
    dict(log2_buckets=2, oversample=1, base_capacity=256),  # poor samples: bad splits likely
    dict(log2_buckets=3, base_capacity=512),
    dict(log2_buckets=9, base_capacity=256),                # widest level
    dict(bad_allowed=-1, base_capacity=256),                # counter starts at 0: fallback only
    dict(bad_allowed=1, log2_buckets=1, oversample=1, base_capacity=256),  # early fallback
    dict(probe=-1),
]


@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(i) for i in range(len(TUNINGS))])
@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
@pytest.mark.parametrize("name", ["random", "mod8", "organ", "dupsq", "sawtooth"])
def test_knobs_force_rare_paths(tuning, dtype, name):
    n = 40000
    if name == "random":
        a = keys_for(dtype, n, 5)
    else:
        a = workloads.pattern(name, n, 5, dtype=np.int64).astype(dtype)
    got, _, st = gpu_sort(a, tuning=tuning)
    assert np.array_equal(bits(got), bits(oracle_sorted(a)))
    if tuning.get("bad_allowed") == -1:
        assert st["fallback_buckets"] >= 1


@pytest.mark.parametrize("vdtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("kdtype", DTYPES)
@pytest.mark.parametrize("n", [5, 8193, 200001])
def test_pairs_values_stay_attached(kdtype, vdtype, n):
    if kdtype == np.float32:
        keys, _ = workloads.normal_f32_specials(n, 3, frac=0.01)
    else:
        keys = (workloads.splitmix64(3, n) % np.uint64(997)).astype(kdtype)  # many ties
    vals = np.arange(n, dtype=vdtype)
    gk, gv, _ = gpu_sort(keys, vals)
    ok, ov = keys.copy(), vals.copy()
    oracle.pdqsort_pairs(ok, ov)
    assert np.array_equal(bits(gk), bits(ok))
    idx = gv.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))          # a permutation of the values
    assert np.array_equal(bits(keys[idx]), bits(gk))           # each value with its own key


@pytest.mark.parametrize("tuning", [None, dict(bad_allowed=-1, base_capacity=256),
                                    dict(log2_buckets=1, base_capacity=256)])
def test_pairs_through_fallback_and_levels(tuning):
    n = 100000
    keys = workloads.pattern("dupsq", n, 9, dtype=np.int32)
    vals = np.arange(n, dtype=np.uint32)
    gk, gv, _ = gpu_sort(keys, vals, tuning=tuning)
    ok, ov = keys.copy(), vals.copy()
    oracle.pdqsort_pairs(ok, ov)
    assert np.array_equal(gk, ok)
    assert np.array_equal(keys[gv.astype(np.int64)], gk)
    assert np.array_equal(np.sort(gv), vals)


def test_float_golden_total_order():
    import os
    words = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "float32_total_order.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                words.append(int(line, 16))
    want = np.array(words, dtype=np.uint32)
    big = np.tile(want, 2000)[workloads.permutation(want.size * 2000, 4)]
    got, _, _ = gpu_sort(big.view(np.float32).copy())
    assert np.array_equal(bits(got), np.repeat(want, 2000))


# ------------------------------------------------------------------- heuristics (stats)
def test_sorted_exit_and_reverse():
    n = 1 << 20
    asc = np.arange(n, dtype=np.int32)
    got, _, st = gpu_sort(asc)
    assert np.array_equal(got, asc) and st["sorted_exit"] == 1 and st["passes"] == 0
    desc = asc[::-1].copy()
    got, _, st = gpu_sort(desc)
    assert np.array_equal(got, asc) and st["reversed"] == 1 and st["passes"] == 0
    ones = np.ones(n, dtype=np.int32)
    got, _, st = gpu_sort(ones)
    assert st["sorted_exit"] == 1 and st["passes"] == 0
    # non-increasing with equal runs is reversed too (unstable order is allowed)
    steps = (np.arange(n)[::-1] // 7).astype(np.int32)
    got, _, st = gpu_sort(steps)
    assert np.array_equal(got, oracle_sorted(steps)) and st["reversed"] == 1


def test_equal_keys_are_final_after_one_level():
    """The equal-key rule (Sec. 3): with k = 16 distinct keys every key lands in an equality
    bucket on the first level, so one distribution pass finishes the sort (O(nk), Theorem 1)."""
    n = 1 << 20
    a = workloads.pattern("mod16", n, 2, dtype=np.int32)
    got, _, st = gpu_sort(a)
    assert np.array_equal(got, oracle_sorted(a))
    assert st["passes"] == 1 and st["equal_buckets"] == 16 and st["base_buckets"] == 0


@pytest.mark.parametrize("k", [2, 3, 5, 40])
def test_few_distinct_passes_bounded(k):
    n = 300000
    a = (workloads.splitmix64(11, n) % np.uint64(k)).astype(np.int64) * 1000003
    got, _, st = gpu_sort(a, tuning=dict(log2_buckets=1, base_capacity=256))
    assert np.array_equal(got, oracle_sorted(a))
    assert st["passes"] <= k


def test_fallback_when_budget_is_zero():
    n = 50000
    a = workloads.pattern("random", n, 8, dtype=np.int32)
    got, _, st = gpu_sort(a, tuning=dict(bad_allowed=-1, base_capacity=256))
    assert np.array_equal(got, oracle_sorted(a))
    assert st["fallback_buckets"] == 1 and st["passes"] == 0


@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
@pytest.mark.parametrize("lo,hi", [(1, 0), (3, -2), (2, -1), (5, -7)])
def test_misaligned_subarrays(dtype, lo, hi):
    """Sorting a slice that starts off a 16-byte boundary: only the slice changes, bit-exact."""
    import torch
    import paper_2106_05123_gb300 as pdq
    from gpu_helpers import CODE, to_device, to_host
    n = 200003
    a = keys_for(dtype, n, 77)
    d = to_device(a)
    end = n + hi if hi else n
    sub = d[lo:end]
    pdq.pdq_sort_keys(sub, key_dtype=CODE[np.dtype(dtype)])
    torch.cuda.synchronize()
    got = to_host(d, dtype)
    want = a.copy()
    want[lo:end] = oracle_sorted(a[lo:end])
    assert np.array_equal(bits(got), bits(want))
    # pairs: keys and values sliced at the same element offset
    if dtype != np.float32:
        v = np.arange(n, dtype=np.uint32 if np.dtype(dtype).itemsize == 4 else np.uint64)
        dk, dv = to_device(a), to_device(v)
        pdq.pdq_sort_pairs(dk[lo:end], dv[lo:end], key_dtype=CODE[np.dtype(dtype)])
        torch.cuda.synchronize()
        gk, gv = to_host(dk, dtype), to_host(dv, v.dtype).astype(np.int64)
        assert np.array_equal(bits(gk), bits(want))
        assert np.array_equal(a[gv], gk) and np.array_equal(gv[:lo], np.arange(lo))


# ---------------------------------------------------------------- nearly-sorted fix-up
FIXUP = {"fixup": 1}

@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.int64, np.uint64, np.float32])
@pytest.mark.parametrize("n", [1 << 16, (1 << 20) + 17, 3_000_001])
def test_nearly_sorted_fixup_exact(dtype, n):
    """Ascending with 1% random transpositions: the probe sees few descents, the fix-up peels,
    sorts and merges them; the keys match the oracle."""
    a = workloads.pattern("asc_swaps", n, workloads.config_seed(80), dtype=np.int64)
    a = (a - n // 2).astype(dtype) if dtype in (np.int32, np.int64, np.float32) else a.astype(dtype)
    got, _, st = gpu_sort(a, tuning=FIXUP)
    want = a.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(got), bits(want))
    assert st["fixup_peeled"] > 0
    _, _, st_on = gpu_sort(a)  # on by default
    assert st_on["fixup_peeled"] > 0
    got_off, _, st_off = gpu_sort(a, tuning={"fixup": -1})
    assert st_off["fixup_peeled"] == 0 and np.array_equal(bits(got_off), bits(want))


@pytest.mark.parametrize("name", ["sort99", "merge", "sawtooth", "asc_swaps"])
def test_nearly_sorted_patterns_pairs(name):
    """Pairs through the fix-up (or through its give-up path back to the ordinary sort)."""
    n = (1 << 20) + 3
    k = workloads.pattern(name, n, workloads.config_seed(81), dtype=np.int32)
    v = np.arange(n, dtype=np.uint32)
    ko, vo, st = gpu_sort(k, v, tuning=FIXUP)
    want = k.copy()
    oracle.pdqsort(want)
    assert np.array_equal(ko, want)
    assert np.array_equal(k[vo.astype(np.int64)], ko)
    if name == "asc_swaps":
        assert st["fixup_peeled"] > 0
    elif name in ("merge", "sawtooth"):  # long runs: peeling does not converge, the sort takes over
        assert st["fixup_peeled"] == 0


@pytest.mark.parametrize("kind", ["reversed_triples", "rotated_blocks"])
def test_nearly_sorted_clustered_displacements(kind):
    """Displaced blocks every 40 elements: reversed triples peel in one round; rotated blocks of
    six need one round per pair and make the fix-up give up.  Either way the keys are exact."""
    n = 1 << 20
    a = np.arange(n, dtype=np.int64)
    for s0 in range(7, n - 8, 40):
        if kind == "reversed_triples":
            a[s0:s0 + 3] = a[s0:s0 + 3][::-1].copy()
        else:
            a[s0:s0 + 6] = np.concatenate([a[s0 + 3:s0 + 6], a[s0:s0 + 3]])
    a = a.astype(np.int32)
    got, _, st = gpu_sort(a, tuning=FIXUP)
    assert np.array_equal(got, oracle_sorted(a))


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
@pytest.mark.parametrize("lo,hi", [(1, 0), (3, -2)])
def test_nearly_sorted_fixup_on_misaligned_subarrays(dtype, lo, hi):
    """The fix-up on a slice that starts off a 16-byte boundary, keys and pairs: only the slice
    changes, bit-exact, values attached."""
    import torch
    import paper_2106_05123_gb300 as pdq
    from gpu_helpers import CODE, to_device, to_host
    n = 700_001
    a = workloads.pattern("asc_swaps", n, workloads.config_seed(82), dtype=np.int64).astype(dtype)
    end = n + hi if hi else n
    want = a.copy()
    want[lo:end] = oracle_sorted(a[lo:end])
    d = to_device(a)
    st = pdq.pdq_sort_keys(d[lo:end], key_dtype=CODE[np.dtype(dtype)])
    torch.cuda.synchronize()
    assert np.array_equal(to_host(d, dtype), want)
    assert st["fixup_peeled"] > 0
    v = np.arange(n, dtype=np.uint32 if np.dtype(dtype).itemsize == 4 else np.uint64)
    dk, dv = to_device(a), to_device(v)
    pdq.pdq_sort_pairs(dk[lo:end], dv[lo:end], key_dtype=CODE[np.dtype(dtype)])
    torch.cuda.synchronize()
    gk, gv = to_host(dk, dtype), to_host(dv, v.dtype).astype(np.int64)
    assert np.array_equal(gk, want)
    assert np.array_equal(a[gv], gk)  # every key kept its value (untouched outside the slice)


def test_nearly_sorted_huge_segment():
    """A segment above the persistent kernel's limit takes the plain path, fix-up included."""
    from gpu_helpers import gpu_sort_segmented
    big = (1 << 20) + 77
    a = np.concatenate([workloads.pattern("asc_swaps", big, workloads.config_seed(83), dtype=np.int64),
                        workloads.uniform_bits(5000, np.int64, workloads.config_seed(84))]).astype(np.int32)
    offs = np.array([0, big, big + 5000], dtype=np.int64)
    got, _, _, rc = gpu_sort_segmented(a, offs)
    assert rc == 0
    want = a.copy()
    oracle.pdqsort_segmented(want, offs)
    assert np.array_equal(got, want)


def with_largest_code(dtype, n, frac, seed):
    """Keys of which about `frac` hold the largest code of their order (the base sort's sentinel
    value: INT_MAX, UINT_MAX, or the float32 +NaN with all payload bits set)."""
    a = keys_for(dtype, n, seed)
    m = int(n * frac) + 1
    pos = (workloads.splitmix64(workloads.substream(seed, 9), m) % np.uint64(max(n, 1))).astype(np.int64)
    if dtype == np.float32:
        a.view(np.uint32)[pos] = np.uint32(0x7FFFFFFF)
    else:
        a[pos] = np.iinfo(dtype).max
    return a


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [31, 1000, 4097, 16383, 100003])
@pytest.mark.parametrize("frac", [0.01, 0.3])
def test_keys_holding_the_sentinel_value(dtype, n, frac):
    # ragged sizes leave padding in the base sort, which ties with these keys
    a = with_largest_code(dtype, n, frac, n)
    got, _, _ = gpu_sort(a)
    assert np.array_equal(bits(got), bits(oracle_sorted(a)))
    vals = np.arange(n, dtype=np.uint32)
    gk, gv, _ = gpu_sort(a, vals)
    assert np.array_equal(bits(gk), bits(oracle_sorted(a)))
    idx = gv.astype(np.int64)
    assert np.array_equal(np.sort(idx), np.arange(n))
    assert np.array_equal(bits(a[idx]), bits(gk))


# ------------------------------------------------------------ bad-split rule (Sec. 4.1)
def _big_equality_bin(n, seed):
    """90% of the keys equal 0, the other 10% are distinct and positive, shuffled.  With two
    buckets per level the one splitter is 0: the zeros fill the equality bin and every other
    key lands in the bucket above it."""
    m = n // 10
    a = np.zeros(n, dtype=np.int32)
    a[:m] = np.arange(1, m + 1, dtype=np.int32)
    return a[workloads.permutation(n, seed)].copy()


BAD_ONLY_BY_NONEQUAL = dict(log2_buckets=1, base_capacity=256, bad_allowed=1)


def test_bad_split_counts_the_parents_non_equal_keys():
    """The child above the splitter keeps all of its parent's non-equal keys (10% of the
    parent): a bad split under the rule "more than 7/8 of the parent's non-equal keys", which the
    parent's total size (90% of it final in the equality bin) would hide.  With a budget of 1 the
    child goes straight to the merge-path fallback."""
    n = 200_000
    a = _big_equality_bin(n, 131)
    got, _, st = gpu_sort(a, tuning=BAD_ONLY_BY_NONEQUAL)
    assert np.array_equal(got, oracle_sorted(a))
    assert st["bad_splits"] >= 1 and st["fallback_buckets"] >= 1
    vals = np.arange(n, dtype=np.uint32)
    gk, gv, st = gpu_sort(a, vals, tuning=BAD_ONLY_BY_NONEQUAL)
    ok, ov = a.copy(), vals.copy()
    oracle.pdqsort_pairs(ok, ov)
    assert np.array_equal(gk, ok) and np.array_equal(a[gv.astype(np.int64)], gk)
    assert st["bad_splits"] >= 1 and st["fallback_buckets"] >= 1


def test_bad_split_rule_in_the_segmented_path():
    from gpu_helpers import gpu_sort_segmented
    n = 300_000  # 30 000 non-equal keys per segment: above the largest base-sort size
    a = np.concatenate([_big_equality_bin(n, 132), _big_equality_bin(n, 133)])
    offs = np.array([0, n, 2 * n], dtype=np.int64)
    got, _, st, rc = gpu_sort_segmented(a, offs, tuning=BAD_ONLY_BY_NONEQUAL)
    assert rc == 0
    want = a.copy()
    oracle.pdqsort_segmented(want, offs)
    assert np.array_equal(got, want)
    assert st["bad_splits"] >= 2 and st["fallback_buckets"] >= 2
