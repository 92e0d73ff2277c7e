"""Seeded synthetic inputs for the sort (shared by the oracle side and the GPU side).

This module holds no sorting arithmetic: it only draws numbers.  Every generator is a pure
function of (size, seed) built on SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): output i of a stream with seed s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15) with the published 64-bit finaliser.

Workloads follow the input distributions of the paper's evaluation (Sec. 6.1: uniform, dupsq,
dup8, mod8, ones, sort50/90/99, organ, merge, asc, desc) and the measured configurations
(uniform int32 keys; a pattern sweep; Zipf uint64 and N(0,1) float32 key/value pairs with
special floats; log-uniform segment lengths; an 8-component Gaussian/lognormal mixture).
"""

from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

CONFIG_SEED_BASE = 0x9E3779B97F4A7C15


def config_seed(config_id: int) -> int:
    """Fixed seed per measured configuration."""
    return (CONFIG_SEED_BASE ^ int(config_id)) & 0xFFFFFFFFFFFFFFFF


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the SplitMix64 stream with the given seed (uint64)."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, n, _CHUNK):
            hi = min(n, lo + _CHUNK)
            ctr = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix(s + ctr * GOLDEN)
    return out


def substream(seed: int, tag: int) -> int:
    """Derive an independent seed for a named purpose (tag) from a base seed."""
    with np.errstate(over="ignore"):
        v = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(tag) * _M2)],
                          dtype=np.uint64))
    return int(v[0])


def uniform01(seed: int, n: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_bits(n: int, dtype, seed: int) -> np.ndarray:
    """i.i.d. uniform keys over the full range of an integer dtype (or all float32 bit patterns)."""
    dtype = np.dtype(dtype)
    r = splitmix64(seed, n)
    if dtype.itemsize == 4:
        return (r >> np.uint64(32)).astype(np.uint32).view(dtype)
    return r.view(dtype)


def permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1 (int64): rank order of n SplitMix64 draws."""
    return np.argsort(splitmix64(seed, n), kind="stable").astype(np.int64)


def shuffle(a: np.ndarray, seed: int, perm=None) -> np.ndarray:
    return a[(perm or permutation)(a.size, seed)]


# ------------------------------------------------------------------ paper distributions (Sec. 6.1)
def pattern(name: str, n: int, seed: int, dtype=np.int32, perm=None) -> np.ndarray:
    """One named input pattern of n keys.  `perm(n, seed)` may replace `permutation` by a
    faster routine that returns the same permutation (used for very large n)."""
    i = np.arange(n, dtype=np.int64)

    def shuffle(a, seed):
        return a[(perm or permutation)(a.size, seed)]

    if name == "uniform":        # A[i] = i, shuffled
        a = shuffle(i, seed)
    elif name == "random":       # i.i.d. uniform over the dtype's full range
        return uniform_bits(n, dtype, seed)
    elif name == "ones":         # all equal
        a = np.ones(n, dtype=np.int64)
    elif name == "asc":
        a = i
    elif name == "desc":
        a = n - 1 - i
    elif name == "organ":        # ascending first half, descending second half
        h = n // 2
        a = np.where(i < h, i, n - 1 - i)
    elif name == "asc_swaps":    # ascending, then n/100 transpositions of random index pairs
        a = i.copy()
        m = n // 100
        if m and n > 1:
            r = splitmix64(seed, 2 * m) % np.uint64(n)
            x, y = r[:m].astype(np.int64), r[m:].astype(np.int64)
            for p, q in zip(x, y):  # sequential, as a series of transpositions
                a[p], a[q] = a[q], a[p]
    elif name.startswith("mod"):  # i mod k, shuffled (k distinct values)
        k = int(name[3:])
        a = shuffle(i % k, seed)
    elif name == "sawtooth":     # 64 ascending runs, each value 64 times
        period = max(1, n // 64)
        a = i % period
    elif name == "dupsq":        # i mod floor(sqrt(n)), shuffled
        a = shuffle(i % max(1, int(np.floor(np.sqrt(n)))), seed)
    elif name == "dup8":         # (i^8 + n/2) mod n, shuffled, computed modulo n exactly
        mod = np.uint64(max(n, 1))
        x = i.astype(np.uint64) % mod
        p = np.ones_like(x)
        for _ in range(8):
            p = (p * x) % mod if n < (1 << 32) else _mulmod(p, x, int(mod))
        a = shuffle(((p + np.uint64(n // 2)) % mod).astype(np.int64), seed)
    elif name.startswith("sort"):  # first x% ascending, rest shuffled
        frac = int(name[4:]) / 100.0
        k = int(n * frac)
        a = i.copy()
        a[k:] = shuffle(a[k:], seed)
    elif name == "merge":        # two ascending halves concatenated
        h = n // 2
        a = np.concatenate([np.arange(h), np.arange(n - h)]).astype(np.int64)
    else:
        raise ValueError(f"unknown pattern {name!r}")
    return a.astype(dtype)


def _mulmod(a: np.ndarray, b: np.ndarray, m: int) -> np.ndarray:
    return np.array([(int(x) * int(y)) % m for x, y in zip(a, b)], dtype=np.uint64)


SWEEP_PATTERNS = ["uniform", "ones", "asc", "desc", "organ", "asc_swaps", "mod16", "sawtooth"]


# ------------------------------------------------------------------ key/value configurations
def zipf_u64_pairs(n: int, seed: int, s: float = 1.1, ranks: int = 256):
    """uint64 keys: Zipf(s) over `ranks` distinct seeded 64-bit values; uint32 payload = index."""
    vals = splitmix64(substream(seed, 1), ranks)
    w = 1.0 / np.arange(1, ranks + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w) / w.sum()
    u = uniform01(substream(seed, 2), n)
    rank = np.minimum(np.searchsorted(cdf, u, side="right"), ranks - 1)
    keys = vals[rank]
    return keys, np.arange(n, dtype=np.uint32)


def normal_f32_specials(n: int, seed: int, frac: float = 0.001):
    """float32 N(0,1) keys (Box-Muller in double, rounded) with frac NaN (half each sign, quiet,
    random 22-bit payload), frac -0.0 and frac +-inf at disjoint seeded positions; uint32
    payload = index."""
    h = (n + 1) // 2
    u1 = uniform01(substream(seed, 3), h)
    u2 = uniform01(substream(seed, 4), h)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:n]
    keys = z.astype(np.float32)
    m = int(n * frac)
    if m and 3 * m <= n:
        cand = (splitmix64(substream(seed, 5), 4 * m) % np.uint64(n)).astype(np.int64)
        _, first = np.unique(cand, return_index=True)
        pos = cand[np.sort(first)][: 3 * m]
        assert pos.size == 3 * m
        bits = keys.view(np.uint32)
        nan_pos, zero_pos, inf_pos = pos[:m], pos[m:2 * m], pos[2 * m:]
        payload = (splitmix64(substream(seed, 6), m) >> np.uint64(42)).astype(np.uint32)
        sign = (np.arange(m) % 2).astype(np.uint32) << np.uint32(31)
        bits[nan_pos] = sign | np.uint32(0x7FC00000) | payload
        bits[zero_pos] = np.uint32(0x80000000)
        bits[inf_pos] = sign | np.uint32(0x7F800000)
    return keys, np.arange(n, dtype=np.uint32)


# ------------------------------------------------------------------ segmented configuration
# composite keys: records of two 4-byte fields (field 0 at the lower address)
COMPOSITE_DTYPES = {
    "i32i32": np.dtype([("first", "<i4"), ("second", "<i4")]),
    "f32u32": np.dtype([("first", "<f4"), ("second", "<u4")]),
}


def composite_keys(kind: str, n: int, seed: int, first_distinct: int = 0) -> np.ndarray:
    """n records of the composite key type `kind` ("i32i32" or "f32u32").  Field 0: uniform bits
    (i32i32) or N(0,1) float32 with 1% NaN / -0.0 / +-inf (f32u32); with first_distinct > 0 it is
    drawn from that many distinct values, so long runs of equal first fields are decided by field
    1.  Field 1: uniform bits."""
    dt = COMPOSITE_DTYPES[kind]
    out = np.empty(n, dtype=dt)
    if kind == "i32i32":
        first = uniform_bits(n, np.int32, substream(seed, 21))
    else:
        first, _ = normal_f32_specials(n, substream(seed, 22), frac=0.01)
    if first_distinct > 0 and n:
        pool = first[: min(n, first_distinct)].copy()
        pick = (splitmix64(substream(seed, 23), n) % np.uint64(pool.size)).astype(np.int64)
        first = pool[pick]
    out["first"] = first
    out["second"] = uniform_bits(n, dt["second"], substream(seed, 24))
    return out


def segment_offsets(num_segments: int, seed: int, max_log2: int = 16) -> np.ndarray:
    """Offsets (int64, num_segments + 1) for lengths clamp(round(2^(max_log2 * U)), 1, 2^max_log2)."""
    u = uniform01(substream(seed, 7), num_segments)
    lens = np.clip(np.rint(np.exp2(max_log2 * u)), 1, 1 << max_log2).astype(np.int64)
    off = np.zeros(num_segments + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


# ------------------------------------------------------------------ learned-CDF configuration
def mixture_f32(n: int, seed: int, components: int = 8):
    """float32 keys drawn i.i.d. from a mixture of 4 Gaussian N(mu, sigma^2) components and 4
    shifted lognormal components mu + sigma * exp(Z); mu ~ U[-1e3, 1e3], sigma = 10^U[-2, 2],
    weights Dirichlet(1) (normalised Exp(1) draws).  Returns (keys, component parameters)."""
    p = uniform01(substream(seed, 8), 3 * components)
    mu = -1e3 + 2e3 * p[:components]
    sigma = 10.0 ** (-2.0 + 4.0 * p[components:2 * components])
    e = -np.log1p(-p[2 * components:])
    w = e / e.sum()
    cdf = np.cumsum(w)
    cdf[-1] = 1.0
    out = np.empty(n, dtype=np.float32)
    s_comp, s_u1, s_u2 = substream(seed, 10), substream(seed, 11), substream(seed, 12)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        m = hi - lo
        c = np.minimum(np.searchsorted(cdf, _u01_at(s_comp, lo, m), side="right"), components - 1)
        u1 = _u01_at(s_u1, lo, m)
        u2 = _u01_at(s_u2, lo, m)
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2 * np.pi * u2)
        x = mu[c] + sigma[c] * np.where(c < components // 2, z, np.exp(z))
        out[lo:hi] = x.astype(np.float32)
    return out, {"mu": mu, "sigma": sigma, "weights": w}


def _u01_at(seed: int, start: int, n: int) -> np.ndarray:
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
