"""CPU oracle for the pdqsort hot path (Peters, arXiv 2106.05123).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs may import this package.  The GPU library never imports it, and
it never imports the GPU library.

Contents (all compiled from the C++ sources beside this file into ``liboracle.so``):

* ``pdqsort(a)``: the paper's sort, in place, on a numpy array of int32/uint32/int64/uint64/
  float32 (float32 under IEEE 754 totalOrder) or of the composite records TUPLE_I32I32 /
  TUPLE_F32U32 (two 4-byte fields, lexicographic).  Returns the instrumentation counters
  (comparisons, heapsort fallbacks, bad partitions, ...).
* ``pdqsort_pairs(keys, vals)``: the same on key/value records (values ride with their key).
* ``pdqsort_segmented(a, offsets)``: each segment sorted independently.
* ``mergesort_check(keys, vals=None)``: independent naive merge sort (separate code).
* ``killer_adversary(n)``: McIlroy's adaptive adversary run against the oracle.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["pdq_oracle.cpp", "mergesort_check.cpp", "adversary.cpp"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Thresholds the paper leaves open (Sec. 5.1, Sec. 2, Sec. 5.2, Sec. 4.1)."""

    _fields_ = [
        ("insertion_threshold", ctypes.c_int64),
        ("ninther_threshold", ctypes.c_int64),
        ("partial_limit", ctypes.c_int64),
        ("bad_allowed_override", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("comparisons", ctypes.c_int64),
        ("heapsort_calls", ctypes.c_int64),
        ("bad_partitions", ctypes.c_int64),
        ("partition_right_calls", ctypes.c_int64),
        ("partition_left_calls", ctypes.c_int64),
        ("partial_insertion_successes", ctypes.c_int64),
        ("insertion_sort_calls", ctypes.c_int64),
        ("max_depth", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (plain -O2, no architecture-specific flags)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_mtime = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_mtime for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


# composite keys: records of two 4-byte fields, ordered lexicographically (first, then second)
TUPLE_I32I32 = np.dtype([("first", "<i4"), ("second", "<i4")])
TUPLE_F32U32 = np.dtype([("first", "<f4"), ("second", "<u4")])

_DT = {
    np.dtype(np.int32): "i32",
    np.dtype(np.uint32): "u32",
    np.dtype(np.int64): "i64",
    np.dtype(np.uint64): "u64",
    np.dtype(np.float32): "f32",
    TUPLE_I32I32: "i32i32",
    TUPLE_F32U32: "f32u32",
}


def _declare(L: ctypes.CDLL) -> None:
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    for name in _DT.values():
        f = getattr(L, f"oracle_pdqsort_{name}")
        f.argtypes = [vp, ctypes.c_int64, P(Params), P(Stats)]
        f.restype = None
        for vb in ("v32", "v64"):
            g = getattr(L, f"oracle_pdqsort_pairs_{name}_{vb}")
            g.argtypes = [vp, vp, ctypes.c_int64, P(Params), P(Stats)]
            g.restype = None
        s = getattr(L, f"oracle_pdqsort_segmented_{name}")
        s.argtypes = [vp, vp, ctypes.c_int64, P(Params)]
        s.restype = None
        m = getattr(L, f"check_mergesort_{name}")
        m.argtypes = [vp, vp, ctypes.c_int64]
        m.restype = None
    L.oracle_default_params.argtypes = [P(Params)]
    L.oracle_default_params.restype = None
    L.oracle_killer_adversary.argtypes = [ctypes.c_int64, P(Params), P(Stats), vp]
    L.oracle_killer_adversary.restype = None


def default_params() -> Params:
    p = Params()
    lib().oracle_default_params(ctypes.byref(p))
    return p


def make_params(insertion_threshold=None, ninther_threshold=None, partial_limit=None,
                bad_allowed_override=None) -> Params:
    p = default_params()
    if insertion_threshold is not None:
        p.insertion_threshold = insertion_threshold
    if ninther_threshold is not None:
        p.ninther_threshold = ninther_threshold
    if partial_limit is not None:
        p.partial_limit = partial_limit
    if bad_allowed_override is not None:
        p.bad_allowed_override = bad_allowed_override
    return p


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def pdqsort(a: np.ndarray, params: Params | None = None) -> dict:
    """Sort ``a`` in place with the oracle; return its counters."""
    name = _DT[a.dtype]
    st = Stats()
    p = params if params is not None else default_params()
    getattr(lib(), f"oracle_pdqsort_{name}")(_ptr(a), a.size, ctypes.byref(p), ctypes.byref(st))
    return st.as_dict()


def pdqsort_pairs(keys: np.ndarray, vals: np.ndarray, params: Params | None = None) -> dict:
    """Sort key/value records in place by key (values ride along)."""
    assert keys.shape == vals.shape
    name = _DT[keys.dtype]
    vb = {4: "v32", 8: "v64"}[vals.dtype.itemsize]
    st = Stats()
    p = params if params is not None else default_params()
    getattr(lib(), f"oracle_pdqsort_pairs_{name}_{vb}")(
        _ptr(keys), _ptr(vals), keys.size, ctypes.byref(p), ctypes.byref(st))
    return st.as_dict()


def pdqsort_segmented(a: np.ndarray, offsets: np.ndarray, params: Params | None = None) -> None:
    """Sort every segment [offsets[s], offsets[s+1]) of ``a`` independently, in place."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    name = _DT[a.dtype]
    p = params if params is not None else default_params()
    getattr(lib(), f"oracle_pdqsort_segmented_{name}")(
        _ptr(a), _ptr(offsets), offsets.size - 1, ctypes.byref(p))


def mergesort_check(keys: np.ndarray, vals: np.ndarray | None = None) -> None:
    """Independent stable merge sort (separate code), in place."""
    name = _DT[keys.dtype]
    if vals is not None:
        assert vals.dtype == np.uint32 and vals.shape == keys.shape
    getattr(lib(), f"check_mergesort_{name}")(
        _ptr(keys), _ptr(vals) if vals is not None else None, keys.size)


def killer_adversary(n: int, params: Params | None = None) -> tuple[np.ndarray, dict]:
    """Run McIlroy's adversary against the oracle; return (concrete input, counters)."""
    out = np.empty(n, dtype=np.int64)
    st = Stats()
    p = params if params is not None else default_params()
    lib().oracle_killer_adversary(n, ctypes.byref(p), ctypes.byref(st), _ptr(out))
    return out, st.as_dict()
