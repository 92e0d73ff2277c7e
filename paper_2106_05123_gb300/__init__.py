"""Python binding of the GB300 pattern-defeating sort library (libpdq.so, C ABI in include/pdq.h).

Argument marshalling only: every step of the sort runs in the library's CUDA kernels.  PyTorch
provides device memory and streams.  The library must have been built (``__graft_entry__.build()``
or ``python paper_2106_05123_gb300/_build.py``); there is no CPU fallback, and every call raises
``PdqError`` when the library or a CUDA device is missing.

Names follow the C ABI: ``pdq_sort_keys``, ``pdq_sort_pairs``, ``pdq_sort_segmented``,
``pdq_sort_host``, ``pdq_workspace_bytes``, ``pdq_reverse``, ``pdq_sort_keys_noalloc``.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdq.so")

PDQ_I32, PDQ_U32, PDQ_I64, PDQ_U64, PDQ_F32 = 0, 1, 2, 3, 4
# composite keys: 8-byte records {field 0, field 1}, ordered by field 0, then field 1
PDQ_I32I32, PDQ_F32U32 = 5, 6
KEY_BYTES = {PDQ_I32: 4, PDQ_U32: 4, PDQ_F32: 4, PDQ_I64: 8, PDQ_U64: 8, PDQ_I32I32: 8, PDQ_F32U32: 8}
_STATUS = {0: "PDQ_OK", -1: "PDQ_ERR_ARG", -2: "PDQ_ERR_DTYPE", -3: "PDQ_ERR_WORKSPACE",
           -4: "PDQ_ERR_CUDA", -5: "PDQ_ERR_TIMEOUT", -6: "PDQ_ERR_INTERNAL"}

_TORCH_DT = {
    torch.int32: PDQ_I32,
    torch.int64: PDQ_I64,
    torch.float32: PDQ_F32,
}
if hasattr(torch, "uint32"):
    _TORCH_DT[torch.uint32] = PDQ_U32
if hasattr(torch, "uint64"):
    _TORCH_DT[torch.uint64] = PDQ_U64


class PdqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "passes", "equal_buckets", "fallback_buckets", "reversed", "sorted_exit",
        "learned_overflow", "bad_splits", "base_buckets", "kernel_launches", "fixup_peeled")]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("log2_buckets", ctypes.c_int32), ("oversample", ctypes.c_int32),
                ("base_capacity", ctypes.c_int32), ("bad_allowed", ctypes.c_int32),
                ("probe", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("inject_wait", ctypes.c_int32), ("seg_block", ctypes.c_int32), ("fixup", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libpdq.so (raises PdqError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PdqError(-4, f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
            P = ctypes.POINTER
            L.pdq_workspace_bytes.argtypes = [i64, i64, i32, i32]
            L.pdq_workspace_bytes.restype = sz
            L.pdq_sort_keys.argtypes = [vp, i64, i32, vp, sz, vp, P(Tuning), P(Stats)]
            L.pdq_sort_keys.restype = i32
            L.pdq_sort_pairs.argtypes = [vp, vp, i32, i64, i32, vp, sz, vp, P(Tuning), P(Stats)]
            L.pdq_sort_pairs.restype = i32
            L.pdq_sort_host.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp, sz, vp, P(Tuning), P(Stats)]
            L.pdq_sort_segmented.argtypes = [vp, vp, i32, vp, i64, i64, i32, vp, sz, vp, P(Tuning), P(Stats)]
            L.pdq_sort_segmented.restype = i32
            L.pdq_sort_host.restype = i32
            L.pdq_sort_keys_learned.argtypes = [vp, i64, i32, vp, sz, vp, P(Tuning), P(Stats)]
            L.pdq_sort_keys_learned.restype = i32
            L.pdq_workspace_bytes_learned.argtypes = [i64]
            L.pdq_workspace_bytes_learned.restype = sz
            fp = P(ctypes.c_float)
            L.pdq_learned_loss_grad.argtypes = [vp, vp, i64, fp, ctypes.c_float, ctypes.c_float, fp, vp, vp]
            L.pdq_learned_loss_grad.restype = i32
            L.pdq_learned_train.argtypes = [vp, i64, i32, i32, ctypes.c_float, vp, fp, fp, fp, vp]
            L.pdq_learned_train.restype = i32
            L.pdq_sort_keys_noalloc.argtypes = [vp, i64, i32, vp, P(Stats)]
            L.pdq_sort_keys_noalloc.restype = i32
            L.pdq_reverse.argtypes = [vp, i64, i32, vp]
            L.pdq_reverse.restype = i32
            L.pdq_last_error.argtypes = []
            L.pdq_last_error.restype = ctypes.c_char_p
            L.pdq_launch_count.argtypes = []
            L.pdq_launch_count.restype = i64
            L.pdq_profile_enable.argtypes = [i32]
            L.pdq_profile_enable.restype = None
            L.pdq_profile_read.argtypes = [ctypes.c_char_p, P(ctypes.c_double), P(i64),
                                           P(ctypes.c_double), i32]
            L.pdq_profile_read.restype = i32
            L.pdq_profile_reset.argtypes = []
            L.pdq_profile_reset.restype = None
            L.pdq_autotune_scratch_bytes.argtypes = [i64, i64, i32, i32]
            L.pdq_autotune_scratch_bytes.restype = sz
            L.pdq_autotune.argtypes = [vp, vp, i32, vp, i64, i64, i32, vp, sz, vp, P(Tuning),
                                       P(ctypes.c_float)]
            L.pdq_autotune.restype = i32
            L.pdq_autotune_lookup.argtypes = [i64, i64, i32, i32, P(Tuning)]
            L.pdq_autotune_lookup.restype = i32
            L.pdq_autotune_reset.argtypes = []
            L.pdq_autotune_reset.restype = None
            _lib = L
        return _lib


def _check(rc: int) -> None:
    if rc != 0:
        raise PdqError(rc, lib().pdq_last_error().decode())


def key_dtype_code(t: torch.dtype) -> int:
    if t not in _TORCH_DT:
        raise PdqError(-2, f"unsupported key dtype {t}")
    return _TORCH_DT[t]


def _stream_ptr(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _tuning(t) -> ctypes.POINTER(Tuning) | None:
    if t is None:
        return None
    if isinstance(t, Tuning):
        return ctypes.pointer(t)
    tt = Tuning()
    for k, v in dict(t).items():
        setattr(tt, k, int(v))
    return ctypes.pointer(tt)


def pdq_workspace_bytes(n: int, key_dtype, value_bytes: int = 0, num_segments: int = 0) -> int:
    """Workspace bytes for a call; key_dtype is a torch dtype or a PDQ_* code; num_segments is
    0 for the single-array calls and the segment count for pdq_sort_segmented."""
    code = key_dtype if isinstance(key_dtype, int) else key_dtype_code(key_dtype)
    return int(lib().pdq_workspace_bytes(int(n), int(num_segments), code, int(value_bytes)))


def workspace_for(n: int, key_dtype, value_bytes: int = 0, num_segments: int = 0,
                  device="cuda") -> torch.Tensor:
    """A uint8 device tensor large enough (and 256-byte aligned) for the call."""
    nbytes = pdq_workspace_bytes(n, key_dtype, value_bytes, num_segments)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def _require_cuda(t: torch.Tensor, what: str) -> None:
    if not t.is_cuda:
        raise PdqError(-1, f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise PdqError(-1, f"{what} must be contiguous")


def _key_code(keys: torch.Tensor, key_dtype: int | None) -> int:
    """The PDQ_* code of the keys: the tensor's own dtype, or the override, whose key width must
    match the tensor's element size (composite keys are passed as an 8-byte view)."""
    if key_dtype is None:
        return key_dtype_code(keys.dtype)
    code = int(key_dtype)
    if code in KEY_BYTES and KEY_BYTES[code] != keys.element_size():
        raise PdqError(-1, f"key_dtype {code} needs {KEY_BYTES[code]}-byte elements, "
                           f"the tensor has {keys.element_size()}-byte elements")
    return code


def composite_keys(fields: torch.Tensor) -> torch.Tensor:
    """View an (n, 2) contiguous tensor of 4-byte fields (int32 for PDQ_I32I32; float32 field 0
    and uint32 bits of field 1 for PDQ_F32U32, e.g. an int32 or float32 tensor holding both) as
    the 1-D tensor of n 8-byte records that the composite key types sort."""
    if fields.dim() != 2 or fields.shape[1] != 2 or fields.element_size() != 4:
        raise PdqError(-1, "composite keys are an (n, 2) tensor of 4-byte fields")
    if not fields.is_contiguous():
        raise PdqError(-1, "composite keys must be contiguous")
    return fields.view(torch.int64).view(-1)


def pdq_sort_keys(keys: torch.Tensor, workspace: torch.Tensor | None = None, tuning=None,
                  stream=None, key_dtype: int | None = None) -> dict:
    """Sort a 1-D CUDA tensor in place (ascending; float32 in IEEE totalOrder).  ``key_dtype``
    (a PDQ_* code) overrides the tensor's dtype, e.g. to sort an int32 view as uint32."""
    _require_cuda(keys, "keys")
    dt = _key_code(keys, key_dtype)
    n = keys.numel()
    ws = workspace if workspace is not None else workspace_for(n, dt, 0, 0, keys.device)
    st = Stats()
    _check(lib().pdq_sort_keys(keys.data_ptr(), n, dt, ws.data_ptr(), ws.numel(),
                               _stream_ptr(stream), _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()


def pdq_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, workspace: torch.Tensor | None = None,
                   tuning=None, stream=None, key_dtype: int | None = None) -> dict:
    """Sort (key, value) pairs in place by key; values (4- or 8-byte elements) follow keys."""
    _require_cuda(keys, "keys")
    _require_cuda(vals, "vals")
    if vals.numel() != keys.numel():
        raise PdqError(-1, "keys and vals differ in length")
    vb = vals.element_size()
    dt = _key_code(keys, key_dtype)
    n = keys.numel()
    ws = workspace if workspace is not None else workspace_for(n, dt, vb, 0, keys.device)
    st = Stats()
    _check(lib().pdq_sort_pairs(keys.data_ptr(), vals.data_ptr(), vb, n, dt, ws.data_ptr(),
                                ws.numel(), _stream_ptr(stream), _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()


def pdq_sort_segmented(keys: torch.Tensor, offsets: torch.Tensor, vals: torch.Tensor | None = None,
                       workspace: torch.Tensor | None = None, tuning=None, stream=None,
                       key_dtype: int | None = None) -> dict:
    """Sort every segment [offsets[s], offsets[s+1]) of ``keys`` (and ``vals``) in place in one
    call; ``offsets`` is a CUDA int64 tensor of num_segments + 1 non-decreasing entries."""
    _require_cuda(keys, "keys")
    _require_cuda(offsets, "offsets")
    if offsets.dtype != torch.int64:
        raise PdqError(-1, "offsets must be int64")
    if vals is not None:
        _require_cuda(vals, "vals")
        if vals.numel() != keys.numel():
            raise PdqError(-1, "keys and vals differ in length")
    dt = _key_code(keys, key_dtype)
    vb = vals.element_size() if vals is not None else 0
    n = keys.numel()
    nseg = max(0, offsets.numel() - 1)
    ws = workspace if workspace is not None else workspace_for(n, dt, vb, max(1, nseg), keys.device)
    st = Stats()
    _check(lib().pdq_sort_segmented(keys.data_ptr(), vals.data_ptr() if vals is not None else None, vb,
                                    offsets.data_ptr(), nseg, n, dt, ws.data_ptr(), ws.numel(),
                                    _stream_ptr(stream), _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()


def _tuning_dict(t: Tuning) -> dict:
    return {name: int(getattr(t, name)) for name, _ in Tuning._fields_}


def pdq_autotune(keys: torch.Tensor, vals: torch.Tensor | None = None, offsets: torch.Tensor | None = None,
                 key_dtype: int | None = None, stream=None) -> tuple[dict, float]:
    """Time the candidate tunings on a scratch copy of ``keys`` (and ``vals``; per segment of
    ``offsets`` when given) and record the fastest for this call shape; later sorts of the same
    shape class that pass no tuning use it.  Returns (tuning, milliseconds)."""
    _require_cuda(keys, "keys")
    dt = _key_code(keys, key_dtype)
    vb = vals.element_size() if vals is not None else 0
    n = keys.numel()
    nseg = max(0, offsets.numel() - 1) if offsets is not None else 0
    need = lib().pdq_autotune_scratch_bytes(n, nseg, dt, vb)
    if need == 0:
        raise PdqError(-1, "no autotune scratch size for these arguments")
    scratch = torch.empty(need, dtype=torch.uint8, device=keys.device)
    best = Tuning()
    ms = ctypes.c_float(0.0)
    _check(lib().pdq_autotune(keys.data_ptr(), vals.data_ptr() if vals is not None else None, vb,
                              offsets.data_ptr() if offsets is not None else None, nseg, n, dt,
                              scratch.data_ptr(), scratch.numel(), _stream_ptr(stream), ctypes.byref(best),
                              ctypes.byref(ms)))
    return _tuning_dict(best), float(ms.value)


def pdq_autotune_lookup(n: int, key_dtype: int, value_bytes: int = 0, num_segments: int = 0) -> dict | None:
    """The tuning recorded for this call shape, or None."""
    t = Tuning()
    if lib().pdq_autotune_lookup(n, num_segments, int(key_dtype), value_bytes, ctypes.byref(t)):
        return _tuning_dict(t)
    return None


def pdq_autotune_reset() -> None:
    """Forget every recorded tuning."""
    lib().pdq_autotune_reset()


def pdq_sort_host(h_keys: torch.Tensor, d_keys: torch.Tensor, workspace: torch.Tensor,
                  h_vals: torch.Tensor | None = None, d_vals: torch.Tensor | None = None,
                  tuning=None, stream=None) -> dict:
    """Sort host tensors through caller-provided device buffers (copies in, sorts, copies out)."""
    if h_keys.is_cuda or not d_keys.is_cuda:
        raise PdqError(-1, "h_keys must be a host tensor and d_keys a CUDA tensor")
    dt = key_dtype_code(h_keys.dtype)
    vb = h_vals.element_size() if h_vals is not None else 0
    st = Stats()
    _check(lib().pdq_sort_host(h_keys.data_ptr(), h_vals.data_ptr() if h_vals is not None else None,
                               vb, h_keys.numel(), dt, d_keys.data_ptr(),
                               d_vals.data_ptr() if d_vals is not None else None,
                               workspace.data_ptr(), workspace.numel(), _stream_ptr(stream),
                               _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()


def pdq_sort_keys_learned(keys: torch.Tensor, workspace: torch.Tensor | None = None, tuning=None,
                          stream=None) -> dict:
    """Learned-CDF sort of a float32 CUDA tensor in place (bit-identical to pdq_sort_keys)."""
    _require_cuda(keys, "keys")
    if keys.dtype != torch.float32:
        raise PdqError(-2, "the learned path sorts float32 keys")
    n = keys.numel()
    ws = workspace if workspace is not None else torch.empty(
        max(256, int(lib().pdq_workspace_bytes_learned(n))), dtype=torch.uint8, device=keys.device)
    st = Stats()
    _check(lib().pdq_sort_keys_learned(keys.data_ptr(), n, PDQ_F32, ws.data_ptr(), ws.numel(),
                                       _stream_ptr(stream), _tuning(tuning), ctypes.byref(st)))
    return st.as_dict()


def pdq_workspace_bytes_learned(n: int) -> int:
    return int(lib().pdq_workspace_bytes_learned(int(n)))


def _fbuf(k):
    return (ctypes.c_float * k)()


def pdq_learned_loss_grad(x: torch.Tensor, targets: torch.Tensor, theta, mu: float, sigma: float,
                          stream=None):
    """Loss and gradient of the learned model's objective on the device (test probe)."""
    th = _fbuf(48)
    for i, v in enumerate(theta):
        th[i] = float(v)
    out = _fbuf(49)
    ws = torch.empty(1024, dtype=torch.uint8, device=x.device)
    _check(lib().pdq_learned_loss_grad(x.data_ptr(), targets.data_ptr(), x.numel(), th, float(mu),
                                       float(sigma), out, ws.data_ptr(), _stream_ptr(stream)))
    return float(out[48]), [float(out[i]) for i in range(48)]


def pdq_learned_train(sorted_sample: torch.Tensor, steps: int = 64, batch: int = 16384, lr: float = 0.05,
                      stream=None) -> dict:
    """Train the learned model on a sorted float32 sample on the device (test probe)."""
    th, nl, wba = _fbuf(48), _fbuf(4), _fbuf(48)
    ws = torch.empty(4096, dtype=torch.uint8, device=sorted_sample.device)
    _check(lib().pdq_learned_train(sorted_sample.data_ptr(), sorted_sample.numel(), int(steps), int(batch),
                                   float(lr), ws.data_ptr(), th, nl, wba, _stream_ptr(stream)))
    return {"theta": list(th), "mu": nl[0], "sigma": nl[1], "loss_first": nl[2], "loss_last": nl[3],
            "w": list(wba[:16]), "t": list(wba[16:32]), "a": list(wba[32:48])}


def pdq_sort_keys_noalloc(keys: torch.Tensor, stream=None, key_dtype: int | None = None) -> dict:
    """Keys-only sort that allocates nothing: its scratch is the library's fixed 64 MiB device
    array (n <= 2^20).  For callers that cannot allocate device memory."""
    _require_cuda(keys, "keys")
    dt = _key_code(keys, key_dtype)
    st = Stats()
    _check(lib().pdq_sort_keys_noalloc(keys.data_ptr(), keys.numel(), dt, _stream_ptr(stream),
                                       ctypes.byref(st)))
    return st.as_dict()


def pdq_reverse(t: torch.Tensor, stream=None) -> None:
    _require_cuda(t, "t")
    _check(lib().pdq_reverse(t.data_ptr(), t.numel(), t.element_size(), _stream_ptr(stream)))


def launch_count() -> int:
    return int(lib().pdq_launch_count())


def profile_enable(on: bool = True) -> None:
    lib().pdq_profile_enable(1 if on else 0)


def profile_reset() -> None:
    lib().pdq_profile_reset()


def profile_read(cap: int = 64) -> dict:
    """Per-kernel {name: (total_ms, launches, algorithmic_bytes)} since the last reset."""
    names = ctypes.create_string_buffer(64 * cap)
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_int64 * cap)()
    by = (ctypes.c_double * cap)()
    k = min(cap, lib().pdq_profile_read(names, ms, cnt, by, cap))
    out = {}
    for i in range(k):
        nm = names.raw[64 * i:64 * i + 64].split(b"\0", 1)[0].decode()
        out[nm] = (ms[i], int(cnt[i]), by[i])
    return out
