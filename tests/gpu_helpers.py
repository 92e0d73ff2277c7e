"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on numpy inputs."""

import numpy as np
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads

CODE = {
    np.dtype(np.int32): pdq.PDQ_I32,
    np.dtype(np.uint32): pdq.PDQ_U32,
    np.dtype(np.int64): pdq.PDQ_I64,
    np.dtype(np.uint64): pdq.PDQ_U64,
    np.dtype(np.float32): pdq.PDQ_F32,
    workloads.COMPOSITE_DTYPES["i32i32"]: pdq.PDQ_I32I32,
    workloads.COMPOSITE_DTYPES["f32u32"]: pdq.PDQ_F32U32,
}
# transport dtypes: unsigned keys travel as same-width signed tensors (the ABI takes raw bits)
CARRIER = {4: (np.int32, torch.int32), 8: (np.int64, torch.int64)}


def to_device(a: np.ndarray) -> torch.Tensor:
    npdt, _ = CARRIER[a.dtype.itemsize]
    if a.dtype == np.float32:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a).view(npdt)).cuda()


def to_host(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def gpu_sort(keys: np.ndarray, vals: np.ndarray | None = None, tuning=None):
    """Sort keys (and values) with the CUDA path; returns (keys, vals, stats) as numpy."""
    code = CODE[keys.dtype]
    dk = to_device(keys)
    n = keys.size
    vb = vals.dtype.itemsize if vals is not None else 0
    ws = torch.empty(max(256, pdq.pdq_workspace_bytes(n, code, vb, 0)), dtype=torch.uint8, device="cuda")
    if vals is None:
        st = pdq.pdq_sort_keys(dk, workspace=ws, tuning=tuning, key_dtype=code)
        torch.cuda.synchronize()
        return to_host(dk, keys.dtype), None, st
    dv = to_device(vals)
    st = pdq.pdq_sort_pairs(dk, dv, workspace=ws, tuning=tuning, key_dtype=code)
    torch.cuda.synchronize()
    return to_host(dk, keys.dtype), to_host(dv, vals.dtype), st


def bits(a: np.ndarray) -> np.ndarray:
    return a.view({4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


def gpu_sort_segmented(keys: np.ndarray, offsets: np.ndarray, vals: np.ndarray | None = None, tuning=None,
                       raise_on_error=True):
    """Segmented sort on the GPU; returns (keys, vals, stats, status)."""
    code = CODE[keys.dtype]
    dk = to_device(keys) if keys.size else torch.empty(16, dtype=CARRIER[keys.dtype.itemsize][1], device="cuda")
    doff = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).cuda()
    dv = to_device(vals) if vals is not None and vals.size else None
    n = keys.size
    nseg = max(0, offsets.size - 1)
    vb = vals.dtype.itemsize if vals is not None else 0
    ws = torch.empty(max(256, pdq.pdq_workspace_bytes(n, code, vb, max(1, nseg))), dtype=torch.uint8,
                     device="cuda")
    import ctypes
    st = pdq.Stats()
    L = pdq.lib()
    rc = L.pdq_sort_segmented(dk.data_ptr(), dv.data_ptr() if dv is not None else None, vb, doff.data_ptr(),
                              nseg, n, code, ws.data_ptr(), ws.numel(),
                              torch.cuda.current_stream().cuda_stream, pdq._tuning(tuning), ctypes.byref(st))
    torch.cuda.synchronize()
    if rc and raise_on_error:
        raise pdq.PdqError(rc, L.pdq_last_error().decode())
    kout = to_host(dk, keys.dtype)[:n]
    vout = to_host(dv, vals.dtype)[:n] if dv is not None else None
    return kout, vout, st.as_dict(), rc


def oracle_sorted(a: np.ndarray) -> np.ndarray:
    """The expected keys: the CPU oracle's pdqsort of a copy of `a`."""
    b = np.ascontiguousarray(a).copy()
    oracle.pdqsort(b)
    return b
