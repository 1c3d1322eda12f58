"""qdot on one GB300: Python binding of libqdot.so.

Thin marshalling layer over the C ABI in include/qdot.h: every step of the
method runs in the library's CUDA kernels; PyTorch only provides device
memory (tensors, workspaces) and streams.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _abi
from ._abi import Params, QdotError, Result, Selection, TraceUnit, check, load

__all__ = ["QdotResult", "QdotError", "qdot", "qdot_async", "explain", "trace", "dot_fp64", "from_host",
           "workspace_size",
           "load", "params", "decode_result", "Batch", "Csr", "cg", "cg_batched", "power"]

CLASS_NAMES = ("perforate", "half", "single", "double", "zero")


def _torch():
    import torch
    return torch


@dataclass
class QdotResult:
    value: float
    bound: float
    n_bins: int
    count: tuple
    e_max: int
    e_min: int
    f: int
    status: int


# qdot_status values (include/qdot.h)
QDOT_OK, QDOT_ERR_ARG, QDOT_ERR_NONFINITE, QDOT_ERR_CUDA, QDOT_ERR_TIMEOUT, QDOT_ERR_WORKSPACE, QDOT_ERR_NOCONV = range(7)


def params(eps=1e-16, block=32, split_budget=1, mant_reading=0, path="auto") -> Params:
    return Params(float(eps), int(block), int(split_budget), int(mant_reading), _abi.PATHS[path])


def decode_result(buf) -> QdotResult:
    """Parse an 80-byte qdot_result (host bytes / numpy / CPU tensor)."""
    raw = bytes(np.asarray(buf, dtype=np.uint8).tobytes())
    r = Result.from_buffer_copy(raw[: ctypes.sizeof(Result)])
    return QdotResult(r.value, r.bound, r.n_bins, tuple(r.count), r.e_max, r.e_min, r.f, r.status)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_vec(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float64 or t.dim() != 1:
        raise TypeError(f"{name} must be a 1-D float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def workspace_size(n: int, p: Params) -> int:
    return int(load().qdot_workspace_size(int(n), ctypes.byref(p)))


def _workspace(nbytes, device, ws=None):
    torch = _torch()
    nbytes = max(int(nbytes), 256)
    if ws is not None and ws.numel() >= nbytes:
        return ws
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def qdot_async(x, y, eps=1e-16, block=32, split_budget=1, mant_reading=0, path="auto", out=None, ws=None,
               selection=None, stream=None):
    """Launch qdot(x, y) on ``stream``; returns the 80-byte device result tensor.
    ``selection`` (uint8 CUDA tensor of sizeof(qdot_selection) bytes) receives
    the parameter selection when given."""
    torch = _torch()
    lib = load()
    _check_vec(x, "x")
    _check_vec(y, "y")
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same length")
    p = params(eps, block, split_budget, mant_reading, path)
    n = x.numel()
    need = lib.qdot_workspace_size(n, ctypes.byref(p))
    if need == 0:
        raise QdotError(1, "invalid qdot parameters")
    ws = _workspace(need, x.device, ws)
    if out is None:
        out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=x.device)
    st = lib.qdot(_ptr(x), _ptr(y), n, ctypes.byref(p), _ptr(out), _ptr(selection), _ptr(ws), ws.numel(),
                  _stream_ptr(stream))
    check(st, lib)
    return out


def qdot(x, y, eps=1e-16, block=32, split_budget=1, mant_reading=0, path="auto", stream=None) -> QdotResult:
    """qdot(x, y, eps) on the GPU (Algorithm 3); synchronises and returns the result."""
    out = qdot_async(x, y, eps, block, split_budget, mant_reading, path, stream=stream)
    r = decode_result(out.cpu().numpy())
    if r.status != 0:
        raise QdotError(r.status, "non-finite component in x or y")
    return r


def explain(x, y, eps=1e-16, block=32, split_budget=1, mant_reading=0, stream=None):
    """qdot plus the per-component class map and quantized vectors (device tensors)."""
    torch = _torch()
    lib = load()
    _check_vec(x, "x")
    _check_vec(y, "y")
    p = params(eps, block, split_budget, mant_reading, "two_pass")
    n = x.numel()
    need = lib.qdot_workspace_size(n, ctypes.byref(p))
    if need == 0:
        raise QdotError(1, "invalid qdot parameters")
    ws = _workspace(need, x.device)
    out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=x.device)
    cls = torch.empty(n, dtype=torch.uint8, device=x.device)
    qx = torch.empty(n, dtype=torch.float64, device=x.device)
    qy = torch.empty(n, dtype=torch.float64, device=x.device)
    st = lib.qdot_explain(_ptr(x), _ptr(y), n, ctypes.byref(p), _ptr(out), _ptr(cls), _ptr(qx), _ptr(qy),
                          _ptr(ws), ws.numel(), _stream_ptr(stream))
    check(st, lib)
    return decode_result(out.cpu().numpy()), cls, qx, qy


TRACE_DTYPE = np.dtype([("value", "<i8"), ("grid", "<i4"), ("cls", "u1"), ("source", "u1"), ("reserved", "<u2")])


def trace(x, y, eps=1e-16, block=32, split_budget=1, mant_reading=0, path="auto", want_cls=True, stream=None):
    """qdot on the fused or one-pass path, exactly as ``qdot`` runs it, plus
    what its kernels decided: returns (result, units, unit_components, cls).

    ``units`` is a numpy record array (value, grid, cls, source) with one
    record per block (or per warp item of 256 components on the item-record
    paths): the unit contributed value * 2**grid to the sum.  ``cls`` is the
    per-component class map (uint8 CUDA tensor) on item-record paths (when
    ``want_cls``), else None.  Raises QdotError when the arguments take the
    two-pass path."""
    torch = _torch()
    lib = load()
    _check_vec(x, "x")
    _check_vec(y, "y")
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same length")
    p = params(eps, block, split_budget, mant_reading, path)
    n = x.numel()
    al16 = int((x.data_ptr() | y.data_ptr()) % 16 == 0)
    per = ctypes.c_int32(0)
    nunits = int(lib.qdot_trace_units(n, ctypes.byref(p), al16, ctypes.byref(per)))
    if nunits == 0 and n > 0:
        raise QdotError(1, "these arguments take the two-pass path (use explain)")
    ws = _workspace(lib.qdot_workspace_size(n, ctypes.byref(p)), x.device)
    out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=x.device)
    units = torch.zeros(max(nunits, 1) * ctypes.sizeof(TraceUnit), dtype=torch.uint8, device=x.device)
    cls = None
    if want_cls and per.value == 256 and block != 256:  # item units: per-component classes too
        cls = torch.full((n,), 255, dtype=torch.uint8, device=x.device)
    st = lib.qdot_trace(_ptr(x), _ptr(y), n, ctypes.byref(p), _ptr(out), _ptr(units), nunits, _ptr(cls), _ptr(ws),
                        ws.numel(), _stream_ptr(stream))
    check(st, lib)
    rec = units.cpu().numpy().view(TRACE_DTYPE)[:nunits]
    return decode_result(out.cpu().numpy()), rec, per.value, cls


def dot_fp64(x, y, stream=None) -> float:
    """Plain FP64 dot product on the GPU (the speedup comparator)."""
    torch = _torch()
    lib = load()
    _check_vec(x, "x")
    _check_vec(y, "y")
    ws = _workspace(lib.qdot_dot_fp64_workspace_size(), x.device)
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    check(lib.qdot_dot_fp64(_ptr(x), _ptr(y), x.numel(), _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream)), lib)
    return float(out.item())


def from_host(x_host, y_host, eps=1e-16, block=32, split_budget=1, mant_reading=0, path="auto", x_dev=None,
              y_dev=None, ws=None, stream=None) -> QdotResult:
    """End-to-end qdot from CPU float64 tensors.  Pinned (page-locked) tensors
    are read in place by the kernels over the host link; others are copied into
    x_dev, y_dev first."""
    torch = _torch()
    lib = load()
    n = x_host.numel()
    dev = torch.device("cuda", torch.cuda.current_device())
    if x_dev is None:
        x_dev = torch.empty(n, dtype=torch.float64, device=dev)
    if y_dev is None:
        y_dev = torch.empty(n, dtype=torch.float64, device=dev)
    p = params(eps, block, split_budget, mant_reading, path)
    ws = _workspace(lib.qdot_workspace_size(n, ctypes.byref(p)), dev, ws)
    out_dev = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=dev)
    res = Result()
    st = lib.qdot_from_host(ctypes.c_void_p(x_host.data_ptr()), ctypes.c_void_p(y_host.data_ptr()), n,
                            ctypes.byref(p), ctypes.byref(res), _ptr(x_dev), _ptr(y_dev), _ptr(out_dev), _ptr(ws),
                            ws.numel(), _stream_ptr(stream))
    check(st, lib)
    return QdotResult(res.value, res.bound, res.n_bins, tuple(res.count), res.e_max, res.e_min, res.f, res.status)


def _decode_results(buf, count):
    raw = np.asarray(buf, dtype=np.uint8).reshape(count, ctypes.sizeof(Result))
    return [decode_result(raw[i]) for i in range(count)]


class Batch:
    """A batch of independent qdot problems on the GPU (one persistent launch).

    ``xs``/``ys`` are lists of 1-D float64 CUDA tensors (16-byte aligned);
    the pointer and length arrays and the workspace are built once, so
    ``launch()`` can be recorded in a CUDA graph and replayed."""

    def __init__(self, xs, ys, eps=1e-8, block=32, split_budget=1, mant_reading=0, grid_ctas=0):
        torch = _torch()
        lib = load()
        if len(xs) != len(ys):
            raise ValueError("xs and ys must have the same number of vectors")
        for i, (a, b) in enumerate(zip(xs, ys)):
            _check_vec(a, f"xs[{i}]")
            _check_vec(b, f"ys[{i}]")
            if a.numel() != b.numel():
                raise ValueError(f"pair {i}: lengths differ")
        self.count = len(xs)
        self.p = params(eps, block, split_budget, mant_reading, "auto")
        self.grid_ctas = int(grid_ctas)
        dev = xs[0].device if xs else torch.device("cuda")
        self._keep = (xs, ys)
        self.ns_host = np.array([a.numel() for a in xs], dtype=np.int64)
        self.xs_dev = torch.tensor([a.data_ptr() for a in xs], dtype=torch.int64, device=dev)
        self.ys_dev = torch.tensor([b.data_ptr() for b in ys], dtype=torch.int64, device=dev)
        self.ns_dev = torch.from_numpy(self.ns_host).to(dev)
        need = lib.qdot_batched_workspace_size(self.ns_host.ctypes.data, self.count, ctypes.byref(self.p))
        if need == 0 and self.count > 0:
            raise QdotError(1, "invalid batched qdot parameters (block must be a power of two in [32, 256])")
        self.ws = _workspace(need, dev)
        self.outs = torch.empty(max(self.count, 1) * ctypes.sizeof(Result), dtype=torch.uint8, device=dev)
        self.tuning = None  # an _abi.BatchedTuning, set by autotune()

    def launch(self, stream=None):
        lib = load()
        st = lib.qdot_batched_tuned(_ptr(self.xs_dev), _ptr(self.ys_dev), _ptr(self.ns_dev), self.count,
                                    ctypes.byref(self.p), _ptr(self.outs),
                                    ctypes.byref(self.tuning) if self.tuning is not None else None, self.grid_ctas,
                                    _ptr(self.ws), self.ws.numel(), _stream_ptr(stream))
        check(st, lib)

    def autotune(self, reps=5, use_cache=True, path=None):
        """Time every launch shape on this batch and keep the fastest (cached)."""
        from .tune import tune_batched
        return tune_batched(self, reps=reps, use_cache=use_cache, path=path)

    def results(self):
        return _decode_results(self.outs.cpu().numpy()[: self.count * ctypes.sizeof(Result)], self.count)


class Csr:
    """A CSR matrix in device memory (int64 row pointers, int32 columns, float64 values)."""

    def __init__(self, rowptr, col, val, device="cuda"):
        torch = _torch()
        self.rowptr = torch.as_tensor(np.asarray(rowptr, dtype=np.int64)).to(device)
        self.col = torch.as_tensor(np.asarray(col, dtype=np.int32)).to(device)
        self.val = torch.as_tensor(np.asarray(val, dtype=np.float64)).to(device)
        self.n = self.rowptr.numel() - 1
        self.abi = _abi.Csr(self.n, self.col.numel(), self.rowptr.data_ptr(), self.col.data_ptr(),
                            self.val.data_ptr())


def _solver_path(dot):
    if dot not in ("qdot", "fp64"):
        raise ValueError("dot must be 'qdot' or 'fp64'")
    return "auto" if dot == "qdot" else "fp64_dot"


def cg(A: Csr, b, x0=None, rel_tol=1e-10, max_it=50000, eps=1e-16, block=0, split_budget=1, mant_reading=0,
       history=False, dot="qdot", stream=None):
    """ACG (Algorithm 4) on the GPU.  Returns (x, info dict, history or None).

    dot="fp64" runs the same solver with plain FP64 dot products (the comparator)."""
    torch = _torch()
    lib = load()
    _check_vec(b, "b")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    p = params(eps, block, split_budget, mant_reading, _solver_path(dot))
    ws = _workspace(lib.qdot_cg_workspace_size(A.n, ctypes.byref(p)), b.device)
    info = torch.empty(64, dtype=torch.uint8, device=b.device)
    hist = torch.zeros(max(max_it, 1) * 10, dtype=torch.int64, device=b.device) if history else None
    check(lib.qdot_cg(ctypes.byref(A.abi), _ptr(b), _ptr(x), float(rel_tol), int(max_it), ctypes.byref(p),
                      _ptr(info), _ptr(hist), _ptr(ws), ws.numel(), _stream_ptr(stream)), lib)
    raw = _abi.CgInfo.from_buffer_copy(bytes(info.cpu().numpy()))
    out = {"iters": raw.iters, "status": raw.status, "relres": raw.relres, "true_relres": raw.true_relres,
           "counts": tuple(raw.counts)}
    h = hist[: raw.iters * 10].view(raw.iters, 2, 5).cpu().numpy() if history else None
    return x, out, h


def cg_batched(A: Csr, row_off, b, x0=None, rel_tol=1e-10, max_it=50000, eps=1e-16, block=32, split_budget=1,
               mant_reading=0, dot="qdot", stream=None):
    """Batched ACG on the diagonal blocks of A (system s owns rows
    [row_off[s], row_off[s+1])).  Returns (x, list of per-system info dicts)."""
    torch = _torch()
    lib = load()
    _check_vec(b, "b")
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    count = ro.shape[0] - 1
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    p = params(eps, block, split_budget, mant_reading, _solver_path(dot))
    need = lib.qdot_cg_batched_workspace_size(ro.ctypes.data, count, ctypes.byref(p))
    if need == 0:
        raise QdotError(1, "invalid batched CG arguments (row offsets, or block outside [32, 256])")
    ws = _workspace(need, b.device)
    infos = torch.empty(max(count, 1) * 64, dtype=torch.uint8, device=b.device)
    check(lib.qdot_cg_batched(ctypes.byref(A.abi), ro.ctypes.data, count, _ptr(b), _ptr(x), float(rel_tol),
                              int(max_it), ctypes.byref(p), _ptr(infos), _ptr(ws), ws.numel(), _stream_ptr(stream)),
          lib)
    raw = bytes(infos.cpu().numpy())
    out = []
    for s in range(count):
        r = _abi.CgInfo.from_buffer_copy(raw[64 * s: 64 * (s + 1)])
        out.append({"iters": r.iters, "status": r.status, "relres": r.relres, "true_relres": r.true_relres,
                    "counts": tuple(r.counts)})
    return x, out


def power(A: Csr, x0, iters=500, tau=0.0, eps=1e-16, block=0, split_budget=1, mant_reading=0, history=False,
          dot="qdot", stream=None):
    """APM (Algorithm 5) on the GPU.  Returns (lambda, x, info dict, history or None).

    dot="fp64" runs the same iteration with plain FP64 dot products."""
    torch = _torch()
    lib = load()
    _check_vec(x0, "x0")
    x = x0.clone()
    p = params(eps, block, split_budget, mant_reading, _solver_path(dot))
    ws = _workspace(lib.qdot_power_workspace_size(A.n, ctypes.byref(p)), x.device)
    info = torch.empty(56, dtype=torch.uint8, device=x.device)
    hist = torch.zeros(max(iters, 1) * 10, dtype=torch.int64, device=x.device) if history else None
    check(lib.qdot_power(ctypes.byref(A.abi), _ptr(x), int(iters), float(tau), ctypes.byref(p), _ptr(info),
                         _ptr(hist), _ptr(ws), ws.numel(), _stream_ptr(stream)), lib)
    raw = _abi.PowerInfo.from_buffer_copy(bytes(info.cpu().numpy()))
    out = {"iters": raw.iters, "status": raw.status, "lambda": raw.lambda_, "counts": tuple(raw.counts)}
    h = hist[: raw.iters * 10].view(raw.iters, 2, 5).cpu().numpy() if history else None
    return raw.lambda_, x, out, h
