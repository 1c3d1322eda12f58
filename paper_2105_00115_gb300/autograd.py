"""torch.autograd.Function wrappers of qdot: the forward runs qdot, the backward
runs the library's backward kernel, which re-derives every component's class
from the forward's selection (the class map is held fixed).

    z = qdot_fn(x, y, eps, block)        # x, y: 1-D float64 CUDA tensors
    z = qdot_batch_fn(X, Y, eps, block)  # X, Y: [B, L] float64 CUDA tensors

Gradients: dz/dx_i = q_c(y_i), dz/dy_i = q_c(x_i) for kept components (class
half / single / double), 0 for perforated and zero ones.  Nothing here
synchronises with the host; double backward is not supported.
"""
import ctypes

import torch
from torch.autograd.function import once_differentiable

from . import _abi
from . import (load, params, check, _ptr, _stream_ptr, _workspace, _check_vec, QdotError)

_SEL_BYTES = 4272


def _value_of(results: torch.Tensor, count: int) -> torch.Tensor:
    """The z fields of `count` packed 80-byte qdot_result records (a device copy)."""
    return results[: count * 80].view(torch.float64).view(count, 10)[:, 0].clone()


class QdotFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, eps, block, split_budget, mant_reading):
        lib = load()
        _check_vec(x, "x")
        _check_vec(y, "y")
        if x.numel() != y.numel():
            raise ValueError("x and y must have the same length")
        p = params(eps, block, split_budget, mant_reading, "auto")
        n = x.numel()
        need = lib.qdot_workspace_size(n, ctypes.byref(p))
        if need == 0:
            raise QdotError(1, "invalid qdot parameters")
        ws = _workspace(need, x.device)
        out = torch.empty(80, dtype=torch.uint8, device=x.device)
        sel = torch.empty(_SEL_BYTES, dtype=torch.uint8, device=x.device)
        check(lib.qdot(_ptr(x), _ptr(y), n, ctypes.byref(p), _ptr(out), _ptr(sel), _ptr(ws), ws.numel(),
                       _stream_ptr(None)), lib)
        ctx.save_for_backward(x, y, sel)
        ctx.prm = (eps, block, split_budget, mant_reading)
        return _value_of(out, 1)[0]

    @staticmethod
    @once_differentiable
    def backward(ctx, gz):
        x, y, sel = ctx.saved_tensors
        lib = load()
        p = params(*ctx.prm, "auto")
        g = gz.detach().to(torch.float64).reshape(1).contiguous()
        gx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        gy = torch.empty_like(y) if ctx.needs_input_grad[1] else None
        check(lib.qdot_backward(_ptr(x), _ptr(y), x.numel(), ctypes.byref(p), _ptr(sel), _ptr(g), _ptr(gx),
                                _ptr(gy), _stream_ptr(None)), lib)
        return gx, gy, None, None, None, None


class QdotBatchFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, Y, eps, block, split_budget, mant_reading, grid_ctas):
        lib = load()
        if X.dim() != 2 or X.shape != Y.shape or X.dtype != torch.float64 or Y.dtype != torch.float64 \
                or not X.is_cuda or not Y.is_cuda:
            raise TypeError("X and Y must be [B, L] float64 CUDA tensors of the same shape")
        X = X.contiguous()
        Y = Y.contiguous()
        Bn, L = X.shape
        if L % 2:
            raise ValueError("row length must be even (each row 16-byte aligned)")
        p = params(eps, block, split_budget, mant_reading, "auto")
        dev = X.device
        stride = L * 8
        rows = torch.arange(Bn, device=dev, dtype=torch.int64) * stride
        xs = rows + X.data_ptr()
        ys = rows + Y.data_ptr()
        ns = torch.full((Bn,), L, dtype=torch.int64, device=dev)
        ns_host = torch.full((Bn,), L, dtype=torch.int64).numpy()
        need = lib.qdot_batched_workspace_size(ns_host.ctypes.data, Bn, ctypes.byref(p))
        if need == 0 and Bn > 0:
            raise QdotError(1, "invalid batched qdot parameters (block must be a power of two in [32, 256])")
        ws = _workspace(need, dev)
        outs = torch.empty(max(Bn, 1) * 80, dtype=torch.uint8, device=dev)
        check(lib.qdot_batched(_ptr(xs), _ptr(ys), _ptr(ns), Bn, ctypes.byref(p), _ptr(outs), int(grid_ctas),
                               _ptr(ws), ws.numel(), _stream_ptr(None)), lib)
        ctx.save_for_backward(X, Y, outs, xs, ys, ns)
        ctx.prm = (eps, block, split_budget, mant_reading)
        ctx.grid_ctas = int(grid_ctas)
        return _value_of(outs, Bn)

    @staticmethod
    @once_differentiable
    def backward(ctx, gz):
        X, Y, outs, xs, ys, ns = ctx.saved_tensors
        lib = load()
        p = params(*ctx.prm, "auto")
        Bn, L = X.shape
        dev = X.device
        g = gz.detach().to(torch.float64).contiguous()
        stride = L * 8
        rows = torch.arange(Bn, device=dev, dtype=torch.int64) * stride
        GX = torch.empty_like(X) if ctx.needs_input_grad[0] else None
        GY = torch.empty_like(Y) if ctx.needs_input_grad[1] else None
        gxs = rows + GX.data_ptr() if GX is not None else None
        gys = rows + GY.data_ptr() if GY is not None else None
        ws = _workspace(lib.qdot_batched_backward_workspace_size(Bn), dev)
        check(lib.qdot_batched_backward(_ptr(xs), _ptr(ys), _ptr(ns), Bn, ctypes.byref(p), _ptr(outs), _ptr(g),
                                        _ptr(gxs), _ptr(gys), ctx.grid_ctas, _ptr(ws), ws.numel(),
                                        _stream_ptr(None)), lib)
        return GX, GY, None, None, None, None, None


def qdot_fn(x, y, eps=1e-16, block=32, split_budget=1, mant_reading=0):
    """Differentiable qdot(x, y) -> 0-dim float64 CUDA tensor."""
    return QdotFunction.apply(x, y, float(eps), int(block), int(split_budget), int(mant_reading))


def qdot_batch_fn(X, Y, eps=1e-8, block=32, split_budget=1, mant_reading=0, grid_ctas=0):
    """Differentiable row-wise qdot of [B, L] tensors -> [B] float64 CUDA tensor
    (one batched launch forward, one backward)."""
    return QdotBatchFunction.apply(X, Y, float(eps), int(block), int(split_budget), int(mant_reading),
                                   int(grid_ctas))


assert ctypes.sizeof(_abi.Result) == 80
