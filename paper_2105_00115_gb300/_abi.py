"""ctypes view of include/qdot.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqdot.so")

KEY_MIN = -2148
KEY_COUNT = 4224
PATHS = {"auto": 0, "two_pass": 1, "one_pass": 2, "fp64_dot": 3, "fused": 4}
STATUS = {0: "QDOT_OK", 1: "QDOT_ERR_ARG", 2: "QDOT_ERR_NONFINITE", 3: "QDOT_ERR_CUDA", 4: "QDOT_ERR_TIMEOUT",
          5: "QDOT_ERR_WORKSPACE", 6: "QDOT_ERR_NOCONV"}


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("block", ctypes.c_int32), ("split_budget", ctypes.c_int32),
                ("mant_reading", ctypes.c_int32), ("path", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("value", ctypes.c_double), ("bound", ctypes.c_double), ("n_bins", ctypes.c_int64),
                ("count", ctypes.c_int64 * 5), ("e_max", ctypes.c_int32), ("e_min", ctypes.c_int32),
                ("f", ctypes.c_int32), ("status", ctypes.c_int32)]


class Selection(ctypes.Structure):
    _fields_ = [("e_max", ctypes.c_int32), ("e_min", ctypes.c_int32), ("f", ctypes.c_int32),
                ("status", ctypes.c_int32), ("n_bins", ctypes.c_int64), ("block", ctypes.c_int32),
                ("key_min", ctypes.c_int32), ("m_half", ctypes.c_int32), ("m_single", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2), ("cls", ctypes.c_uint8 * KEY_COUNT)]


class TraceUnit(ctypes.Structure):
    _fields_ = [("value", ctypes.c_int64), ("grid", ctypes.c_int32), ("cls", ctypes.c_uint8),
                ("source", ctypes.c_uint8), ("reserved", ctypes.c_uint16)]


# qdot_trace_unit sources (include/qdot.h)
TRACE_SOURCES = {0: "none", 1: "slot0", 2: "slot1", 3: "slot3", 4: "recomputed", 5: "fused", 6: "item",
                 7: "item_recomputed", 8: "item_fixed"}


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class BatchedTuning(ctypes.Structure):
    _fields_ = [("threads_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("staged", ctypes.c_int32)]


class CgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("counts", ctypes.c_int64 * 5)]


class PowerInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("counts", ctypes.c_int64 * 5)]


assert ctypes.sizeof(Result) == 80
assert ctypes.sizeof(CgInfo) == 64
assert ctypes.sizeof(PowerInfo) == 56
assert ctypes.sizeof(Params) == 24
assert ctypes.sizeof(TraceUnit) == 16

# (name, restype, argtypes) for every entry point of include/qdot.h
_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double
_PP = ctypes.POINTER(Params)
SIGNATURES = {
    "qdot_workspace_size": (_SZ, [_I64, _PP]),
    "qdot": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP, _VP, _SZ, _VP]),
    "qdot_explain": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "qdot_batched_workspace_size": (_SZ, [_VP, _I32, _PP]),
    "qdot_batched": (ctypes.c_int, [_VP, _VP, _VP, _I32, _PP, _VP, _I32, _VP, _SZ, _VP]),
    "qdot_backward": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP, _VP, _VP, _VP]),
    "qdot_batched_backward_workspace_size": (_SZ, [_I32]),
    "qdot_batched_backward": (ctypes.c_int, [_VP, _VP, _VP, _I32, _PP, _VP, _VP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "qdot_batched_tuned": (ctypes.c_int, [_VP, _VP, _VP, _I32, _PP, _VP, _VP, _I32, _VP, _SZ, _VP]),
    "qdot_cg_workspace_size": (_SZ, [_I64, _PP]),
    "qdot_cg": (ctypes.c_int, [_VP, _VP, _VP, _D, _I32, _PP, _VP, _VP, _VP, _SZ, _VP]),
    "qdot_cg_batched_workspace_size": (_SZ, [_VP, _I32, _PP]),
    "qdot_cg_batched": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP, _D, _I32, _PP, _VP, _VP, _SZ, _VP]),
    "qdot_power_workspace_size": (_SZ, [_I64, _PP]),
    "qdot_power": (ctypes.c_int, [_VP, _VP, _I32, _D, _PP, _VP, _VP, _VP, _SZ, _VP]),
    "qdot_dot_fp64_workspace_size": (_SZ, []),
    "qdot_dot_fp64": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _SZ, _VP]),
    "qdot_from_host": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "qdot_static_scratch": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP]),
    "qdot_trace_units": (_I64, [_I64, _PP, _I32, _VP]),
    "qdot_trace": (ctypes.c_int, [_VP, _VP, _I64, _PP, _VP, _VP, _I64, _VP, _VP, _SZ, _VP]),
    "qdot_kernel_launches": (_I32, [_I64, _PP, _I32]),
    "qdot_select_path": (_I32, [_I64, _PP, _I32]),
    "qdot_stream_kernel": (ctypes.c_char_p, [_I64, _PP, _I32]),
    "qdot_set_kernel_events": (None, [_VP, _VP]),
    "qdot_last_error": (ctypes.c_char_p, []),
    "qdot_version": (ctypes.c_char_p, []),
}

_lib = None


class QdotError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libqdot.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2105_00115_gb300.build.build() "
                              "(the qdot path has no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, lib=None) -> None:
    if status != 0:
        lib = lib or load()
        raise QdotError(status, lib.qdot_last_error().decode())
