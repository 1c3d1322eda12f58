"""qdot CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python view of the plain-C oracle in ``qdot_oracle.c`` (exact integer
arithmetic, one rounding per result).  Only the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import this package; the GPU
library never does, and this package never imports the GPU library.

Each function follows the paper's definitions (arXiv 2105.00115):
``qdot`` is Algorithm 3 (Algorithm 2 then Algorithm 1), ``cg`` is Algorithm 4,
``power`` is Algorithm 5, ``backward`` is the derivative of the computation
phase with the class map held fixed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdot_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PERF, HALF, SINGLE, DOUBLE, ZERO = 0, 1, 2, 3, 4
CLASS_NAMES = ("perforate", "half", "single", "double", "zero")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (plain C11)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "qdot_oracle.h")))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP only spreads the CPU-baseline helpers over host threads; without
        # it they run on one thread and every result is the same
        if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("block", ctypes.c_int32), ("split_budget", ctypes.c_int32),
                ("mant_reading", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("value", ctypes.c_double), ("value_ld", ctypes.c_double),
                ("class_sum", ctypes.c_double * 4), ("bound_elem", ctypes.c_double),
                ("bound_bins", ctypes.c_double), ("bound_apriori", ctypes.c_double),
                ("e_max", ctypes.c_int32), ("e_min", ctypes.c_int32), ("n_bins", ctypes.c_int64),
                ("f", ctypes.c_int32), ("status", ctypes.c_int32), ("count", ctypes.c_int64 * 5)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_qdot.argtypes = [dp, dp, ctypes.c_int64, ctypes.POINTER(_Params), ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_Result)]
        lib.orc_qdot.restype = ctypes.c_int
        lib.orc_quantize.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.orc_quantize.restype = ctypes.c_double
        lib.orc_floor_log2_ratio.argtypes = [ctypes.c_double, ctypes.c_int64]
        lib.orc_floor_log2_ratio.restype = ctypes.c_int
        for name in ("orc_dot_exact", "orc_abs_dot_exact"):
            getattr(lib, name).argtypes = [dp, dp, ctypes.c_int64]
            getattr(lib, name).restype = ctypes.c_double
        lib.orc_unit_sums.argtypes = [dp, dp, ctypes.c_int64, ctypes.POINTER(_Params), ctypes.c_int64, dp, dp]
        lib.orc_unit_sums.restype = ctypes.c_int
        lib.orc_sum_exact.argtypes = [dp, ctypes.c_int64]
        lib.orc_sum_exact.restype = ctypes.c_double
        lib.orc_spmv.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, dp, dp, dp]
        lib.orc_spmv.restype = None
        lib.orc_cg.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, dp, dp, dp, ctypes.c_double,
                               ctypes.c_int32, ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_int32),
                               dp, ctypes.c_void_p]
        lib.orc_cg.restype = ctypes.c_int
        lib.orc_power.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, dp, dp, ctypes.c_int32,
                                  ctypes.c_double, ctypes.POINTER(_Params), dp, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.c_void_p]
        lib.orc_power.restype = ctypes.c_int
        lib.orc_qdot_threads.argtypes = [dp, dp, ctypes.c_int64, ctypes.POINTER(_Params), ctypes.c_int,
                                         ctypes.POINTER(_Result)]
        lib.orc_qdot_threads.restype = ctypes.c_int
        lib.orc_dot_fp64.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int]
        lib.orc_dot_fp64.restype = ctypes.c_double
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_backward.argtypes = [dp, dp, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, dp, dp]
        lib.orc_backward.restype = None
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(eps, block, split_budget, mant_reading) -> _Params:
    return _Params(float(eps), int(block), int(split_budget), int(mant_reading), 0)


@dataclass
class OracleResult:
    value: float
    value_ld: float
    class_sum: tuple
    bound_elem: float
    bound_bins: float
    bound_apriori: float
    e_max: int
    e_min: int
    n_bins: int
    f: int
    status: int
    count: tuple
    cls: np.ndarray | None = None
    qx: np.ndarray | None = None
    qy: np.ndarray | None = None


def qdot(x, y, eps: float = 1e-16, block: int = 0, split_budget: int = 1, mant_reading: int = 0,
         explain: bool = False) -> OracleResult:
    """Algorithm 3: qdot(x, y, eps).  With ``explain`` also returns the class
    map and the quantized vectors (0 for perforated and zero components)."""
    lib = _load()
    x = _f64(x)
    y = _f64(y)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("x and y must be 1-D arrays of equal length")
    n = x.shape[0]
    res = _Result()
    prm = _params(eps, block, split_budget, mant_reading)
    cls = qx = qy = None
    if explain:
        cls = np.zeros(n, dtype=np.uint8)
        qx = np.zeros(n, dtype=np.float64)
        qy = np.zeros(n, dtype=np.float64)
    st = lib.orc_qdot(_dp(x), _dp(y), n, ctypes.byref(prm),
                      cls.ctypes.data if explain else None,
                      qx.ctypes.data if explain else None,
                      qy.ctypes.data if explain else None, ctypes.byref(res))
    return OracleResult(res.value, res.value_ld, tuple(res.class_sum), res.bound_elem, res.bound_bins,
                        res.bound_apriori, res.e_max, res.e_min, res.n_bins, res.f, st, tuple(res.count),
                        cls, qx, qy)


def unit_sums(x, y, unit: int, eps: float = 1e-16, block: int = 0, split_budget: int = 1, mant_reading: int = 0):
    """Algorithm 1's partial sums over the index ranges [k*unit, (k+1)*unit):
    per range the exact sum of q(x_i) q(y_i) (classes of Algorithm 2 on the
    whole vectors) and the exact sum of |x_i y_i|, each rounded once.
    Returns (sums, abs_sums) as float64 arrays of ceil(n / unit)."""
    lib = _load()
    x = _f64(x)
    y = _f64(y)
    n = x.shape[0]
    m = (n + unit - 1) // unit
    sums = np.zeros(max(m, 1))
    abss = np.zeros(max(m, 1))
    prm = _params(eps, block, split_budget, mant_reading)
    st = lib.orc_unit_sums(_dp(x), _dp(y), n, ctypes.byref(prm), int(unit), _dp(sums), _dp(abss))
    if st != 0:
        raise ValueError(f"oracle status {st}")
    return sums[:m], abss[:m]


def qdot_threads(x, y, eps: float = 1e-16, block: int = 0, split_budget: int = 1, mant_reading: int = 0,
                 threads: int = 0) -> OracleResult:
    """qdot with the components split over host threads (CPU baseline): the
    same value, counts and statistics as ``qdot``; bound fields are 0."""
    lib = _load()
    x = _f64(x)
    y = _f64(y)
    res = _Result()
    prm = _params(eps, block, split_budget, mant_reading)
    nt = threads or lib.orc_max_threads()
    st = lib.orc_qdot_threads(_dp(x), _dp(y), x.shape[0], ctypes.byref(prm), int(nt), ctypes.byref(res))
    return OracleResult(res.value, res.value_ld, tuple(res.class_sum), res.bound_elem, res.bound_bins,
                        res.bound_apriori, res.e_max, res.e_min, res.n_bins, res.f, st, tuple(res.count))


def dot_fp64(x, y, threads: int = 1) -> float:
    """Plain FP64 dot on the host: one fused multiply-add chain per thread."""
    x = _f64(x)
    y = _f64(y)
    return _load().orc_dot_fp64(_dp(x), _dp(y), x.shape[0], int(threads))


def max_threads() -> int:
    """Host threads the threaded helpers use by default (1 without OpenMP)."""
    return int(_load().orc_max_threads())


def quantize(v: float, cls: int) -> float:
    return _load().orc_quantize(float(v), int(cls))


def floor_log2_ratio(eps: float, n_bins: int) -> int:
    """Largest integer k with n_bins * 2**k <= eps."""
    return _load().orc_floor_log2_ratio(float(eps), int(n_bins))


def dot_exact(x, y) -> float:
    x = _f64(x)
    y = _f64(y)
    return _load().orc_dot_exact(_dp(x), _dp(y), x.shape[0])


def abs_dot_exact(x, y) -> float:
    x = _f64(x)
    y = _f64(y)
    return _load().orc_abs_dot_exact(_dp(x), _dp(y), x.shape[0])


def sum_exact(v) -> float:
    v = _f64(v)
    return _load().orc_sum_exact(_dp(v), v.shape[0])


def spmv(rowptr, col, val, x) -> np.ndarray:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    x = _f64(x)
    y = np.zeros(rowptr.shape[0] - 1, dtype=np.float64)
    _load().orc_spmv(y.shape[0], rowptr.ctypes.data, col.ctypes.data, _dp(val), _dp(x), _dp(y))
    return y


def cg(rowptr, col, val, b, x0=None, rel_tol=1e-10, max_it=50000, eps=1e-16, block=0, split_budget=1,
       mant_reading=0):
    """Algorithm 4 (ACG).  Returns (x, iterations, sqrt(c_k)/||b||, class counts, status)."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    b = _f64(b)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int32(0)
    rr = np.zeros(1)
    counts = np.zeros(5, dtype=np.int64)
    prm = _params(eps, block, split_budget, mant_reading)
    st = lib.orc_cg(n, rowptr.ctypes.data, col.ctypes.data, _dp(val), _dp(b), _dp(x), float(rel_tol),
                    int(max_it), ctypes.byref(prm), ctypes.byref(it), _dp(rr), counts.ctypes.data)
    return x, it.value, float(rr[0]), counts, st


def power(rowptr, col, val, x0, iters=500, tau=0.0, eps=1e-16, block=0, split_budget=1, mant_reading=0):
    """Algorithm 5 (APM), Rayleigh-quotient reading.  Returns (lambda, x, iterations, class counts, status)."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64(val)
    x = _f64(x0).copy()
    lam = np.zeros(1)
    it = ctypes.c_int32(0)
    counts = np.zeros(5, dtype=np.int64)
    prm = _params(eps, block, split_budget, mant_reading)
    st = lib.orc_power(x.shape[0], rowptr.ctypes.data, col.ctypes.data, _dp(val), _dp(x), int(iters),
                       float(tau), ctypes.byref(prm), _dp(lam), ctypes.byref(it), counts.ctypes.data)
    return float(lam[0]), x, it.value, counts, st


def backward(x, y, cls, g: float):
    """Gradient of qdot with the class map held fixed: (g*q(y), g*q(x))."""
    x = _f64(x)
    y = _f64(y)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    gx = np.zeros_like(x)
    gy = np.zeros_like(y)
    _load().orc_backward(_dp(x), _dp(y), cls.ctypes.data, x.shape[0], float(g), _dp(gx), _dp(gy))
    return gx, gy
