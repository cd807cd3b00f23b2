"""ctypes wrappers over the C exact-PMP oracle (test infrastructure only).

The shared library is compiled from ``pmp_exact.c`` with gcc/OpenMP on first
use (or by ``build()``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmp_exact.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_pmp.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O3 -fopenmp); returns the .so path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            L.oracle_moments.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, dp, dp, u8p]
            L.oracle_dist.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]
            L.oracle_dist.restype = ctypes.c_double
            for name in ("oracle_pmp_direct", "oracle_pmp_diag"):
                getattr(L, name).argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, dp, i64p, ctypes.c_int32]
            L.oracle_pmp_cells.argtypes = [dp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i64p,
                                           ctypes.c_int64, dp, i64p, ctypes.c_int32]
            L.oracle_max_threads.restype = ctypes.c_int32
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def moments(x, m: int):
    """Two-pass FP64 (mu, population sigma, is_constant) of every length-m window."""
    x = _f64(x)
    nw = x.shape[0] - m + 1
    mu = np.empty(nw)
    sg = np.empty(nw)
    cst = np.empty(nw, dtype=np.uint8)
    rc = lib().oracle_moments(_dp(x), x.shape[0], m, _dp(mu), _dp(sg),
                              cst.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    assert rc == 0
    return mu, sg, cst.astype(bool)


def dist(x, m: int, i: int, j: int) -> float:
    """Direct FP64 z-normalised distance d_m(i, j) (Sec. 2); inf if a window is constant."""
    x = _f64(x)
    return float(lib().oracle_dist(_dp(x), x.shape[0], m, i, j))


def pmp(x, m_min: int, m_max: int, excl: int, tier: str = "direct", threads: int = 0):
    """Exact pan matrix profile rows P[L][n], I[L][n] (Sec. 2)."""
    x = _f64(x)
    n = x.shape[0]
    L = m_max - m_min + 1
    P = np.empty((L, n))
    I = np.empty((L, n), dtype=np.int64)
    fn = lib().oracle_pmp_direct if tier == "direct" else lib().oracle_pmp_diag
    rc = fn(_dp(x), n, m_min, m_max, excl, _dp(P), _ip(I), threads)
    if rc != 0:
        raise RuntimeError(f"oracle failed rc={rc}")
    return P, I


def pmp_cells(x, m: int, excl: int, rows, threads: int = 0):
    """Exact (P_m[i], I_m[i]) for the listed starts i only (tier i)."""
    x = _f64(x)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    P = np.empty(rows.shape[0])
    I = np.empty(rows.shape[0], dtype=np.int64)
    rc = lib().oracle_pmp_cells(_dp(x), x.shape[0], m, excl, _ip(rows), rows.shape[0],
                                _dp(P), _ip(I), threads)
    if rc != 0:
        raise RuntimeError(f"oracle failed rc={rc}")
    return P, I
