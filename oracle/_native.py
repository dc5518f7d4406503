"""Build and load the oracle's plain-C direct NUDFT (oracle/nudft.c).

Test infrastructure only.  The library is compiled with gcc on the machine
that runs it (no architecture-specific flags) into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nudft.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libm2oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile nudft.c into a shared library; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            L.m2o_nudft.argtypes = [ctypes.c_int64, dp, ctypes.c_int, dp, dp,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64), dp, dp, ctypes.c_int]
            L.m2o_nudft.restype = None
            L.m2o_num_threads.argtypes = []
            L.m2o_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nudft(t: np.ndarray, c: np.ndarray, f_lo: float, df: float, idx: np.ndarray,
          nthreads: int = 0) -> np.ndarray:
    """J[k, j] = sum_n c[k, n] exp(-i 2 pi (f_lo + idx[j] df) t_n), FP64."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    c = np.atleast_2d(np.asarray(c))
    K, N = c.shape
    assert N == t.shape[0]
    cre = np.ascontiguousarray(c.real, dtype=np.float64)
    cim = np.ascontiguousarray(c.imag, dtype=np.float64) if np.iscomplexobj(c) else None
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    Jre = np.zeros((K, idx.shape[0]))
    Jim = np.zeros((K, idx.shape[0]))
    lib().m2o_nudft(N, _dptr(t), K, _dptr(cre), _dptr(cim) if cim is not None else None,
                    float(f_lo), float(df), idx.shape[0],
                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                    _dptr(Jre), _dptr(Jim), int(nthreads))
    return Jre + 1j * Jim


def num_threads() -> int:
    return int(lib().m2o_num_threads())
