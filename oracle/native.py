"""Builds and loads the oracle's C helper (cyclic Jacobi).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).  Compiled with the host gcc into
oracle/_build/; nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jacobi.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_jacobi.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.oracle_jacobi_eig.restype = ctypes.c_int
            _lib.oracle_jacobi_eig.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_double, ctypes.c_int]
    return _lib


def jacobi_eigh(A, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigen-decomposition of symmetric A by cyclic Jacobi: (w, V), w ascending."""
    n = A.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    a = np.ascontiguousarray(0.5 * (A + A.T), dtype=np.float64).copy()
    v = np.zeros((n, n))
    sweeps = lib().oracle_jacobi_eig(n, a.ctypes.data, v.ctypes.data, tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    w = np.diag(a).copy()
    order = np.argsort(w)
    return w[order], v[:, order]
