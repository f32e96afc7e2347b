"""Python entry to the C FP64 Jacobi-PCG oracle (test infrastructure; see ``oracle/__init__``).

``build()`` compiles ``oracle/pcg.c`` with gcc (-O2, OpenMP, no fast-math, no
machine-specific flags) into ``oracle/_build/liboracle_pcg.so``; ``ge_d2_cg`` calls
it through ctypes.  The C code follows the textbook PCG with the Jacobi
preconditioner (Section 3.2, the "CG" solver of Table 1) applied to the GE
equation of Section 3.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcg.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_pcg.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (idempotent unless ``force``).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p = ctypes.c_void_p
            lib.oracle_ge_pcg.argtypes = [ctypes.c_int64, p, p, p, ctypes.c_int64, p, p,
                                          ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                          p, p, p, p]
            lib.oracle_ge_pcg.restype = ctypes.c_int
            lib.oracle_components.argtypes = [ctypes.c_int64, p, p, p]
            lib.oracle_components.restype = ctypes.c_int64
            _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ge_d2_cg(n, rowptr, colidx, w, X, Y, rtol=1e-12, max_iter=200000, threads=None,
             return_z=False):
    """d^2 for every row pair of X, Y by FP64 Jacobi-PCG on L z = P(x - y).

    Returns ``(d2 [k], iters [k], relres [k])`` and ``Z [k, n]`` if ``return_z``.
    ``iters[j] == -1`` marks a pair that did not reach ``rtol`` (true residual).
    """
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
    k = X.shape[0]
    d2 = np.zeros(k)
    it = np.zeros(k, dtype=np.int64)
    rr = np.zeros(k)
    Z = np.zeros((k, n)) if return_z else None
    th = threads or default_threads()
    rc = lib.oracle_ge_pcg(int(n), _ptr(rowptr), _ptr(colidx), _ptr(w), int(k), _ptr(X), _ptr(Y),
                           float(rtol), int(max_iter), int(th), _ptr(d2),
                           _ptr(Z) if return_z else None, _ptr(it), _ptr(rr))
    if rc < 0:
        raise ValueError("oracle_ge_pcg: bad arguments")
    if return_z:
        return d2, it, rr, Z
    return d2, it, rr


def components(n, rowptr, colidx):
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    comp = np.zeros(n, dtype=np.int32)
    c = lib.oracle_components(int(n), _ptr(rowptr), _ptr(colidx), _ptr(comp))
    return comp, int(c)
