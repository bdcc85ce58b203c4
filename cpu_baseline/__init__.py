"""The benchmark's second CPU baseline: the paper's own algorithm on the host
(the depth-first Schur-complement tree with pivot correction of Section II,
then the CDet recursion of Section V.A), in plain C with OpenMP over matrices.

It is a timing reference, not the oracle: the oracle evaluates every minor by
its own elimination, and the tests check this code against it. Only the
benchmark's CPU-baseline leg and the tests use it; the CUDA library never does.

``fpm_sc.c`` is compiled on first use (gcc -O3, OpenMP, no target-specific
flags) into ``cpu_baseline/_build/libfpm_sc.so``; ``build()`` does this
explicitly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpm_sc.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfpm_sc.so")
_lock = threading.Lock()
_lib = None

DEFAULT_PIV_THRESHOLD = 1e-6
DEFAULT_PIV_SHIFT = 1.0


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.fpm_sc_batch.argtypes = [P, i32, i64, P, P, d, d, P, i32]
            lib.fpm_sc_batch.restype = None
            lib.fpm_sc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().fpm_sc_max_threads())


def fpm_sc(A, nthreads: int = 0, piv_threshold: float = DEFAULT_PIV_THRESHOLD,
           piv_shift: float = DEFAULT_PIV_SHIFT):
    """All 2^n principal minors and the connected sums c (a[S] = det(A[S])^2)
    of each matrix of A (batch, n, n); returns (minors, c, status), status bit 0
    = a pivot was corrected, bit 1 = more corrections than recorded."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    single = A.ndim == 2
    if single:
        A = A[None]
    b, n, _ = A.shape
    assert A.shape[2] == n and 1 <= n <= 20
    minors = np.empty((b, 1 << n))
    c = np.empty((b, 1 << n))
    status = np.zeros(b, dtype=np.int32)
    _load().fpm_sc_batch(A.ctypes.data, n, b, minors.ctypes.data, c.ctypes.data, piv_threshold, piv_shift,
                         status.ctypes.data, nthreads)
    if single:
        return minors[0], c[0], status[0]
    return minors, c, status
