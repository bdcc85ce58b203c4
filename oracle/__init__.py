"""Plain FP64 CPU oracle for the all-principal-minor path (test infrastructure).

Only the tests, the smoke check (``smoke()`` of the repository's build/smoke
entry module) and the benchmark's CPU-baseline leg may import this package. The product path (the CUDA library and its Python
binding) never does: it shares no code with the oracle.

The C source ``oracle.c`` is compiled on first use (gcc, OpenMP, no fast-math,
no FMA contraction so that x86 and Arm hosts round identically) into
``oracle/_build/liboracle.so``; ``build()`` does this explicitly.

Functions (numpy in, numpy out; FP64 / complex128):
  minors_lu(A)              all 2^n principal minors, one partial-pivot LU each (Section II)
  perm_ryser(A, absval)     all 2^n principal permanents by Ryser per subset (Eq. ryser)
  perm_ryser_term_scale(A)  sum of |terms| of Ryser's formula per subset (error scale)
  cdet_recursion(a)         connected sums by Eq. recursion, plain loops
  cdet_partition(a)         connected sums by the set-partition Moebius formula
  cdet_scale(ahat)          the recursion with all terms taken positive (error scale)
  keldysh(Mt, signed)       sum over 2^n Keldysh assignments of separate complex LUs
  keldysh_scale(Mt)         error scale for the Keldysh sum
  minors_scale(A)           perm(|A[S]|): sum of |Leibniz terms| of every minor
  minors_rowsum_bound(A)    prod_{i in S} sum_{j in S} |A_ij| (a cheaper upper bound)
  xnor_minors(M)            all 2^n XNOR minors of 2n x 2n block matrices, one LU per
                            kept submatrix (Section III.B)
  xnor_scale(M)             error scale of the XNOR minors
  nand(M, minors)           the 3^n NAND minors (Section III.C) or their sums over the
                            two types of every subset (Section V.C), with their scale
  keldysh2(Mu, Md, signed)  sum over shared Keldysh assignments of the product of the
                            two spins' determinants (Section V.D), separate LUs
  keldysh2_scale(Mu, Md)    error scale of that sum
The surrogate network's FP64 forward and backward pass is in ``oracle/mlp.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, P = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            for name, args in {
                "oracle_minors_lu": [P, i32, i64, P, i32],
                "oracle_perm_ryser": [P, i32, i64, P, i32, i32],
                "oracle_cdet_recursion": [P, i32, i64, P, i32],
                "oracle_cdet_scale": [P, i32, i64, P, i32],
                "oracle_cdet_partition": [P, i32, i64, P, i32],
                "oracle_keldysh": [P, i32, i64, i32, P, P, i32],
                "oracle_keldysh_scale": [P, i32, i64, i32, P, i32],
                "oracle_xnor_minors": [P, i32, i64, P, i32],
                "oracle_xnor_scale": [P, i32, i64, i32, P, i32],
                "oracle_nand": [P, i32, i64, P, P, P, i32],
                "oracle_keldysh2": [P, P, i32, i64, i32, P, P, i32],
                "oracle_keldysh2_scale": [P, P, i32, i64, P, i32],
            }.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = None
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _mat_batch(A, dtype=np.float64):
    A = np.ascontiguousarray(A, dtype=dtype)
    single = A.ndim == 2
    if single:
        A = A[None]
    assert A.ndim == 3 and A.shape[1] == A.shape[2], A.shape
    return A, single


def _vec_batch(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    single = a.ndim == 1
    if single:
        a = a[None]
    assert a.shape[-1] == 1 << n
    return a, single


def minors_lu(A, nthreads: int = 0) -> np.ndarray:
    A, single = _mat_batch(A)
    b, n, _ = A.shape
    out = np.empty((b, 1 << n))
    _load().oracle_minors_lu(A.ctypes.data, n, b, out.ctypes.data, nthreads)
    return out[0] if single else out


def perm_ryser(A, absval: bool = False, nthreads: int = 0) -> np.ndarray:
    A, single = _mat_batch(A)
    b, n, _ = A.shape
    out = np.empty((b, 1 << n))
    _load().oracle_perm_ryser(A.ctypes.data, n, b, out.ctypes.data, int(absval), nthreads)
    return out[0] if single else out


def perm_ryser_term_scale(A, nthreads: int = 0) -> np.ndarray:
    """sum_{T subset of S} |prod_{i in S} sum_{j in T} A_ij| for every S: the sum
    of the absolute values of the terms of Ryser's formula (its rounding scale)."""
    A, single = _mat_batch(A)
    b, n, _ = A.shape
    out = np.empty((b, 1 << n))
    _load().oracle_perm_ryser(A.ctypes.data, n, b, out.ctypes.data, 2, nthreads)
    return out[0] if single else out


def minors_scale(A, nthreads: int = 0) -> np.ndarray:
    """perm(|A[S]|) for every S: the sum of the absolute values of all Leibniz
    terms of each principal minor."""
    return perm_ryser(A, absval=True, nthreads=nthreads)


def minors_rowsum_bound(A) -> np.ndarray:
    """prod_{i in S} sum_{j in S} |A_ij| for every S (>= perm(|A[S]|))."""
    A, single = _mat_batch(A)
    b, n, _ = A.shape
    N = 1 << n
    absA = np.abs(A)
    out = np.ones((b, N))
    masks = np.arange(N)
    member = ((masks[:, None] >> np.arange(n)[None, :]) & 1).astype(np.float64)   # (N, n)
    rs = np.einsum("bij,Sj->bSi", absA, member)                                     # (b, N, n)
    rs = np.where(member[None] > 0, rs, 1.0)
    out = np.prod(rs, axis=2)
    return out[0] if single else out


def cdet_recursion(a, nthreads: int = 0) -> np.ndarray:
    a = np.asarray(a)
    n = int(np.log2(a.shape[-1]))
    a, single = _vec_batch(a, n)
    out = np.empty_like(a)
    _load().oracle_cdet_recursion(a.ctypes.data, n, a.shape[0], out.ctypes.data, nthreads)
    return out[0] if single else out


def cdet_scale(ahat, nthreads: int = 0) -> np.ndarray:
    ahat = np.asarray(ahat)
    n = int(np.log2(ahat.shape[-1]))
    ahat, single = _vec_batch(ahat, n)
    out = np.empty_like(ahat)
    _load().oracle_cdet_scale(ahat.ctypes.data, n, ahat.shape[0], out.ctypes.data, nthreads)
    return out[0] if single else out


def cdet_partition(a, nthreads: int = 0) -> np.ndarray:
    a = np.asarray(a)
    n = int(np.log2(a.shape[-1]))
    if n > 12:
        raise ValueError("set-partition route is exponential in Bell numbers; n <= 12")
    a, single = _vec_batch(a, n)
    out = np.empty_like(a)
    _load().oracle_cdet_partition(a.ctypes.data, n, a.shape[0], out.ctypes.data, nthreads)
    return out[0] if single else out


def keldysh(Mt, signed: bool = False, partial: bool = False, nthreads: int = 0):
    """Returns sum (complex, shape (batch,)) and, if partial, the per-depth sums
    (complex, shape (batch, n+1))."""
    Mt, single = _mat_batch(Mt, np.complex128)
    b, n2, _ = Mt.shape
    n = n2 // 2
    s = np.empty((b, 2))
    p = np.empty((b, n + 1, 2)) if partial else None
    _load().oracle_keldysh(Mt.ctypes.data, n, b, int(signed), s.ctypes.data,
                           p.ctypes.data if partial else None, nthreads)
    s = s[:, 0] + 1j * s[:, 1]
    if partial:
        p = p[..., 0] + 1j * p[..., 1]
        return (s[0], p[0]) if single else (s, p)
    return s[0] if single else s


def keldysh_scale(Mt, use_perm: bool | None = None, nthreads: int = 0) -> np.ndarray:
    Mt, single = _mat_batch(Mt, np.complex128)
    b, n2, _ = Mt.shape
    n = n2 // 2
    if use_perm is None:
        use_perm = n <= 10
    out = np.empty(b)
    _load().oracle_keldysh_scale(Mt.ctypes.data, n, b, int(use_perm), out.ctypes.data, nthreads)
    return out[0] if single else out


def _xnor_batch(M):
    M = np.ascontiguousarray(M, dtype=np.float64)
    single = M.ndim == 2
    if single:
        M = M[None]
    assert M.ndim == 3 and M.shape[1] == M.shape[2] and M.shape[1] % 2 == 0, M.shape
    n = M.shape[1] // 2
    assert 1 <= n <= 16, n
    return M, single, n


def xnor_minors(M, nthreads: int = 0) -> np.ndarray:
    """All 2^n XNOR principal minors of 2n x 2n matrices (Section III.B): out[S]
    is the determinant of the rows and columns 2i, 2i+1 of every i in S."""
    M, single, n = _xnor_batch(M)
    out = np.empty((M.shape[0], 1 << n))
    _load().oracle_xnor_minors(M.ctypes.data, n, M.shape[0], out.ctypes.data, nthreads)
    return out[0] if single else out


def xnor_scale(M, use_perm: bool | None = None, nthreads: int = 0) -> np.ndarray:
    """Rounding scale of each XNOR minor: perm(|M[S]|) of the 2|S| x 2|S|
    submatrix (n <= 8 by default), else prod_r sum_q |M_rq| over it."""
    M, single, n = _xnor_batch(M)
    if use_perm is None:
        use_perm = n <= 8
    out = np.empty((M.shape[0], 1 << n))
    _load().oracle_xnor_scale(M.ctypes.data, n, M.shape[0], int(use_perm), out.ctypes.data, nthreads)
    return out[0] if single else out


def nand(M, minors: bool = False, nthreads: int = 0):
    """NAND minors of 2n x 2n matrices (Section III.C). Returns (abar, scale):
    abar[S] = sum over the 2^|S| type assignments of S of the minor keeping row
    and column 2i (type 1) or 2i+1 (type 2) of each i in S; scale[S] the sum of
    the matching row-sum bounds. With minors=True also the 3^n minors, indexed
    by the base-3 digits (vertex i <-> digit i; 0 none, 1 row 2i, 2 row 2i+1)."""
    M, single, n = _xnor_batch(M)
    assert n <= (13 if minors else 16), n
    b = M.shape[0]
    abar = np.empty((b, 1 << n))
    scale = np.empty((b, 1 << n))
    out3 = np.empty((b, 3 ** n)) if minors else None
    _load().oracle_nand(M.ctypes.data, n, b, None if out3 is None else out3.ctypes.data, abar.ctypes.data,
                        scale.ctypes.data, nthreads)
    res = [abar[0] if single else abar, scale[0] if single else scale]
    if minors:
        res.append(out3[0] if single else out3)
    return tuple(res)


def keldysh2(Mu, Md, signed: bool = False, partial: bool = False, nthreads: int = 0):
    """Two-spin Keldysh sum: sum over alpha of det(Mu_alpha) det(Md_alpha);
    returns the complex sums (batch,) and, if partial, the per-depth sums."""
    Mu, single = _mat_batch(Mu, np.complex128)
    Md, _ = _mat_batch(Md, np.complex128)
    assert Mu.shape == Md.shape
    b, n2, _ = Mu.shape
    n = n2 // 2
    s = np.empty((b, 2))
    p = np.empty((b, n + 1, 2)) if partial else None
    _load().oracle_keldysh2(Mu.ctypes.data, Md.ctypes.data, n, b, int(signed), s.ctypes.data,
                            p.ctypes.data if partial else None, nthreads)
    s = s[:, 0] + 1j * s[:, 1]
    if partial:
        p = p[..., 0] + 1j * p[..., 1]
        return (s[0], p[0]) if single else (s, p)
    return s[0] if single else s


def keldysh2_scale(Mu, Md, nthreads: int = 0) -> np.ndarray:
    """Rounding scale of the two-spin sum: sum over alpha of the products of the
    two row-sum bounds."""
    Mu, single = _mat_batch(Mu, np.complex128)
    Md, _ = _mat_batch(Md, np.complex128)
    b, n2, _ = Mu.shape
    out = np.empty(b)
    _load().oracle_keldysh2_scale(Mu.ctypes.data, Md.ctypes.data, n2 // 2, b, out.ctypes.data, nthreads)
    return out[0] if single else out
