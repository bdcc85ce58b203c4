"""Thin Python binding of libapm.so (ctypes). Argument marshalling only.

Every function takes CUDA tensors (torch is used for device memory and the
current stream), checks shapes and dtypes, allocates the outputs with torch and
calls the C ABI declared in include/apm.h with raw device pointers. All
computation happens in the CUDA kernels of the library; there is no CPU or
PyTorch fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

APM_OK, APM_ERR_ARG, APM_ERR_UNSUPPORTED_N, APM_ERR_CUDA, APM_ERR_NUMERIC, APM_ERR_TIMEOUT, \
    APM_ERR_WORKSPACE = range(7)
ST_PIVOT_CORRECTED, ST_NONFINITE_INPUT, ST_ZERO_PIVOT, ST_CORRECTION_OVERFLOW = 1, 2, 4, 8
CDET_SINGLE_DET = 1
KELDYSH_SIGNED = 1
OP_ALL_MINORS, OP_CDET, OP_CDET_FROM_WEIGHTS, OP_PERM_MINORS, OP_CDET_VARLEN, OP_KELDYSH, \
    OP_KELDYSH_VARLEN, OP_XNOR_MINORS, OP_NAMBU_CDET, OP_NAND_MINORS, OP_TWO_TYPE_CDET, OP_KELDYSH2, \
    OP_CDET_FSC = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13
ST_BAD_ORDER = 16


class ApmError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _lib
        msg = lib.apm_status_string(code).decode() if lib is not None else str(code)
        if code == APM_ERR_CUDA and lib is not None:
            msg += f" (cudaError {lib.apm_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libapm.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if _build.needs_build():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libapm.so missing at {path}: the CUDA library was not built")
            L = ctypes.CDLL(path)
            P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
            OPT = ctypes.POINTER(PivotOpts)
            sig = {
                "apm_all_minors": [P, i32, i64, P, OPT, P, P, sz, P],
                "apm_cdet_connected": [P, P, i32, i64, i32, P, P, OPT, P, P, sz, P],
                "apm_cdet_connected_host": [P, P, i32, i64, i32, P, P, OPT, P, i64, i32, P, sz, P],
                "apm_cdet_connected_host_workspace_size": [i32, i64, i32, i32, ctypes.POINTER(sz)],
                "apm_cdet_from_weights": [P, i32, i64, P, P, sz, P],
                "apm_cdet_from_weights_fsc": [P, i32, i64, P, P, sz, P],
                "apm_keldysh_sum": [P, i32, i64, i32, P, P, P, P, sz, P],
                "apm_perm_minors": [P, i32, i64, P, P, sz, P],
                "apm_keldysh_sum_noalloc": [P, i32, i64, i32, P, P, P, P],
                "apm_cdet_connected_varlen": [P, P, P, P, i64, i32, i32, P, P, P, OPT, P, P, sz, P],
                "apm_keldysh_sum_varlen": [P, P, P, i64, i32, i32, P, P, P, P, sz, P],
                "apm_xnor_minors": [P, i32, i64, P, P, P, sz, P],
                "apm_nambu_cdet": [P, i32, i64, P, P, P, P, sz, P],
                "apm_nand_minors": [P, i32, i64, P, OPT, P, P, sz, P],
                "apm_two_type_cdet": [P, i32, i64, P, P, OPT, P, P, sz, P],
                "apm_keldysh2_sum": [P, P, i32, i64, i32, P, P, P, P, sz, P],
                "apm_cdet_tune_set": [P],
                "apm_cdet_tune_get": [i32, ctypes.POINTER(ctypes.c_uint64)],
                "apm_workspace_size": [i32, i32, i64, i32, ctypes.POINTER(sz)],
                "apm_status_reduce": [P, i64, ctypes.POINTER(ctypes.c_uint32), P],
                "apm_fp64_fma_probe": [P, i32, i32, i32, P],
                "apm_order_sums": [P, i32, P, P, i64, i32, P, P],
                "apm_tune_options_set": [i32, i32, i32],
                "apm_tune_options_get": [P, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.apm_status_string.argtypes = [ctypes.c_int]
            L.apm_status_string.restype = ctypes.c_char_p
            L.apm_last_cuda_error.restype = ctypes.c_int
            L.apm_version.restype = ctypes.c_int
            _lib = L
    return _lib


class PivotOpts(ctypes.Structure):
    _fields_ = [("piv_threshold", ctypes.c_double), ("piv_shift", ctypes.c_double)]


def _check(code: int, where: str):
    if code != APM_OK:
        raise ApmError(code, where)


def _stream(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _mat_batch(A: torch.Tensor, dtype=torch.float64, name="A"):
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if A.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if A.dim() == 2:
        A = A.unsqueeze(0)
    if A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError(f"{name} must be (batch, n, n)")
    return A.contiguous()


def _opts(piv_threshold, piv_shift):
    if piv_threshold is None and piv_shift is None:
        return None
    return ctypes.pointer(PivotOpts(1e-4 if piv_threshold is None else piv_threshold,
                                    1.0 if piv_shift is None else piv_shift))


def workspace_size(op: int, n: int, batch: int, two_mats: bool = False) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().apm_workspace_size(op, n, batch, int(two_mats), ctypes.byref(out)),
           "apm_workspace_size")
    return int(out.value)


def _workspace(op, n, batch, device, two_mats=False):
    nb = workspace_size(op, n, batch, two_mats)
    if nb == 0:
        return None, 0
    return torch.empty(nb, dtype=torch.uint8, device=device), nb


def all_minors(A: torch.Tensor, piv_threshold=None, piv_shift=None, return_status=False):
    """All 2^n principal minors of each matrix of A (batch, n, n) float64."""
    A = _mat_batch(A)
    b, n, _ = A.shape
    out = torch.empty((b, 1 << n), dtype=torch.float64, device=A.device)
    st = torch.zeros(b, dtype=torch.int32, device=A.device) if return_status else None
    ws, nb = _workspace(OP_ALL_MINORS, n, b, A.device)
    _check(lib().apm_all_minors(_ptr(A), n, b, _ptr(out), _opts(piv_threshold, piv_shift),
                                _ptr(st), _ptr(ws), nb, _stream(A)), "apm_all_minors")
    return (out, st) if return_status else out


def cdet_connected(A_up: torch.Tensor, A_dn: torch.Tensor | None = None, single_det=False,
                   return_minors=False, return_status=False, piv_threshold=None, piv_shift=None,
                   out_c=None, out_minors=None, workspace=None):
    """Connected sums c[S] (Eq. recursion) of a[S] = det(A_up[S]) det(A_dn[S])
    (A_dn None: det(A_up[S])^2; single_det: det(A_up[S])). out_c / out_minors /
    workspace may pass preallocated tensors."""
    A_up = _mat_batch(A_up, name="A_up")
    b, n, _ = A_up.shape
    if A_dn is not None:
        A_dn = _mat_batch(A_dn, name="A_dn")
        if A_dn.shape != A_up.shape:
            raise ValueError("A_dn must match A_up")
    dev = A_up.device
    c = out_c if out_c is not None else torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    mo = None
    if return_minors or out_minors is not None:
        shape = (b, 2, 1 << n) if A_dn is not None else (b, 1 << n)
        mo = out_minors if out_minors is not None else torch.empty(shape, dtype=torch.float64,
                                                                   device=dev)
        if tuple(mo.shape) != shape or not mo.is_contiguous() or mo.dtype != torch.float64:
            raise ValueError("out_minors has the wrong shape/dtype")
    if tuple(c.shape) != (b, 1 << n) or not c.is_contiguous() or c.dtype != torch.float64:
        raise ValueError("out_c has the wrong shape/dtype")
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    if workspace is not None:
        ws, nb = workspace, workspace.numel()
    else:
        ws, nb = _workspace(OP_CDET, n, b, dev, A_dn is not None)
    flags = CDET_SINGLE_DET if single_det else 0
    _check(lib().apm_cdet_connected(_ptr(A_up), _ptr(A_dn), n, b, flags, _ptr(c), _ptr(mo),
                                    _opts(piv_threshold, piv_shift), _ptr(st), _ptr(ws), nb,
                                    _stream(A_up)), "apm_cdet_connected")
    res = [c]
    if return_minors:
        res.append(mo)
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def _host_mat_batch(A: torch.Tensor, name="A"):
    if not isinstance(A, torch.Tensor) or A.device.type != "cpu":
        raise TypeError(f"{name} must be a CPU (host) tensor")
    if A.dtype != torch.float64:
        raise TypeError(f"{name} must be torch.float64")
    if A.dim() == 2:
        A = A.unsqueeze(0)
    if A.dim() != 3 or A.shape[-1] != A.shape[-2]:
        raise ValueError(f"{name} must be (batch, n, n)")
    return A.contiguous()


def cdet_connected_host_workspace_size(n: int, chunk: int, nstreams: int = 4, two_mats=False) -> int:
    nb = ctypes.c_size_t(0)
    _check(lib().apm_cdet_connected_host_workspace_size(n, chunk, nstreams, 1 if two_mats else 0,
                                                        ctypes.byref(nb)),
           "apm_cdet_connected_host_workspace_size")
    return nb.value


def cdet_connected_host(A_up: torch.Tensor, A_dn: torch.Tensor | None = None, single_det=False,
                        return_minors=False, return_status=False, chunk=2048, nstreams=4, out_c=None,
                        out_minors=None, workspace=None, device=None, piv_threshold=None, piv_shift=None):
    """cdet_connected on matrices in host memory through apm_cdet_connected_host:
    the library copies chunks in, runs the kernels and copies the outputs back
    on its own streams, and returns when the outputs (CPU tensors, page-locked
    when A_up is) are filled. workspace: a uint8 CUDA tensor of at least
    cdet_connected_host_workspace_size bytes, allocated here when None."""
    A_up = _host_mat_batch(A_up, "A_up")
    b, n, _ = A_up.shape
    if A_dn is not None:
        A_dn = _host_mat_batch(A_dn, "A_dn")
        if A_dn.shape != A_up.shape:
            raise ValueError("A_dn must match A_up")
    pin = A_up.is_pinned()
    N = 1 << n

    def host_out(t, shape, dtype, what):
        if t is None:
            return torch.empty(shape, dtype=dtype, pin_memory=pin)
        if t.device.type != "cpu" or tuple(t.shape) != shape or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous CPU tensor {shape} {dtype}")
        return t

    c = host_out(out_c, (b, N), torch.float64, "out_c")
    mo = None
    if return_minors or out_minors is not None:
        mo = host_out(out_minors, (b, 2, N) if A_dn is not None else (b, N), torch.float64, "out_minors")
    st = torch.zeros(b, dtype=torch.int32, pin_memory=pin) if return_status else None
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        if workspace is None:
            nb = cdet_connected_host_workspace_size(n, min(chunk, max(b, 1)), nstreams, A_dn is not None)
            workspace = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        if not workspace.is_cuda or workspace.dtype != torch.uint8:
            raise TypeError("workspace must be a uint8 CUDA tensor")
        flags = CDET_SINGLE_DET if single_det else 0
        _check(lib().apm_cdet_connected_host(_ptr(A_up), _ptr(A_dn), n, b, flags, _ptr(c), _ptr(mo),
                                             _opts(piv_threshold, piv_shift), _ptr(st), chunk, nstreams,
                                             _ptr(workspace), workspace.numel(), _stream(workspace)),
               "apm_cdet_connected_host")
    res = [c]
    if return_minors:
        res.append(mo)
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def cdet_from_weights(a: torch.Tensor):
    """Eq. recursion applied to given weights a (batch, 2^n)."""
    if not a.is_cuda or a.dtype != torch.float64:
        raise TypeError("a must be a CUDA float64 tensor")
    if a.dim() == 1:
        a = a.unsqueeze(0)
    a = a.contiguous()
    b, N = a.shape
    n = N.bit_length() - 1
    if 1 << n != N:
        raise ValueError("last dimension must be 2^n")
    c = torch.empty_like(a)
    ws, nb = _workspace(OP_CDET_FROM_WEIGHTS, n, b, a.device)
    _check(lib().apm_cdet_from_weights(_ptr(a), n, b, _ptr(c), _ptr(ws), nb, _stream(a)),
           "apm_cdet_from_weights")
    return c


def cdet_from_weights_fsc(a: torch.Tensor):
    """The connected sums of cdet_from_weights by the fast subset convolution."""
    if not a.is_cuda or a.dtype != torch.float64:
        raise TypeError("a must be a CUDA float64 tensor")
    if a.dim() == 1:
        a = a.unsqueeze(0)
    a = a.contiguous()
    b, N = a.shape
    n = N.bit_length() - 1
    if 1 << n != N:
        raise ValueError("last dimension must be 2^n")
    c = torch.empty_like(a)
    ws, nb = _workspace(OP_CDET_FSC, n, b, a.device)
    _check(lib().apm_cdet_from_weights_fsc(_ptr(a), n, b, _ptr(c), _ptr(ws), nb, _stream(a)),
           "apm_cdet_from_weights_fsc")
    return c


def keldysh_sum(Mt: torch.Tensor, signed=False, partial=False, return_status=False):
    """Sum over the 2^n Keldysh assignments; Mt (batch, 2n, 2n) complex128."""
    Mt = _mat_batch(Mt, torch.complex128, "Mt")
    b, n2, _ = Mt.shape
    if n2 % 2:
        raise ValueError("Mt must be 2n x 2n")
    n = n2 // 2
    dev = Mt.device
    s = torch.empty((b, 2), dtype=torch.float64, device=dev)
    p = torch.empty((b, n + 1, 2), dtype=torch.float64, device=dev) if partial else None
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_KELDYSH, n, b, dev)
    _check(lib().apm_keldysh_sum(_ptr(Mt), n, b, KELDYSH_SIGNED if signed else 0, _ptr(s), _ptr(p),
                                 _ptr(st), _ptr(ws), nb, _stream(Mt)), "apm_keldysh_sum")
    res = [torch.view_as_complex(s)]
    if partial:
        res.append(torch.view_as_complex(p))
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def _nambu_batch(M: torch.Tensor):
    M = _mat_batch(M, torch.float64, "M")
    b, n2, _ = M.shape
    if n2 % 2:
        raise ValueError("M must be 2n x 2n")
    return M, b, n2 // 2


def xnor_minors(M: torch.Tensor, return_status=False):
    """All 2^n XNOR principal minors (apm_xnor_minors); M (batch, 2n, 2n) float64."""
    M, b, n = _nambu_batch(M)
    dev = M.device
    out = torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_XNOR_MINORS, n, b, dev)
    _check(lib().apm_xnor_minors(_ptr(M), n, b, _ptr(out), _ptr(st), _ptr(ws), nb, _stream(M)),
           "apm_xnor_minors")
    return (out, st) if return_status else out


def nambu_cdet(M: torch.Tensor, return_minors=False, return_status=False):
    """Connected sums c[S] of the Nambu CDet (apm_nambu_cdet): weights = XNOR
    minors of M (batch, 2n, 2n) float64, then the CDet recursion."""
    M, b, n = _nambu_batch(M)
    dev = M.device
    minors = torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    c = torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_NAMBU_CDET, n, b, dev)
    _check(lib().apm_nambu_cdet(_ptr(M), n, b, _ptr(minors), _ptr(c), _ptr(st), _ptr(ws), nb, _stream(M)),
           "apm_nambu_cdet")
    res = [c]
    if return_minors:
        res.append(minors)
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def nand_minors(M: torch.Tensor, return_status=False, piv_threshold=None, piv_shift=None):
    """All 3^n NAND principal minors (apm_nand_minors); M (batch, 2n, 2n) float64;
    index sum_i sigma_i 3^i (0 none, 1 row/column 2i, 2 row/column 2i+1)."""
    M, b, n = _nambu_batch(M)
    dev = M.device
    out = torch.empty((b, 3 ** n), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_NAND_MINORS, n, b, dev)
    _check(lib().apm_nand_minors(_ptr(M), n, b, _ptr(out), _opts(piv_threshold, piv_shift), _ptr(st), _ptr(ws),
                                 nb, _stream(M)),
           "apm_nand_minors")
    return (out, st) if return_status else out


def two_type_cdet(M: torch.Tensor, return_weights=False, return_status=False, piv_threshold=None,
                  piv_shift=None):
    """CDet summed over two vertex types (apm_two_type_cdet): weights abar[S] =
    NAND minors summed over the types of S, then the CDet recursion."""
    M, b, n = _nambu_batch(M)
    dev = M.device
    abar = torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    c = torch.empty((b, 1 << n), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_TWO_TYPE_CDET, n, b, dev)
    _check(lib().apm_two_type_cdet(_ptr(M), n, b, _ptr(abar), _ptr(c), _opts(piv_threshold, piv_shift), _ptr(st),
                                   _ptr(ws), nb, _stream(M)),
           "apm_two_type_cdet")
    res = [c]
    if return_weights:
        res.append(abar)
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def keldysh2_sum(Mu: torch.Tensor, Md: torch.Tensor, signed=False, partial=False, return_status=False):
    """Two-spin Keldysh sum (apm_keldysh2_sum): sum over the shared assignments
    of det(Mu_alpha) det(Md_alpha); Mu, Md (batch, 2n, 2n) complex128."""
    Mu = _mat_batch(Mu, torch.complex128, "Mu")
    Md = _mat_batch(Md, torch.complex128, "Md")
    if Mu.shape != Md.shape or Mu.shape[1] % 2:
        raise ValueError("Mu and Md must both be (batch, 2n, 2n)")
    b, n = Mu.shape[0], Mu.shape[1] // 2
    dev = Mu.device
    s = torch.empty((b, 2), dtype=torch.float64, device=dev)
    p = torch.empty((b, n + 1, 2), dtype=torch.float64, device=dev) if partial else None
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    ws, nb = _workspace(OP_KELDYSH2, n, b, dev)
    _check(lib().apm_keldysh2_sum(_ptr(Mu), _ptr(Md), n, b, KELDYSH_SIGNED if signed else 0, _ptr(s), _ptr(p),
                                  _ptr(st), _ptr(ws), nb, _stream(Mu)), "apm_keldysh2_sum")
    res = [torch.view_as_complex(s)]
    if partial:
        res.append(torch.view_as_complex(p))
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def order_sums(c: torch.Tensor, n: int | None = None, n_arr: torch.Tensor | None = None,
               c_off: torch.Tensor | None = None, n_max: int | None = None) -> torch.Tensor:
    """apm_order_sums: a (n_max+1, 4) float64 device tensor whose row m holds
    (count, sum c, sum |c|, sum c^2) of c_m = c[2^m - 1], the connected sum of
    the whole vertex set, over the rows of order m. c is (batch, 2^n) for a
    fixed order n, or the packed rows of an uneven batch with n_arr (int32) and
    c_off (int64) as in cdet_connected_varlen."""
    if not isinstance(c, torch.Tensor) or not c.is_cuda or c.dtype != torch.float64 or not c.is_contiguous():
        raise TypeError("c must be a contiguous float64 CUDA tensor")
    if n_arr is None:
        if n is None or c.dim() != 2 or c.shape[1] != 1 << n:
            raise ValueError("fixed order: c must be (batch, 2^n)")
        b, n_max = c.shape[0], n if n_max is None else n_max
    else:
        if c_off is None or n_arr.dtype != torch.int32 or c_off.dtype != torch.int64:
            raise TypeError("uneven batch: n_arr int32 and c_off int64")
        b = n_arr.numel()
        n_max = int(n_arr.max()) if n_max is None else n_max
    out = torch.empty((n_max + 1, 4), dtype=torch.float64, device=c.device)
    with torch.cuda.device(c.device):
        _check(lib().apm_order_sums(_ptr(c), 0 if n is None else n, _ptr(n_arr), _ptr(c_off), b, n_max, _ptr(out),
                                    _stream(c)), "apm_order_sums")
    return out


def keldysh_sum_noalloc(Mt: torch.Tensor, signed=False, partial=False, return_status=False):
    """apm_keldysh_sum_noalloc: the Keldysh sum without a caller workspace (the
    library's fixed device array serves as scratch; orders 1..14; calls that
    overlap on the GPU must not share a device)."""
    Mt = _mat_batch(Mt, torch.complex128, "Mt")
    b, n2, _ = Mt.shape
    if n2 % 2:
        raise ValueError("Mt must be 2n x 2n")
    n = n2 // 2
    dev = Mt.device
    s = torch.empty((b, 2), dtype=torch.float64, device=dev)
    p = torch.empty((b, n + 1, 2), dtype=torch.float64, device=dev) if partial else None
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    with torch.cuda.device(dev):   # the library resolves its array on the current device
        _check(lib().apm_keldysh_sum_noalloc(_ptr(Mt), n, b, KELDYSH_SIGNED if signed else 0, _ptr(s),
                                             _ptr(p), _ptr(st), _stream(Mt)), "apm_keldysh_sum_noalloc")
    res = [torch.view_as_complex(s)]
    if partial:
        res.append(torch.view_as_complex(p))
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def varlen_out_offsets(n: torch.Tensor) -> torch.Tensor:
    """Exclusive prefix sum of 2^n (int64): output row offsets of an uneven batch."""
    sizes = torch.ones_like(n, dtype=torch.int64) << n.to(torch.int64)
    return torch.cumsum(sizes, 0) - sizes


def cdet_connected_varlen(A: torch.Tensor, a_off: torch.Tensor, n: torch.Tensor, n_max: int | None = None,
                          A_dn: torch.Tensor | None = None, c_off: torch.Tensor | None = None,
                          single_det=False, return_minors=False, return_status=False,
                          out_c=None, out_minors=None, workspace=None, piv_threshold=None,
                          piv_shift=None):
    """apm_cdet_connected_varlen. A: packed float64 matrices (1-D), a_off: int64
    offsets, n: int32 orders. Returns packed c (and minors/status) with row
    offsets c_off (varlen_out_offsets(n) when not given)."""
    for t, nm in ((A, "A"), (a_off, "a_off"), (n, "n")):
        if not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{nm} must be a contiguous CUDA tensor")
    if A.dtype != torch.float64 or a_off.dtype != torch.int64 or n.dtype != torch.int32:
        raise TypeError("A float64, a_off int64, n int32 expected")
    b = n.numel()
    if n_max is None:
        n_max = int(n.max().item()) if b else 1
    if c_off is None:
        c_off = varlen_out_offsets(n)
    total = int((c_off[-1] + (1 << int(n[-1].item()))).item()) if b else 0
    dev = A.device
    c = out_c if out_c is not None else torch.empty(total, dtype=torch.float64, device=dev)
    mo = None
    if return_minors or out_minors is not None:
        mo = out_minors if out_minors is not None else torch.empty(
            total * (2 if A_dn is not None else 1), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    if workspace is None:
        nb = workspace_size(OP_CDET_VARLEN, n_max, b, A_dn is not None)
        workspace = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
    _check(lib().apm_cdet_connected_varlen(_ptr(A), _ptr(A_dn), _ptr(a_off), _ptr(n), b, n_max,
                                           CDET_SINGLE_DET if single_det else 0, _ptr(c), _ptr(mo),
                                           _ptr(c_off), _opts(piv_threshold, piv_shift), _ptr(st),
                                           _ptr(workspace), workspace.numel(), _stream(A)),
           "apm_cdet_connected_varlen")
    res = [c]
    if return_minors:
        res.append(mo)
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def keldysh_sum_varlen(Mt: torch.Tensor, m_off: torch.Tensor, n: torch.Tensor, n_max: int | None = None,
                       signed=False, partial=False, return_status=False, out_sum=None, out_partial=None,
                       workspace=None):
    """apm_keldysh_sum_varlen. Mt: packed complex128 (1-D), m_off: int64 offsets
    in complex entries, n: int32 orders."""
    if Mt.dtype != torch.complex128 or m_off.dtype != torch.int64 or n.dtype != torch.int32:
        raise TypeError("Mt complex128, m_off int64, n int32 expected")
    b = n.numel()
    if n_max is None:
        n_max = int(n.max().item()) if b else 1
    dev = Mt.device
    s = out_sum if out_sum is not None else torch.empty((b, 2), dtype=torch.float64, device=dev)
    p = None
    if partial or out_partial is not None:
        p = out_partial if out_partial is not None else torch.empty((b, 17, 2), dtype=torch.float64, device=dev)
    st = torch.zeros(b, dtype=torch.int32, device=dev) if return_status else None
    if workspace is None:
        nb = workspace_size(OP_KELDYSH_VARLEN, n_max, b)
        workspace = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
    _check(lib().apm_keldysh_sum_varlen(_ptr(Mt), _ptr(m_off), _ptr(n), b, n_max,
                                        KELDYSH_SIGNED if signed else 0, _ptr(s), _ptr(p), _ptr(st),
                                        _ptr(workspace), workspace.numel(), _stream(Mt)),
           "apm_keldysh_sum_varlen")
    res = [torch.view_as_complex(s)]
    if partial:
        res.append(torch.view_as_complex(p))
    if return_status:
        res.append(st)
    return res[0] if len(res) == 1 else tuple(res)


def tune_set(table):
    """Install per-order lane-group tables (17 packed uint64; 0 = cost model);
    None restores the cost model everywhere."""
    if table is None:
        _check(lib().apm_cdet_tune_set(None), "apm_cdet_tune_set")
        return
    arr = (ctypes.c_uint64 * 17)(*[int(x) for x in table])
    _check(lib().apm_cdet_tune_set(ctypes.cast(arr, ctypes.c_void_p)), "apm_cdet_tune_set")


def tune_get(n: int) -> int:
    out = ctypes.c_uint64(0)
    _check(lib().apm_cdet_tune_get(n, ctypes.byref(out)), "apm_cdet_tune_get")
    return int(out.value)


def tune_options_set(fsc_from_n: int = 0, cdet_ctas_per_sm: int = 0, keldysh_warps: int = 0):
    """apm_tune_options_set: the order from which connected sums take the fast
    subset convolution (13..16, 17 never, 0 default), the resident CTAs per SM
    of the uneven connected-sum batch (1..3, 0 all), and the warps per CTA of
    the uneven Keldysh batch (4..12, 0 default)."""
    _check(lib().apm_tune_options_set(fsc_from_n, cdet_ctas_per_sm, keldysh_warps), "apm_tune_options_set")


def tune_options_get() -> tuple[int, int, int]:
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().apm_tune_options_get(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "apm_tune_options_get")
    return a.value, b.value, c.value


def perm_minors(A: torch.Tensor):
    """All 2^n permanent principal minors of A (batch, n, n) float64."""
    A = _mat_batch(A)
    b, n, _ = A.shape
    out = torch.empty((b, 1 << n), dtype=torch.float64, device=A.device)
    ws, nb = _workspace(OP_PERM_MINORS, n, b, A.device)
    _check(lib().apm_perm_minors(_ptr(A), n, b, _ptr(out), _ptr(ws), nb, _stream(A)),
           "apm_perm_minors")
    return out


def status_reduce(status: torch.Tensor) -> tuple[int, int]:
    """(return code, OR of bits) of a per-matrix status tensor; synchronises."""
    bits = ctypes.c_uint32(0)
    code = lib().apm_status_reduce(_ptr(status), status.numel(), ctypes.byref(bits), _stream(status))
    return code, int(bits.value)


def fp64_probe(blocks: int, threads: int, iters: int, device="cuda") -> torch.Tensor:
    sink = torch.empty(blocks * threads, dtype=torch.float64, device=device)
    _check(lib().apm_fp64_fma_probe(_ptr(sink), blocks, threads, iters, _stream(sink)),
           "apm_fp64_fma_probe")
    return sink
