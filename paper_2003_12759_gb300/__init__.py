"""GB300 library for the shifted-solve hot path of projection-based model
order reduction with reused SPAI preconditioners (Singh & Ahuja).

This module is a thin ctypes binding of the C ABI declared in
include/mor_spai.h: the functions below carry the same names and only
marshal arguments (NumPy arrays as host pointers; torch CUDA tensors as
device pointers with MOR_DEVICE_PTRS).  Every step of the path runs in the
CUDA library libmor_spai.so; if it is missing or cannot be loaded, importing
the functions raises -- there is no CPU fallback.

Typical use (one IRKA iteration, Algorithm 2 with the reuse of Algorithm 4):

    import paper_2003_12759_gb300 as mor
    h = mor.mor_create(0)
    mor.mor_set_system(h, A, B, C, E_diag=e)
    shifts, rom, st = mor.mor_irka_step(h, shifts, opts=mor.default_opts())
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmor_spai.so")

# --------------------------------------------------------------------------
# constants (include/mor_spai.h)
# --------------------------------------------------------------------------
MOR_OK, MOR_EINVAL, MOR_ENOMEM, MOR_ECUDA, MOR_ENOCONV, MOR_EBREAKDOWN, MOR_ESINGULAR, MOR_ETIMEOUT, MOR_ESTATE = range(9)
STATUS_NAMES = {0: "MOR_OK", 1: "MOR_EINVAL", 2: "MOR_ENOMEM", 3: "MOR_ECUDA", 4: "MOR_ENOCONV",
                5: "MOR_EBREAKDOWN", 6: "MOR_ESINGULAR", 7: "MOR_ETIMEOUT", 8: "MOR_ESTATE"}
MOR_DEVICE_PTRS = 1
MOR_REAL_VECTORS = 2
MOR_FP64, MOR_MIXED = 0, 1
MOR_BICGSTAB = 0
MOR_GMRES = 1
MOR_BGMRES = 2
MOR_FMT_AUTO, MOR_FMT_CSR, MOR_FMT_SELL, MOR_FMT_DIA = 0, 1, 2, 3
MOR_REUSE_CHAIN, MOR_REUSE_FIRST, MOR_REUSE_AUTO = 0, 1, 2
MOR_MAX_R = 64
MOR_MAX_IO = 8


class mor_c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class mor_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class mor_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("solver", C.c_int), ("tol", C.c_double), ("maxit", C.c_int),
                ("inner_tol", C.c_double), ("max_refine", C.c_int), ("batch", C.c_int), ("use_graph", C.c_int),
                ("graph_chunk", C.c_int), ("precond", C.c_int), ("max_chain", C.c_int), ("restart", C.c_int),
                ("precond_precision", C.c_int), ("fp64_fallback", C.c_int), ("concurrent_sweeps", C.c_int),
                ("reuse", C.c_int), ("moments", C.c_int)]


MOR_MAX_R2 = 32


class mor_reduced2(C.Structure):
    _fields_ = [("r", C.c_int), ("m", C.c_int), ("q", C.c_int), ("alpha", C.c_double), ("beta", C.c_double),
                ("Mr", C.c_double * (MOR_MAX_R2 * MOR_MAX_R2)), ("Kr", C.c_double * (MOR_MAX_R2 * MOR_MAX_R2)),
                ("Fr", C.c_double * (MOR_MAX_R2 * MOR_MAX_IO)), ("Cr", C.c_double * (MOR_MAX_R2 * MOR_MAX_IO))]

    def arrays(self):
        """(M_r, D_r, K_r, F_r, C_r) as NumPy arrays (D_r = alpha M_r + beta K_r)."""
        r, m, q = self.r, self.m, self.q
        Mr = np.ctypeslib.as_array(self.Mr)[: r * r].reshape(r, r, order="F").copy()
        Kr = np.ctypeslib.as_array(self.Kr)[: r * r].reshape(r, r, order="F").copy()
        Fr = np.ctypeslib.as_array(self.Fr)[: r * m].reshape(r, m, order="F").copy()
        Cr = np.ctypeslib.as_array(self.Cr)[: r * q].reshape(r, q, order="F").copy()
        return Mr, self.alpha * Mr + self.beta * Kr, Kr, Fr, Cr


class mor_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("relres", C.c_double), ("status", C.c_int),
                ("fallback", C.c_int)]


class mor_reduced(C.Structure):
    _fields_ = [("r", C.c_int), ("m", C.c_int), ("q", C.c_int),
                ("Ar", C.c_double * (MOR_MAX_R * MOR_MAX_R)), ("Er", C.c_double * (MOR_MAX_R * MOR_MAX_R)),
                ("Br", C.c_double * (MOR_MAX_R * MOR_MAX_IO)), ("Cr", C.c_double * (MOR_MAX_R * MOR_MAX_IO))]

    def arrays(self):
        """(Ar, Er, Br, Cr) as NumPy arrays (column-major storage, leading dimension r)."""
        r, m, q = self.r, self.m, self.q
        Ar = np.ctypeslib.as_array(self.Ar)[: r * r].reshape(r, r, order="F").copy()
        Er = np.ctypeslib.as_array(self.Er)[: r * r].reshape(r, r, order="F").copy()
        Br = np.ctypeslib.as_array(self.Br)[: r * m].reshape(r, m, order="F").copy()
        Cr = np.ctypeslib.as_array(self.Cr)[: r * q].reshape(r, q, order="F").copy()
        return Ar, Er, Br, Cr


class mor_irka_stats(C.Structure):
    _fields_ = [("z", C.c_int), ("nsolve", C.c_int), ("builds_spai", C.c_int), ("builds_reuse", C.c_int),
                ("chain_len", C.c_int), ("iters_V", C.c_int), ("iters_W", C.c_int), ("max_relres", C.c_double),
                ("shift_change", C.c_double), ("ms_precond", C.c_double), ("ms_solve", C.c_double),
                ("ms_orth", C.c_double), ("ms_reduce", C.c_double), ("status", C.c_int), ("fallbacks", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# the exported entry points of include/mor_spai.h with their ctypes signatures
_P = C.c_void_p
SIGNATURES = {
    "mor_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _P]),
    "mor_destroy": (C.c_int, [_P]),
    "mor_last_error": (C.c_char_p, [_P]),
    "mor_default_opts": (None, [C.POINTER(mor_solve_opts)]),
    "mor_set_system": (C.c_int, [_P, C.POINTER(mor_csr), C.POINTER(mor_csr), _P, _P, C.c_int, _P, C.c_int,
                                 C.c_int, C.c_uint]),
    "mor_set_system_2nd": (C.c_int, [_P, C.POINTER(mor_csr), _P, C.c_double, C.c_double, _P, C.c_int, _P,
                                     C.c_int, C.c_int, C.c_uint]),
    "mor_get_io": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mor_get_info": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                               C.POINTER(C.c_int)]),
    "mor_build_precond": (C.c_int, [_P, mor_c64, C.c_int, C.c_int]),
    "mor_update_precond": (C.c_int, [_P, mor_c64, C.c_int]),
    "mor_truncate_precond": (C.c_int, [_P, C.c_int, C.c_int]),
    "mor_chain_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mor_get_factor": (C.c_int, [_P, C.c_int, C.c_int, _P, C.POINTER(mor_c64), C.POINTER(mor_c64)]),
    "mor_get_pattern": (C.c_int, [_P, C.c_int, _P, _P]),
    "mor_apply_operator": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, _P, C.c_uint]),
    "mor_apply_precond": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, C.c_uint]),
    "mor_solve_shifts": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(mor_solve_opts), _P, _P,
                                   C.POINTER(mor_solve_stats), C.c_uint]),
    "mor_orthonormalize": (C.c_int, [_P, _P, C.c_int, C.c_uint]),
    "mor_moment_blocks": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.POINTER(mor_solve_opts), _P, C.c_int, _P,
                                    C.POINTER(mor_solve_stats), C.c_uint]),
    "mor_project": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(mor_reduced), C.c_uint]),
    "mor_reduced_poles": (C.c_int, [_P, C.POINTER(mor_reduced), _P, _P]),
    "mor_irka_step": (C.c_int, [_P, _P, C.c_int, C.POINTER(mor_solve_opts), C.POINTER(mor_reduced),
                                C.POINTER(mor_irka_stats)]),
    "mor_irka_step_tangential": (C.c_int, [_P, _P, _P, _P, C.c_int, C.POINTER(mor_solve_opts), C.POINTER(mor_reduced),
                                            C.POINTER(mor_irka_stats)]),
    "mor_irka_reset": (C.c_int, [_P]),
    "mor_airga_step": (C.c_int, [_P, _P, C.c_int, C.POINTER(mor_solve_opts), C.POINTER(mor_reduced2),
                                 C.POINTER(mor_irka_stats)]),
    "mor_eval_tf2": (C.c_int, [_P, C.POINTER(mor_reduced2), _P, C.c_int, _P, C.c_uint]),
    "mor_eval_tf": (C.c_int, [_P, C.POINTER(mor_reduced), _P, C.c_int, _P, C.c_uint]),
    "mor_launch_count": (C.c_int, [C.POINTER(C.c_int64)]),
    "mor_kernel_tally": (C.c_int, [C.c_int, C.c_int, _P]),
    "mor_time_kernel": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "mor_orthonormalize_noalloc": (C.c_int, [_P, C.c_int64, C.c_int, _P]),
    "mor_set_batch": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int, C.c_uint]),
    "mor_batch_info": (C.c_int, [_P, C.POINTER(C.c_int), _P]),
    "mor_batch_solve": (C.c_int, [_P, _P, C.c_int, C.c_int, C.POINTER(mor_solve_opts), _P,
                                  C.POINTER(mor_solve_stats), C.c_uint]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libmor_spai.so (build it with paper_2003_12759_gb300.build).
    Raises OSError if it is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libmor_spai.so not found at %s; run `python -m paper_2003_12759_gb300.build`" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MorError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


def _check(h, code: int, allow=()):
    if code != MOR_OK and code not in allow:
        msg = load_library().mor_last_error(h)
        raise MorError(code, msg.decode() if msg else "")
    return code


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


_HANDLE_DEVICE = {}        # handle address -> CUDA device it was created on


def _check_cuda_tensor(x, dtype=None, rows=None, device=None):
    """Reject a CUDA tensor whose dtype, device or layout differs from what
    the C side will read through its raw pointer: an n x k block must be
    column-major (stride (1, n); a single column needs only stride(0) == 1),
    a vector contiguous."""
    import torch
    want = {np.dtype(np.float64): torch.float64, np.dtype(np.complex128): torch.complex128,
            np.dtype(np.int32): torch.int32}.get(np.dtype(dtype)) if dtype is not None else None
    if want is not None and x.dtype != want:
        raise ValueError("device tensor has dtype %s, the library reads %s" % (x.dtype, want))
    if device is not None and x.device.index != device:
        raise ValueError("device tensor is on cuda:%s, the handle on cuda:%d" % (x.device.index, device))
    if rows is not None and (x.dim() == 0 or x.shape[0] != rows):
        raise ValueError("device tensor has %s rows, expected %d" % (tuple(x.shape)[:1], rows))
    if x.dim() == 1:
        if x.numel() > 1 and x.stride(0) != 1:
            raise ValueError("device vector must be contiguous")
    elif x.dim() == 2:
        n, k = x.shape
        if (n > 1 and x.stride(0) != 1) or (k > 1 and x.stride(1) != n):
            raise ValueError("device block must be column-major n x k (stride (1, n))")
    else:
        raise ValueError("device tensor must be 1-D or 2-D")


def _ptr(x, dtype=None, fortran=True, rows=None, device=None):
    """(pointer, keep-alive object, is_device) for a NumPy array or torch tensor.
    CUDA tensors are passed by address after a check of dtype, rows, device
    and layout (see _check_cuda_tensor)."""
    if x is None:
        return None, None, False
    if _is_torch(x):
        if x.is_cuda:
            _check_cuda_tensor(x, dtype, rows, device)
            return C.c_void_p(x.data_ptr()), x, True
        x = x.numpy()
    a = np.asarray(x, dtype=dtype)
    a = np.asfortranarray(a) if fortran else np.ascontiguousarray(a)
    return a.ctypes.data_as(C.c_void_p), a, False


def _csr_struct(M):
    """mor_csr from a scipy.sparse matrix (host) or a (n, rowptr, col, val) tuple."""
    if M is None:
        return None, None
    if isinstance(M, tuple):
        n, rowptr, col, val = M
    else:
        import scipy.sparse as sp
        M = sp.csr_matrix(M)
        M.sort_indices()
        n, rowptr, col, val = M.shape[0], M.indptr, M.indices, M.data
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    vl = np.ascontiguousarray(val, dtype=np.float64)
    s = mor_csr(int(n), int(cl.shape[0]), rp.ctypes.data_as(C.c_void_p), cl.ctypes.data_as(C.c_void_p),
                vl.ctypes.data_as(C.c_void_p))
    return s, (rp, cl, vl)


def _shifts(sig):
    s = np.ascontiguousarray(np.asarray(sig, dtype=np.complex128).ravel())
    return s, s.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# --------------------------------------------------------------------------
def mor_default_opts(**kw) -> mor_solve_opts:
    o = mor_solve_opts()
    load_library().mor_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


default_opts = mor_default_opts


def mor_create(device: int = 0, stream=None):
    """Handle on `device`; `stream` may be a torch.cuda.Stream (its cuda_stream
    is used) or an int handle; None lets the library create its own stream."""
    lib = load_library()
    h = C.c_void_p()
    sp_ = None
    if stream is not None:
        sp_ = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    code = lib.mor_create(C.byref(h), int(device), sp_)
    if code != MOR_OK:
        raise MorError(code, "mor_create failed")
    _HANDLE_DEVICE[h.value] = int(device)
    return h


def mor_destroy(h):
    _HANDLE_DEVICE.pop(getattr(h, "value", None), None)
    return load_library().mor_destroy(h)


def _hdev(h):
    return _HANDLE_DEVICE.get(getattr(h, "value", None))


def mor_last_error(h) -> str:
    m = load_library().mor_last_error(h)
    return m.decode() if m else ""


def mor_set_system(h, A, B, C_, E=None, E_diag=None, fmt: int = MOR_FMT_AUTO):
    """First-order system E x' = A x + B u, y = C^T x.  A, E: scipy sparse;
    E_diag: 1-D array; B, C_: n x m / n x q arrays (NumPy or torch CUDA)."""
    lib = load_library()
    As, keepA = _csr_struct(A)
    Es, keepE = _csr_struct(E)
    Bp, Bk, dev = _ptr(np.asarray(B).reshape(As.n, -1) if not _is_torch(B) else B, np.float64, rows=As.n,
                       device=_hdev(h))
    Cp, Ck, devc = _ptr(np.asarray(C_).reshape(As.n, -1) if not _is_torch(C_) else C_, np.float64, rows=As.n,
                        device=_hdev(h))
    Dp, Dk, devd = _ptr(E_diag, np.float64, rows=As.n, device=_hdev(h))
    if dev != devc or (E_diag is not None and devd != dev):
        raise ValueError("B, C and E_diag must all be host arrays or all device tensors")
    m = Bk.shape[1] if Bk.ndim == 2 else 1
    q = Ck.shape[1] if Ck.ndim == 2 else 1
    code = lib.mor_set_system(h, C.byref(As), C.byref(Es) if Es is not None else None, Dp, Bp, m, Cp, q, fmt,
                              MOR_DEVICE_PTRS if dev else 0)
    return _check(h, code)


def mor_set_system_2nd(h, K, M_diag, alpha, beta, F, C_, fmt: int = MOR_FMT_AUTO):
    lib = load_library()
    Ks, keepK = _csr_struct(K)
    Mp, Mk, _ = _ptr(M_diag, np.float64)
    Fp, Fk, dev = _ptr(np.asarray(F).reshape(Ks.n, -1), np.float64)
    Cp, Ck, _ = _ptr(np.asarray(C_).reshape(Ks.n, -1), np.float64)
    code = lib.mor_set_system_2nd(h, C.byref(Ks), Mp, float(alpha), float(beta), Fp, Fk.shape[1], Cp,
                                  Ck.shape[1], fmt, 0)
    return _check(h, code)


def mor_get_info(h):
    n, nnz, fmt, sym = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
    _check(h, load_library().mor_get_info(h, C.byref(n), C.byref(nnz), C.byref(fmt), C.byref(sym)))
    return {"n": n.value, "nnz": nnz.value, "format": fmt.value, "symmetric": bool(sym.value)}


def mor_get_io(h):
    """(m, q): the numbers of inputs and outputs of the system."""
    m, q = C.c_int(), C.c_int()
    _check(h, load_library().mor_get_io(h, C.byref(m), C.byref(q)))
    return m.value, q.value


def mor_build_precond(h, sigma, transpose: int = 0, precision: int = MOR_MIXED, allow=()):
    s = complex(sigma)
    return _check(h, load_library().mor_build_precond(h, mor_c64(s.real, s.imag), int(transpose), int(precision)),
                  allow)


def mor_update_precond(h, sigma_new, transpose: int = 0, allow=()):
    s = complex(sigma_new)
    return _check(h, load_library().mor_update_precond(h, mor_c64(s.real, s.imag), int(transpose)), allow)


def mor_truncate_precond(h, transpose: int, length: int):
    return _check(h, load_library().mor_truncate_precond(h, int(transpose), int(length)))


def mor_chain_info(h, transpose: int = 0):
    L, p = C.c_int(), C.c_int()
    _check(h, load_library().mor_chain_info(h, int(transpose), C.byref(L), C.byref(p)))
    return L.value, p.value


def mor_get_pattern(h, transpose: int = 0):
    info = mor_get_info(h)
    rowptr = np.empty(info["n"] + 1, dtype=np.int32)
    col = np.empty(info["nnz"], dtype=np.int32)
    _check(h, load_library().mor_get_pattern(h, int(transpose), rowptr.ctypes.data_as(C.c_void_p),
                                             col.ctypes.data_as(C.c_void_p)))
    return rowptr, col


def mor_get_factor(h, transpose: int, index: int):
    """(values complex128 in the CSR order of mor_get_pattern, sigma_from, sigma_to)."""
    info = mor_get_info(h)
    vals = np.empty(info["nnz"], dtype=np.complex128)
    sf, st = mor_c64(), mor_c64()
    _check(h, load_library().mor_get_factor(h, int(transpose), int(index), vals.ctypes.data_as(C.c_void_p),
                                            C.byref(sf), C.byref(st)))
    return vals, complex(sf.re, sf.im), complex(st.re, st.im)


def _nk_c128(X, n):
    if _is_torch(X):
        return X
    X = np.asarray(X, dtype=np.complex128)
    if X.ndim == 1:
        X = X.reshape(n, 1)
    return np.asfortranarray(X)


def mor_apply_operator(h, sigma, X, transpose: int = 0, precision: int = MOR_FP64, Y=None, real: bool = False):
    lib = load_library()
    n = mor_get_info(h)["n"]
    s, sp_ = _shifts(sigma)
    Xa = _nk_c128(X, n)
    k = Xa.shape[1]
    if Y is None:
        if _is_torch(Xa) and Xa.is_cuda:
            import torch
            Y = torch.empty((k, n), dtype=torch.complex128, device=Xa.device).T    # column-major n x k
        else:
            Y = np.empty((n, k), dtype=np.complex128, order="F")
    Xp, Xk, dev = _ptr(Xa, np.complex128, rows=n, device=_hdev(h))
    Yp, Yk, devy = _ptr(Y, np.complex128, rows=n, device=_hdev(h))
    if devy != dev:
        raise ValueError("X and Y must both be host arrays or both device tensors")
    if (Yk.shape[1] if Yk.ndim == 2 else 1) != k:
        raise ValueError("Y must have k = %d columns" % k)
    _check(h, lib.mor_apply_operator(h, sp_, k, int(transpose), int(precision), Xp, Yp,
                                     (MOR_DEVICE_PTRS if dev else 0) | (MOR_REAL_VECTORS if real else 0)))
    return Y if _is_torch(Y) else Yk


def mor_apply_precond(h, sigma, X, transpose: int = 0, real: bool = False):
    lib = load_library()
    n = mor_get_info(h)["n"]
    s, sp_ = _shifts(sigma)
    Xa = _nk_c128(X, n)
    k = Xa.shape[1]
    Y = np.empty((n, k), dtype=np.complex128, order="F")
    Xp, Xk, dev = _ptr(Xa, np.complex128, rows=n, device=_hdev(h))
    _check(h, lib.mor_apply_precond(h, sp_, k, int(transpose), Xp, Y.ctypes.data_as(C.c_void_p),
                                    MOR_REAL_VECTORS if real else 0))
    return Y


def mor_solve_shifts(h, sigma, transpose: int = 0, opts: Optional[mor_solve_opts] = None, R=None,
                     allow=(MOR_ENOCONV, MOR_EBREAKDOWN)):
    """Solve A(sigma_c) x_c = r_c (or the transposed systems).  Returns
    (X n x k complex128, list of per-column stats dicts, status)."""
    lib = load_library()
    n = mor_get_info(h)["n"]
    s, sp_ = _shifts(sigma)
    k = s.shape[0]
    o = opts if opts is not None else mor_default_opts()
    Rp, Rk, dev = (None, None, False)
    if R is not None:
        Rp, Rk, dev = _ptr(_nk_c128(R, n), np.complex128, rows=n, device=_hdev(h))
        if (Rk.shape[1] if Rk.ndim == 2 else 1) != k:
            raise ValueError("R must have k = %d columns" % k)
    if dev:
        import torch
        X = torch.empty((k, n), dtype=torch.complex128, device=R.device)   # column-major n x k
        Xp = C.c_void_p(X.data_ptr())
    else:
        X = np.empty((n, k), dtype=np.complex128, order="F")
        Xp = X.ctypes.data_as(C.c_void_p)
    st = (mor_solve_stats * k)()
    code = lib.mor_solve_shifts(h, sp_, k, int(transpose), C.byref(o), Rp, Xp, st, MOR_DEVICE_PTRS if dev else 0)
    _check(h, code, allow)
    stats = [{"iters": x.iters, "refinements": x.refinements, "relres": x.relres, "status": x.status,
              "fallback": x.fallback} for x in st]
    if dev:
        X = X.T
    return X, stats, code


def mor_moment_blocks(h, sigma, J: int, transpose: int = 0, opts: Optional[mor_solve_opts] = None, R=None,
                      allow=(MOR_ENOCONV, MOR_EBREAKDOWN)):
    """Moment blocks X_j(s_i) = A(s_i)^{-1} E X_{j-1}(s_i), X_0 = A(s_i)^{-1} R
    (R = None: B, or C for transpose = 1).  Returns (blocks as a list over
    shifts of lists over j of n x m complex128 arrays, stats, status)."""
    lib = load_library()
    n = mor_get_info(h)["n"]
    s, sp_ = _shifts(sigma)
    l = s.shape[0]
    o = opts if opts is not None else mor_default_opts()
    if R is None:
        m = mor_get_io(h)[1 if transpose else 0]
        Rp, Rk = None, None
    else:
        Rk = np.asfortranarray(np.asarray(R, dtype=np.complex128).reshape(n, -1))
        m = Rk.shape[1]
        Rp = Rk.ctypes.data_as(C.c_void_p)
    X = np.empty((n, l * J * m), dtype=np.complex128, order="F")
    st = (mor_solve_stats * (l * J * m))()
    code = lib.mor_moment_blocks(h, sp_, l, int(J), int(transpose), C.byref(o), Rp, int(m),
                                 X.ctypes.data_as(C.c_void_p), st, 0)
    _check(h, code, allow)
    blocks = [[X[:, (i * J + j) * m:(i * J + j + 1) * m] for j in range(J)] for i in range(l)]
    stats = [{"iters": x.iters, "refinements": x.refinements, "relres": x.relres, "status": x.status,
              "fallback": x.fallback} for x in st]
    return blocks, stats, code


def mor_orthonormalize(h, X):
    lib = load_library()
    Xa = np.asfortranarray(np.asarray(X, dtype=np.float64)).copy(order="F")
    code = lib.mor_orthonormalize(h, Xa.ctypes.data_as(C.c_void_p), Xa.shape[1], 0)
    _check(h, code)
    return Xa


def mor_project(h, V, W):
    lib = load_library()
    Va = np.asfortranarray(np.asarray(V, dtype=np.float64))
    Wa = np.asfortranarray(np.asarray(W, dtype=np.float64))
    rom = mor_reduced()
    _check(h, lib.mor_project(h, Va.ctypes.data_as(C.c_void_p), Wa.ctypes.data_as(C.c_void_p), Va.shape[1],
                              C.byref(rom), 0))
    return rom


def reduced_from_arrays(Ar, Er, Br, Cr) -> mor_reduced:
    rom = mor_reduced()
    r = Ar.shape[0]
    Br = np.asarray(Br, dtype=np.float64).reshape(r, -1)
    Cr = np.asarray(Cr, dtype=np.float64).reshape(r, -1)
    rom.r, rom.m, rom.q = r, Br.shape[1], Cr.shape[1]
    for name, M in (("Ar", Ar), ("Er", Er), ("Br", Br), ("Cr", Cr)):
        flat = np.asarray(M, dtype=np.float64).ravel(order="F")
        getattr(rom, name)[: flat.size] = flat.tolist()
    return rom


def mor_reduced_poles(h, rom: mor_reduced):
    lib = load_library()
    lam = np.empty(rom.r, dtype=np.complex128)
    sh = np.empty(rom.r, dtype=np.complex128)
    _check(h, lib.mor_reduced_poles(h, C.byref(rom), lam.ctypes.data_as(C.c_void_p), sh.ctypes.data_as(C.c_void_p)))
    return lam, sh


def mor_irka_step(h, shifts, opts: Optional[mor_solve_opts] = None, allow=()):
    """One IRKA iteration.  Returns (new shifts, mor_reduced, stats dict)."""
    lib = load_library()
    s = np.ascontiguousarray(np.asarray(shifts, dtype=np.complex128).ravel()).copy()
    rom = mor_reduced()
    st = mor_irka_stats()
    o = opts if opts is not None else mor_default_opts()
    code = lib.mor_irka_step(h, s.ctypes.data_as(C.c_void_p), s.shape[0], C.byref(o), C.byref(rom), C.byref(st))
    _check(h, code, allow)
    return s, rom, st.as_dict()


def mor_irka_step_tangential(h, shifts, btil, ctil, opts: Optional[mor_solve_opts] = None, allow=()):
    """One tangential IRKA iteration (MIMO).  btil: r x m, ctil: r x q
    complex directions, row i for shifts[i].  Returns (new shifts, new btil,
    new ctil, mor_reduced, stats dict)."""
    lib = load_library()
    s = np.ascontiguousarray(np.asarray(shifts, dtype=np.complex128).ravel()).copy()
    r = s.shape[0]
    m, q = mor_get_io(h)
    bt = np.ascontiguousarray(np.asarray(btil, dtype=np.complex128).reshape(r, m)).copy()
    ct = np.ascontiguousarray(np.asarray(ctil, dtype=np.complex128).reshape(r, q)).copy()
    rom = mor_reduced()
    st = mor_irka_stats()
    o = opts if opts is not None else mor_default_opts()
    code = lib.mor_irka_step_tangential(h, s.ctypes.data_as(C.c_void_p), bt.ctypes.data_as(C.c_void_p),
                                        ct.ctypes.data_as(C.c_void_p), r, C.byref(o), C.byref(rom), C.byref(st))
    _check(h, code, allow)
    return s, bt, ct, rom, st.as_dict()


def mor_airga_step(h, points, opts: Optional[mor_solve_opts] = None, allow=()):
    """One second-order reduction iteration (mor_set_system_2nd systems).
    Returns (new points, mor_reduced2, stats dict)."""
    lib = load_library()
    p = np.ascontiguousarray(np.asarray(points, dtype=np.complex128).ravel()).copy()
    rom = mor_reduced2()
    st = mor_irka_stats()
    o = opts if opts is not None else mor_default_opts()
    code = lib.mor_airga_step(h, p.ctypes.data_as(C.c_void_p), p.shape[0], C.byref(o), C.byref(rom), C.byref(st))
    _check(h, code, allow)
    return p, rom, st.as_dict()


def mor_eval_tf2(h, rom: mor_reduced2, omega):
    """H_r(i omega) of a reduced second-order system: nw x q x m (complex128)."""
    lib = load_library()
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).ravel())
    nw = w.shape[0]
    H = np.empty(nw * rom.q * rom.m, dtype=np.complex128)
    _check(h, lib.mor_eval_tf2(h, C.byref(rom), w.ctypes.data_as(C.c_void_p), nw, H.ctypes.data_as(C.c_void_p), 0))
    return H.reshape((nw, rom.q, rom.m), order="F")


def mor_irka_reset(h):
    return _check(h, load_library().mor_irka_reset(h))


def mor_eval_tf(h, rom: mor_reduced, omega):
    """H_r(i omega) for each omega: array nw x q x m (complex128)."""
    lib = load_library()
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).ravel())
    nw = w.shape[0]
    H = np.empty(nw * rom.q * rom.m, dtype=np.complex128)
    _check(h, lib.mor_eval_tf(h, C.byref(rom), w.ctypes.data_as(C.c_void_p), nw, H.ctypes.data_as(C.c_void_p), 0))
    return H.reshape((nw, rom.q, rom.m), order="F")


def mor_launch_count() -> int:
    c = C.c_int64()
    load_library().mor_launch_count(C.byref(c))
    return c.value


VEC_F32, VEC_F64, VEC_C64, VEC_C128 = 0, 1, 2, 3


def mor_kernel_tally(which: int, vec_type: int):
    """Launches of the operator (which = 0) or factor (1) SpMV since the
    process started, by number of real shift columns: array of 17 counts."""
    out = np.zeros(17, dtype=np.int64)
    code = load_library().mor_kernel_tally(int(which), int(vec_type), out.ctypes.data_as(C.c_void_p))
    if code != MOR_OK:
        raise MorError(code, "mor_kernel_tally")
    return out


def mor_time_kernel(h, which: int, sigma, precision: int = MOR_MIXED, reps: int = 20) -> float:
    """Mean duration (ms) of one hot-loop kernel launch (0 operator SpMV,
    1 preconditioner-factor SpMV) over k = len(sigma) columns, CUDA events on
    the handle's stream."""
    s, sp_ = _shifts(sigma)
    ms = C.c_double()
    _check(h, load_library().mor_time_kernel(h, int(which), sp_, s.shape[0], int(precision), int(reps),
                                             C.byref(ms)))
    return ms.value


def mor_orthonormalize_noalloc(X, stream=None) -> int:
    """Allocation-free two-pass Gram-Schmidt of a CUDA tensor X (n x k FP64,
    column-major storage, i.e. X.t() contiguous / X with stride (1, n)), in
    place on the current device.  Returns the status code (MOR_OK on success)."""
    if not _is_torch(X) or not X.is_cuda:
        raise ValueError("X must be a CUDA tensor")
    import torch
    if X.dim() != 2:
        raise ValueError("X must be an n x k tensor")
    n, k = X.shape
    # the C side works on the current device and reads n x k FP64, column-major
    _check_cuda_tensor(X, np.float64, rows=n, device=torch.cuda.current_device())
    sp_ = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    return load_library().mor_orthonormalize_noalloc(C.c_void_p(X.data_ptr()), int(n), int(k), sp_)


def mor_set_batch(h, As, Bs, Cs, E_diags=None, fmt: int = MOR_FMT_AUTO):
    """A batch of independent SISO systems (lists of scipy.sparse A_s and
    length-n_s vectors b_s, c_s, optional E_s diagonals)."""
    lib = load_library()
    nsys = len(As)
    structs = (mor_csr * nsys)()
    keep = []
    for i, A in enumerate(As):
        st, kp = _csr_struct(A)
        structs[i] = st
        keep.append(kp)
    def ptrs(vs):
        if vs is None:
            return None, None
        arrs = [None if v is None else np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel()) for v in vs]
        P = (C.c_void_p * nsys)(*[None if a is None else a.ctypes.data for a in arrs])
        return P, arrs
    Bp, Bk = ptrs(Bs)
    Cp, Ck = ptrs(Cs)
    Ep, Ek = ptrs(E_diags)
    code = lib.mor_set_batch(h, nsys, structs, Ep, Bp, Cp, fmt, 0)
    return _check(h, code)


def mor_batch_info(h):
    n = C.c_int()
    _check(h, load_library().mor_batch_info(h, C.byref(n), None))
    off = np.empty(n.value + 1, dtype=np.int64)
    _check(h, load_library().mor_batch_info(h, C.byref(n), off.ctypes.data_as(C.c_void_p)))
    return n.value, off


def mor_batch_solve(h, sigma, transpose: int = 0, opts: Optional[mor_solve_opts] = None,
                    allow=(MOR_ENOCONV, MOR_EBREAKDOWN)):
    """Solve every (system, shift) pair of the batch.  Returns (X N x k
    complex128, stats as an nsys x k list of dicts, status)."""
    lib = load_library()
    nsys, off = mor_batch_info(h)
    N = int(off[-1])
    s, sp_ = _shifts(sigma)
    k = s.shape[0]
    o = opts if opts is not None else mor_default_opts()
    X = np.empty((N, k), dtype=np.complex128, order="F")
    st = (mor_solve_stats * (nsys * k))()
    code = lib.mor_batch_solve(h, sp_, k, int(transpose), C.byref(o), X.ctypes.data_as(C.c_void_p), st, 0)
    _check(h, code, allow)
    stats = [[{"iters": st[i * k + c].iters, "refinements": st[i * k + c].refinements,
               "relres": st[i * k + c].relres, "status": st[i * k + c].status,
               "fallback": st[i * k + c].fallback} for c in range(k)]
             for i in range(nsys)]
    return X, stats, code
