"""Thin ctypes binding of libtqr (include/tqr.h, include/tqr_debug.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names.  Matrix arguments may be

* torch tensors on a CUDA device (the call is asynchronous on the current
  torch stream),
* torch CPU tensors or NumPy arrays (the library stages them through the GPU
  and synchronizes),

and must be float64 and column-major (``x.stride(0) == 1``; the leading
dimension is taken from ``x.stride(1)``).  ``colmajor(x)`` makes such a copy.

The library is loaded on first use; if it is missing the call raises
RuntimeError (there is no fallback).
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtqr.so")

TQR_OK = 0
TQR_ERR_CUDA = 1
TQR_ERR_NOMEM = 2
TQR_ERR_TIMEOUT = 3
TQR_ERR_RANK = 4
TQR_ERR_NOCONV = 5
TQR_ERR_BUSY = 6
TQR_ERR_UNSUPPORTED = 7
TQR_ERR_TOO_LARGE = 8
TQR_ERR_NONFINITE = 9
TQR_PREC_FP64 = 0
TQR_PREC_FP32 = 1
TQR_LS_PATH_FP64 = 0
TQR_LS_PATH_FP32 = 1
TQR_LS_PATH_FP32_SEMINORMAL = 2
TQR_LS_PATH_FP32_AUGMENTED = 3
TQR_LS_PATH_FP32_GMRES = 4
TQR_LS_PATH_FP64_FALLBACK = 5
LS_PATH_NAMES = {0: "fp64", 1: "fp32", 2: "fp32_seminormal", 3: "fp32_augmented", 4: "fp32_gmres",
                 5: "fp64_fallback"}

_ERRNAMES = {1: "TQR_ERR_CUDA", 2: "TQR_ERR_NOMEM", 3: "TQR_ERR_TIMEOUT", 4: "TQR_ERR_RANK",
             5: "TQR_ERR_NOCONV", 6: "TQR_ERR_BUSY", 7: "TQR_ERR_UNSUPPORTED", 8: "TQR_ERR_TOO_LARGE",
             9: "TQR_ERR_NONFINITE"}

_lib = None


class TqrDesc(ctypes.Structure):
    """tqr_desc of include/tqr.h."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("T", ctypes.c_void_p), ("nb", ctypes.c_int32), ("ib", ctypes.c_int32)]

class TqrLsInfo(ctypes.Structure):
    """tqr_ls_info of include/tqr.h."""
    _fields_ = [("path", ctypes.c_int32), ("iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("fp32_status", ctypes.c_int32), ("berr", ctypes.c_double), ("berr_fp32", ctypes.c_double),
                ("gmres_res", ctypes.c_double), ("r_spread", ctypes.c_double)]

    def as_dict(self):
        return dict(path=LS_PATH_NAMES.get(self.path, str(self.path)), iters=self.iters,
                    inner_iters=self.inner_iters, fp32_status=self.fp32_status, berr=self.berr,
                    berr_fp32=self.berr_fp32, gmres_res=self.gmres_res, r_spread=self.r_spread)


_i64 = ctypes.c_int64
_int = ctypes.c_int
_vp = ctypes.c_void_p
_dbl = ctypes.c_double
_size = ctypes.c_size_t

# name -> (restype, argtypes); every declaration of include/*.h
SIGNATURES = {
    "tqr_version": (ctypes.c_char_p, []),
    "tqr_t_size": (_size, [_i64, _i64, _int, _int]),
    "tqr_work_size": (_size, [_i64, _i64, _int, _int]),
    "tqr_factor": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp]),
    "tqr_factor_ws": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _size, _vp]),
    "tqr_apply_qt": (_int, [ctypes.c_char, _i64, _i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _i64, _vp]),
    "tqr_solve_ls": (_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _int, _dbl, _int,
                            ctypes.POINTER(_int), ctypes.POINTER(_dbl), _int, _int, _vp]),
    "tqr_ls_last_info": (_int, [ctypes.POINTER(TqrLsInfo)]),
    "tqr_ls_factor": (_int, [_i64, _i64, _vp, _i64, _int, _int, _int, _i64, _vp, ctypes.POINTER(_vp)]),
    "tqr_ls_solve": (_int, [_vp, _i64, _vp, _i64, _vp, _i64, _dbl, _int, ctypes.POINTER(TqrLsInfo), _vp]),
    "tqr_ls_release": (_int, [_vp, _vp]),
    "tqr_factor_noalloc": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp]),
    "tqr_autotune": (_int, [_i64, _i64, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "tqr_autotune_run": (_int, [_i64, _i64, _vp]),
    "tqr_autotune_save": (_int, [ctypes.c_char_p]),
    "tqr_autotune_load": (_int, [ctypes.c_char_p]),
    "tqr_autotune_clear": (_int, []),
    "tqr_autotune_batch": (_int, [_int, _vp, _vp, _vp]),
    "tqr_debug_autotune_class": (_int, [_i64, _i64, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "tqr_debug_autotune_put": (_int, [_i64, _i64, _int, _int, _dbl]),
    "tqr_server_create": (_int, [_size, _int, _int, ctypes.POINTER(_vp)]),
    "tqr_server_submit": (_int, [_vp, ctypes.c_uint64, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _int,
                                 _dbl, ctypes.POINTER(ctypes.c_uint64)]),
    "tqr_server_poll": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(_int),
                               ctypes.POINTER(_int), ctypes.POINTER(_dbl), ctypes.POINTER(_dbl),
                               ctypes.POINTER(_int)]),
    "tqr_server_wait": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(_int),
                               ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_int)]),
    "tqr_server_wait_info": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(TqrLsInfo),
                                    ctypes.POINTER(_dbl), ctypes.POINTER(_int)]),
    "tqr_server_stats": (_int, [_vp, _vp]),
    "tqr_server_destroy": (_int, [_vp]),
    "tqr_batch_submit": (_int, [_int, _vp, ctypes.POINTER(ctypes.c_uint64), _vp]),
    "tqr_batch_submit_pairs": (_int, [_int, _vp, ctypes.POINTER(ctypes.c_uint64), _vp]),
    "tqr_batch_poll": (_int, [ctypes.c_uint64, ctypes.POINTER(_int), _vp]),
    "tqr_batch_wait": (_int, [ctypes.c_uint64, _vp]),
    "tqr_t_size_tree": (_size, [_i64, _i64, _int, _int]),
    "tqr_factor_tree": (_int, [_i64, _i64, _vp, _i64, _int, _int, ctypes.POINTER(_int), _vp, _vp]),
    "tqr_apply_qt_tree": (_int, [ctypes.c_char, _i64, _i64, _i64, _vp, _i64, _int, _int, _int, _vp, _vp, _i64, _vp]),
    "tqr_ormqr": (_int, [ctypes.c_char, ctypes.c_char, _i64, _i64, _vp, _i64, _int, _int, _int, _vp, _i64, _i64, _vp,
                         _i64, _vp]),
    "tqr_orgqr": (_int, [_i64, _i64, _vp, _i64, _int, _int, _int, _vp, _i64, _vp, _i64, _vp]),
    "tqr_lu_piv_size": (ctypes.c_size_t, [_i64, _i64, _int]),
    "tqr_release_memory": (_int, []),
    "tqr_factor_pairs": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp]),
    "tqr_apply_qt_pairs": (_int, [ctypes.c_char, _i64, _i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _i64, _vp]),
    "tqr_debug_critical_path": (_int, [_int, _i64, _i64, _int, _int, _int, _int, _int, _int, _vp]),
    "tqr_lu_factor": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _vp]),
    "tqr_lu_solve": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _vp, _i64, _vp]),
    "tqr_lu_factor_pairs": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _vp]),
    "tqr_lu_solve_pairs": (_int, [_i64, _i64, _vp, _i64, _int, _int, _vp, _vp, _vp, _i64, _vp]),
    "tqr_stream_status": (_int, [_vp]),
    "tqr_set_wait_limit_ms": (_i64, [_i64]),
    "tqr_debug_plan": (_i64, [_int, _i64, _i64, _int, _int, _int, _int, _int, _int, _int, _int, _vp, _i64, _vp]),
    "tqr_debug_rules": (_int, [_int, _i64, _i64, _int, _int, _int, _int, _int, _vp, _vp, _vp]),
    "tqr_debug_set_schedule": (_int, [_int, _int]),
    "tqr_debug_stalled_launch": (_int, [_i64, _vp]),
    "tqr_debug_timing": (_int, [_int]),
    "tqr_debug_timing_read": (_int, [ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
    "tqr_debug_fp64_peak": (_int, [ctypes.POINTER(_dbl), _vp]),
    "tqr_debug_trace": (_int, [_vp, _i64]),
    "tqr_debug_set_shape": (_int, [_int, _int]),
    "tqr_debug_last_error": (ctypes.c_char_p, []),
    "tqr_debug_server_last_failure": (_int, [_vp, ctypes.c_char_p, ctypes.c_size_t]),
}


class TqrError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        name = _ERRNAMES.get(code, "invalid argument %d" % -code if code < 0 else str(code))
        super().__init__("%s failed: %s (%d)" % (fn, name, code))


def lib():
    """The loaded libtqr (ctypes.CDLL); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtqr.so is not built (run paper_0707_3548_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------------ marshalling
def _torch():
    import torch
    return torch


def colmajor(x):
    """Column-major float64 copy of a 2-D torch tensor or array (same device)."""
    if isinstance(x, np.ndarray):
        return np.asfortranarray(x, dtype=np.float64)
    torch = _torch()
    x = x.to(torch.float64)
    if x.dim() == 1:
        x = x[:, None]
    return x.t().contiguous().t()


def _mat(x, name):
    """(pointer, rows, cols, ld, is_cuda) of a column-major float64 matrix."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64:
            raise TypeError("%s must be float64" % name)
        if x.ndim == 1:
            return x.ctypes.data, x.shape[0], 1, max(1, x.shape[0]), False
        if not x.flags.f_contiguous and x.shape[1] > 1:
            raise ValueError("%s must be column-major (np.asfortranarray)" % name)
        return x.ctypes.data, x.shape[0], x.shape[1], max(1, x.shape[0]), False
    torch = _torch()
    if x.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    if x.dim() == 1:
        return x.data_ptr(), x.shape[0], 1, max(1, x.shape[0]), x.is_cuda
    if x.shape[0] > 1 and x.stride(0) != 1:
        raise ValueError("%s must be column-major (use tqr.colmajor)" % name)
    ld = x.stride(1) if x.shape[1] > 1 else max(1, x.shape[0])
    return x.data_ptr(), x.shape[0], x.shape[1], ld, x.is_cuda


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(is_cuda, stream=None):
    if stream is not None:
        return stream
    if not is_cuda:
        return None
    return _torch().cuda.current_stream().cuda_stream


def _check(fn, code):
    if code != TQR_OK:
        raise TqrError(fn, code)
    return code


# ------------------------------------------------------------------ API
def tqr_version():
    return lib().tqr_version().decode()


def tqr_t_size(m, n, nb, ib):
    return lib().tqr_t_size(m, n, nb, ib)


def tqr_work_size(m, n, nb, ib):
    return lib().tqr_work_size(m, n, nb, ib)


def new_t(m, n, nb, ib, like):
    """A T buffer (float64, flat) for tqr_factor on the device/host of `like`."""
    cnt = tqr_t_size(m, n, nb, ib) // 8
    if isinstance(like, np.ndarray):
        return np.zeros(cnt)
    return _torch().zeros(cnt, dtype=_torch().float64, device=like.device)


def tqr_factor(A, nb, ib, T=None, stream=None, check=True):
    """Factors column-major A in place; returns T (allocated if not given)."""
    pa, m, n, lda, cuda = _mat(A, "A")
    if T is None:
        T = new_t(m, n, nb, ib, A)
    rc = lib().tqr_factor(m, n, pa, lda, nb, ib, _ptr(T), _stream(cuda, stream))
    if check:
        _check("tqr_factor", rc)
    return T if check else (T, rc)


def tqr_t_size_tree(m, n, nb, ib):
    return lib().tqr_t_size_tree(m, n, nb, ib)


def tqr_factor_tree(A, nb, ib, D=0, T=None, stream=None):
    """Reduction-tree factorization in place; returns (T, D) with the domain
    size used (D = 0 lets the library choose)."""
    pa, m, n, lda, cuda = _mat(A, "A")
    if T is None:
        cnt = tqr_t_size_tree(m, n, nb, ib) // 8
        T = np.zeros(cnt) if isinstance(A, np.ndarray) else _torch().zeros(cnt, dtype=_torch().float64,
                                                                             device=A.device)
    d = _int(D)
    _check("tqr_factor_tree", lib().tqr_factor_tree(m, n, pa, lda, nb, ib, ctypes.byref(d), _ptr(T),
                                                     _stream(cuda, stream)))
    return T, d.value


def tqr_apply_qt_tree(trans, A, nb, ib, D, T, B, stream=None):
    pa, m, n, lda, cuda = _mat(A, "A")
    pb, mb, nrhs, ldb, _ = _mat(B, "B")
    _check("tqr_apply_qt_tree", lib().tqr_apply_qt_tree(trans.encode() if isinstance(trans, str) else trans, m, n,
                                                         nrhs, pa, lda, nb, ib, D, _ptr(T), pb, ldb,
                                                         _stream(cuda, stream)))
    return B


def _ch(c):
    return c.encode() if isinstance(c, str) else c


def tqr_ormqr(side, trans, A, nb, ib, T, C, D=0, stream=None):
    """C <- op(Q) C (side 'L') or C op(Q) (side 'R') in place, for the
    factorization held in (A, nb, ib, T, D); returns C."""
    pa, m, n, lda, cuda = _mat(A, "A")
    pc, mc, nc, ldc, _ = _mat(C, "C")
    _check("tqr_ormqr", lib().tqr_ormqr(_ch(side), _ch(trans), m, n, pa, lda, nb, ib, D, _ptr(T), mc, nc, pc, ldc,
                                        _stream(cuda, stream)))
    return C


def tqr_orgqr(A, nb, ib, T, ncols=None, D=0, Q=None, stream=None):
    """The first ncols columns of Q (default n: the thin Q), written to Q
    (allocated column-major on A's device if not given); returns Q."""
    pa, m, n, lda, cuda = _mat(A, "A")
    if ncols is None:
        ncols = n
    if Q is None:
        if isinstance(A, np.ndarray):
            Q = np.zeros((m, ncols), order="F")
        else:
            Q = colmajor(_torch().zeros((m, ncols), dtype=_torch().float64, device=A.device))
    pq, mq, nq, ldq, _ = _mat(Q, "Q")
    _check("tqr_orgqr", lib().tqr_orgqr(m, n, pa, lda, nb, ib, D, _ptr(T), nq, pq, ldq, _stream(cuda, stream)))
    return Q


def tqr_factor_pairs(A, nb, ib, T=None, stream=None):
    """Tiled QR with 2b x b bottoms (pairs of tile rows), A in place; returns T."""
    pa, m, n, lda, cuda = _mat(A, "A")
    if T is None:
        T = new_t(m, n, nb, ib, A)
    _check("tqr_factor_pairs", lib().tqr_factor_pairs(m, n, pa, lda, nb, ib, _ptr(T), _stream(cuda, stream)))
    return T


def tqr_apply_qt_pairs(trans, A, nb, ib, T, B, stream=None):
    pa, m, n, lda, cuda = _mat(A, "A")
    pb, mb, nrhs, ldb, _ = _mat(B, "B")
    _check("tqr_apply_qt_pairs", lib().tqr_apply_qt_pairs(_ch(trans), m, n, nrhs, pa, lda, nb, ib, _ptr(T), pb, ldb,
                                                           _stream(cuda, stream)))
    return B


def tqr_release_memory():
    """Return the library's cached workspace memory to the driver."""
    _check("tqr_release_memory", lib().tqr_release_memory())


def tqr_lu_piv_size(m, n, nb):
    return lib().tqr_lu_piv_size(m, n, nb)


def tqr_lu_factor(A, nb, ib, L=None, piv=None, stream=None, pairs=False):
    """Tiled LU (pairwise pivoting) of column-major A in place; returns
    (L, piv), allocated on A's device (or host) if not given.  pairs: 2b x b
    bottoms (tqr_lu_factor_pairs)."""
    pa, m, n, lda, cuda = _mat(A, "A")
    if L is None:
        L = new_t(m, n, nb, ib, A)
    if piv is None:
        cnt = tqr_lu_piv_size(m, n, nb) // 4
        piv = np.zeros(cnt, dtype=np.int32) if isinstance(A, np.ndarray) else \
            _torch().zeros(cnt, dtype=_torch().int32, device=A.device)
    fn = "tqr_lu_factor_pairs" if pairs else "tqr_lu_factor"
    _check(fn, getattr(lib(), fn)(m, n, pa, lda, nb, ib, _ptr(L), _ptr(piv), _stream(cuda, stream)))
    return L, piv


def tqr_lu_solve(A, nb, ib, L, piv, B, stream=None, pairs=False):
    """B <- A^-1 B in place from tqr_lu_factor's (A, L, piv); returns B."""
    pa, n, n2, lda, cuda = _mat(A, "A")
    pb, nb_rows, nrhs, ldb, _ = _mat(B, "B")
    fn = "tqr_lu_solve_pairs" if pairs else "tqr_lu_solve"
    _check(fn, getattr(lib(), fn)(n, nrhs, pa, lda, nb, ib, _ptr(L), _ptr(piv), pb, ldb, _stream(cuda, stream)))
    return B


def tqr_factor_noalloc(A, nb, ib, T, stream=None, check=True):
    """tqr_factor with no allocation at all (static device scratch).  A (in
    place) and T must be CUDA tensors; returns the status code."""
    pa, m, n, lda, cuda = _mat(A, "A")
    rc = lib().tqr_factor_noalloc(m, n, pa, lda, nb, ib, _ptr(T), _stream(cuda, stream))
    if check:
        _check("tqr_factor_noalloc", rc)
    return rc


def tqr_autotune(m, n):
    nb = _int(0)
    ib = _int(0)
    _check("tqr_autotune", lib().tqr_autotune(m, n, ctypes.byref(nb), ctypes.byref(ib)))
    return nb.value, ib.value


def tqr_autotune_run(m, n, stream=None):
    """Measure the size class of m x n on the device (no-op if tuned)."""
    _check("tqr_autotune_run", lib().tqr_autotune_run(m, n, _stream(True, stream)))


def tqr_autotune_batch(shapes, stream=None):
    """Tune the tile policy for a batch of (m, n) shapes on the device."""
    ms = np.asarray([m for m, n in shapes], dtype=np.int64)
    ns = np.asarray([n for m, n in shapes], dtype=np.int64)
    _check("tqr_autotune_batch", lib().tqr_autotune_batch(len(shapes), ms.ctypes.data, ns.ctypes.data,
                                                           _stream(True, stream)))


def tqr_autotune_save(path):
    _check("tqr_autotune_save", lib().tqr_autotune_save(os.fsencode(path)))


def tqr_autotune_load(path):
    _check("tqr_autotune_load", lib().tqr_autotune_load(os.fsencode(path)))


def tqr_autotune_clear():
    _check("tqr_autotune_clear", lib().tqr_autotune_clear())


def tqr_debug_autotune_class(m, n):
    a, b = _int(0), _int(0)
    _check("tqr_debug_autotune_class", lib().tqr_debug_autotune_class(m, n, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def tqr_debug_autotune_put(m, n, nb, ib, us=1.0):
    _check("tqr_debug_autotune_put", lib().tqr_debug_autotune_put(m, n, nb, ib, us))


def tqr_batch_submit(mats, Ts, tiles=None, stream=None, pairs=False):
    """Submit column-major CUDA float64 matrices (factored in place) with T
    buffers; tiles: list of (nb, ib) or None for the autotuner; pairs: 2b x b
    bottoms (tqr_batch_submit_pairs).  Returns the ticket."""
    n = len(mats)
    descs = (TqrDesc * n)()
    for a, (A, T) in enumerate(zip(mats, Ts)):
        pa, m, nn, lda, _ = _mat(A, "A")
        nb, ib = tiles[a] if tiles is not None else (0, 0)
        descs[a] = TqrDesc(m, nn, pa, lda, _ptr(T), nb, ib)
    ticket = ctypes.c_uint64(0)
    fn = "tqr_batch_submit_pairs" if pairs else "tqr_batch_submit"
    _check(fn, getattr(lib(), fn)(n, ctypes.cast(descs, _vp), ctypes.byref(ticket), _stream(True, stream)))
    return ticket.value


def tqr_batch_poll(ticket, count):
    done = _int(0)
    st = np.zeros(count, dtype=np.int32)
    rc = lib().tqr_batch_poll(ticket, ctypes.byref(done), st.ctypes.data)
    return bool(done.value), rc, st


def tqr_batch_wait(ticket, count):
    st = np.zeros(count, dtype=np.int32)
    rc = lib().tqr_batch_wait(ticket, st.ctypes.data)
    return rc, st


def tqr_factor_ws(A, nb, ib, T, work, stream=None):
    pa, m, n, lda, cuda = _mat(A, "A")
    nbytes = work.numel() * work.element_size()
    _check("tqr_factor_ws", lib().tqr_factor_ws(m, n, pa, lda, nb, ib, _ptr(T), _ptr(work), nbytes,
                                                 _stream(cuda, stream)))
    return T


def tqr_apply_qt(trans, A, nb, ib, T, B, stream=None):
    """B <- Q^T B ('T') or Q B ('N') in place, from tqr_factor's A and T."""
    pa, m, n, lda, cuda = _mat(A, "A")
    pb, mb, nrhs, ldb, _ = _mat(B, "B")
    if mb != m:
        raise ValueError("B must have m rows")
    _check("tqr_apply_qt", lib().tqr_apply_qt(trans.encode() if isinstance(trans, str) else trans, m, n, nrhs,
                                               pa, lda, nb, ib, _ptr(T), pb, ldb, _stream(cuda, stream)))
    return B


def tqr_solve_ls(A, B, X=None, prec=TQR_PREC_FP64, tol=1e-12, maxit=30, nb=0, ib=0, stream=None, check=True):
    """Least squares min ||A x - b|| per column of B; returns (X, iters, berr, status)."""
    pa, m, n, lda, cuda = _mat(A, "A")
    pb, mb, nrhs, ldb, _ = _mat(B, "B")
    if X is None:
        if isinstance(A, np.ndarray):
            X = np.zeros((n, nrhs), order="F")
        else:
            X = colmajor(_torch().zeros((n, nrhs), dtype=_torch().float64, device=A.device))
    px, _, _, ldx, _ = _mat(X, "X")
    iters = _int(0)
    berr = _dbl(0.0)
    rc = lib().tqr_solve_ls(m, n, nrhs, pa, lda, pb, ldb, px, ldx, prec, tol, maxit, ctypes.byref(iters),
                            ctypes.byref(berr), nb, ib, _stream(cuda, stream))
    if check and rc not in (TQR_OK,):
        raise TqrError("tqr_solve_ls", rc)
    return X, iters.value, berr.value, rc


def tqr_ls_last_info():
    """tqr_ls_info (as a dict) of this thread's last tqr_solve_ls / LsHandle.solve."""
    info = TqrLsInfo()
    _check("tqr_ls_last_info", lib().tqr_ls_last_info(ctypes.byref(info)))
    return info.as_dict()


class LsHandle:
    """A resident least-squares factorization (tqr_ls_factor / tqr_ls_solve /
    tqr_ls_release); A is a CUDA tensor, copied by the library."""

    def __init__(self, A, prec=TQR_PREC_FP64, rhs_cap=16, nb=0, ib=0, stream=None):
        pa, m, n, lda, cuda = _mat(A, "A")
        if not cuda:
            raise ValueError("LsHandle takes device tensors")
        self.m, self.n, self.rhs_cap = m, n, rhs_cap
        h = _vp()
        self.stream = stream
        _check("tqr_ls_factor", lib().tqr_ls_factor(m, n, pa, lda, prec, nb, ib, rhs_cap, _stream(True, stream),
                                                     ctypes.byref(h)))
        self.h = h

    def solve(self, B, X=None, tol=1e-12, maxit=30, check=True):
        """Returns (X, info dict, status)."""
        pb, mb, nrhs, ldb, _ = _mat(B, "B")
        if X is None:
            X = colmajor(_torch().zeros((self.n, nrhs), dtype=_torch().float64, device=B.device))
        px, _, _, ldx, _ = _mat(X, "X")
        info = TqrLsInfo()
        rc = lib().tqr_ls_solve(self.h, nrhs, pb, ldb, px, ldx, tol, maxit, ctypes.byref(info),
                                _stream(True, self.stream))
        if check and rc != TQR_OK:
            raise TqrError("tqr_ls_solve", rc)
        return X, info.as_dict(), rc

    def release(self):
        if self.h:
            _check("tqr_ls_release", lib().tqr_ls_release(self.h, _stream(True, self.stream)))
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def tqr_stream_status(stream=None):
    return lib().tqr_stream_status(_stream(True, stream))


def tqr_set_wait_limit_ms(ms):
    return lib().tqr_set_wait_limit_ms(ms)


# ------------------------------------------------------------------ host-only introspection
def tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs=0, trsm=0, workers=8, policy=-1, D=0):
    """(tasks int32[N, 8], stats float64[6]) of the ordered plan of one launch."""
    L = lib()
    cnt = L.tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs, trsm, D, workers, policy, None, 0, None)
    if cnt < 0:
        raise RuntimeError("tqr_debug_plan: %d %s" % (cnt, L.tqr_debug_last_error().decode()))
    out = np.zeros((cnt, 8), dtype=np.int32)
    stats = np.zeros(6)
    L.tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs, trsm, D, workers, policy, out.ctypes.data, cnt,
                     stats.ctypes.data)
    return out, stats


def tqr_debug_critical_path(mode, m, n, nb, ib, cs, nrhs=0, trsm=0, D=0):
    """(critical path, work) in seconds of the cost model, one-pass estimate."""
    out = np.zeros(2)
    rc = lib().tqr_debug_critical_path(mode, m, n, nb, ib, cs, nrhs, trsm, D, out.ctypes.data)
    if rc != 0:
        raise RuntimeError("tqr_debug_critical_path: %d" % rc)
    return float(out[0]), float(out[1])


def tqr_debug_rules(mode, m, n, nb, ib, cs, nrhs, task, D=0):
    """(waits [(ctr, cnt, ver)], signals [(ctr, cnt)]) of one task."""
    t = np.asarray(list(task) + [0] * (8 - len(task)), dtype=np.int32)
    w = np.zeros(12, dtype=np.int32)
    s = np.zeros(6, dtype=np.int32)
    r = lib().tqr_debug_rules(mode, m, n, nb, ib, cs, nrhs, D, t.ctypes.data, w.ctypes.data, s.ctypes.data)
    nw, ns = r % 16, r // 16
    return [tuple(w[3 * a:3 * a + 3]) for a in range(nw)], [tuple(s[2 * a:2 * a + 2]) for a in range(ns)]


def tqr_debug_set_schedule(policy=-1, max_ctas=0):
    return lib().tqr_debug_set_schedule(policy, max_ctas)


def tqr_debug_set_shape(cs=0, D=-1):
    return lib().tqr_debug_set_shape(cs, D)


def tqr_debug_stalled_launch(limit_ms, stream=None):
    return lib().tqr_debug_stalled_launch(limit_ms, _stream(True, stream))


def tqr_debug_timing(enable):
    return lib().tqr_debug_timing(1 if enable else 0)


def tqr_debug_timing_read():
    """(milliseconds, launches) of the persistent kernel since the last read."""
    ms = _dbl(0)
    n = _i64(0)
    _check("tqr_debug_timing_read", lib().tqr_debug_timing_read(ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def tqr_debug_fp64_peak(stream=None):
    t = _dbl(0)
    _check("tqr_debug_fp64_peak", lib().tqr_debug_fp64_peak(ctypes.byref(t), _stream(True, stream)))
    return t.value


def tqr_debug_trace(buffer):
    """Traces later task-kernel launches into a device int64 tensor of shape
    (capacity, 8) (None stops tracing); decode with trace_records."""
    if buffer is None:
        _check("tqr_debug_trace", lib().tqr_debug_trace(None, 0))
        return
    if (not getattr(buffer, "is_cuda", False) or buffer.dim() != 2 or buffer.shape[1] != 8
            or buffer.element_size() != 8 or not buffer.is_contiguous()):
        raise ValueError("trace buffer must be a contiguous (capacity, 8) 64-bit device tensor")
    _check("tqr_debug_trace", lib().tqr_debug_trace(_vp(buffer.data_ptr()), buffer.shape[0]))


def trace_records(words):
    """Decodes an (n, 8) array of trace words into a dict of columns, keeping
    the rows that were written (nonzero end time)."""
    w = np.asarray(words).astype(np.uint64)
    w = w[w[:, 2] != 0]
    return {
        "ticket_ns": w[:, 0].astype(np.int64), "start_ns": w[:, 1].astype(np.int64),
        "end_ns": w[:, 2].astype(np.int64), "sm": (w[:, 3] & 0xffff).astype(np.int64),
        "kind": ((w[:, 3] >> 16) & 0xffff).astype(np.int64), "inst": (w[:, 3] >> 32).astype(np.int64),
        "k": w[:, 4].astype(np.int64), "i": w[:, 5].astype(np.int64), "j": w[:, 6].astype(np.int64),
        "s": (w[:, 7] & 0xffffffff).astype(np.int64), "l": (w[:, 7] >> 32).astype(np.int64),
    }


TASK_KIND_NAMES = ("GEQRT", "TSQRT", "LARFB", "SSRFB", "LARFB_N", "SSRFB_N", "TRSM_UPD", "TRSM_SOLVE",
                   "TRSMT_UPD", "TRSMT_SOLVE", "TTQRT", "TTMQR", "TTMQR_N", "GETRF", "GESSM", "TSTRF", "SSSSM",
                   "TSQRT2", "SSRFB2", "SSRFB2_N", "TSTRF2", "SSSSM2")


def trace_chrome(words, path=None):
    """Chrome-trace ("traceEvents") form of a task trace: one complete event
    per task on a row of its SM (tasks that overlap on one SM -- its two CTAs
    -- go to separate rows), times in microseconds from the first ticket, the
    task's indices and its dependency wait in args.  Written as JSON to path
    when given; returns the dict."""
    import json

    r = trace_records(words)
    n = len(r["kind"])
    t0 = int(r["ticket_ns"].min()) if n else 0
    rows_end = {}
    events = []
    for a in np.argsort(r["start_ns"], kind="stable"):
        sm, st, en = int(r["sm"][a]), int(r["start_ns"][a]), int(r["end_ns"][a])
        lanes = rows_end.setdefault(sm, [])
        lane = next((x for x, e in enumerate(lanes) if e <= st), len(lanes))
        if lane == len(lanes):
            lanes.append(en)
        else:
            lanes[lane] = en
        kind = int(r["kind"][a])
        events.append({
            "name": TASK_KIND_NAMES[kind] if kind < len(TASK_KIND_NAMES) else str(kind), "ph": "X",
            "ts": (st - t0) / 1e3, "dur": (en - st) / 1e3, "pid": 0, "tid": sm * 4 + lane,
            "args": {"k": int(r["k"][a]), "i": int(r["i"][a]), "j": int(r["j"][a]), "s": int(r["s"][a]),
                     "l": int(r["l"][a]), "inst": int(r["inst"][a]),
                     "wait_us": (st - int(r["ticket_ns"][a])) / 1e3},
        })
    out = {"traceEvents": events, "displayTimeUnit": "ms"}
    if path is not None:
        with open(path, "w") as f:
            json.dump(out, f)
    return out


def trace_summary(words, ctas=None):
    """Per task kind: count, mean / total execution time and mean dependency
    wait (microseconds), plus the launch's span (first ticket to last end)
    and, given the number of CTAs, the fraction of CTA time spent
    executing."""
    r = trace_records(words)
    n = len(r["kind"])
    if n == 0:
        return {"tasks": 0, "span_us": 0.0, "kinds": {}}
    t0 = int(r["ticket_ns"].min())
    span = (int(r["end_ns"].max()) - t0) / 1e3
    ex = (r["end_ns"] - r["start_ns"]) / 1e3
    wt = (r["start_ns"] - r["ticket_ns"]) / 1e3
    kinds = {}
    for k in np.unique(r["kind"]):
        sel = r["kind"] == k
        name = TASK_KIND_NAMES[int(k)] if int(k) < len(TASK_KIND_NAMES) else str(int(k))
        kinds[name] = {"count": int(sel.sum()), "mean_us": float(ex[sel].mean()), "total_us": float(ex[sel].sum()),
                       "mean_wait_us": float(wt[sel].mean())}
    out = {"tasks": n, "span_us": span, "kinds": kinds}
    if ctas:
        out["busy_fraction"] = float(ex.sum() / (span * ctas)) if span > 0 else 0.0
    return out


class Server:
    """Thin wrapper of the tqr_server_* calls (device tensors only)."""

    def __init__(self, budget_bytes, slots=4, grid_cap=0):
        h = _vp()
        _check("tqr_server_create", lib().tqr_server_create(int(budget_bytes), slots, grid_cap, ctypes.byref(h)))
        self.h = h

    def submit(self, matrix_id, A, B, X, prec=TQR_PREC_FP64, tol=1e-12):
        pa, m, n, lda, _ = _mat(A, "A")
        pb, mb, nrhs, ldb, _ = _mat(B, "B")
        px, _, _, ldx, _ = _mat(X, "X")
        r = ctypes.c_uint64(0)
        _check("tqr_server_submit", lib().tqr_server_submit(self.h, matrix_id, m, n, nrhs, pa, lda, pb, ldb, px, ldx,
                                                             prec, tol, ctypes.byref(r)))
        return r.value

    def _out(self):
        return _int(0), _int(0), _dbl(0), _dbl(0), _int(0)

    def poll(self, request):
        done = _int(0)
        st, it, be, lat, ru = self._out()
        rc = lib().tqr_server_poll(self.h, request, ctypes.byref(done), ctypes.byref(st), ctypes.byref(it),
                                   ctypes.byref(be), ctypes.byref(lat), ctypes.byref(ru))
        if rc != 0:
            raise TqrError("tqr_server_poll", rc)
        if not done.value:
            return None
        return dict(status=st.value, iters=it.value, berr=be.value, latency_ms=lat.value, reused=ru.value)

    def wait(self, request):
        st, it, be, lat, ru = self._out()
        rc = lib().tqr_server_wait(self.h, request, ctypes.byref(st), ctypes.byref(it), ctypes.byref(be),
                                   ctypes.byref(lat), ctypes.byref(ru))
        if rc != 0:
            raise TqrError("tqr_server_wait", rc)
        return dict(status=st.value, iters=it.value, berr=be.value, latency_ms=lat.value, reused=ru.value)

    def wait_info(self, request):
        """Blocking; (status, tqr_ls_info dict, latency_ms, reused)."""
        st, lat, ru = _int(0), _dbl(0), _int(0)
        info = TqrLsInfo()
        rc = lib().tqr_server_wait_info(self.h, request, ctypes.byref(st), ctypes.byref(info), ctypes.byref(lat),
                                        ctypes.byref(ru))
        if rc != 0:
            raise TqrError("tqr_server_wait_info", rc)
        return st.value, info.as_dict(), lat.value, ru.value

    def stats(self):
        out = np.zeros(8)
        _check("tqr_server_stats", lib().tqr_server_stats(self.h, out.ctypes.data))
        keys = ("completed", "p50_ms", "p99_ms", "bytes_in_use", "reused", "failed", "queued", "resident")
        return dict(zip(keys, out.tolist()))

    def last_failure(self):
        """Description of the latest failed request ("" if none)."""
        buf = ctypes.create_string_buffer(512)
        _check("tqr_debug_server_last_failure", lib().tqr_debug_server_last_failure(self.h, buf, len(buf)))
        return buf.value.decode()

    def close(self):
        if self.h:
            lib().tqr_server_destroy(self.h)
            self.h = None
