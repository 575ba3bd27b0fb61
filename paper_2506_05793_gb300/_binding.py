"""ctypes binding of include/mfchol.h -- argument marshalling only.

Every function has the name of the C entry point it calls.  Host arrays are
numpy arrays; device arrays are torch CUDA tensors (torch is used only for
device memory and streams).  Matrices of right-hand sides are column-major:
numpy arrays are converted with ``np.asfortranarray``; device tensors must
have unit row stride (e.g. the transpose of a contiguous (nrhs, n) tensor).

The library must be built (``paper_2506_05793_gb300.build.build()``); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

MF_OK, MF_ERR_INVALID, MF_ERR_NOT_SPD, MF_ERR_OOM, MF_ERR_CUDA, MF_ERR_TIMEOUT, \
    MF_ERR_STAGNATION, MF_ERR_INTERNAL = range(8)
MF_FP64, MF_FP32 = 0, 1
FACTOR_KINDS = ("small_front", "assemble", "potrf", "trsm", "syrk", "syrk_tc")

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


class mf_options(ctypes.Structure):
    _fields_ = [("small_front_max", _I32), ("use_graphs", _I32), ("profile", _I32),
                ("relax", _I32), ("budget_bytes", _I64), ("tc", _I32), ("sptrsv", _I32),
                ("small_queue", _I32), ("update_tile", _I32 * 4)]


class mf_symbolic_info(ctypes.Structure):
    _fields_ = [("n", _I64), ("nnz_lower", _I64), ("nsuper", _I64), ("nnz_L", _I64),
                ("flops", _D), ("nlevels", _I64), ("max_front", _I64), ("max_k", _I64),
                ("factor_bytes_fp64", _I64), ("factor_bytes_fp32", _I64), ("nfronts", _I64),
                ("front_flops", _D), ("queued_fronts", _I64)]


class mf_ir_report(ctypes.Structure):
    _fields_ = [("iterations", _I32), ("fell_back", _I32), ("berr", _D), ("berr_first", _D)]


class mf_server_stats(ctypes.Structure):
    _fields_ = [("completed", _I64), ("failed", _I64), ("p50_ms", _D), ("p99_ms", _D),
                ("mean_ms", _D), ("solves_per_s", _D), ("resident_bytes", _I64),
                ("peak_resident_bytes", _I64)]


class MFError(RuntimeError):
    def __init__(self, code, msg, column=-1):
        super().__init__("mfchol error %d: %s" % (code, msg))
        self.code = code
        self.column = column


_lib = None

_SIGS = {
    "mf_options_default": [_P],
    "mf_create": [_P, _P],
    "mf_destroy": [_P],
    "mf_symbolic_analyze": [_P, _I64, _P, _P, _P, _P],
    "mf_symbolic_analyze_batch": [_P, _I32, _P, _P, _P, _P, _P],
    "mf_symbolic_analyze_condensed": [_P, _I64, _P, _P, _P, _P, _I32, _P],
    "mf_symbolic_save": [_P, ctypes.c_char_p],
    "mf_symbolic_check": [_P],
    "mf_symbolic_load": [_P, ctypes.c_char_p, _P],
    "mf_symbolic_free": [_P],
    "mf_symbolic_get_info": [_P, _P],
    "mf_symbolic_etree": [_P, _P],
    "mf_symbolic_colcounts": [_P, _P],
    "mf_symbolic_supernodes": [_P, _P],
    "mf_symbolic_pattern": [_P, _P, _P],
    "mf_symbolic_supernode_tree": [_P, _P, _P],
    "mf_factor_create": [_P, _P, _I32, _P],
    "mf_factor_numeric": [_P, _P, _I32, _P, _I32],
    "mf_factor_check": [_P, _P],
    "mf_factor_free": [_P],
    "mf_factor_export_L": [_P, _P],
    "mf_factor_launch_counts": [_P, _P, _P],
    "mf_factor_profile": [_P, _P, _P, _P],
    "mf_solve": [_P, _I32, _P, _I64, _P, _I64, _I32, _P],
    "mf_solve_refined": [_P, _I32, _P, _I64, _P, _I64, _I32, _D, _I32, _I32, _P, _P],
    "mf_solve_noalloc": [_P, _I32, _P, _I64, _P, _I64, _P],
    "mf_autotune": [_P, _I64, _P, _P, _P, _P, _I32, _I32, _I32, _P, _P],
    "mf_server_create": [_P, _I32, _I64, _P],
    "mf_server_submit_factor": [_P, _P, _P, _I32, _I32, _P, _I64, _P, _I64, _P, _P],
    "mf_server_submit_solve": [_P, _I64, _I32, _P, _I64, _P, _I64, _P],
    "mf_server_poll": [_P, _I64, _P, _P, _P],
    "mf_server_wait": [_P, _I64, _P, _P],
    "mf_server_release_factor": [_P, _I64],
    "mf_server_get_stats": [_P, _P],
    "mf_server_free": [_P],
    "mf_diag_wait_timeout": [_I32, _P],
    "mf_solve_check": [_P, _P],
    "mf_factor_export_columns": [_P, _I64, _I64, _P],
    "mf_diag_fp64_peak": [_I32, _P, _P],
    "mf_diag_small_queue": [_P, _I32, _P],
    "mf_symbolic_options": [_P, _P],
    "mf_factor_create_ldlt": [_P, _P, _I32, _P],
    "mf_factor_export_D": [_P, _P],
    "mf_factor_create_lu": [_P, _P, _I32, _I32, _P],
    "mf_factor_create_ldlt_piv": [_P, _P, _I32, _P],
    "mf_factor_export_U": [_P, _P],
    "mf_factor_export_pivots": [_P, _P],
    "mf_symbolic_fronts": [_P, _P],
    "mf_factor_kind_items": [_P, _P, _P],
    "mf_ilu_symbolic": [_P, _I64, _P, _P, _I32, _P],
    "mf_ilu_info": [_P, _P, _P],
    "mf_ilu_pattern": [_P, _P, _P, _P],
    "mf_ilu_numeric": [_P, _P, _I32, _I32, _D, _D, _I32, _I32, _P],
    "mf_ilu_export": [_P, _P],
    "mf_ilu_trsv": [_P, _I32, _I32, _D, _P, _P, _I32, _P],
    "mf_ilu_apply": [_P, _I32, _D, _P, _P, _I32, _P],
    "mf_ilu_free": [_P],
    "mf_factor_set_wait_limit": [_P, _I32],
    "mf_factor_solve_work_bytes": [_P, _P],
}


def lib():
    """Load libmfchol.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libmfchol.so is not built (%s); run __graft_entry__.build()" % LIB)
        L = ctypes.CDLL(LIB)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.mf_last_error_string.restype = ctypes.c_char_p
        L.mf_last_error_string.argtypes = []
        L.mf_last_error_column.restype = _I64
        L.mf_last_error_column.argtypes = []
        _lib = L
    return _lib


def _check(rc):
    if rc != MF_OK:
        L = lib()
        raise MFError(rc, L.mf_last_error_string().decode(), int(L.mf_last_error_column()))


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _is_device(a):
    return hasattr(a, "is_cuda") and a.is_cuda


# ---------------------------------------------------------------------------
def mf_options_default():
    o = mf_options()
    _check(lib().mf_options_default(ctypes.byref(o)))
    return o


def mf_create(opt=None):
    h = ctypes.c_void_p()
    _check(lib().mf_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None))
    return h


def mf_destroy(h):
    _check(lib().mf_destroy(h))


def mf_symbolic_analyze(h, rowptr, colind, perm=None):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    s = ctypes.c_void_p()
    _check(lib().mf_symbolic_analyze(h, len(rowptr) - 1, _ptr(rowptr), _ptr(colind), _ptr(perm),
                                     ctypes.byref(s)))
    return s


def mf_symbolic_analyze_condensed(h, rowptr, colind, perm=None, node_of=None, block=1):
    """Symbolic analysis on the condensed (node) graph: node_of[i] is the node
    of DoF i, else fixed blocks of `block` consecutive DoFs."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    node_of = None if node_of is None else np.ascontiguousarray(node_of, dtype=np.int32)
    s = ctypes.c_void_p()
    _check(lib().mf_symbolic_analyze_condensed(h, len(rowptr) - 1, _ptr(rowptr), _ptr(colind),
                                               _ptr(perm), _ptr(node_of), int(block),
                                               ctypes.byref(s)))
    return s


def mf_symbolic_check(s):
    _check(lib().mf_symbolic_check(s))


def mf_symbolic_save(s, path):
    _check(lib().mf_symbolic_save(s, os.fsencode(path)))


def mf_symbolic_load(h, path):
    s = ctypes.c_void_p()
    _check(lib().mf_symbolic_load(h, os.fsencode(path), ctypes.byref(s)))
    return s


def mf_symbolic_analyze_batch(h, mats):
    """mats: list of (rowptr, colind, perm or None)."""
    keep = []
    ns = np.array([len(m[0]) - 1 for m in mats], dtype=np.int64)
    rps = (ctypes.c_void_p * len(mats))()
    cis = (ctypes.c_void_p * len(mats))()
    pms = (ctypes.c_void_p * len(mats))()
    for b, (rp, ci, pm) in enumerate(mats):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        keep += [rp, ci]
        rps[b] = rp.ctypes.data
        cis[b] = ci.ctypes.data
        if pm is not None:
            pm = np.ascontiguousarray(pm, dtype=np.int32)
            keep.append(pm)
            pms[b] = pm.ctypes.data
        else:
            pms[b] = None
    s = ctypes.c_void_p()
    _check(lib().mf_symbolic_analyze_batch(h, len(mats), _ptr(ns), rps, cis, pms, ctypes.byref(s)))
    return s


def mf_symbolic_free(s):
    _check(lib().mf_symbolic_free(s))


def mf_symbolic_get_info(s):
    info = mf_symbolic_info()
    _check(lib().mf_symbolic_get_info(s, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in mf_symbolic_info._fields_}


def mf_symbolic_etree(s):
    n = mf_symbolic_get_info(s)["n"]
    out = np.empty(n, dtype=np.int32)
    _check(lib().mf_symbolic_etree(s, _ptr(out)))
    return out


def mf_symbolic_colcounts(s):
    n = mf_symbolic_get_info(s)["n"]
    out = np.empty(n, dtype=np.int64)
    _check(lib().mf_symbolic_colcounts(s, _ptr(out)))
    return out


def mf_symbolic_supernodes(s):
    ns = mf_symbolic_get_info(s)["nsuper"]
    out = np.empty(ns + 1, dtype=np.int32)
    _check(lib().mf_symbolic_supernodes(s, _ptr(out)))
    return out


def mf_symbolic_pattern(s):
    info = mf_symbolic_get_info(s)
    Lp = np.empty(info["n"] + 1, dtype=np.int64)
    Li = np.empty(info["nnz_L"], dtype=np.int32)
    _check(lib().mf_symbolic_pattern(s, _ptr(Lp), _ptr(Li)))
    return Lp, Li


def mf_symbolic_supernode_tree(s):
    ns = mf_symbolic_get_info(s)["nsuper"]
    par = np.empty(ns, dtype=np.int32)
    lev = np.empty(ns, dtype=np.int32)
    _check(lib().mf_symbolic_supernode_tree(s, _ptr(par), _ptr(lev)))
    return par, lev


def mf_autotune(h, rowptr, colind, perm, values, prec=MF_FP64, reps=2):
    """Fastest options for this matrix (see the C header).  Returns (mf_options, ms)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    dev = _is_device(values)
    if not dev:
        values = np.ascontiguousarray(values, dtype=np.float64)
    best = mf_options()
    ms = ctypes.c_double()
    _check(lib().mf_autotune(h, len(rowptr) - 1, _ptr(rowptr), _ptr(colind), _ptr(perm),
                             _ptr(values), 1 if dev else 0, prec, reps, ctypes.byref(best),
                             ctypes.byref(ms)))
    return best, ms.value


def mf_factor_create(h, s, prec=MF_FP64):
    f = ctypes.c_void_p()
    _check(lib().mf_factor_create(h, s, prec, ctypes.byref(f)))
    return f


def mf_factor_numeric(f, values, stream=None, async_=False):
    """values: float64 numpy array (host) or torch CUDA tensor (device)."""
    dev = _is_device(values)
    if not dev:
        values = np.ascontiguousarray(values, dtype=np.float64)
    _check(lib().mf_factor_numeric(f, _ptr(values), 1 if dev else 0, _stream(stream),
                                   1 if async_ else 0))


def mf_factor_check(f, stream=None):
    _check(lib().mf_factor_check(f, _stream(stream)))


def mf_factor_free(f):
    _check(lib().mf_factor_free(f))


def mf_factor_set_wait_limit(f, polls):
    """Bound of the solve's flag waits on f in polls (0: the default)."""
    _check(lib().mf_factor_set_wait_limit(f, polls))


def mf_factor_solve_work_bytes(f):
    out = _I64(0)
    _check(lib().mf_factor_solve_work_bytes(f, ctypes.byref(out)))
    return int(out.value)


def mf_solve_check(f, stream=None):
    """Wait for ``stream`` and raise MFError(MF_ERR_TIMEOUT) if a bounded wait
    of the last solve call on f gave up."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    _check(lib().mf_solve_check(f, _stream(stream)))


def mf_factor_export_L(f, nnz_L):
    out = np.empty(nnz_L, dtype=np.float64)
    _check(lib().mf_factor_export_L(f, _ptr(out)))
    return out


def mf_factor_export_columns(f, j0, j1, count):
    """Values of columns j0..j1-1 of L (``count`` = sum of their column counts)."""
    out = np.empty(count, dtype=np.float64)
    _check(lib().mf_factor_export_columns(f, j0, j1, _ptr(out)))
    return out


def mf_factor_launch_counts(f):
    a, b = _I64(), _I64()
    _check(lib().mf_factor_launch_counts(f, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mf_factor_profile(f):
    ms = np.zeros(6)
    n = np.zeros(6, dtype=np.int64)
    fl = np.zeros(6)
    _check(lib().mf_factor_profile(f, _ptr(ms), _ptr(n), _ptr(fl)))
    return {k: {"ms": float(ms[i]), "launches": int(n[i]), "flops": float(fl[i])}
            for i, k in enumerate(FACTOR_KINDS)}


def mf_diag_wait_timeout(polls=1 << 14, stream=None):
    """Run the solve's bounded device wait on a flag nothing sets; returns the
    status code (MF_ERR_TIMEOUT expected) instead of raising."""
    return int(lib().mf_diag_wait_timeout(polls, _stream(stream)))


def mf_diag_small_queue(f, skip, stream=None):
    """Run f's small-front queue with its first ``skip`` tickets skipped;
    returns the status code (MF_ERR_TIMEOUT expected) instead of raising."""
    return int(lib().mf_diag_small_queue(f, skip, _stream(stream)))


def mf_diag_fp64_peak(kind, stream=None):
    """Measured FP64 peak in TFLOP/s: kind 0 DFMA loop, 1 DMMA loop."""
    out = _D(0.0)
    _check(lib().mf_diag_fp64_peak(kind, _stream(stream), ctypes.byref(out)))
    return float(out.value)


def _rhs_layout(B):
    """(pointer holder, nrhs, ld, on_device, one_dim) for a column-major RHS."""
    if _is_device(B):
        if B.dim() == 1:
            return B, 1, B.shape[0], 1, True
        if B.stride(0) != 1:
            raise ValueError("device RHS must be column-major (unit row stride)")
        return B, B.shape[1], B.stride(1) if B.shape[1] > 1 else B.shape[0], 1, False
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        return np.ascontiguousarray(B), 1, B.shape[0], 0, True
    B = np.asfortranarray(B)
    return B, B.shape[1], B.shape[0], 0, False


def _alloc_like(B, on_dev):
    if on_dev:
        import torch
        if B.dim() == 1:
            return torch.empty_like(B)
        return torch.empty((B.shape[1], B.shape[0]), dtype=B.dtype, device=B.device).t()
    return np.empty_like(B, order="F")


def mf_solve(f, B, X=None, stream=None):
    """X = A^{-1} B.  Returns X (allocated like B if not given)."""
    Bh, nrhs, ldb, dev, _ = _rhs_layout(B)
    if X is None:
        X = _alloc_like(Bh, dev)
    Xh, _, ldx, _, _ = _rhs_layout(X)
    if dev and stream is None:
        import torch
        stream = torch.cuda.current_stream()
    _check(lib().mf_solve(f, nrhs, _ptr(Bh), ldb, _ptr(Xh), ldx, dev, _stream(stream)))
    return Xh


def mf_solve_noalloc(f, B, X, stream=None):
    """X = A^{-1} B with device tensors B, X and no allocation (see the C
    header); enqueued on ``stream`` (default: torch's current stream)."""
    Bh, nrhs, ldb, dev, _ = _rhs_layout(B)
    Xh, _, ldx, devx, _ = _rhs_layout(X)
    if not (dev and devx):
        raise ValueError("mf_solve_noalloc takes device tensors")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    _check(lib().mf_solve_noalloc(f, nrhs, _ptr(Bh), ldb, _ptr(Xh), ldx, _stream(stream)))
    return Xh


def mf_solve_refined(f, B, X=None, tol=1e-13, max_iter=30, allow_fallback=True, stream=None):
    """Mixed-precision refinement (FP32 factor, FP64 residual).  Returns (X, report)."""
    Bh, nrhs, ldb, dev, _ = _rhs_layout(B)
    if X is None:
        X = _alloc_like(Bh, dev)
    Xh, _, ldx, _, _ = _rhs_layout(X)
    if dev and stream is None:
        import torch
        stream = torch.cuda.current_stream()
    rep = mf_ir_report()
    _check(lib().mf_solve_refined(f, nrhs, _ptr(Bh), ldb, _ptr(Xh), ldx, dev, tol, max_iter,
                                  1 if allow_fallback else 0, ctypes.byref(rep), _stream(stream)))
    return Xh, {k: getattr(rep, k) for k, _ in mf_ir_report._fields_}


# ---------------------------------------------------------------------------
# serving loop.  Host arrays handed to a request are kept alive by the
# binding until the request is waited on.
_keep = {}


def mf_server_create(h, workers=4, budget_bytes=0):
    sv = ctypes.c_void_p()
    _check(lib().mf_server_create(h, workers, budget_bytes, ctypes.byref(sv)))
    return sv


def mf_server_submit_factor(sv, s, values, prec, B=None, X=None):
    """Returns (req, factor_id, X); B/X column-major host arrays or None."""
    values = np.ascontiguousarray(values, dtype=np.float64)
    nrhs, ldb = 0, 1
    if B is not None:
        B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(B.shape[0], -1))
        nrhs, ldb = B.shape[1], B.shape[0]
        if X is None:
            X = np.empty_like(B, order="F")
    req, fid = _I64(), _I64()
    _check(lib().mf_server_submit_factor(sv, s, _ptr(values), prec, nrhs, _ptr(B), ldb, _ptr(X),
                                         ldb, ctypes.byref(req), ctypes.byref(fid)))
    _keep[(sv.value, req.value)] = (values, B, X)
    return req.value, fid.value, X


def mf_server_submit_solve(sv, factor_id, B, X=None):
    B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(B.shape[0], -1))
    if X is None:
        X = np.empty_like(B, order="F")
    req = _I64()
    _check(lib().mf_server_submit_solve(sv, factor_id, B.shape[1], _ptr(B), B.shape[0], _ptr(X),
                                        B.shape[0], ctypes.byref(req)))
    _keep[(sv.value, req.value)] = (B, X)
    return req.value, X


def mf_server_poll(sv, req):
    d, st, ms = _I32(), _I32(), _D()
    _check(lib().mf_server_poll(sv, req, ctypes.byref(d), ctypes.byref(st), ctypes.byref(ms)))
    return bool(d.value), st.value, ms.value


def mf_server_wait(sv, req):
    st, ms = _I32(), _D()
    _check(lib().mf_server_wait(sv, req, ctypes.byref(st), ctypes.byref(ms)))
    _keep.pop((sv.value, req), None)
    return st.value, ms.value


def mf_server_release_factor(sv, factor_id):
    _check(lib().mf_server_release_factor(sv, factor_id))


def mf_server_get_stats(sv):
    out = mf_server_stats()
    _check(lib().mf_server_get_stats(sv, ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in mf_server_stats._fields_}


def mf_server_free(sv):
    _check(lib().mf_server_free(sv))
    for key in [k for k in _keep if k[0] == sv.value]:
        del _keep[key]


def exported_symbols():
    """Names of the C entry points this binding wraps plus the error helpers."""
    return sorted(list(_SIGS) + ["mf_last_error_string", "mf_last_error_column"])


# ---------------------------------------------------------------------------
# FastILU / FastSpTRSV
def mf_ilu_symbolic(h, rowptr, colind, level):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().mf_ilu_symbolic(h, len(rp) - 1, _ptr(rp), _ptr(ci), level, ctypes.byref(out)))
    return out


def mf_ilu_info(ilu):
    n, nnz = _I64(0), _I64(0)
    _check(lib().mf_ilu_info(ilu, ctypes.byref(n), ctypes.byref(nnz)))
    return int(n.value), int(nnz.value)


def mf_ilu_pattern(ilu):
    n, nnz = mf_ilu_info(ilu)
    Sp = np.empty(n + 1, dtype=np.int64)
    Sj = np.empty(nnz, dtype=np.int32)
    Sl = np.empty(nnz, dtype=np.int32)
    _check(lib().mf_ilu_pattern(ilu, _ptr(Sp), _ptr(Sj), _ptr(Sl)))
    return Sp, Sj, Sl


def mf_ilu_numeric(ilu, values, sweeps=2, omega=1.0, shift=0.0, warmup=False, in_place=False,
                   stream=None):
    dev = 1 if _is_device(values) else 0
    v = values if dev else np.ascontiguousarray(values, dtype=np.float64)
    if dev and stream is None:
        import torch
        stream = torch.cuda.current_stream()
    _check(lib().mf_ilu_numeric(ilu, _ptr(v), dev, sweeps, omega, shift, 1 if warmup else 0,
                                1 if in_place else 0, _stream(stream)))


def mf_ilu_export(ilu):
    _, nnz = mf_ilu_info(ilu)
    out = np.empty(nnz, dtype=np.float64)
    _check(lib().mf_ilu_export(ilu, _ptr(out)))
    return out


def _ilu_vec(ilu, fn, b, x, stream, *args):
    dev = 1 if _is_device(b) else 0
    if x is None:
        x = _alloc_like(b, dev) if dev else np.empty(len(b))
    bb = b if dev else np.ascontiguousarray(b, dtype=np.float64)
    if dev and stream is None:
        import torch
        stream = torch.cuda.current_stream()
    _check(fn(ilu, *args, _ptr(bb), _ptr(x), dev, _stream(stream)))
    return x


def mf_ilu_trsv(ilu, b, upper, sweeps, omega=1.0, x=None, stream=None):
    return _ilu_vec(ilu, lib().mf_ilu_trsv, b, x, stream, 1 if upper else 0, sweeps, omega)


def mf_ilu_apply(ilu, b, sweeps, omega=1.0, x=None, stream=None):
    return _ilu_vec(ilu, lib().mf_ilu_apply, b, x, stream, sweeps, omega)


def mf_ilu_free(ilu):
    _check(lib().mf_ilu_free(ilu))


def mf_symbolic_options(s):
    """The options the analysis was made with (mf_options)."""
    o = mf_options()
    _check(lib().mf_symbolic_options(s, ctypes.byref(o)))
    return o


def mf_factor_create_ldlt(h, s, prec=MF_FP64):
    """LDL^T factor object (see the C header)."""
    f = ctypes.c_void_p()
    _check(lib().mf_factor_create_ldlt(h, s, prec, ctypes.byref(f)))
    return f


def mf_factor_create_lu(h, s, prec=MF_FP64, pivot=0):
    """LU factor object, pivot 0 (none) or 1 (within diagonal blocks); see the C header."""
    f = ctypes.c_void_p()
    _check(lib().mf_factor_create_lu(h, s, prec, pivot, ctypes.byref(f)))
    return f


def mf_factor_create_ldlt_piv(h, s, prec=MF_FP64):
    """LDL^T factor with symmetric pivoting within the diagonal blocks (see the C header)."""
    f = ctypes.c_void_p()
    _check(lib().mf_factor_create_ldlt_piv(h, s, prec, ctypes.byref(f)))
    return f


def mf_factor_export_U(f, nnz_L):
    out = np.empty(nnz_L, dtype=np.float64)
    _check(lib().mf_factor_export_U(f, _ptr(out)))
    return out


def mf_factor_export_pivots(f, n):
    out = np.empty(n, dtype=np.int32)
    _check(lib().mf_factor_export_pivots(f, _ptr(out)))
    return out


def mf_symbolic_fronts(s):
    nf = mf_symbolic_get_info(s)["nfronts"]
    out = np.empty(nf + 1, dtype=np.int32)
    _check(lib().mf_symbolic_fronts(s, _ptr(out)))
    return out


def mf_factor_export_D(f, n):
    out = np.empty(n, dtype=np.float64)
    _check(lib().mf_factor_export_D(f, _ptr(out)))
    return out


def mf_factor_kind_items(f):
    """{kind: (items, launches)} of one numeric factorization."""
    items = np.zeros(6, dtype=np.int64)
    launches = np.zeros(6, dtype=np.int64)
    _check(lib().mf_factor_kind_items(f, _ptr(items), _ptr(launches)))
    return {k: (int(items[i]), int(launches[i])) for i, k in enumerate(FACTOR_KINDS)}
