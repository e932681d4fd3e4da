"""FP64 CPU oracle for sparse CP-ALS (test infrastructure only).

Thin ctypes wrapper over ``oracle.c``. Only ``tests/``, the smoke check in
``__graft_entry__`` and the benchmark's CPU-baseline leg may import this
module. The product library (the CUDA path) never uses it and shares no code
with it.

What each function computes, and the reading of the paper behind it, is in the
header of ``oracle.c`` (arXiv:1812.05961, Section III and Algorithm 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc, no GPU),
    with OpenMP when the compiler has it (the threaded MTTKRP; see
    ``set_threads``), else without."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Host threads of the oracle's MTTKRP (1 = the literal single loop, the
    default). Returns the number in effect (1 without OpenMP). Only the FP64
    summation order depends on it."""
    _threads_now[0] = int(_load().oracle_set_threads(int(n)))
    return _threads_now[0]


def threads() -> int:
    """The number of threads the MTTKRP currently uses."""
    return _threads_now[0]


_threads_now = [1]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_philox4x64.argtypes = [_u64p, _u64p, _u64p]
            lib.oracle_init_factor.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int32, _f64p]
            lib.oracle_coalesce.restype = ctypes.c_int64
            lib.oracle_coalesce.argtypes = [ctypes.c_int32, ctypes.c_int64, _i64p,
                                            ctypes.POINTER(_i32p), _f32p, _i32p,
                                            ctypes.POINTER(_i32p), _f32p]
            lib.oracle_csf.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(_i32p),
                                       _i32p, _i64p, ctypes.POINTER(_i32p),
                                       ctypes.POINTER(_i32p)]
            lib.oracle_mttkrp.argtypes = [ctypes.c_int32, ctypes.c_int64, _i64p,
                                          ctypes.POINTER(_i32p), _f32p, ctypes.POINTER(_f64p),
                                          ctypes.c_int32, ctypes.c_int32, _f64p, _f64p, _u8p]
            lib.oracle_gram.argtypes = [ctypes.c_int64, ctypes.c_int32, _f64p, _f64p]
            lib.oracle_cholesky.restype = ctypes.c_int
            lib.oracle_cholesky.argtypes = [ctypes.c_int32, _f64p, _f64p]
            lib.oracle_sym_eig.argtypes = [ctypes.c_int32, _f64p, _f64p, _f64p]
            lib.oracle_pinv_sym.argtypes = [ctypes.c_int32, _f64p, _f64p]
            lib.oracle_solve_normals.restype = ctypes.c_int
            lib.oracle_solve_normals.argtypes = [ctypes.c_int64, ctypes.c_int32, _f64p, _f64p]
            lib.oracle_normalize.argtypes = [ctypes.c_int64, ctypes.c_int32, _f64p, _f64p]
            lib.oracle_fit.restype = ctypes.c_double
            lib.oracle_fit.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.POINTER(_f64p), _f64p, ctypes.c_int64, _f64p,
                                       _f64p]
            lib.oracle_als_mode_update.restype = ctypes.c_int
            lib.oracle_als_mode_update.argtypes = [ctypes.c_int32, ctypes.c_int64, _i64p,
                                                   ctypes.POINTER(_i32p), _f32p, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.POINTER(_f64p),
                                                   ctypes.POINTER(_f64p), _f64p, _f64p]
            lib.oracle_cpd_als.restype = ctypes.c_int32
            lib.oracle_cpd_als.argtypes = [ctypes.c_int32, ctypes.c_int64, _i64p,
                                           ctypes.POINTER(_i32p), _f32p, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_f64p),
                                           _f64p, _f64p]
            lib.oracle_mlp_forward.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f64p,
                                               ctypes.c_int64, _f64p, _f64p]
            lib.oracle_mlp_loss_grad.restype = ctypes.c_double
            lib.oracle_set_threads.restype = ctypes.c_int32
            lib.oracle_set_threads.argtypes = [ctypes.c_int32]
            lib.oracle_mlp_loss_grad.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _f64p,
                                                 ctypes.c_int64, _f64p, _f64p, _f64p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr_array(arrs, t, elem):
    return (elem * len(arrs))(*[_p(a, t) for a in arrs])


def _coo(inds, vals, dims):
    inds = [_c(x, np.int32) for x in inds]
    vals = _c(vals, np.float32)
    dims = _c(dims, np.int64)
    if len(inds) != len(dims):
        raise ValueError("one index array per mode")
    for x in inds:
        if x.shape != vals.shape:
            raise ValueError("index and value arrays differ in length")
    return inds, vals, dims


def default_order(dims, root: int):
    """Level order of a CSF rooted at ``root``: the root, then the other modes
    by ascending length, ties broken by the lower mode id."""
    rest = sorted((m for m in range(len(dims)) if m != root), key=lambda m: (int(dims[m]), m))
    return [root] + rest


# --------------------------------------------------------------------------
# Generator
# --------------------------------------------------------------------------

def philox4x64(counter, key) -> np.ndarray:
    """Philox4x64-10 of one 4-word counter under a 2-word key."""
    lib = _load()
    c = np.array([int(x) for x in counter], dtype=np.uint64)
    k = np.array([int(x) for x in key], dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib.oracle_philox4x64(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def init_factor(seed: int, mode: int, rows: int, rank: int) -> np.ndarray:
    """U(0,1) initial factor (rows x rank, FP64) from the Philox stream."""
    lib = _load()
    A = np.zeros((rows, rank), np.float64)
    lib.oracle_init_factor(ctypes.c_uint64(seed), mode, rows, rank, _p(A, _f64p))
    return A


# --------------------------------------------------------------------------
# Sort / coalesce / CSF
# --------------------------------------------------------------------------

def coalesce(inds, vals, dims, order=None):
    """Sort non-zeros lexicographically in ``order`` and sum duplicates.

    Returns (inds_sorted: list of int32 arrays per mode, vals_sorted float32)."""
    lib = _load()
    inds, vals, dims = _coo(inds, vals, dims)
    n = len(dims)
    order = _c(list(range(n)) if order is None else order, np.int32)
    nnz = vals.shape[0]
    out_inds = [np.zeros(max(nnz, 1), np.int32) for _ in range(n)]
    out_vals = np.zeros(max(nnz, 1), np.float32)
    u = lib.oracle_coalesce(n, nnz, _p(dims, _i64p), _ptr_array(inds, _i32p, _i32p),
                            _p(vals, _f32p), _p(order, _i32p),
                            _ptr_array(out_inds, _i32p, _i32p), _p(out_vals, _f32p))
    if u < 0:
        raise ValueError("index out of range")
    return [x[:u].copy() for x in out_inds], out_vals[:u].copy()


def csf(inds, vals, dims, root: int, order=None):
    """CSF of the tensor rooted at ``root`` (coalesces first).

    Returns dict(order, nfibs, fptr[l] for l < N-1, fids[l] for all l, vals)."""
    lib = _load()
    dims = _c(dims, np.int64)
    n = len(dims)
    order = default_order(dims, root) if order is None else list(order)
    if order[0] != root or sorted(order) != list(range(n)):
        raise ValueError("order must be a permutation of the modes starting at root")
    s_inds, s_vals = coalesce(inds, vals, dims, order)
    nnz = s_vals.shape[0]
    ordc = _c(order, np.int32)
    nfibs = np.zeros(n, np.int64)
    fptr = [np.zeros(nnz + 1, np.int32) for _ in range(n - 1)]
    fids = [np.zeros(max(nnz, 1), np.int32) for _ in range(n)]
    lib.oracle_csf(n, nnz, _ptr_array(s_inds, _i32p, _i32p), _p(ordc, _i32p),
                   _p(nfibs, _i64p), _ptr_array(fptr, _i32p, _i32p),
                   _ptr_array(fids, _i32p, _i32p))
    return {
        "order": order,
        "nfibs": [int(x) for x in nfibs],
        "fptr": [fptr[l][: nfibs[l] + 1].copy() for l in range(n - 1)],
        "fids": [fids[l][: nfibs[l]].copy() for l in range(n)],
        "vals": s_vals,
    }


# --------------------------------------------------------------------------
# MTTKRP and dense algebra
# --------------------------------------------------------------------------

def mttkrp(inds, vals, dims, factors, mode: int, with_abs: bool = False, rows=None):
    """FP64 MTTKRP by the element definition. ``factors`` are per-mode
    (dims[m] x R) arrays (the root mode's may be None). ``rows`` restricts the
    work to a subset of output rows (others are zero)."""
    lib = _load()
    inds, vals, dims = _coo(inds, vals, dims)
    n = len(dims)
    rank = None
    fac = []
    for m in range(n):
        if factors[m] is None:
            fac.append(np.zeros((1, 1), np.float64))
        else:
            f = _c(factors[m], np.float64)
            rank = f.shape[1]
            fac.append(f)
    if rank is None:
        raise ValueError("need at least one non-root factor")
    for m in range(n):
        if factors[m] is not None and fac[m].shape != (dims[m], rank):
            raise ValueError("factor %d has shape %s, want %s" % (m, fac[m].shape, (dims[m], rank)))
    out = np.zeros((int(dims[mode]), rank), np.float64)
    out_abs = np.zeros_like(out) if with_abs else None
    mask = None
    if rows is not None:
        mask = np.zeros(int(dims[mode]), np.uint8)
        mask[np.asarray(rows, np.int64)] = 1
    lib.oracle_mttkrp(n, vals.shape[0], _p(dims, _i64p), _ptr_array(inds, _i32p, _i32p),
                      _p(vals, _f32p), _ptr_array(fac, _f64p, _f64p), rank, mode,
                      _p(out, _f64p), None if out_abs is None else _p(out_abs, _f64p),
                      None if mask is None else _p(mask, _u8p))
    return (out, out_abs) if with_abs else out


def gram(A):
    lib = _load()
    A = _c(A, np.float64)
    rank = A.shape[1]
    G = np.zeros((rank, rank), np.float64)
    lib.oracle_gram(A.shape[0], rank, _p(A, _f64p), _p(G, _f64p))
    return G


def cholesky(V):
    """Lower Cholesky factor, or None when V fails the positive-definite test."""
    lib = _load()
    V = _c(V, np.float64)
    L = np.zeros_like(V)
    return L if lib.oracle_cholesky(V.shape[0], _p(V, _f64p), _p(L, _f64p)) == 0 else None


def sym_eig(V):
    lib = _load()
    V = _c(V, np.float64)
    n = V.shape[0]
    w = np.zeros(n, np.float64)
    Q = np.zeros((n, n), np.float64)
    lib.oracle_sym_eig(n, _p(V, _f64p), _p(w, _f64p), _p(Q, _f64p))
    return w, Q


def pinv_sym(V):
    lib = _load()
    V = _c(V, np.float64)
    P = np.zeros_like(V)
    lib.oracle_pinv_sym(V.shape[0], _p(V, _f64p), _p(P, _f64p))
    return P


def solve_normals(M, V):
    """A = M V^dagger row-wise. Returns (A, branch) with branch 0 = Cholesky,
    1 = pseudo-inverse."""
    lib = _load()
    A = _c(M, np.float64).copy()
    V = _c(V, np.float64)
    b = lib.oracle_solve_normals(A.shape[0], V.shape[0], _p(V, _f64p), _p(A, _f64p))
    return A, b


def normalize(A):
    lib = _load()
    A = _c(A, np.float64).copy()
    lam = np.zeros(A.shape[1], np.float64)
    lib.oracle_normalize(A.shape[0], A.shape[1], _p(A, _f64p), _p(lam, _f64p))
    return A, lam


def fit(normx_sq, grams, lam, M, A):
    lib = _load()
    grams = [_c(g, np.float64) for g in grams]
    lam = _c(lam, np.float64)
    M = _c(M, np.float64)
    A = _c(A, np.float64)
    return lib.oracle_fit(len(grams), lam.shape[0], float(normx_sq),
                          _ptr_array(grams, _f64p, _f64p), _p(lam, _f64p), M.shape[0],
                          _p(M, _f64p), _p(A, _f64p))


def als_mode_update(inds, vals, dims, factors, grams, mode: int):
    """One factor update of Algorithm 1 for ``mode``. Returns
    (new_factor, lambda, new_gram, mttkrp, branch); inputs are not modified."""
    lib = _load()
    inds, vals, dims = _coo(inds, vals, dims)
    n = len(dims)
    fac = [_c(f, np.float64).copy() for f in factors]
    grs = [_c(g, np.float64).copy() for g in grams]
    rank = fac[0].shape[1]
    lam = np.zeros(rank, np.float64)
    M = np.zeros((int(dims[mode]), rank), np.float64)
    b = lib.oracle_als_mode_update(n, vals.shape[0], _p(dims, _i64p),
                                   _ptr_array(inds, _i32p, _i32p), _p(vals, _f32p), rank, mode,
                                   _ptr_array(fac, _f64p, _f64p), _ptr_array(grs, _f64p, _f64p),
                                   _p(lam, _f64p), _p(M, _f64p))
    return fac[mode], lam, grs[mode], M, b


def cpd_als(inds, vals, dims, rank: int, max_iters: int, tol: float = 0.0, seed: int = 0,
            init=None, coalesce_first: bool = True):
    """CP-ALS (Algorithm 1, N modes). ``init`` gives the initial factors
    (default: the Philox U(0,1) stream from ``seed``). Returns
    dict(factors, lam, fits, iters)."""
    lib = _load()
    if coalesce_first:
        inds, vals = coalesce(inds, vals, dims)
    inds, vals, dims = _coo(inds, vals, dims)
    n = len(dims)
    if init is None:
        fac = [init_factor(seed, m, int(dims[m]), rank) for m in range(n)]
    else:
        fac = [_c(f, np.float64).copy() for f in init]
    lam = np.zeros(rank, np.float64)
    fits = np.zeros(max(max_iters, 1), np.float64)
    it = lib.oracle_cpd_als(n, vals.shape[0], _p(dims, _i64p), _ptr_array(inds, _i32p, _i32p),
                            _p(vals, _f32p), rank, max_iters, float(tol),
                            _ptr_array(fac, _f64p, _f64p), _p(lam, _f64p), _p(fits, _f64p))
    return {"factors": fac, "lam": lam, "fits": fits[:it].copy(), "iters": int(it)}


# --------------------------------------------------------------------------
# Scheduler MLP (FP64 reference for the GPU training kernels)
# --------------------------------------------------------------------------

def mlp_nparams(nin, nh, nout):
    return nh * nin + nh + nh * nh + nh + nout * nh + nout


def mlp_forward(P, x, nin, nh, nout):
    lib = _load()
    P = _c(P, np.float64)
    x = _c(x, np.float64).reshape(-1, nin)
    y = np.zeros((x.shape[0], nout), np.float64)
    lib.oracle_mlp_forward(nin, nh, nout, _p(P, _f64p), x.shape[0], _p(x, _f64p), _p(y, _f64p))
    return y


def mlp_loss_grad(P, x, t, nin, nh, nout):
    """MSE loss 1/(n*nout) sum (y - t)^2 and its gradient (same layout as P)."""
    lib = _load()
    P = _c(P, np.float64)
    x = _c(x, np.float64).reshape(-1, nin)
    t = _c(t, np.float64).reshape(-1, nout)
    G = np.zeros_like(P)
    L = lib.oracle_mlp_loss_grad(nin, nh, nout, _p(P, _f64p), x.shape[0], _p(x, _f64p), _p(t, _f64p),
                                 _p(G, _f64p))
    return L, G
