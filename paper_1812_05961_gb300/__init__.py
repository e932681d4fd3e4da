"""Python binding of libsptt (sparse CP-ALS over CSF on one GB300 GPU).

Argument marshalling only: every function forwards to the C ABI declared in
``include/sptt.h`` under the same name, passing torch tensors as raw device
pointers and torch's current CUDA stream. All compute runs in the library's
CUDA kernels; there is no CPU fallback, and loading fails loudly when the
compiled library is missing (run ``build()`` first).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsptt.so")

SPTT_OK = 0
SPTT_ERR_BAD_ARG = -1
SPTT_ERR_OOM = -2
SPTT_ERR_CUDA = -3
SPTT_ERR_TIMEOUT = -4
SPTT_ERR_NOT_PD = -5
SPTT_ERR_UNSUPPORTED = -6
SPTT_ERR_INTERNAL = -7
SPTT_MAX_MODES = 5
SPTT_MAX_RANK_ALS = 64
SPTT_F32 = 0
SPTT_BF16 = 1
SPTT_NUM_TIMERS = 5
TIMER_NAMES = ("mttkrp", "inverse", "solve_gram", "mat_norm", "cpd_fit")


class SpttError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__("%s failed: %s (%s)" % (where, _status_name(status), detail))
        self.status = status


class sptt_coo(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("inds", ctypes.POINTER(ctypes.c_void_p)),
                ("vals", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class sptt_sched(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("block", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("order", ctypes.c_int32)]

    def as_tuple(self):
        return (self.chunk, self.block, self.variant, self.order)


class sptt_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("refine_iters", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("sched", ctypes.POINTER(sptt_sched)),
                ("mode_sched", ctypes.POINTER(sptt_sched)), ("plan", ctypes.c_int32),
                ("mlp", ctypes.c_void_p), ("csf_mode", ctypes.c_int32), ("leaf_tile_rows", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_ST = ctypes.c_int32


def build(**kw) -> str:
    """Compile libsptt.so in-tree (nvcc, sm_103a)."""
    from . import buildlib
    return buildlib.build(**kw)


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsptt.so is not built (%s); call paper_1812_05961_gb300.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sptt_status_str": (ctypes.c_char_p, [_ST]),
            "sptt_last_error": (ctypes.c_char_p, []),
            "sptt_version": (_I32, []),
            "sptt_csf_build": (_ST, [ctypes.POINTER(sptt_coo), _I32, _P, _P, ctypes.POINTER(_P)]),
            "sptt_csf_free": (None, [_P]),
            "sptt_csf_shape": (_ST, [_P, _P, _P, _P]),
            "sptt_csf_copy_level": (_ST, [_P, _I32, _P, _P, _P, _P]),
            "sptt_csf_check": (_ST, [_P, _P]),
            "sptt_mttkrp": (_ST, [_P, _P, _I32, _I32, _P, _P, _P]),
            "sptt_mttkrp_mode": (_ST, [_P, _I32, _P, _I32, _I32, _P, _P, _P]),
            "sptt_cpd_save": (_ST, [_P, _P, ctypes.c_size_t, _P]),
            "sptt_cpd_load": (_ST, [_P, _P, ctypes.c_size_t]),
            "sptt_gram": (_ST, [_P, _I64, _I32, _I32, _P, _P]),
            "sptt_gram_noalloc": (_ST, [_P, _I64, _I32, _I32, _P, _P]),
            "sptt_cpd_create": (_ST, [ctypes.POINTER(sptt_coo), _I32, ctypes.POINTER(sptt_opts), _P,
                                      ctypes.POINTER(_P)]),
            "sptt_cpd_free": (None, [_P]),
            "sptt_cpd_init": (_ST, [_P, _P]),
            "sptt_cpd_iterate": (_ST, [_P, _I32, ctypes.c_double, _P]),
            "sptt_cpd_refine": (_ST, [_P, _I32]),
            "sptt_cpd_fit": (_ST, [_P, _P, _P]),
            "sptt_cpd_fit_history": (_ST, [_P, _P, _I32, _P]),
            "sptt_cpd_lambda": (_ST, [_P, _P]),
            "sptt_cpd_factor": (_ST, [_P, _I32, _P]),
            "sptt_cpd_gram": (_ST, [_P, _I32, _P]),
            "sptt_cpd_solve_branch": (_ST, [_P, _P, _P]),
            "sptt_cpd_timers": (_ST, [_P, _P, _P]),
            "sptt_cpd_als": (_ST, [ctypes.POINTER(sptt_coo), _I32, _I32, ctypes.c_double,
                                   ctypes.POINTER(sptt_opts), _P, _P, _P, _P, _P]),
            "sptt_debug_fail_alloc_after": (None, [_I64]),
            "sptt_debug_launch_count": (_I64, []),
            "sptt_sched_candidates": (_I32, [_I64, _P, _I32]),
            "sptt_sched_default": (_ST, [_P, _I32, _I32, _I32, _I32, _I64, _P]),
            "sptt_level_order": (_ST, [_P, _I32, _I32, _I32, _P]),
            "sptt_autotune": (_ST, [ctypes.POINTER(sptt_coo), _I32, _I32, _I32, _I32, _P, _P]),
            "sptt_csf_features": (_ST, [_P, _I32, _I32, _P, _P]),
            "sptt_mlp_create": (_ST, [ctypes.c_uint64, ctypes.POINTER(_P)]),
            "sptt_mlp_free": (None, [_P]),
            "sptt_mlp_nparams": (_I32, []),
            "sptt_mlp_get": (_ST, [_P, _P, _P, _P]),
            "sptt_mlp_set": (_ST, [_P, _P, _P, _P]),
            "sptt_mlp_forward": (_ST, [_P, _P, _I64, _P, _P]),
            "sptt_mlp_loss_grad": (_ST, [_P, _P, _P, _I64, _P, _P, _P]),
            "sptt_mlp_train": (_ST, [_P, _P, _P, _I64, _I32, ctypes.c_float, _P, _P]),
            "sptt_mlp_predict": (_ST, [_P, _P, _I64, _P, _P, _P]),
            "sptt_batch_create": (_ST, [_P, _I32, _I32, ctypes.POINTER(sptt_opts), _P, ctypes.POINTER(_P)]),
            "sptt_batch_free": (None, [_P]),
            "sptt_batch_init": (_ST, [_P]),
            "sptt_batch_run": (_ST, [_P, _I32]),
            "sptt_batch_fit_history": (_ST, [_P, _I32, _P, _I32, _P]),
            "sptt_batch_factor": (_ST, [_P, _I32, _I32, _P]),
            "sptt_batch_lambda": (_ST, [_P, _I32, _P]),
            "sptt_batch_info": (_ST, [_P, _P, _P, _P]),
            "sptt_debug_batch_stall": (_ST, [_P, _I32, _I64]),
            "sptt_batch_phase_ms": (_ST, [_P, _P]),
            "sptt_batch_schedule": (_ST, [_P, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    try:
        return lib().sptt_status_str(s).decode()
    except Exception:  # pragma: no cover - only when the library itself is absent
        return str(s)


def _check(status: int, where: str):
    if status != SPTT_OK:
        raise SpttError(status, where, lib().sptt_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


class _Coo:
    """Holds an sptt_coo and the arrays it points to."""

    def __init__(self, dims, inds: Sequence[torch.Tensor], vals: torch.Tensor):
        if len(inds) != len(dims):
            raise ValueError("one index array per mode")
        self.dims = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
        self.inds_t = [x.contiguous() for x in inds]
        self.vals_t = vals.contiguous()
        for x in self.inds_t:
            if x.dtype != torch.int32:
                raise TypeError("indices must be int32")
        if self.vals_t.dtype != torch.float32:
            raise TypeError("values must be float32")
        on_dev = self.vals_t.is_cuda
        if any(x.is_cuda != on_dev for x in self.inds_t):
            raise ValueError("indices and values must all be on the host or all on the device")
        self.ptrs = (ctypes.c_void_p * len(dims))(*[x.data_ptr() for x in self.inds_t])
        self.c = sptt_coo(len(dims), int(self.vals_t.numel()), self.dims, self.ptrs,
                          self.vals_t.data_ptr(), 1 if on_dev else 0)


def _sched(s):
    return s if isinstance(s, sptt_sched) else sptt_sched(*s)


def _opts(seed=0, precision=SPTT_F32, refine_iters=0, use_graph=0, profile=0, sched=None,
          mode_sched=None, plan=0, mlp=None, csf_mode=0, leaf_tile_rows=0):
    o = sptt_opts(seed, precision, refine_iters, use_graph, profile, None, None, plan,
                  None if mlp is None else (mlp.handle if hasattr(mlp, "handle") else mlp), csf_mode,
                  leaf_tile_rows)
    keep = []
    if sched is not None:
        one = _sched(sched)
        keep.append(one)
        o.sched = ctypes.pointer(one)
    if mode_sched is not None:
        arr = (sptt_sched * len(mode_sched))(*[_sched(x) for x in mode_sched])
        keep.append(arr)
        o.mode_sched = ctypes.cast(arr, ctypes.POINTER(sptt_sched))
    return o, keep


# ---------------------------------------------------------------------------
# Same-name wrappers of the C ABI
# ---------------------------------------------------------------------------

def sptt_version() -> int:
    return lib().sptt_version()


def sptt_status_str(status: int) -> str:
    return lib().sptt_status_str(status).decode()


def sptt_last_error() -> str:
    return lib().sptt_last_error().decode()


def sptt_csf_build(dims, inds, vals, root_mode: int, level_order=None, stream=None) -> int:
    coo = _Coo(dims, inds, vals)
    order = None
    if level_order is not None:
        order = (ctypes.c_int32 * len(dims))(*level_order)
    out = ctypes.c_void_p()
    _check(lib().sptt_csf_build(ctypes.byref(coo.c), root_mode, order, _stream(stream),
                                ctypes.byref(out)), "sptt_csf_build")
    return out.value


def sptt_csf_free(csf: int):
    lib().sptt_csf_free(csf)


def sptt_csf_shape(csf: int):
    n = ctypes.c_int32()
    order = (ctypes.c_int32 * SPTT_MAX_MODES)()
    nfibs = (ctypes.c_int64 * SPTT_MAX_MODES)()
    _check(lib().sptt_csf_shape(csf, ctypes.byref(n), order, nfibs), "sptt_csf_shape")
    return n.value, list(order[:n.value]), list(nfibs[:n.value])


def sptt_csf_check(csf: int, stream=None):
    _check(lib().sptt_csf_check(csf, _stream(stream)), "sptt_csf_check")


def sptt_csf_copy_level(csf: int, level: int, stream=None):
    """Returns (fptr or None, fids, vals or None) as host int32/float32 tensors."""
    n, order, nfibs = sptt_csf_shape(csf)
    nl = nfibs[level]
    fptr = torch.empty(nl + 1, dtype=torch.int32) if level < n - 1 else None
    fids = torch.empty(max(nl, 1), dtype=torch.int32)
    vals = torch.empty(max(nl, 1), dtype=torch.float32) if level == n - 1 else None
    _check(lib().sptt_csf_copy_level(csf, level, _ptr(fptr), _ptr(fids), _ptr(vals), _stream(stream)),
           "sptt_csf_copy_level")
    return fptr, fids[:nl], None if vals is None else vals[:nl]


def sptt_mttkrp(csf: int, factors: Sequence[Optional[torch.Tensor]], out: torch.Tensor,
                factor_dtype: int = SPTT_F32, sched=None, stream=None):
    """out (dims[root] x ld float32, device) = MTTKRP of the CSF's root mode.
    factors: per mode (dims[m] x ld) device tensors (float32 or bfloat16)."""
    ld = out.shape[1]
    arr = (ctypes.c_void_p * len(factors))(*[0 if f is None else f.data_ptr() for f in factors])
    for f in factors:
        if f is not None and (not f.is_contiguous() or f.shape[1] != ld):
            raise ValueError("factors must be contiguous with ld = out.shape[1] columns")
    s = None
    if sched is not None:
        s = _sched(sched)
    _check(lib().sptt_mttkrp(csf, arr, factor_dtype, ld, out.data_ptr(),
                             None if s is None else ctypes.byref(s), _stream(stream)), "sptt_mttkrp")
    return out


def sptt_mttkrp_mode(csf: int, mode: int, factors: Sequence[Optional[torch.Tensor]], out: torch.Tensor,
                     factor_dtype: int = SPTT_F32, sched=None, stream=None):
    """out (dims[mode] x ld float32, device) = MTTKRP of any mode from one CSF."""
    ld = out.shape[1]
    arr = (ctypes.c_void_p * len(factors))(*[0 if f is None else f.data_ptr() for f in factors])
    for f in factors:
        if f is not None and (not f.is_contiguous() or f.shape[1] != ld):
            raise ValueError("factors must be contiguous with ld = out.shape[1] columns")
    s = None
    if sched is not None:
        s = _sched(sched)
    _check(lib().sptt_mttkrp_mode(csf, mode, arr, factor_dtype, ld, out.data_ptr(),
                                  None if s is None else ctypes.byref(s), _stream(stream)), "sptt_mttkrp_mode")
    return out


def sptt_gram(A: torch.Tensor, rank: int, G: Optional[torch.Tensor] = None, stream=None):
    if G is None:
        G = torch.empty((rank, rank), dtype=torch.float64, device=A.device)
    _check(lib().sptt_gram(A.data_ptr(), A.shape[0], rank, A.shape[1], G.data_ptr(), _stream(stream)),
           "sptt_gram")
    return G


def sptt_gram_noalloc(A: torch.Tensor, rank: int, G: torch.Tensor, stream=None):
    """sptt_gram without device allocation (static device workspace; see
    include/sptt.h). G must be a preallocated rank x rank float64 tensor."""
    _check(lib().sptt_gram_noalloc(A.data_ptr(), A.shape[0], rank, A.shape[1], G.data_ptr(),
                                   _stream(stream)), "sptt_gram_noalloc")
    return G


def sptt_cpd_create(dims, inds, vals, rank: int, stream=None, **opts) -> int:
    coo = _Coo(dims, inds, vals)
    o, keep = _opts(**opts)
    out = ctypes.c_void_p()
    _check(lib().sptt_cpd_create(ctypes.byref(coo.c), rank, ctypes.byref(o), _stream(stream),
                                 ctypes.byref(out)), "sptt_cpd_create")
    del keep
    return out.value


def sptt_cpd_free(cpd: int):
    lib().sptt_cpd_free(cpd)


def sptt_cpd_init(cpd: int, init: Optional[Sequence[torch.Tensor]] = None):
    arr = None
    if init is not None:
        init = [t.contiguous().to(torch.float32) for t in init]
        arr = (ctypes.c_void_p * len(init))(*[t.data_ptr() for t in init])
    _check(lib().sptt_cpd_init(cpd, arr), "sptt_cpd_init")


def sptt_cpd_iterate(cpd: int, iters: int, tol: float = 0.0) -> int:
    done = ctypes.c_int32()
    _check(lib().sptt_cpd_iterate(cpd, iters, tol, ctypes.byref(done)), "sptt_cpd_iterate")
    return done.value


def sptt_cpd_refine(cpd: int, iters: int):
    _check(lib().sptt_cpd_refine(cpd, iters), "sptt_cpd_refine")


def sptt_cpd_fit(cpd: int):
    f = ctypes.c_double()
    it = ctypes.c_int32()
    _check(lib().sptt_cpd_fit(cpd, ctypes.byref(f), ctypes.byref(it)), "sptt_cpd_fit")
    return f.value, it.value


def sptt_cpd_fit_history(cpd: int, cap: int = 4096):
    buf = (ctypes.c_double * cap)()
    n = ctypes.c_int32()
    _check(lib().sptt_cpd_fit_history(cpd, buf, cap, ctypes.byref(n)), "sptt_cpd_fit_history")
    return list(buf[:n.value])


def sptt_cpd_lambda(cpd: int, rank: int) -> torch.Tensor:
    t = torch.empty(rank, dtype=torch.float64)
    _check(lib().sptt_cpd_lambda(cpd, t.data_ptr()), "sptt_cpd_lambda")
    return t


def sptt_cpd_factor(cpd: int, mode: int, rows: int, rank: int, device="cpu") -> torch.Tensor:
    t = torch.empty((rows, rank), dtype=torch.float32, device=device)
    _check(lib().sptt_cpd_factor(cpd, mode, t.data_ptr()), "sptt_cpd_factor")
    return t


def sptt_cpd_gram(cpd: int, mode: int, rank: int) -> torch.Tensor:
    t = torch.empty((rank, rank), dtype=torch.float64)
    _check(lib().sptt_cpd_gram(cpd, mode, t.data_ptr()), "sptt_cpd_gram")
    return t


def sptt_cpd_solve_branch(cpd: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sptt_cpd_solve_branch(cpd, ctypes.byref(a), ctypes.byref(b)), "sptt_cpd_solve_branch")
    return a.value, b.value


def sptt_cpd_timers(cpd: int):
    ms = (ctypes.c_double * SPTT_NUM_TIMERS)()
    cnt = (ctypes.c_int64 * SPTT_NUM_TIMERS)()
    _check(lib().sptt_cpd_timers(cpd, ms, cnt), "sptt_cpd_timers")
    return {n: (ms[i], cnt[i]) for i, n in enumerate(TIMER_NAMES)}


def sptt_cpd_als(dims, inds, vals, rank: int, max_iters: int, tol: float = 0.0,
                 factors_out: Optional[Sequence[torch.Tensor]] = None,
                 lambda_out: Optional[torch.Tensor] = None, stream=None, **opts):
    """One-shot CP-ALS. Inputs may be host or device tensors (host ones are
    copied inside the call); outputs are written into the given tensors.
    Returns (fit, iters)."""
    coo = _Coo(dims, inds, vals)
    o, keep = _opts(**opts)
    fo = None
    if factors_out is not None:
        fo = (ctypes.c_void_p * len(dims))(*[0 if t is None else t.data_ptr() for t in factors_out])
    fit = ctypes.c_double()
    it = ctypes.c_int32()
    _check(lib().sptt_cpd_als(ctypes.byref(coo.c), rank, max_iters, tol, ctypes.byref(o),
                              _stream(stream), fo, _ptr(lambda_out), ctypes.byref(fit),
                              ctypes.byref(it)), "sptt_cpd_als")
    del keep
    return fit.value, it.value


def sptt_cpd_save(cpd: int) -> bytes:
    """The run's state as a checkpoint (see include/sptt.h)."""
    need = ctypes.c_size_t()
    _check(lib().sptt_cpd_save(cpd, None, 0, ctypes.byref(need)), "sptt_cpd_save")
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().sptt_cpd_save(cpd, buf, need.value, ctypes.byref(need)), "sptt_cpd_save")
    return buf.raw


def sptt_cpd_load(cpd: int, data: bytes):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib().sptt_cpd_load(cpd, buf, len(data)), "sptt_cpd_load")


def sptt_debug_fail_alloc_after(countdown: int):
    lib().sptt_debug_fail_alloc_after(countdown)


def sptt_debug_launch_count() -> int:
    return lib().sptt_debug_launch_count()


def sptt_batch_create(tensors, rank: int, stream=None, **opts):
    """tensors: list of (dims, inds, vals). Returns (handle, keepalive)."""
    coos = [_Coo(d, i, v) for (d, i, v) in tensors]
    arr = (sptt_coo * len(coos))(*[c.c for c in coos])
    o, keep = _opts(**opts)
    out = ctypes.c_void_p()
    _check(lib().sptt_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(coos), rank, ctypes.byref(o),
                                   _stream(stream), ctypes.byref(out)), "sptt_batch_create")
    del keep, coos
    return out.value


def sptt_batch_free(b: int):
    lib().sptt_batch_free(b)


def sptt_batch_init(b: int):
    _check(lib().sptt_batch_init(b), "sptt_batch_init")


def sptt_batch_run(b: int, iters: int):
    _check(lib().sptt_batch_run(b, iters), "sptt_batch_run")


def sptt_batch_fit_history(b: int, t: int, cap: int = 4096):
    buf = (ctypes.c_double * cap)()
    n = ctypes.c_int32()
    _check(lib().sptt_batch_fit_history(b, t, buf, cap, ctypes.byref(n)), "sptt_batch_fit_history")
    return list(buf[:n.value])


def sptt_batch_factor(b: int, t: int, mode: int, rows: int, rank: int) -> torch.Tensor:
    out = torch.empty((rows, rank), dtype=torch.float32)
    _check(lib().sptt_batch_factor(b, t, mode, out.data_ptr()), "sptt_batch_factor")
    return out


def sptt_batch_lambda(b: int, t: int, rank: int) -> torch.Tensor:
    out = torch.empty(rank, dtype=torch.float64)
    _check(lib().sptt_batch_lambda(b, t, out.data_ptr()), "sptt_batch_lambda")
    return out


def sptt_batch_info(b: int):
    grid = ctypes.c_int32()
    chunks = (ctypes.c_int64 * SPTT_MAX_MODES)()
    tiles = (ctypes.c_int64 * SPTT_MAX_MODES)()
    _check(lib().sptt_batch_info(b, ctypes.byref(grid), chunks, tiles), "sptt_batch_info")
    return grid.value, list(chunks), list(tiles)


def sptt_batch_schedule(b: int):
    """(chunk, block, variant, order) the batch runs with, the plan-1 timed
    run of the chosen candidate (ms) and how many candidates were timed."""
    out = sptt_sched()
    ms = ctypes.c_float()
    n = ctypes.c_int32()
    _check(lib().sptt_batch_schedule(b, ctypes.byref(out), ctypes.byref(ms), ctypes.byref(n)), "sptt_batch_schedule")
    return out.as_tuple(), ms.value, n.value


def sptt_batch_phase_ms(b: int):
    ms = (ctypes.c_double * 10)()
    _check(lib().sptt_batch_phase_ms(b, ms), "sptt_batch_phase_ms")
    names = ("mttkrp", "normal_eq", "row_solve", "finalize_fit", "normalize")
    out = dict(zip(names, list(ms)[:5]))
    out.update({k + "_barrier_wait": v for k, v in zip(names, list(ms)[5:])})
    return out


def sptt_debug_batch_stall(b: int, skip_block: int, timeout_ns: int):
    _check(lib().sptt_debug_batch_stall(b, skip_block, timeout_ns), "sptt_debug_batch_stall")


def sptt_sched_candidates(nnz: int = 1 << 30):
    """The candidate schedules (chunk, block, variant, order) for a tensor of nnz non-zeros."""
    n = lib().sptt_sched_candidates(int(nnz), None, 0)
    arr = (sptt_sched * n)()
    lib().sptt_sched_candidates(int(nnz), arr, n)
    return [arr[i].as_tuple() for i in range(n)]


def sptt_level_order(dims, root: int, kind: int):
    """The CSF level order of kind 0 / 1 / 2 (see sptt_sched::order)."""
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    out = (ctypes.c_int32 * len(dims))()
    _check(lib().sptt_level_order(d, len(dims), root, kind, out), "sptt_level_order")
    return list(out)


def sptt_sched_default(dims, root: int, rank: int, dtype: int = SPTT_F32, nnz: int = 1 << 30):
    """The library's default schedule (chunk, block, variant, order) for this tensor shape."""
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    out = sptt_sched()
    _check(lib().sptt_sched_default(d, len(dims), root, rank, dtype, int(nnz), ctypes.byref(out)),
           "sptt_sched_default")
    return out.as_tuple()


def sptt_autotune(dims, inds, vals, root: int, rank: int, dtype: int = SPTT_F32, reps: int = 3, stream=None):
    """Median time (ms) of the root-mode MTTKRP under every candidate schedule."""
    coo = _Coo(dims, inds, vals)
    n = lib().sptt_sched_candidates(int(vals.numel()), None, 0)
    ms = (ctypes.c_float * n)()
    _check(lib().sptt_autotune(ctypes.byref(coo.c), root, rank, dtype, reps, ms, _stream(stream)),
           "sptt_autotune")
    return list(ms)


def sptt_csf_features(csf: int, rank: int, factor_dtype: int = SPTT_F32, stream=None):
    f = (ctypes.c_float * 16)()
    _check(lib().sptt_csf_features(csf, rank, factor_dtype, f, _stream(stream)), "sptt_csf_features")
    return list(f)


def sptt_mlp_create(seed: int = 0) -> int:
    out = ctypes.c_void_p()
    _check(lib().sptt_mlp_create(ctypes.c_uint64(seed), ctypes.byref(out)), "sptt_mlp_create")
    return out.value


def sptt_mlp_free(m: int):
    lib().sptt_mlp_free(m)


def sptt_mlp_nparams() -> int:
    return lib().sptt_mlp_nparams()


def sptt_mlp_get(m: int):
    P = torch.empty(sptt_mlp_nparams(), dtype=torch.float32)
    mu = torch.empty(16, dtype=torch.float32)
    sd = torch.empty(16, dtype=torch.float32)
    _check(lib().sptt_mlp_get(m, P.data_ptr(), mu.data_ptr(), sd.data_ptr()), "sptt_mlp_get")
    return P, mu, sd


def sptt_mlp_set(m: int, params=None, mu=None, sd=None):
    keep = [None if x is None else x.contiguous().to(torch.float32) for x in (params, mu, sd)]
    _check(lib().sptt_mlp_set(m, *[_ptr(x) for x in keep]), "sptt_mlp_set")


def sptt_mlp_forward(m: int, X: torch.Tensor, stream=None) -> torch.Tensor:
    Y = torch.empty((X.shape[0], 16), dtype=torch.float32, device=X.device)
    _check(lib().sptt_mlp_forward(m, X.data_ptr(), X.shape[0], Y.data_ptr(), _stream(stream)),
           "sptt_mlp_forward")
    return Y


def sptt_mlp_loss_grad(m: int, X: torch.Tensor, T: torch.Tensor, stream=None):
    loss = ctypes.c_float()
    G = torch.empty(sptt_mlp_nparams(), dtype=torch.float32)
    _check(lib().sptt_mlp_loss_grad(m, X.data_ptr(), T.data_ptr(), X.shape[0], ctypes.byref(loss),
                                    G.data_ptr(), _stream(stream)), "sptt_mlp_loss_grad")
    return loss.value, G


def sptt_mlp_train(m: int, X: torch.Tensor, T: torch.Tensor, steps: int, lr: float = 1e-3, stream=None):
    hist = torch.empty(max(steps, 1), dtype=torch.float32)
    _check(lib().sptt_mlp_train(m, X.data_ptr(), T.data_ptr(), X.shape[0], steps, ctypes.c_float(lr),
                                hist.data_ptr(), _stream(stream)), "sptt_mlp_train")
    return hist[:steps]


def sptt_mlp_predict(m: int, feats, stream=None):
    F = torch.as_tensor(feats, dtype=torch.float32).reshape(-1, 16).contiguous()
    n = F.shape[0]
    choice = (ctypes.c_int32 * n)()
    pred = torch.empty((n, 16), dtype=torch.float32)
    _check(lib().sptt_mlp_predict(m, F.data_ptr(), n, choice, pred.data_ptr(), _stream(stream)),
           "sptt_mlp_predict")
    return list(choice), pred


class Mlp:
    """The learned scheduler (freed with the object)."""

    def __init__(self, seed: int = 0):
        self.handle = sptt_mlp_create(seed)

    def close(self):
        if self.handle:
            sptt_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Owning wrappers
# ---------------------------------------------------------------------------

class Csf:
    """A CSF tree on the device (freed with the object)."""

    def __init__(self, dims, inds, vals, root_mode: int, level_order=None, stream=None):
        self.dims = [int(d) for d in dims]
        self.handle = sptt_csf_build(dims, inds, vals, root_mode, level_order, stream)
        self.nmodes, self.order, self.nfibs = sptt_csf_shape(self.handle)
        self.root = root_mode

    def levels(self):
        return [sptt_csf_copy_level(self.handle, l) for l in range(self.nmodes)]

    def mttkrp(self, factors, out=None, ld=None, factor_dtype=SPTT_F32, sched=None, stream=None):
        if out is None:
            if ld is None:
                ld = next(f.shape[1] for f in factors if f is not None)
            dev = next(f.device for f in factors if f is not None)
            out = torch.empty((self.dims[self.root], ld), dtype=torch.float32, device=dev)
        return sptt_mttkrp(self.handle, factors, out, factor_dtype, sched, stream)

    def mttkrp_mode(self, mode, factors, out=None, ld=None, factor_dtype=SPTT_F32, sched=None, stream=None):
        if out is None:
            if ld is None:
                ld = next(f.shape[1] for f in factors if f is not None)
            dev = next(f.device for f in factors if f is not None)
            out = torch.empty((self.dims[mode], ld), dtype=torch.float32, device=dev)
        return sptt_mttkrp_mode(self.handle, mode, factors, out, factor_dtype, sched, stream)

    def close(self):
        if self.handle:
            sptt_csf_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched CP-ALS of many small tensors (freed with the object)."""

    def __init__(self, tensors, rank: int, stream=None, **opts):
        self.dims = [list(map(int, d)) for (d, _, _) in tensors]
        self.rank = rank
        self.handle = sptt_batch_create(tensors, rank, stream, **opts)

    def init(self):
        sptt_batch_init(self.handle)
        return self

    def run(self, iters: int):
        sptt_batch_run(self.handle, iters)

    def fit_history(self, t: int):
        return sptt_batch_fit_history(self.handle, t)

    def factor(self, t: int, mode: int):
        return sptt_batch_factor(self.handle, t, mode, self.dims[t][mode], self.rank)

    def lam(self, t: int):
        return sptt_batch_lambda(self.handle, t, self.rank)

    def info(self):
        return sptt_batch_info(self.handle)

    def schedule(self):
        return sptt_batch_schedule(self.handle)

    def close(self):
        if self.handle:
            sptt_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cpd:
    """A CP-ALS run on the device (freed with the object)."""

    def __init__(self, dims, inds, vals, rank: int, stream=None, **opts):
        self.dims = [int(d) for d in dims]
        self.rank = rank
        self.handle = sptt_cpd_create(dims, inds, vals, rank, stream, **opts)

    def init(self, init=None):
        sptt_cpd_init(self.handle, init)
        return self

    def iterate(self, iters: int, tol: float = 0.0) -> int:
        return sptt_cpd_iterate(self.handle, iters, tol)

    def refine(self, iters: int = 1):
        sptt_cpd_refine(self.handle, iters)

    def fit(self):
        return sptt_cpd_fit(self.handle)

    def fit_history(self):
        return sptt_cpd_fit_history(self.handle)

    def lam(self):
        return sptt_cpd_lambda(self.handle, self.rank)

    def save(self) -> bytes:
        return sptt_cpd_save(self.handle)

    def load(self, data: bytes):
        sptt_cpd_load(self.handle, data)
        return self

    def factor(self, mode: int, device="cpu"):
        return sptt_cpd_factor(self.handle, mode, self.dims[mode], self.rank, device)

    def gram(self, mode: int):
        return sptt_cpd_gram(self.handle, mode, self.rank)

    def solve_branch(self):
        return sptt_cpd_solve_branch(self.handle)

    def timers(self):
        return sptt_cpd_timers(self.handle)

    def close(self):
        if self.handle:
            sptt_cpd_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
