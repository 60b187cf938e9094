"""Argument marshalling from torch tensors to the C ABI (same names as the C calls).

Matrices are column-major: a tensor of shape (rows, cols) with stride
(1, ld), ld >= rows -- e.g. ``colmajor(rows, cols)`` below, or
``torch.from_numpy(np.asfortranarray(a)).cuda()``.
"""
from __future__ import annotations

import ctypes

import torch

from ._lib import LU_F32, LU_F64, LU_WARN_NOT_CONVERGED, LuError, LuOpts, lib

_DT = {torch.float64: LU_F64, torch.float32: LU_F32}


def colmajor(rows: int, cols: int, dtype=torch.float64, device="cuda", ld: int | None = None):
    """An uninitialised column-major (rows x cols) tensor with leading dimension ld."""
    ld = rows if ld is None else ld
    buf = torch.empty((max(cols, 1), max(ld, 1)), dtype=dtype, device=device)
    return buf.t()[:rows, :cols]


def to_colmajor(t: torch.Tensor, ld: int | None = None) -> torch.Tensor:
    out = colmajor(t.shape[0], t.shape[1], t.dtype, t.device, ld)
    out.copy_(t)
    return out


def _ld(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return max(int(t.stride(1)) if t.shape[1] > 1 else int(t.shape[0]), 1)


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


def _check(name: str, rc: int, ok_positive: bool = False) -> int:
    if rc < 0 or (rc > 0 and not ok_positive):
        detail = lib().lu_last_error().decode(errors="replace")
        raise LuError(name, rc, detail)
    return rc


def default_opts(**kw) -> LuOpts:
    o = LuOpts()
    lib().lu_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "sched":
            o.set_schedule(v)
        else:
            setattr(o, k, int(v))
    return o


class Handle:
    """Owns an lu_handle (workspace and internal streams)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check("lu_create", lib().lu_create(ctypes.byref(h)))
        self._h = h

    @property
    def ptr(self):
        return self._h

    def set_stream(self, stream: torch.cuda.Stream | None = None):
        s = stream if stream is not None else torch.cuda.current_stream()
        _check("lu_set_stream", lib().lu_set_stream(self._h, ctypes.c_void_p(s.cuda_stream)))

    def close(self):
        if self._h:
            lib().lu_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles: dict[int, Handle] = {}


def _handle(h: Handle | None) -> Handle:
    if h is None:
        dev = torch.cuda.current_device()
        h = _handles.get(dev)
        if h is None:
            h = _handles[dev] = Handle()
    h.set_stream()
    return h


def lu_launch_count() -> int:
    return int(lib().lu_launch_count())


def lu_factor(A: torch.Tensor, ipiv: torch.Tensor, nb: int = 256) -> int:
    """In-place FP64 LU (synchronous).  Returns info (0 or first zero pivot)."""
    n = A.shape[0]
    return _check("lu_factor", lib().lu_factor(n, _p(A), _ld(A, "A"), _p(ipiv), nb), ok_positive=True)


def lu_solve(LU: torch.Tensor, ipiv: torch.Tensor, B: torch.Tensor) -> None:
    """In-place FP64 solve of B (n x nrhs, ld n) with lu_factor output (ld n)."""
    n, nrhs = B.shape
    _check("lu_solve", lib().lu_solve(n, nrhs, _p(LU), _p(ipiv), _p(B)))


def lu_factor_ex(A: torch.Tensor, ipiv: torch.Tensor, info: torch.Tensor, opts: LuOpts | None = None,
                 handle: Handle | None = None) -> None:
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    _check("lu_factor_ex", lib().lu_factor_ex(h.ptr, _DT[A.dtype], A.shape[0], _p(A), _ld(A, "A"), _p(ipiv),
                                               ctypes.byref(o), _p(info)))


def lu_solve_ex(LU: torch.Tensor, ipiv: torch.Tensor, B: torch.Tensor, handle: Handle | None = None) -> None:
    h = _handle(handle)
    n, nrhs = B.shape
    _check("lu_solve_ex", lib().lu_solve_ex(h.ptr, _DT[LU.dtype], n, nrhs, _p(LU), _ld(LU, "LU"), _p(ipiv),
                                             _p(B), _ld(B, "B")))


def lu_panel_factor_ex(P: torch.Tensor, ipiv: torch.Tensor, info: torch.Tensor, opts: LuOpts | None = None,
                       handle: Handle | None = None) -> None:
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    m, w = P.shape
    _check("lu_panel_factor_ex", lib().lu_panel_factor_ex(h.ptr, _DT[P.dtype], m, w, _p(P), _ld(P, "P"),
                                                           _p(ipiv), ctypes.byref(o), _p(info)))


def lu_laswp_ex(A: torch.Tensor, k1: int, k2: int, ipiv: torch.Tensor, handle: Handle | None = None) -> None:
    h = _handle(handle)
    _check("lu_laswp_ex", lib().lu_laswp_ex(h.ptr, _DT[A.dtype], A.shape[1], _p(A), _ld(A, "A"), k1, k2,
                                             _p(ipiv)))


def lu_trsm_ex(L: torch.Tensor, B: torch.Tensor, handle: Handle | None = None) -> None:
    h = _handle(handle)
    m, n = B.shape
    _check("lu_trsm_ex", lib().lu_trsm_ex(h.ptr, _DT[B.dtype], m, n, _p(L), _ld(L, "L"), _p(B), _ld(B, "B")))


def lu_gemm_update_ex(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, handle: Handle | None = None) -> None:
    h = _handle(handle)
    m, n = C.shape
    k = A.shape[1]
    _check("lu_gemm_update_ex", lib().lu_gemm_update_ex(h.ptr, _DT[C.dtype], m, n, k, _p(A), _ld(A, "A"), _p(B),
                                                         _ld(B, "B"), _p(C), _ld(C, "C")))


def lu_gemm_update_tc_ex(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, prec: int, info: torch.Tensor,
                         handle: Handle | None = None) -> None:
    """C := C - round(A) round(B) on the tensor cores (FP32 C, A, B; k % 64 == 0)."""
    h = _handle(handle)
    m, n = C.shape
    k = A.shape[1]
    _check("lu_gemm_update_tc_ex", lib().lu_gemm_update_tc_ex(h.ptr, prec, m, n, k, _p(A), _ld(A, "A"), _p(B),
                                                               _ld(B, "B"), _p(C), _ld(C, "C"), _p(info)))


def lu_factor_mixed_ex(A: torch.Tensor, ipiv: torch.Tensor, info: torch.Tensor, prec: int, opts: LuOpts | None = None,
                       handle: Handle | None = None) -> None:
    """FP32 LU with the tensor-core trailing update (prec: LU_TU_BF16 / LU_TU_FP16 / LU_TU_F32)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    _check("lu_factor_mixed_ex", lib().lu_factor_mixed_ex(h.ptr, prec, A.shape[0], _p(A), _ld(A, "A"), _p(ipiv),
                                                           ctypes.byref(o), _p(info)))


def lu_gesv_mixed(A: torch.Tensor, B: torch.Tensor, X: torch.Tensor, prec: int, tol: float = 1e-14,
                  max_iter: int = 30, opts: LuOpts | None = None, handle: Handle | None = None):
    """Mixed-precision solve with FP64 refinement.  Returns (status, iters, eta);
    status is 0 or LU_WARN_NOT_CONVERGED (other codes raise)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    n, nrhs = B.shape
    iters = ctypes.c_int(0)
    eta = ctypes.c_double(0.0)
    rc = lib().lu_gesv_mixed(h.ptr, prec, n, nrhs, _p(A), _ld(A, "A"), _p(B), _ld(B, "B"), _p(X), _ld(X, "X"),
                             float(tol), int(max_iter), ctypes.byref(o), ctypes.byref(iters), ctypes.byref(eta))
    if rc != 0 and rc != LU_WARN_NOT_CONVERGED:
        _check("lu_gesv_mixed", rc)
    return rc, iters.value, eta.value


def lu_panel_factor_noalloc(P: torch.Tensor, ipiv: torch.Tensor, info: torch.Tensor, opts: LuOpts | None = None,
                            stream: torch.cuda.Stream | None = None) -> None:
    """Panel factorization that allocates no device memory (scratch in a static
    device array inside the library; concurrent calls on one device race)."""
    o = opts if opts is not None else default_opts()
    s = stream if stream is not None else torch.cuda.current_stream()
    m, w = P.shape
    _check("lu_panel_factor_noalloc", lib().lu_panel_factor_noalloc(_DT[P.dtype], m, w, _p(P), _ld(P, "P"),
                                                                     _p(ipiv), ctypes.byref(o), _p(info),
                                                                     ctypes.c_void_p(s.cuda_stream)))


class Batch:
    """Device-side descriptor arrays for lu_gesv_batched built from lists of
    column-major tensors (all of one dtype)."""

    def __init__(self, mats, ipivs, rhs=None):
        dev = mats[0].device
        self.mats, self.ipivs, self.rhs = mats, ipivs, rhs
        self.n = torch.tensor([m.shape[0] for m in mats], dtype=torch.int32, device=dev)
        self.A = torch.tensor([m.data_ptr() for m in mats], dtype=torch.int64, device=dev)
        self.lda = torch.tensor([_ld(m, "A") for m in mats], dtype=torch.int64, device=dev)
        self.ipiv = torch.tensor([p.data_ptr() for p in ipivs], dtype=torch.int64, device=dev)
        self.info = torch.zeros(len(mats), dtype=torch.int32, device=dev)
        if rhs is not None:
            self.nrhs = torch.tensor([b.shape[1] for b in rhs], dtype=torch.int32, device=dev)
            self.B = torch.tensor([b.data_ptr() for b in rhs], dtype=torch.int64, device=dev)
            self.ldb = torch.tensor([_ld(b, "B") for b in rhs], dtype=torch.int64, device=dev)
        self.dtype = _DT[mats[0].dtype]


def lu_gesv_batched(batch: Batch, handle: Handle | None = None) -> None:
    h = _handle(handle)
    has_b = batch.rhs is not None
    _check("lu_gesv_batched", lib().lu_gesv_batched(
        h.ptr, batch.dtype, len(batch.mats), _p(batch.n), _p(batch.A), _p(batch.lda), _p(batch.ipiv),
        _p(batch.nrhs) if has_b else None, _p(batch.B) if has_b else None, _p(batch.ldb) if has_b else None,
        _p(batch.info)))


def lu_factor_batched(batch: Batch, handle: Handle | None = None) -> None:
    h = _handle(handle)
    _check("lu_factor_batched", lib().lu_factor_batched(
        h.ptr, batch.dtype, len(batch.mats), _p(batch.n), _p(batch.A), _p(batch.lda), _p(batch.ipiv),
        _p(batch.info)))


def lu_solve_batched(batch: Batch, handle: Handle | None = None) -> None:
    """B_i := A_i^{-1} B_i from the factors lu_factor_batched left in batch.mats."""
    if batch.rhs is None:
        raise ValueError("lu_solve_batched needs right-hand sides")
    h = _handle(handle)
    _check("lu_solve_batched", lib().lu_solve_batched(
        h.ptr, batch.dtype, len(batch.mats), _p(batch.n), _p(batch.A), _p(batch.lda), _p(batch.ipiv),
        _p(batch.nrhs), _p(batch.B), _p(batch.ldb), _p(batch.info)))


def lu_potrf_ex(A: torch.Tensor, info: torch.Tensor, opts: LuOpts | None = None,
                handle: Handle | None = None) -> None:
    """In-place Cholesky A = L L^T (A symmetric positive definite, both triangles
    stored, FP64 or FP32); L in the lower triangle, the strict upper overwritten."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    _check("lu_potrf_ex", lib().lu_potrf_ex(h.ptr, _DT[A.dtype], A.shape[0], _p(A), _ld(A, "A"), ctypes.byref(o), _p(info)))


def lu_tune_nb(kind: int, n: int, candidates, reps: int = 3, opts: LuOpts | None = None,
               handle: Handle | None = None):
    """Times the factorization of `kind` (an lu_prec, LU_TUNE_F64 or LU_TUNE_F32) on
    a synthetic n x n matrix for each candidate nb; returns (best_nb, ms list, -1 for
    a skipped candidate) and stores best_nb in the library's table."""
    h = _handle(handle)
    cand = (ctypes.c_int * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_float * len(candidates))()
    best = ctypes.c_int(0)
    o = opts if opts is not None else default_opts()
    _check("lu_tune_nb", lib().lu_tune_nb(h.ptr, int(kind), int(n), cand, len(candidates), int(reps),
                                          ctypes.byref(o), ctypes.byref(best), ms))
    return best.value, [float(t) for t in ms]


def _dev(device):
    return None if device is None else device.encode()


def lu_tune_get(kind: int, n: int, device: str | None = None) -> int:
    """The tuned nb for (device, kind, ceil(log2 n)), 0 if none (device None = current GPU)."""
    return int(lib().lu_tune_get(_dev(device), int(kind), int(n)))


def lu_tune_set(kind: int, n: int, nb: int, ms: float = 0.0, device: str | None = None) -> None:
    _check("lu_tune_set", lib().lu_tune_set(_dev(device), int(kind), int(n), int(nb), float(ms)))


def lu_tune_clear() -> None:
    _check("lu_tune_clear", lib().lu_tune_clear())


def lu_tune_save(path: str) -> None:
    _check("lu_tune_save", lib().lu_tune_save(path.encode()))


def lu_tune_load(path: str) -> None:
    _check("lu_tune_load", lib().lu_tune_load(path.encode()))


def lu_tune_plan(kind: int, n: int, reps: int = 3, opts: LuOpts | None = None, handle: Handle | None = None,
                 cap: int = 4096):
    """Tunes the whole plan of the factorization of `kind` at order n (block size,
    the right update's SM reserve, look-ahead depth, a per-step schedule) and
    stores it in the table.  Returns (best opts, schedule list (empty: fixed nb),
    best ms, best ms without a schedule)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    best = LuOpts()
    buf = (ctypes.c_int32 * cap)()
    bms, fms = ctypes.c_float(0), ctypes.c_float(0)
    _check("lu_tune_plan", lib().lu_tune_plan(h.ptr, int(kind), int(n), int(reps), ctypes.byref(o),
                                              ctypes.byref(best), buf, cap, ctypes.byref(bms), ctypes.byref(fms)))
    sched = [int(buf[i]) for i in range(best.nsched)]
    best.set_schedule(sched)
    return best, sched, float(bms.value), float(fms.value)


def lu_tune_plan_get(kind: int, n: int, device: str | None = None):
    """(nb, reserve, depth, schedule, pf_sms) stored for (device, kind, ceil(log2 n)), or None."""
    nb, res, dep, cnt, pf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    L = lib()
    if not L.lu_tune_plan_get(_dev(device), int(kind), int(n), ctypes.byref(nb), ctypes.byref(res),
                              ctypes.byref(dep), None, 0, ctypes.byref(cnt), ctypes.byref(pf)):
        return None
    buf = (ctypes.c_int32 * max(cnt.value, 1))()
    L.lu_tune_plan_get(_dev(device), int(kind), int(n), None, None, None, buf, cnt.value, None, None)
    return nb.value, res.value, dep.value, [int(buf[i]) for i in range(cnt.value)], pf.value


def lu_step_trace(enable: bool, handle: Handle | None = None) -> Handle:
    """Turns the per-step trace of later factorizations on this handle on or off."""
    h = _handle(handle)
    _check("lu_step_trace", lib().lu_step_trace(h.ptr, 1 if enable else 0))
    return h


def lu_step_trace_read(handle: Handle | None = None):
    """Per-step records of the last traced factorization: a list of dicts with
    k0, kb, span_ms, pu_ms and tu_ms."""
    h = _handle(handle)
    L = lib()
    cnt = int(L.lu_step_trace_read(h.ptr, 0, None, None, None, None, None))
    if cnt < 0:
        raise LuError("lu_step_trace_read", cnt)
    k0 = (ctypes.c_int64 * max(cnt, 1))()
    kb = (ctypes.c_int32 * max(cnt, 1))()
    sp, pu, tu = ((ctypes.c_float * max(cnt, 1))() for _ in range(3))
    L.lu_step_trace_read(h.ptr, cnt, k0, kb, sp, pu, tu)
    return [{"k0": int(k0[i]), "kb": int(kb[i]), "span_ms": float(sp[i]), "pu_ms": float(pu[i]),
             "tu_ms": float(tu[i])} for i in range(cnt)]


def lu_geqrf_ex(A: torch.Tensor, tau: torch.Tensor, info: torch.Tensor, opts: LuOpts | None = None,
                handle: Handle | None = None) -> None:
    """In-place Householder QR (LAPACK geqrf layout) of a column-major FP64/FP32
    m x n matrix; tau receives min(m, n) reflector scalars (nb <= 128)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts(nb=128)
    m, n = A.shape
    _check("lu_geqrf_ex", lib().lu_geqrf_ex(h.ptr, _DT[A.dtype], m, n, _p(A), _ld(A, "A"), _p(tau),
                                            ctypes.byref(o), _p(info)))


def lu_potrf_mixed_ex(A: torch.Tensor, info: torch.Tensor, prec: int, opts: LuOpts | None = None,
                      handle: Handle | None = None) -> None:
    """In-place Cholesky of an FP32 symmetric positive definite matrix with the
    trailing update on the tensor cores in precision `prec` (an lu_prec)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts()
    _check("lu_potrf_mixed_ex", lib().lu_potrf_mixed_ex(h.ptr, int(prec), A.shape[0], _p(A), _ld(A, "A"),
                                                        ctypes.byref(o), _p(info)))


def lu_geqrf_mixed_ex(A: torch.Tensor, tau: torch.Tensor, info: torch.Tensor, prec: int,
                      opts: LuOpts | None = None, handle: Handle | None = None) -> None:
    """Householder QR of an FP32 matrix with the update's last product on the
    tensor cores in precision `prec` (an lu_prec other than FP8)."""
    h = _handle(handle)
    o = opts if opts is not None else default_opts(nb=128)
    m, n = A.shape
    _check("lu_geqrf_mixed_ex", lib().lu_geqrf_mixed_ex(h.ptr, int(prec), m, n, _p(A), _ld(A, "A"), _p(tau),
                                                        ctypes.byref(o), _p(info)))


def lu_tune_batched(dtype: int, sizes, nrhs, cuts, reps: int = 3, handle: Handle | None = None):
    """Times lu_gesv_batched of `dtype` (LU_F64/LU_F32) on a synthetic batch with these
    orders and right-hand-side counts for each tile cut-over; returns (best, ms list)
    and stores the best in the table (kinds LU_TUNE_BATCHED_F64/F32)."""
    h = _handle(handle)
    b = len(sizes)
    nn = (ctypes.c_int * b)(*[int(v) for v in sizes])
    rr = (ctypes.c_int * b)(*[int(v) for v in nrhs])
    cc = (ctypes.c_int * len(cuts))(*[int(v) for v in cuts])
    ms = (ctypes.c_float * len(cuts))()
    best = ctypes.c_int(0)
    _check("lu_tune_batched", lib().lu_tune_batched(h.ptr, int(dtype), b, nn, rr, int(reps), cc, len(cuts),
                                                    ctypes.byref(best), ms))
    return best.value, [float(t) for t in ms]
