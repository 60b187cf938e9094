"""CPU oracle for blocked LU with partial pivoting (arXiv 1804.07017).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; never
by the GPU library.  The arithmetic lives in ``oracle.c`` (plain C, FP64,
``-ffp-contract=off``); this module compiles it with gcc and marshals numpy
arrays to it with ctypes.

Each routine states the passage of the paper it restates:

* ``getrf``  -- LU_unb of algorithm LU_blk (RL1, Sec. 3): unblocked
  right-looking elimination with partial pivoting; blocking (RL1-RL3) and the
  static look-ahead (Sec. 4, Listing 5) only re-order these operations.
* ``laswp``  -- the row permutation of the getrf decomposition (Sec. 3.4).
* ``trsm_lower_unit`` -- RL2, ``A12 := trilu(A11)^{-1} A12``.
* ``gemm_update``     -- RL3, ``A22 := A22 - A21 A12``.
* ``getrs``  -- the triangular solves paired with getrf (not in the paper).
* ``backward_error`` / ``factor_error`` -- the normwise backward errors used
  as pass criteria (definitions, compensated sums).
* ``potrf`` -- Cholesky A = L L^T (unblocked, right-looking), the factorization
  the paper names as fitting the same blocked / look-ahead skeleton (Sec. 1, 7).
* ``chol_error`` -- ||A0 - L L^T|| / (n ||A0||) (compensated sums).
* ``geqr2`` -- Householder QR, the unblocked form of the geqrf the paper's QR
  experiments reorganise with look-ahead (Sec. 6); ``qr_q`` forms Q from the
  reflectors and ``qr_error`` gives ||A0 - Q R|| / (n ||A0||) and ||Q^T Q - I||.
* ``round_*`` -- ties-to-even rounding onto bf16 / fp16 / e4m3 / fp32.
* ``quant_e4m3_rows`` / ``quant_e4m3_cols`` -- power-of-two block scaling onto
  e4m3 (one scale per row of L21 / per column of U12) for the FP8 update.

Parity status: every function here is pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so with gcc (OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        sig = {
            "oracle_num_threads": (i32, []),
            "oracle_getrf": (i32, [i64, i64, vp, i64, vp, vp, i32]),
            "oracle_getrf_steps": (i32, [i64, i64, vp, i64, vp, vp, i32, i64]),
            "oracle_laswp": (None, [i64, vp, i64, i64, i64, vp]),
            "oracle_trsm_lower_unit": (None, [i64, i64, vp, i64, vp, i64]),
            "oracle_trsm_upper": (None, [i64, i64, vp, i64, vp, i64]),
            "oracle_gemm_update": (None, [i64, i64, i64, vp, i64, vp, i64, vp, i64]),
            "oracle_getrs": (None, [i64, i64, vp, i64, vp, vp, i64]),
            "oracle_norm_inf": (dbl, [i64, i64, vp, i64]),
            "oracle_backward_error": (dbl, [i64, i64, vp, i64, vp, i64, vp, i64, vp, i64]),
            "oracle_factor_error": (dbl, [i64, vp, i64, vp, i64, vp]),
            "oracle_round_bf16": (None, [i64, vp, vp]),
            "oracle_round_fp16": (None, [i64, vp, vp]),
            "oracle_round_e4m3": (None, [i64, vp, vp]),
            "oracle_round_fp32": (None, [i64, vp, vp]),
            "oracle_quant_e4m3_blocks": (None, [i64, i64, vp, i64, i64, vp, vp]),
            "oracle_potrf": (i32, [i64, vp, i64]),
            "oracle_chol_error": (dbl, [i64, vp, i64, vp, i64]),
            "oracle_geqr2": (None, [i64, i64, vp, i64, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    return _load().oracle_num_threads()


def getrf(A, nthreads: int = 0):
    """Unblocked GEPP of an m x n matrix (RL1).  Returns (LU, ipiv, info, gap).

    ``ipiv`` is int32, 1-based, LAPACK sequential-interchange form; ``gap[j]``
    is the relative separation of the two largest pivot candidates at step j.
    """
    lib = _load()
    LU = _f64(A)
    m, n = LU.shape
    k = min(m, n)
    ipiv = np.zeros(max(k, 1), dtype=np.int32)
    gap = np.zeros(max(k, 1), dtype=np.float64)
    info = lib.oracle_getrf(m, n, _ptr(LU), max(m, 1), _ptr(ipiv), _ptr(gap), int(nthreads))
    return LU, ipiv[:k].copy(), int(info), gap[:k].copy()


def getrf_steps_inplace(A: np.ndarray, steps: int, nthreads: int = 0) -> int:
    """Run the first `steps` elimination steps of getrf in place on a
    Fortran-ordered float64 array (no copy; used to time a bounded sample)."""
    lib = _load()
    assert A.dtype == np.float64 and A.flags["F_CONTIGUOUS"]
    m, n = A.shape
    ipiv = np.zeros(max(min(m, n), 1), dtype=np.int32)
    return int(lib.oracle_getrf_steps(m, n, _ptr(A), max(m, 1), _ptr(ipiv), None, int(nthreads), int(steps)))


def laswp(A, k1: int, k2: int, ipiv):
    """Apply interchanges ipiv[k1:k2] (1-based) to all columns of a copy of A."""
    lib = _load()
    out = _f64(A)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_laswp(out.shape[1], _ptr(out), max(out.shape[0], 1), k1, k2, _ptr(piv))
    return out


def trsm_lower_unit(L, B):
    """Return trilu(L)^{-1} B (RL2)."""
    lib = _load()
    Lf, out = _f64(L), _f64(B)
    m = Lf.shape[0]
    lib.oracle_trsm_lower_unit(m, out.shape[1], _ptr(Lf), max(m, 1), _ptr(out), max(m, 1))
    return out


def trsm_upper(U, B):
    """Return triu(U)^{-1} B."""
    lib = _load()
    Uf, out = _f64(U), _f64(B)
    m = Uf.shape[0]
    lib.oracle_trsm_upper(m, out.shape[1], _ptr(Uf), max(m, 1), _ptr(out), max(m, 1))
    return out


def gemm_update(C, A, B):
    """Return C - A B (RL3), plain loops in FP64."""
    lib = _load()
    Cf, Af, Bf = _f64(C), _f64(A), _f64(B)
    m, n = Cf.shape
    k = Af.shape[1]
    lib.oracle_gemm_update(m, n, k, _ptr(Af), max(m, 1), _ptr(Bf), max(k, 1), _ptr(Cf), max(m, 1))
    return Cf


def getrs(LU, ipiv, B):
    """Solve A X = B from getrf factors; B may be a vector or an n x nrhs array."""
    lib = _load()
    LUf = _f64(LU)
    vec = np.asarray(B).ndim == 1
    X = _f64(B)
    n = LUf.shape[0]
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    lib.oracle_getrs(n, X.shape[1], _ptr(LUf), max(n, 1), _ptr(piv), _ptr(X), max(n, 1))
    return X[:, 0].copy() if vec else X


def norm_inf(A) -> float:
    lib = _load()
    Af = _f64(A)
    return float(lib.oracle_norm_inf(Af.shape[0], Af.shape[1], _ptr(Af), max(Af.shape[0], 1)))


def backward_error(A, X, B) -> float:
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    lib = _load()
    Af, Xf, Bf = _f64(A), _f64(X), _f64(B)
    n = Af.shape[0]
    return float(lib.oracle_backward_error(n, Xf.shape[1], _ptr(Af), max(n, 1), _ptr(Xf),
                                           max(n, 1), _ptr(Bf), max(n, 1), None, 1))


def factor_error(A0, LU, ipiv) -> float:
    """||P A0 - L U||_inf / (n ||A0||_inf) for getrf output (LU, ipiv)."""
    lib = _load()
    Af, LUf = _f64(A0), _f64(LU)
    n = Af.shape[0]
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    return float(lib.oracle_factor_error(n, _ptr(Af), max(n, 1), _ptr(LUf), max(n, 1), _ptr(piv)))


def _round(name, x):
    lib = _load()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.empty_like(a)
    getattr(lib, name)(a.size, _ptr(a), _ptr(out))
    return out


def round_bf16(x):
    return _round("oracle_round_bf16", x)


def round_fp16(x):
    return _round("oracle_round_fp16", x)


def round_e4m3(x):
    return _round("oracle_round_e4m3", x)


def round_fp32(x):
    return _round("oracle_round_fp32", x)


def quant_e4m3_rows(X):
    """Per-row power-of-two scaled e4m3 quantisation.  Returns (Q, s) with
    X ~= diag(s) Q; Q holds e4m3 values, s powers of two."""
    lib = _load()
    Xf = _f64(X)
    m, k = Xf.shape
    Q = np.zeros_like(Xf)
    sc = np.zeros(max(m, 1))
    lib.oracle_quant_e4m3_blocks(m, k, _ptr(Xf), 1, max(m, 1), _ptr(Q), _ptr(sc))
    return Q, sc[:m]


def quant_e4m3_cols(X):
    """Per-column power-of-two scaled e4m3 quantisation: X ~= Q diag(t)."""
    lib = _load()
    Xf = _f64(X)
    k, n = Xf.shape
    Q = np.zeros_like(Xf)
    sc = np.zeros(max(n, 1))
    lib.oracle_quant_e4m3_blocks(n, k, _ptr(Xf), max(k, 1), 1, _ptr(Q), _ptr(sc))
    return Q, sc[:n]


def potrf(A):
    """Cholesky factor of a symmetric positive definite matrix.  Returns (L, info):
    L is the lower triangle (strict upper part zero) and info is 0, or j when
    the leading j x j minor is not positive definite (L is then not meaningful)."""
    lib = _load()
    W = _f64(A)
    n = W.shape[0]
    info = lib.oracle_potrf(n, _ptr(W), max(n, 1))
    return np.tril(W), int(info)


def chol_error(A0, L) -> float:
    """||A0 - L L^T||_inf / (n ||A0||_inf) with the lower triangle of L."""
    lib = _load()
    A0f, Lf = _f64(A0), _f64(L)
    n = A0f.shape[0]
    return float(lib.oracle_chol_error(n, _ptr(A0f), max(n, 1), _ptr(Lf), max(Lf.shape[0], 1)))


def geqr2(A):
    """Householder QR of an m x n matrix.  Returns (QR, tau): R in the upper
    triangle, the reflectors' vectors (unit first entry implied) below it, and
    tau[j] the reflectors' scalars (LAPACK geqrf layout)."""
    lib = _load()
    W = _f64(A)
    m, n = W.shape
    tau = np.zeros(max(min(m, n), 1), dtype=np.float64)
    lib.oracle_geqr2(m, n, _ptr(W), max(m, 1), _ptr(tau))
    return W, tau[:min(m, n)].copy()


def qr_q(QR, tau):
    """Q (m x m) = H_0 H_1 ... H_{k-1} from geqr2's reflectors, H_j = I - tau_j v_j v_j^T."""
    QR = np.asarray(QR, dtype=np.float64)
    m = QR.shape[0]
    Q = np.eye(m)
    for j in range(len(tau) - 1, -1, -1):
        v = np.zeros(m)
        v[j] = 1.0
        v[j + 1:] = QR[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return Q


def qr_error(A0, QR, tau):
    """(||A0 - Q R||_inf / (n ||A0||_inf), ||Q^T Q - I||_inf) for square or tall A0."""
    A0 = np.asarray(A0, dtype=np.float64)
    n = A0.shape[1]
    Q = qr_q(QR, tau)
    R = np.triu(np.asarray(QR, dtype=np.float64))
    res = np.abs(A0 - Q @ R).sum(axis=1).max()
    anorm = np.abs(A0).sum(axis=1).max()
    orth = np.abs(Q.T @ Q - np.eye(Q.shape[0])).sum(axis=1).max()
    return (res / (max(n, 1) * anorm) if anorm > 0 else res), orth
