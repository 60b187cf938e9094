"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module holds only input construction: random draws and the fixed recipes
that shape them.  It contains none of the factorization's arithmetic, and it
imports neither the oracle nor the GPU library.

Random numbers come from numpy's counter-based Philox bit generator keyed by
(seed, stream), so any matrix can be regenerated bit-identically on any host.
The recipes mirror the paper's workload -- square matrices with random,
uniformly distributed entries (Sec. 6.1) -- plus the variants used to stress
the mixed-precision solver (normal entries, row scaling, diagonal scaling) and
a family with well-separated pivot candidates for bit-exact pivot checks.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int = 0, stream: int = 0) -> np.random.Generator:
    """Philox generator for (seed, stream); distinct streams never overlap."""
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def _pad(A: np.ndarray, lda: int | None) -> np.ndarray:
    """Return a column-major (Fortran) array; with ``lda`` > rows, embed A in
    an lda x n buffer whose padding rows hold NaN so reads of them show."""
    m, n = A.shape
    if lda is None or lda == m:
        return np.asfortranarray(A)
    assert lda >= m
    buf = np.full((lda, n), np.nan, dtype=A.dtype, order="F")
    buf[:m, :] = A
    return buf


def uniform_matrix(m: int, n: int | None = None, seed: int = 0, stream: int = 0,
                   lo: float = -1.0, hi: float = 1.0, lda: int | None = None) -> np.ndarray:
    """iid U[lo, hi) entries, FP64, column-major (the paper's workload)."""
    n = m if n is None else n
    A = rng(seed, stream).uniform(lo, hi, size=(n, m)).T  # column-major fill order
    return _pad(np.asfortranarray(A), lda)


def normal_matrix(m: int, n: int | None = None, seed: int = 0, stream: int = 0,
                  lda: int | None = None) -> np.ndarray:
    """iid N(0, 1) entries, FP64, column-major."""
    n = m if n is None else n
    A = rng(seed, stream).standard_normal(size=(n, m)).T
    return _pad(np.asfortranarray(A), lda)


def row_scaled(A: np.ndarray, seed: int = 0, stream: int = 3, lo: float = -3.0,
               hi: float = 3.0) -> np.ndarray:
    """Multiply row i of A by 10**u_i, u_i ~ U[lo, hi) (a badly row-scaled input)."""
    u = rng(seed, stream).uniform(lo, hi, size=A.shape[0])
    return np.asfortranarray(A * (10.0 ** u)[:, None])


def diag_scaled_normal(n: int, seed: int = 0, stream: int = 0, lo: float = -2.0,
                       hi: float = 2.0) -> np.ndarray:
    """diag(d) G with G iid N(0,1) and d_i = 10**u_i, u_i ~ U[lo, hi).

    d is rounded to single precision: pow is not correctly rounded, so its last
    bit differs between math libraries (x86 SIMD, aarch64 libm); after the
    rounding every platform builds the same matrix bit for bit."""
    G = normal_matrix(n, seed=seed, stream=stream)
    u = rng(seed, stream + 4).uniform(lo, hi, size=n)
    d = (10.0 ** u).astype(np.float32).astype(np.float64)
    return np.asfortranarray(G * d[:, None])


def ones_rhs(A: np.ndarray, nrhs: int = 1) -> np.ndarray:
    """b = A * ones(n) (so the exact solution is all ones), as an n x nrhs array."""
    n = A.shape[0]
    b = A[:n, :n] @ np.ones(n)
    return np.asfortranarray(np.repeat(b[:, None], nrhs, axis=1))


def random_rhs(A: np.ndarray, nrhs: int, seed: int = 0, stream: int = 1):
    """B = A X_true with X_true iid U[-1, 1); returns (B, X_true)."""
    n = A.shape[0]
    X = np.asfortranarray(rng(seed, stream).uniform(-1.0, 1.0, size=(nrhs, n)).T)
    return np.asfortranarray(A[:n, :n] @ X), X


def separated_matrix(n: int, seed: int = 0, stream: int = 2, factor: float = 4.0, perm=None):
    """A = Pi D with D strictly column diagonally dominant by ``factor``.

    D has off-diagonal entries iid U[-1, 1) and d_jj = +-factor * (sum of
    |d_ij| over i != j).  Row i of A is row perm[i] of D, i.e. A[i] = D[perm[i]];
    perm is drawn at random unless given.  Returns (A, perm).  Elimination with partial pivoting on such a matrix
    picks, at step j, the row holding D's diagonal entry of column j, so the
    pivot sequence is a closed-form function of perm and every pivot choice has
    a wide margin.
    """
    g = rng(seed, stream)
    D = g.uniform(-1.0, 1.0, size=(n, n))
    np.fill_diagonal(D, 0.0)
    colsum = np.abs(D).sum(axis=0)
    sign = np.where(g.uniform(size=n) < 0.5, -1.0, 1.0)
    D[np.arange(n), np.arange(n)] = sign * factor * np.maximum(colsum, 1.0)
    drawn = g.permutation(n)
    perm = drawn if perm is None else np.asarray(perm, dtype=np.int64)
    A = np.asfortranarray(D[perm, :])
    return A, perm


def spd_matrix(n: int, seed: int = 0, stream: int = 7):
    """Symmetric positive definite A = G G^T / n + I with G iid U[-1, 1)
    (eigenvalues in [1, about 1 + 4/3]); both triangles stored, exactly symmetric."""
    g = rng(seed, stream)
    G = g.uniform(-1.0, 1.0, size=(n, n))
    A = (G @ G.T) / max(n, 1)
    A = 0.5 * (A + A.T) + np.eye(n)
    return np.asfortranarray(A)


def batched_sizes(count: int, seed: int = 0, stream: int = 5, lo: int = 16, hi: int = 512):
    """Sizes n_i = round(exp(U[ln lo, ln hi])) (log-uniform), and nrhs_i ~ U{1..8}."""
    g = rng(seed, stream)
    n = np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    n = np.clip(n, lo, hi)
    nrhs = g.integers(1, 9, size=count).astype(np.int64)
    return n, nrhs


def batched_matrices(sizes, seed: int = 0, stream: int = 6):
    """One iid U[-1,1) matrix per size, each from its own stream."""
    return [uniform_matrix(int(s), seed=seed, stream=stream * 100003 + i)
            for i, s in enumerate(sizes)]
