"""Row orders that make partial pivoting take a chosen sequence of interchanges.

For A = Pi D with D strictly column diagonally dominant (synth.separated_matrix),
elimination with partial pivoting picks, at step j, the row that holds D's row j
(Sec. 3, RL1: the pivot is the largest entry of the current column, and the
dominant diagonal entry stays the largest).  So any LAPACK-style sequence
ipiv[j] >= j is produced by the row order obtained from the identity by undoing
those interchanges in reverse order.  The patterns below stress the parts of an
interchange implementation that random matrices rarely reach: swaps inside a
32- or nb-wide panel, one row below the panel reached by many steps, no swap at
all, and long mixed chains.
"""
import numpy as np

import synth

PATTERNS = ("identity", "reverse", "last_row", "in_panel", "random", "mixed")


def perm_for_ipiv(piv0):
    """Row order perm (A[i] = D[perm[i]]) whose pivot sequence is piv0 (0-based)."""
    n = len(piv0)
    rows = np.arange(n)
    for j in range(n - 1, -1, -1):
        p = int(piv0[j])
        assert j <= p < n
        rows[j], rows[p] = rows[p], rows[j]
    return rows


def ipiv_pattern(name: str, n: int, seed: int = 0, panel: int = 32):
    """0-based pivot rows piv0[j] >= j of the named pattern."""
    g = synth.rng(seed, 31)
    j = np.arange(n)
    end = np.minimum((j // panel) * panel + panel - 1, n - 1)  # last row of j's panel
    if name == "identity":
        return j.copy()
    if name == "reverse":
        return np.where(j < n // 2, n - 1 - j, j)
    if name == "last_row":
        return np.full(n, n - 1)
    if name == "in_panel":
        return np.where(j % 3 == 0, end, np.where((j % 3 == 1) & (j + 1 <= end), j + 1, j))
    if name == "random":
        return j + np.floor(g.uniform(size=n) * (n - j)).astype(np.int64)
    if name == "mixed":
        kind = g.integers(0, 4, size=n)
        inside = j + np.floor(g.uniform(size=n) * (end - j + 1)).astype(np.int64)
        below = j + np.floor(g.uniform(size=n) * (n - j)).astype(np.int64)
        return np.select([kind == 0, kind == 1, kind == 2], [j, inside, below], n - 1)
    raise ValueError(name)


def patterned_matrix(name: str, n: int, seed: int = 0, panel: int = 32):
    """(A, ipiv) with A = Pi D and ipiv (1-based) the pivots elimination must take."""
    piv0 = ipiv_pattern(name, n, seed, panel)
    A, _ = synth.separated_matrix(n, seed=seed, perm=perm_for_ipiv(piv0))
    return A, piv0 + 1
