"""Pins for the CPU oracle, each against something other than the oracle itself.

The oracle restates LU_unb (RL1 of LU_blk, Sec. 3 of arXiv 1804.07017) plus the
solve, the backward-error definitions and the narrow-format rounding.  These
tests tie it to hand-worked factorizations (tests/golden), brute force on tiny
inputs (Leibniz determinants, Cramer's rule in exact rationals), invariants
that partial pivoting guarantees, closed-form special cases, and library
routines (LAPACK via scipy, numpy matmul, torch dtype conversions).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    data = {}
    lines = [ln.strip() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        parts = lines[i].split()
        key = parts[0]
        if key in ("A", "LU"):
            r, c = int(parts[1]), int(parts[2])
            rows = [[float(v) for v in lines[i + 1 + k].split()] for k in range(r)]
            data[key] = np.array(rows, dtype=np.float64)
            i += 1 + r
        else:
            data[key] = [float(v) for v in parts[1:]]
            i += 1
    return data


def perm_from_ipiv(ipiv, n):
    """Row order of P A built by applying the interchanges to the identity."""
    order = list(range(n))
    for k, p in enumerate(ipiv):
        p = int(p) - 1
        order[k], order[p] = order[p], order[k]
    return np.array(order)


def split_lu(LU):
    n = LU.shape[0]
    L = np.tril(LU[:, :n], -1) + np.eye(LU.shape[0], min(LU.shape))
    U = np.triu(LU[: min(LU.shape), :])
    return L, U


@pytest.mark.parametrize("name", ["lu_2x2.txt", "lu_3x3.txt", "lu_tie_2x2.txt", "lu_zero_pivot_2x2.txt"])
def test_hand_worked(name):
    g = read_golden(name)
    LU, ipiv, info, _ = oracle.getrf(g["A"])
    assert list(ipiv) == [int(v) for v in g["ipiv"]]
    assert info == int(g.get("info", [0])[0])
    np.testing.assert_array_max_ulp(LU, g["LU"], maxulp=1)
    # determinant from the factors: sign of the interchanges times prod(diag U)
    swaps = sum(1 for k, p in enumerate(ipiv) if p - 1 != k)
    det = (-1) ** swaps * np.prod(np.diag(LU))
    assert det == pytest.approx(g["det"][0], rel=1e-15, abs=0)


def leibniz_det(M):
    n = len(M)
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1
        for i in range(n):
            prod *= M[i][perm[i]]
        total += (-1) ** inv * prod
    return total


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_determinant_brute_force(n):
    g = synth.rng(11, n)
    for trial in range(6):
        M = g.integers(-9, 10, size=(n, n))
        exact = leibniz_det(M.tolist())
        LU, ipiv, info, _ = oracle.getrf(M.astype(np.float64))
        swaps = sum(1 for k, p in enumerate(ipiv) if p - 1 != k)
        d = (-1) ** swaps * np.prod(np.diag(LU))
        scale = np.prod(np.abs(np.diag(LU))) + 1.0
        assert abs(d - exact) <= 8 * n * np.finfo(float).eps * scale, (M, exact, d)
        if exact == 0:
            continue
        assert info == 0


def cramer(M, b):
    n = len(M)
    Mf = [[Fraction(int(v)) for v in row] for row in M]
    D = leibniz_det(Mf)
    xs = []
    for c in range(n):
        Mc = [row[:] for row in Mf]
        for r in range(n):
            Mc[r][c] = Fraction(int(b[r]))
        xs.append(leibniz_det(Mc) / D)
    return xs


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_solve_cramer_exact(n):
    g = synth.rng(12, n)
    done = 0
    while done < 4:
        M = g.integers(-9, 10, size=(n, n))
        if leibniz_det(M.tolist()) == 0:
            continue
        b = g.integers(-9, 10, size=n)
        x_exact = np.array([float(v) for v in cramer(M.tolist(), b.tolist())])
        LU, ipiv, info, _ = oracle.getrf(M.astype(float))
        x = oracle.getrs(LU, ipiv, b.astype(float))
        kappa = np.linalg.cond(M.astype(float), np.inf)
        tol = 16 * n * kappa * np.finfo(float).eps * (np.abs(x_exact).max() + 1)
        assert np.abs(x - x_exact).max() <= tol
        done += 1


@pytest.mark.parametrize("m,n", [(1, 1), (7, 7), (33, 33), (64, 40), (40, 64), (130, 130)])
def test_invariants(m, n):
    A = synth.uniform_matrix(m, n, seed=3, stream=m * 1000 + n)
    LU, ipiv, info, gap = oracle.getrf(A)
    k = min(m, n)
    L, U = split_lu(LU)
    assert info == 0
    # |l_ij| <= 1 exactly (|a| <= |pivot| and division is monotone)
    assert np.all(np.abs(np.tril(LU[:, :k], -1)) <= 1.0)
    assert np.all(ipiv >= np.arange(1, k + 1)) and np.all(ipiv <= m)
    order = perm_from_ipiv(ipiv, m)
    PA = A[order, :]
    R = PA - L @ U
    assert np.abs(R).sum(axis=1).max() / (max(m, n) * np.abs(A).sum(axis=1).max()) <= 4 * np.finfo(float).eps
    # the gap definition: relative distance of the top two candidates
    assert np.all((gap >= 0) & (gap <= 1))


def test_factor_error_definition():
    """oracle.factor_error against the same quantity formed with numpy matmul."""
    for n in (5, 50, 120):
        A = synth.normal_matrix(n, seed=4, stream=n)
        LU, ipiv, _, _ = oracle.getrf(A)
        L, U = split_lu(LU)
        PA = A[perm_from_ipiv(ipiv, n), :]
        ref = np.abs(PA - L @ U).sum(axis=1).max() / (n * np.abs(A).sum(axis=1).max())
        got = oracle.factor_error(A, LU, ipiv)
        assert got <= 1e-15
        assert abs(got - ref) <= 4 * np.finfo(float).eps  # both are tiny rounding residues
    # exactly representable factors -> exactly zero error
    g = read_golden("lu_2x2.txt")
    LU, ipiv, _, _ = oracle.getrf(g["A"])
    assert oracle.factor_error(g["A"], LU, ipiv) == 0.0
    # a planted error of known size is reported exactly
    LU2 = LU.copy()
    LU2[1, 1] += 0.25
    assert oracle.factor_error(g["A"], LU2, ipiv) == pytest.approx(0.25 / (2 * 5.0))


def test_special_identity_and_permutation():
    n = 9
    LU, ipiv, info, _ = oracle.getrf(np.eye(n))
    assert list(ipiv) == list(range(1, n + 1)) and np.array_equal(LU, np.eye(n))
    perm = synth.rng(5, 0).permutation(n)
    P = np.eye(n)[perm]  # row i of P is e_{perm[i]}
    LU, ipiv, info, _ = oracle.getrf(P)
    assert np.array_equal(LU, np.eye(n))
    order = perm_from_ipiv(ipiv, n)
    assert np.array_equal(P[order], np.eye(n))


def test_special_upper_triangular_no_swaps():
    n = 12
    g = synth.rng(6, 0)
    U = np.triu(g.uniform(-1, 1, size=(n, n)), 1) + np.diag(4.0 + g.uniform(0, 1, size=n))
    LU, ipiv, info, _ = oracle.getrf(U)
    assert list(ipiv) == list(range(1, n + 1))
    assert np.array_equal(LU, U)


def expected_pivots_separated(perm):
    """Closed-form pivot sequence for A = Pi D with D column diagonally dominant:
    at step j the pivot is the current position of D's row j."""
    n = len(perm)
    rows = list(perm)  # rows[i] = which D-row sits at position i
    piv = []
    for j in range(n):
        p = rows.index(j)
        piv.append(p + 1)
        rows[j], rows[p] = rows[p], rows[j]
    return piv


@pytest.mark.parametrize("n", [3, 17, 64, 150])
def test_special_separated_pivots(n):
    A, perm = synth.separated_matrix(n, seed=7)
    LU, ipiv, info, gap = oracle.getrf(A)
    assert list(ipiv) == expected_pivots_separated(perm)
    assert gap.min() > 0.1


def test_ones_solution():
    n = 200
    A = synth.uniform_matrix(n, seed=0)
    b = synth.ones_rhs(A)[:, 0]
    LU, ipiv, _, _ = oracle.getrf(A)
    x = oracle.getrs(LU, ipiv, b)
    assert np.abs(x - 1).max() <= 1e-10
    assert oracle.backward_error(A, x, b) <= 1e-15


def test_against_lapack():
    """Third-party cross-check: LAPACK dgetrf (scipy) gives the same pivots on
    matrices whose pivot candidates are separated, and factors within rounding."""
    sl = pytest.importorskip("scipy.linalg")
    for n, seed in ((64, 0), (257, 1)):
        A = synth.uniform_matrix(n, seed=seed, stream=9)
        LU, ipiv, info, gap = oracle.getrf(A)
        lu_ref, piv_ref = sl.lu_factor(A)
        sep = gap > 1e-8
        assert np.array_equal((piv_ref + 1)[sep], ipiv[sep])
        if np.array_equal(piv_ref + 1, ipiv):
            assert np.abs(LU - lu_ref).max() <= 1e-10 * np.abs(lu_ref).max()


def test_laswp_matches_permutation_matrix():
    n, c = 20, 7
    A = synth.uniform_matrix(n, c, seed=8)
    ipiv = np.array([int(synth.rng(8, 1).integers(k, n)) + 1 for k in range(n)], dtype=np.int32)
    P = np.eye(n)[perm_from_ipiv(ipiv, n)]
    np.testing.assert_array_equal(oracle.laswp(A, 0, n, ipiv), P @ A)
    # partial range k1..k2 only applies those interchanges
    part = oracle.laswp(A, 3, 9, ipiv)
    order = list(range(n))
    for k in range(3, 9):
        p = ipiv[k] - 1
        order[k], order[p] = order[p], order[k]
    np.testing.assert_array_equal(part, A[order])


def test_trsm_and_gemm_update_against_numpy():
    g = synth.rng(9, 0)
    m, n, k = 37, 23, 11
    L = np.tril(g.uniform(-1, 1, size=(m, m)), -1) + np.eye(m)
    B = g.uniform(-1, 1, size=(m, n))
    junk = np.tril(L, -1) + np.triu(g.uniform(-5, 5, size=(m, m)), 0)  # diagonal/upper must be ignored
    X = oracle.trsm_lower_unit(junk, B)
    # the strict upper part and the diagonal of the argument must be ignored (unit diag)
    X2 = oracle.trsm_lower_unit(L, B)
    np.testing.assert_array_equal(X, X2)
    assert np.abs(L @ X2 - B).max() <= 1e-13
    U = np.triu(g.uniform(-1, 1, size=(m, m))) + 3 * np.eye(m)
    Y = oracle.trsm_upper(U + np.tril(np.full((m, m), 7.0), -1), B)
    assert np.abs(U @ Y - B).max() <= 1e-13
    C = g.uniform(-1, 1, size=(m, n))
    A = g.uniform(-1, 1, size=(m, k))
    Bk = g.uniform(-1, 1, size=(k, n))
    np.testing.assert_allclose(oracle.gemm_update(C, A, Bk), C - A @ Bk, rtol=0, atol=1e-14)
    # integer operands: exact
    Ai, Bi, Ci = (g.integers(-5, 6, size=s).astype(float) for s in ((m, k), (k, n), (m, n)))
    np.testing.assert_array_equal(oracle.gemm_update(Ci, Ai, Bi), Ci - Ai @ Bi)


def test_getrs_multiple_rhs_and_zero_size():
    n, nrhs = 90, 16
    A = synth.normal_matrix(n, seed=10)
    B, Xt = synth.random_rhs(A, nrhs, seed=10)
    LU, ipiv, _, _ = oracle.getrf(A)
    X = oracle.getrs(LU, ipiv, B)
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=0, atol=1e-10)
    assert oracle.backward_error(A, X, B) <= 1e-15
    LU0, ipiv0, info0, _ = oracle.getrf(np.zeros((0, 0)))
    assert info0 == 0 and ipiv0.size == 0


def test_backward_error_definition():
    A = np.array([[2.0, 0.0], [0.0, 4.0]])
    x = np.array([1.0, 1.0])
    b = np.array([2.0, 4.0])
    assert oracle.backward_error(A, x, b) == 0.0
    b2 = np.array([2.0, 4.5])  # r = (0, 0.5); ||A|| = 4, ||x|| = 1, ||b|| = 4.5
    assert oracle.backward_error(A, x, b2) == pytest.approx(0.5 / (4 + 4.5), rel=1e-15)
    assert oracle.norm_inf(np.array([[1.0, -2.0], [0.5, 0.25]])) == 3.0


def test_rounding_against_torch_conversions():
    torch = pytest.importorskip("torch")
    g = synth.rng(13, 0)
    x = np.concatenate([g.standard_normal(20000) * 10.0 ** g.uniform(-12, 12, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 65519.0, 1e-8, 6e-8]])
    bf = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), bf)
    # torch converts double -> half through float, which can round twice; compare
    # on FP32-representable inputs where one rounding is all there is
    x32 = x.astype(np.float32).astype(np.float64)
    h = torch.from_numpy(x32).to(torch.float16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_fp16(x32), h)
    f = x.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(oracle.round_fp32(x), f)
    if hasattr(torch, "float8_e4m3fn"):
        xs = np.clip(g.standard_normal(20000) * 10.0 ** g.uniform(-4, 2.6, 20000), -448, 448)
        xs = xs.astype(np.float32).astype(np.float64)
        e = torch.from_numpy(xs).to(torch.float8_e4m3fn).to(torch.float64).numpy()
        np.testing.assert_array_equal(oracle.round_e4m3(xs), e)


def test_rounding_hand_values():
    # ties to even at each format's spacing
    assert list(oracle.round_bf16([1.00390625, 1.01171875])) == [1.0, 1.015625]
    assert list(oracle.round_e4m3([1.0625, 1.1875, 500.0, -1000.0, 2.0 ** -10 * 1.5, 2.0 ** -10]))[:5] == \
        [1.0, 1.25, 448.0, -448.0, 2.0 ** -9]
    assert oracle.round_e4m3([2.0 ** -10])[0] == 0.0  # exact tie at half the smallest subnormal -> even (0)
    assert list(oracle.round_fp16([65519.0, 65520.0])) == [65504.0, np.inf]


def test_thread_count_does_not_change_results():
    A = synth.normal_matrix(300, seed=14)
    r1 = oracle.getrf(A, nthreads=1)
    r4 = oracle.getrf(A, nthreads=4)
    np.testing.assert_array_equal(r1[0], r4[0])
    np.testing.assert_array_equal(r1[1], r4[1])


def test_e4m3_block_quantiser():
    """Power-of-two block scaling: the scale is the smallest power of two that
    brings the block maximum to <= 448 (so 224 < amax/s <= 448), the stored
    values are e4m3-representable and equal torch's e4m3 conversion of X/s."""
    g = synth.rng(15, 0)
    X = g.standard_normal((40, 64)) * 10.0 ** g.uniform(-6, 6, size=(40, 1))
    X[3] = 0.0
    X[5, :] = 448.0 * 2.0 ** -7  # amax exactly a power-of-two multiple of 448: no extra halving
    Q, s = oracle.quant_e4m3_rows(X)
    amax = np.abs(X).max(axis=1)
    nz = amax > 0
    assert np.all(np.log2(s) == np.round(np.log2(s)))
    assert np.all((amax[nz] / s[nz] <= 448.0) & (amax[nz] / s[nz] > 224.0))
    assert s[3] == 1.0 and np.all(Q[3] == 0.0)
    assert s[5] == 2.0 ** -7
    np.testing.assert_array_equal(oracle.round_e4m3(Q), Q)
    torch = pytest.importorskip("torch")
    if hasattr(torch, "float8_e4m3fn"):
        ref = torch.from_numpy((X / s[:, None]).astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
        np.testing.assert_array_equal(Q, ref)
    Qc, t = oracle.quant_e4m3_cols(X.T)
    np.testing.assert_array_equal(Qc, Q.T)
    np.testing.assert_array_equal(t, s)


@pytest.mark.parametrize("name", ["identity", "reverse", "last_row", "in_panel", "random", "mixed"])
@pytest.mark.parametrize("n", [1, 31, 70])
def test_designed_pivot_sequences(name, n):
    """Sec. 3 RL1 on A = Pi D (D column diagonally dominant) takes exactly the
    designed interchanges, including repeated targets and swaps inside a panel;
    the row order is built independently of the oracle by undoing the sequence."""
    import pivot_patterns
    A, piv = pivot_patterns.patterned_matrix(name, n, seed=3)
    LU, ipiv, info, gap = oracle.getrf(A)
    assert info == 0
    assert np.array_equal(ipiv, piv)
    assert oracle.factor_error(A, LU, ipiv) <= 1e-15


def test_potrf_integer_factor_exact():
    """A = L0 L0^T with a small integer L0 (positive integer diagonal): every
    step of the elimination is exact in FP64, so the Cholesky oracle must return
    L0 bit for bit."""
    g = synth.rng(12, 0)
    for n in (1, 2, 5, 9):
        L0 = np.tril(g.integers(-3, 4, size=(n, n)).astype(float), -1) + np.diag(g.integers(1, 4, size=n).astype(float))
        A = L0 @ L0.T
        L, info = oracle.potrf(A)
        assert info == 0 and np.array_equal(L, L0)
        assert oracle.chol_error(A, L) == 0.0


@pytest.mark.parametrize("n", [3, 40, 130])
def test_potrf_against_numpy(n):
    A = synth.spd_matrix(n, seed=n)
    assert np.array_equal(A, A.T)
    L, info = oracle.potrf(A)
    R = np.linalg.cholesky(A)  # LAPACK potrf, a third-party routine
    assert info == 0
    assert np.all(np.diag(L) > 0) and np.array_equal(L, np.tril(L))
    assert np.abs(L - R).max() <= 1e-13 * np.abs(R).max()
    assert oracle.chol_error(A, L) <= 4 * np.finfo(float).eps


def test_nan_candidate_never_pivots():
    """Reading of RL1's pivot search for NaN (the paper is silent): NaN is
    unordered, so it maximises nothing and is never chosen; a column whose
    every candidate is NaN keeps its diagonal position.  Worked by hand:
    column 0 holds NaN, 3, 1 -> row 2 wins although the NaN comes first;
    after the swap row 2 becomes [NaN, NaN, NaN] through l = NaN / 3;
    column 1 holds NaN, -2/3 -> row 3; column 2 holds only NaN -> row 3
    stays.  No exactly-zero pivot occurs (NaN == 0 is false)."""
    A = np.array([[np.nan, 1.0, 0.0], [3.0, 2.0, 0.0], [1.0, 0.0, 4.0]])
    LU, ipiv, info, _ = oracle.getrf(A)
    assert list(ipiv) == [2, 3, 3] and info == 0
    np.testing.assert_array_equal(LU[0], [3.0, 2.0, 0.0])
    assert LU[1, 0] == 1.0 / 3.0 and LU[1, 2] == 4.0
    assert abs(LU[1, 1] - (-2.0 / 3.0)) <= np.spacing(2.0 / 3.0)
    assert np.all(np.isnan(LU[2]))
    # every candidate NaN: the diagonal position is kept
    LU, ipiv, info, _ = oracle.getrf(np.array([[np.nan, 1.0], [np.nan, 2.0]]))
    assert list(ipiv) == [1, 2] and info == 0
    # a NaN in the first candidate position loses as a zero there would
    B = synth.uniform_matrix(9, seed=4)
    B[0, 0] = 0.0
    first = oracle.getrf(B)[1][0]
    B[0, 0] = np.nan
    assert first != 1 and oracle.getrf(B)[1][0] == first


def test_potrf_not_positive_definite():
    assert oracle.potrf(np.diag([1.0, 2.0, -1.0, 4.0]))[1] == 3
    assert oracle.potrf(np.ones((2, 2)))[1] == 2  # the leading 2 x 2 minor is singular
    assert oracle.potrf(np.zeros((1, 1)))[1] == 1
    A = synth.spd_matrix(10, seed=1)
    A[6, 6] = -100.0  # the leading 6 x 6 minor is untouched and positive definite
    assert oracle.potrf(A)[1] == 7
    B = A.copy()
    B[6, 6] = np.nan
    assert oracle.potrf(B)[1] == 7


def test_chol_error_planted():
    n, delta = 4, 0.125
    L = np.eye(n)
    L[1, 1] = 1 + delta
    # (L L^T)(1,1) = (1 + delta)^2: one residual entry of 2 delta + delta^2 in row 1
    assert oracle.chol_error(np.eye(n), L) == (2 * delta + delta ** 2) / n


def test_geqr2_upper_triangular_is_untouched():
    """A column that is already zero below the diagonal needs no reflector:
    tau_j = 0 and R = A exactly."""
    g = synth.rng(14, 0)
    U = np.triu(g.uniform(-1, 1, size=(7, 7)))
    QR, tau = oracle.geqr2(U)
    assert np.array_equal(tau, np.zeros(7)) and np.array_equal(QR, U)


def test_geqr2_hand_worked_2x2():
    """A = [[3, 1], [4, 2]], worked by hand from the reflector definition:
    alpha = 3, sigma = 4, beta = -5, tau = 8/5, v = [1, 1/2];
    w = 1 + 2/2 = 2, R = [[-5, 1 - 16/5], [0, 2 - 8/5]] = [[-5, -2.2], [0, 0.4]]."""
    QR, tau = oracle.geqr2(np.array([[3.0, 1.0], [4.0, 2.0]]))
    assert tau[0] == 1.6 and tau[1] == 0.0
    assert QR[0, 0] == -5.0 and QR[1, 0] == 0.5
    assert abs(QR[0, 1] + 2.2) <= 4e-16 and abs(QR[1, 1] - 0.4) <= 4e-16


@pytest.mark.parametrize("m,n", [(5, 5), (60, 60), (90, 40)])
def test_geqr2_against_lapack_raw(m, n):
    """numpy's 'raw' QR is LAPACK dgeqrf's output (reflectors below the diagonal,
    R above, tau): the same convention, so every entry agrees to rounding."""
    A = synth.uniform_matrix(max(m, n), seed=m + n)[:m, :n]
    QR, tau = oracle.geqr2(A)
    h, tau_l = np.linalg.qr(A, mode="raw")
    scale = np.abs(A).max()
    assert np.abs(QR - h.T).max() <= 1e-12 * scale
    assert np.abs(tau - tau_l).max() <= 1e-12
    res, orth = oracle.qr_error(A, QR, tau)
    assert res <= 4 * np.finfo(float).eps and orth <= 8 * m * np.finfo(float).eps


def test_qr_error_planted():
    """For A0 = I the reflectors are identities (Q = I, R = I); a planted error
    delta in R(0, 1) is reported as delta / n, and Q stays exactly orthogonal."""
    n, delta = 5, 0.25
    QR, tau = oracle.geqr2(np.eye(n))
    assert np.array_equal(QR, np.eye(n)) and np.array_equal(tau, np.zeros(n))
    QR[0, 1] += delta
    res, orth = oracle.qr_error(np.eye(n), QR, tau)
    assert res == delta / n and orth == 0.0
