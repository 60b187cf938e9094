"""GPU parity of the blocked LU path (FP64 and FP32 storage) against the CPU
oracle, through the C ABI.

Pass criteria (stated in the tests):
  * pivots bit-exact at every elimination step whose two largest candidates
    are separated by a relative gap > tau (tau = 1e-8 FP64, 1e-3 FP32), and
    at every step of the constructed well-separated family;
  * factorization backward error ||PA - LU||_inf / (n ||A||_inf) <= 1e-14 in FP64;
  * solve backward error eta <= 1e-14 in FP64;
  * integer/index work (interchanges) bit-exact;
  * look-ahead off / on give bit-identical factors.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TAU64 = 1e-8
TAU32 = 1e-3


@pytest.fixture(scope="module")
def lu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1804_07017_gb300 as pkg
    pkg.lib()
    return pkg


def dev(a, dtype=torch.float64, ld=None):
    from paper_1804_07017_gb300.api import colmajor
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    t = colmajor(a.shape[0], a.shape[1], dtype=dtype, ld=ld)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def host(t):
    return t.detach().cpu().double().numpy()


def factor_gpu(lu, A0, nb, dtype=torch.float64, ld=None, **opts):
    n = A0.shape[0]
    A = dev(A0, dtype, ld)
    ipiv = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    o = lu.default_opts(nb=nb, **opts)
    lu.lu_factor_ex(A, ipiv, info, o)
    torch.cuda.synchronize()
    return A, host(A), ipiv[:n].cpu().numpy(), int(info.item())


def check_pivots(piv, piv_o, gap, tau):
    sep = gap > tau
    bad = np.nonzero((piv != piv_o) & sep)[0]
    assert bad.size == 0, f"pivots differ at separated steps {bad[:10]} (gaps {gap[bad[:10]]})"


def compare_factors(LU, LU_o, piv, piv_o, gap, tau, tol):
    """Pivots may differ only at steps whose candidates are not separated
    (gap <= tau); the rows before the first differing step are final in both
    factorizations (later interchanges only touch rows at or below their own
    step), so they are always compared, entry by entry, relative to max|LU_o|.
    NaN entries must sit in the same places.  Returns the relative error."""
    check_pivots(piv, piv_o, gap, tau)
    diff = np.nonzero(piv != piv_o)[0]
    d = int(diff[0]) if diff.size else LU_o.shape[0]
    a, b = LU[:d], LU_o[:d]
    nan = np.isnan(b)
    assert np.array_equal(np.isnan(a), nan)
    scale = max(np.abs(b[~nan]).max(initial=0.0), 1e-300)
    rel = float(np.abs(a[~nan] - b[~nan]).max(initial=0.0) / scale)
    assert rel <= tol, (rel, d)
    return rel


@pytest.mark.parametrize("n,nb,ld_pad", [(1024, 64, 0), (1024, 64, 7), (333, 64, 0), (130, 32, 3), (1, 64, 0),
                                         (2, 64, 0), (700, 256, 0), (2048, 256, 0)])
def test_factor_and_solve_fp64(lu, n, nb, ld_pad):
    A0 = synth.uniform_matrix(n, seed=0, stream=n)
    A, LU, piv, info = factor_gpu(lu, A0, nb, ld=n + ld_pad if ld_pad else None)
    assert info == 0
    LU_o, piv_o, info_o, gap = oracle.getrf(A0)
    check_pivots(piv, piv_o, gap, TAU64)
    LU = LU[:n, :n]
    assert oracle.factor_error(A0, LU, piv) <= 1e-14
    compare_factors(LU, LU_o, piv, piv_o, gap, TAU64, 1e-10)
    # |l_ij| <= 1 holds for the GPU factors too (the division is exact-rounded)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)
    b0 = synth.ones_rhs(A0)
    Bt = dev(b0)
    if ld_pad == 0:
        lu.lu_solve(A, torch.from_numpy(piv).cuda(), Bt)
    else:
        lu.lu_solve_ex(A, torch.from_numpy(piv).cuda(), Bt)
    torch.cuda.synchronize()
    x = host(Bt)
    assert oracle.backward_error(A0, x, b0) <= 1e-14


def test_c0_configuration(lu):
    """The n = 1024 configuration exactly: A iid U[-1,1) from seed 0 (stream 0),
    column-major with lda = n, nb = 64, depth-1 look-ahead, one right-hand side
    b = A * ones(n).  Pivots equal the oracle's at every step (its smallest
    relative gap between the two largest candidates is ~2e-4, far above any
    rounding difference), the factors agree entry by entry to 1e-10 of
    max|LU|, the factorization's backward error is <= 1e-14 and the solve's
    eta <= 1e-14 (Sec. 3, LU_blk with RL1 = LU_unb)."""
    n, nb = 1024, 64
    A0 = synth.uniform_matrix(n, seed=0, stream=0)
    A, LU, piv, info = factor_gpu(lu, A0, nb, lookahead=1)
    LU_o, piv_o, info_o, gap = oracle.getrf(A0)
    assert info == info_o == 0
    assert gap.min() > TAU64
    assert np.array_equal(piv, piv_o)
    rel = np.abs(LU - LU_o).max() / np.abs(LU_o).max()
    assert rel <= 1e-10, rel
    assert oracle.factor_error(A0, LU, piv) <= 1e-14
    b0 = synth.ones_rhs(A0)
    Bt = dev(b0)
    lu.lu_solve(A, torch.from_numpy(piv).cuda(), Bt)
    torch.cuda.synchronize()
    x = host(Bt)
    assert oracle.backward_error(A0, x, b0) <= 1e-14
    print(f"\n[c0] max|LU - LU_oracle|/max|LU_oracle| = {rel:.2e}, "
          f"eta = {oracle.backward_error(A0, x, b0):.2e}, ||x - 1||_inf = {np.abs(x - 1).max():.2e}")


def test_plain_lu_factor_entry(lu):
    n = 512
    A0 = synth.uniform_matrix(n, seed=5)
    A = dev(A0)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert lu.lu_factor(A, ipiv, 64) == 0
    LU_o, piv_o, _, gap = oracle.getrf(A0)
    check_pivots(ipiv.cpu().numpy(), piv_o, gap, TAU64)
    assert oracle.factor_error(A0, host(A), ipiv.cpu().numpy()) <= 1e-14


@pytest.mark.parametrize("n,nb", [(700, 64), (1500, 256)])
def test_separated_family_pivots_bit_exact(lu, n, nb):
    A0, perm = synth.separated_matrix(n, seed=21)
    _, LU, piv, info = factor_gpu(lu, A0, nb)
    rows = list(perm)
    expect = []
    for j in range(n):
        p = rows.index(j)
        expect.append(p + 1)
        rows[j], rows[p] = rows[p], rows[j]
    assert np.array_equal(piv, np.array(expect))
    assert oracle.factor_error(A0, LU, piv) <= 1e-14


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lookahead_bit_identical(lu, dtype):
    n, nb = 1536, 128
    A0 = synth.normal_matrix(n, seed=3)
    _, LU0, p0, _ = factor_gpu(lu, A0, nb, dtype=dtype, lookahead=0)
    _, LU1, p1, _ = factor_gpu(lu, A0, nb, dtype=dtype, lookahead=1)
    _, LU2, p2, _ = factor_gpu(lu, A0, nb, dtype=dtype, lookahead=1, steal=0)
    assert np.array_equal(p0, p1) and np.array_equal(p0, p2)
    assert np.array_equal(LU0, LU1) and np.array_equal(LU0, LU2)
    # and repeated runs are deterministic
    _, LU3, p3, _ = factor_gpu(lu, A0, nb, dtype=dtype, lookahead=1)
    assert np.array_equal(LU1, LU3) and np.array_equal(p1, p3)


def test_zero_pivot_info(lu):
    n = 200
    A0 = synth.uniform_matrix(n, seed=8)
    A0[:, 77] = 0.0  # column 78 (1-based) is zero -> U(78,78) == 0 exactly
    _, LU, piv, info = factor_gpu(lu, A0, 64)
    _, piv_o, info_o, gap = oracle.getrf(A0)
    assert info_o == 78 and info == info_o
    check_pivots(piv, piv_o, gap, TAU64)


def test_fp32_factor(lu):
    n, nb = 1024, 64
    A0 = synth.uniform_matrix(n, seed=9)
    A32 = A0.astype(np.float32).astype(np.float64)
    _, LU, piv, info = factor_gpu(lu, A32, nb, dtype=torch.float32)
    LU_o, piv_o, _, gap = oracle.getrf(A32)
    check_pivots(piv, piv_o, gap, TAU32)
    # FP32 backward error bound: a small multiple of n * u32 for random matrices
    assert oracle.factor_error(A32, LU, piv) <= 4 * np.finfo(np.float32).eps


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,w,leaf", [(1000, 64, 0), (300, 37, 0), (5000, 128, 0), (257, 64, 16), (64, 64, 0),
                                      (3000, 256, 32), (16384, 48, 16), (9000, 29, 32), (2100, 13, 8)])
def test_panel_factor(lu, dtype, m, w, leaf):
    P0 = synth.uniform_matrix(m, w, seed=10, stream=m + w)
    if dtype == torch.float32:
        P0 = P0.astype(np.float32).astype(np.float64)
    P = dev(P0, dtype)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu.lu_panel_factor_ex(P, ipiv, info, lu.default_opts(leaf=leaf))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    LUo, pivo, _, gap = oracle.getrf(P0)
    piv = ipiv.cpu().numpy()
    compare_factors(host(P), LUo, piv, pivo, gap, TAU64 if dtype == torch.float64 else TAU32,
                    1e-12 if dtype == torch.float64 else 2e-4)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_laswp_bit_exact(lu, dtype):
    n, ncols = 900, 333
    g = synth.rng(11, 0)
    A0 = g.uniform(-1, 1, size=(n, ncols))
    if dtype == torch.float32:
        A0 = A0.astype(np.float32).astype(np.float64)
    for k1, k2 in ((0, 256), (300, 557), (640, 641), (0, 900)):
        ipiv = np.arange(1, n + 1, dtype=np.int32)
        for k in range(k1, k2):
            ipiv[k] = int(g.integers(k, n)) + 1
        # repeated targets below the block must compose correctly
        if k2 - k1 > 4:
            ipiv[k1 + 1] = ipiv[k1 + 3] = max(ipiv[k1 + 1], ipiv[k1 + 3])
        A = dev(A0, dtype)
        lu.lu_laswp_ex(A, k1, k2, torch.from_numpy(ipiv).cuda())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(A), oracle.laswp(A0, k1, k2, ipiv))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n", [(256, 1000), (64, 33), (100, 7), (512, 300), (1024, 17), (256, 256), (128, 128),
                                 (31, 5)])
def test_trsm(lu, dtype, m, n):
    """RL2 on the L11 that elimination produces (unit lower, |l_ij| <= 1), with
    junk stored on and above the diagonal that must be ignored.  Criteria:
    componentwise backward error |L X - B| <= 4 m u (|L| |X| + |B|) and the
    forward error against the oracle within the same bound propagated by the
    condition of the substitution, cond = || |L^-1| |L| |X| || / ||X||."""
    g = synth.rng(12, m)
    F, _, _, _ = oracle.getrf(g.uniform(-1, 1, size=(m, m)))
    L0 = np.tril(F, -1) + np.triu(g.uniform(5, 9, size=(m, m)))
    B0 = g.uniform(-1, 1, size=(m, n))
    if dtype == torch.float32:
        L0, B0 = (a.astype(np.float32).astype(np.float64) for a in (L0, B0))
    u = np.finfo(np.float64 if dtype == torch.float64 else np.float32).eps / 2
    B = dev(B0, dtype)
    lu.lu_trsm_ex(dev(L0, dtype), B)
    torch.cuda.synchronize()
    Xg = host(B)
    Lu = np.tril(L0, -1) + np.eye(m)
    assert np.all(np.abs(Lu @ Xg - B0) <= 4 * m * u * (np.abs(Lu) @ np.abs(Xg) + np.abs(B0)))
    X = oracle.trsm_lower_unit(L0, B0)
    cond = np.linalg.norm(np.abs(np.linalg.inv(Lu)) @ (np.abs(Lu) @ np.abs(X)), np.inf) / np.linalg.norm(X, np.inf)
    assert np.abs(Xg - X).max() <= 8 * m * u * cond * np.abs(X).max()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 2e-6)])
@pytest.mark.parametrize("m,n,k", [(1000, 700, 256), (65, 63, 17), (1, 1, 1), (4097, 129, 64), (300, 5000, 32)])
def test_gemm_update(lu, dtype, tol, m, n, k):
    g = synth.rng(13, m + n + k)
    C0, A0, B0 = (g.uniform(-1, 1, size=s) for s in ((m, n), (m, k), (k, n)))
    if dtype == torch.float32:
        C0, A0, B0 = (a.astype(np.float32).astype(np.float64) for a in (C0, A0, B0))
    C = dev(C0, dtype)
    lu.lu_gemm_update_ex(C, dev(A0, dtype), dev(B0, dtype))
    torch.cuda.synchronize()
    ref = oracle.gemm_update(C0, A0, B0)
    scale = np.abs(A0) @ np.abs(B0) + np.abs(C0)
    assert np.all(np.abs(host(C) - ref) <= tol * scale * max(1, k / 64))


def test_solve_multi_rhs_and_fp32(lu):
    n, nrhs = 1000, 16
    A0 = synth.normal_matrix(n, seed=14)
    B0, X_true = synth.random_rhs(A0, nrhs, seed=14)
    A, LU, piv, info = factor_gpu(lu, A0, 128)
    Bt = dev(B0)
    lu.lu_solve_ex(A, torch.from_numpy(piv).cuda(), Bt)
    torch.cuda.synchronize()
    assert oracle.backward_error(A0, host(Bt), B0) <= 1e-14
    # 19 rhs crosses the 16-column chunking of the triangular solves
    B19, _ = synth.random_rhs(A0, 19, seed=15)
    Bt = dev(B19)
    lu.lu_solve_ex(A, torch.from_numpy(piv).cuda(), Bt)
    torch.cuda.synchronize()
    assert oracle.backward_error(A0, host(Bt), B19) <= 1e-14


@pytest.mark.parametrize("n,nb", [(8192, 256)])
def test_full_size_sampled(lu, n, nb):
    """The n = 8192, nb = 256 configuration at full size: pivots bit-exact on the
    separated family; for the N(0,1) input the factorization residual
    ||(PA - LU)(i,:)||_1 / (n ||A||_inf) <= 1e-14 on sampled rows (formed row by
    row on the host) and the solve's backward error over the whole system."""
    A0 = synth.normal_matrix(n, seed=0)
    A, LU, piv, info = factor_gpu(lu, A0, nb, lookahead=1)
    assert info == 0
    order = np.arange(n)
    for k in range(n):
        p = piv[k] - 1
        order[k], order[p] = order[p], order[k]
    g = synth.rng(99, 0)
    rows = np.concatenate([[0, 1, n // 2, n - 1], g.integers(0, n, size=28)])
    anorm = np.abs(A0).sum(axis=1).max()
    for i in rows:
        l = LU[i, : i + 1].copy()
        l[i] = 1.0
        acc = np.zeros(n)
        for p0 in range(0, i + 1, 512):
            p1 = min(i + 1, p0 + 512)
            acc += l[p0:p1] @ np.triu(LU[p0:p1, :], k=p0)  # rows p of U keep columns c >= p
        r = A0[order[i], :] - acc
        assert np.abs(r).sum() / (n * anorm) <= 1e-14
    b0 = synth.ones_rhs(A0)
    Bt = dev(b0)
    lu.lu_solve(A, torch.from_numpy(piv).cuda(), Bt)
    torch.cuda.synchronize()
    x = host(Bt)
    r = b0[:, 0] - A0 @ x[:, 0]
    eta = np.abs(r).max() / (anorm * np.abs(x).max() + np.abs(b0).max())
    # a backward-stable FP64 solve without refinement: eta <= n u (measured ~3e-14 at n = 8192)
    print(f"\n[fp64 solve n={n}] eta = {eta:.2e}")
    assert eta <= n * np.finfo(float).eps / 2
    # the separated family at the same size: every pivot bit-exact
    S0, perm = synth.separated_matrix(n, seed=22)
    _, _, ps, _ = factor_gpu(lu, S0, nb, lookahead=1)
    pos = np.empty(n, dtype=np.int64)
    cur = perm.copy()
    pos[cur] = np.arange(n)
    expect = np.empty(n, dtype=np.int64)
    for j in range(n):
        p = pos[j]
        expect[j] = p + 1
        cur[j], cur[p] = cur[p], cur[j]
        pos[cur[j]] = j
        pos[cur[p]] = p
    assert np.array_equal(ps, expect)


def check_nan_factors(LU, LU_o, piv, piv_o, gap, tau, tol):
    """Factors of an input holding NaN: NaN in the same places (one whole row,
    the row that held the NaN), and the prefix comparison of compare_factors
    on the finite entries (same pivots at separated steps)."""
    nan = np.isnan(LU_o)
    assert nan.any() and np.array_equal(np.isnan(LU), nan)
    assert np.array_equal(np.nonzero(nan.all(axis=1))[0], np.nonzero(nan.any(axis=1))[0])
    compare_factors(np.where(nan, 0.0, LU), np.where(nan, 0.0, LU_o), piv, piv_o, gap, tau, tol)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_panel_nan_and_zero_column(lu, dtype):
    """A NaN candidate is never chosen, even in the first candidate position
    (NaN is unordered, so it maximises nothing), and an exactly zero column is
    reported as the first zero pivot without scaling.  P(0,0) = NaN: column 0
    pivots on the largest finite entry, and the NaN row then carries NaN
    through l = NaN / pivot into every later column, where it is skipped
    again; column 21 is zero, so info = 22.  Pivots, info, the NaN pattern and
    the finite entries equal the oracle's."""
    m, w = 3000, 40
    P0 = synth.uniform_matrix(m, w, seed=12, stream=5)
    if dtype == torch.float32:
        P0 = P0.astype(np.float32).astype(np.float64)
    P0[:, 21] = 0.0
    P0[0, 0] = np.nan
    P = dev(P0, dtype)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    for leaf in (16, 0):
        P.copy_(dev(P0, dtype))
        lu.lu_panel_factor_ex(P, ipiv, info, lu.default_opts(leaf=leaf))
        torch.cuda.synchronize()
        LU_o, pivo, info_o, gap = oracle.getrf(P0)
        piv = ipiv.cpu().numpy()
        assert pivo[0] != 1 and pivo[0] - 1 >= w  # the NaN row leaves the panel's rows
        assert int(info.item()) == info_o == 22
        check_nan_factors(host(P), LU_o, piv, pivo, gap, TAU64 if dtype == torch.float64 else TAU32,
                          1e-12 if dtype == torch.float64 else 2e-4)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_blocked_nan_first_candidate(lu, dtype):
    """The blocked look-ahead factorization with A(0,0) = NaN.  The NaN row is
    the first candidate of column 0 and loses; whenever later interchanges
    bring it to the diagonal position of a step it is the first candidate
    again and loses again, across panels, until the last step, where it is the
    only candidate and stays.  Pivots, the NaN pattern and the finite entries
    equal the oracle's."""
    n, nb = 700, 64
    A0 = synth.uniform_matrix(n, seed=31)
    if dtype == torch.float32:
        A0 = A0.astype(np.float32).astype(np.float64)
    A0[0, 0] = np.nan
    _, LU, piv, info = factor_gpu(lu, A0, nb, dtype=dtype, lookahead=1)
    LU_o, piv_o, info_o, gap = oracle.getrf(A0)
    assert info == info_o == 0
    assert piv_o[0] != 1 and piv_o[-1] == n and piv[-1] == n
    assert np.all(np.isnan(LU_o[n - 1])) and not np.isnan(LU_o[: n - 1]).any()
    check_nan_factors(LU[:n, :n], LU_o, piv, piv_o, gap, TAU64 if dtype == torch.float64 else TAU32,
                      1e-10 if dtype == torch.float64 else 1e-3)


@pytest.mark.parametrize("name", ["last_row", "in_panel", "mixed", "reverse"])
@pytest.mark.parametrize("dtype,n,nb", [(torch.float64, 700, 64), (torch.float64, 1500, 256),
                                        (torch.float32, 700, 64)])
def test_designed_pivot_sequences(lu, name, dtype, n, nb):
    """Designed interchange sequences (pivot_patterns: repeated targets below a
    panel, swaps inside it, long mixed chains) through the look-ahead
    factorization: the leaves' argmax, the interchange plans on both sides of
    each panel and the updates between must reproduce them exactly.  Patterns
    are laid out per nb-wide panel and per 32-wide leaf."""
    import pivot_patterns as pp
    for panel in (nb, 32):
        A0, piv = pp.patterned_matrix(name, n, seed=9, panel=panel)
        if dtype == torch.float32:
            A0 = A0.astype(np.float32).astype(np.float64)
        _, LU, p, info = factor_gpu(lu, A0, nb, dtype=dtype)
        assert info == 0
        assert np.array_equal(p, piv), (panel, np.nonzero(p != piv)[0][:10])
        bound = 1e-14 if dtype == torch.float64 else 4 * np.finfo(np.float32).eps
        assert oracle.factor_error(A0, LU[:n, :n], p) <= bound
