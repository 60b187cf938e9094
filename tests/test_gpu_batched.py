"""GPU parity of the batched factorization + solve (lu_gesv_batched) against the
CPU oracle, matrix by matrix.

Criteria: FP64 -- pivots bit-exact at separated steps (gap > 1e-8),
||PA - LU|| / (n ||A||) <= 1e-14 and solve eta <= 1e-14; FP32 -- pivots at
gap > 1e-3, factorization error <= 4 u32, eta <= 64 n u32 (no refinement).
Per-matrix status codes for out-of-range sizes and singular matrices.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1804_07017_gb300 as pkg
    pkg.lib()
    return pkg


def colmajor_dev(a, dtype, ld=None):
    from paper_1804_07017_gb300.api import colmajor
    t = colmajor(a.shape[0], a.shape[1], dtype=dtype, ld=ld)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_gesv_parity(lu, dtype):
    count = 96
    sizes, nrhs = synth.batched_sizes(count, seed=7)
    sizes[:4] = [512, 16, 1, 33]  # the extremes and a ragged panel
    mats = synth.batched_matrices(sizes, seed=7)
    g = synth.rng(7, 9)
    rhs = [g.uniform(-1, 1, size=(int(n), int(r))) for n, r in zip(sizes, nrhs)]
    if dtype == torch.float32:
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
        rhs = [b.astype(np.float32).astype(np.float64) for b in rhs]
    dA = [colmajor_dev(m, dtype, ld=int(m.shape[0]) + (i % 3)) for i, m in enumerate(mats)]
    dB = [colmajor_dev(b, dtype) for b in rhs]
    piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv, dB)
    lu.lu_gesv_batched(batch)
    torch.cuda.synchronize()
    info = batch.info.cpu().numpy()
    assert np.all(info == 0), info
    u = np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps / 2
    tau = 1e-8 if dtype == torch.float64 else 1e-3
    worst_f, worst_eta = 0.0, 0.0
    for i in range(count):
        n = int(sizes[i])
        LU = dA[i].cpu().double().numpy()[:n, :n]
        p = piv[i].cpu().numpy()
        _, po, _, gap = oracle.getrf(mats[i])
        sep = gap > tau
        assert np.array_equal(p[sep], po[sep]), i
        fe = oracle.factor_error(mats[i], LU, p)
        x = dB[i].cpu().double().numpy()
        eta = oracle.backward_error(mats[i], x, rhs[i])
        worst_f, worst_eta = max(worst_f, fe), max(worst_eta, eta)
        if dtype == torch.float64:
            assert fe <= 1e-14 and eta <= 1e-14, (i, n, fe, eta)
        else:
            assert fe <= 4 * u * 2 and eta <= 64 * n * u, (i, n, fe, eta)
    print(f"\n[batched {dtype}] {count} systems, n in [{sizes.min()}, {sizes.max()}]: "
          f"max factor error {worst_f:.2e}, max eta {worst_eta:.2e}")


def test_batched_status_codes(lu):
    sizes = [8, 513, 20, 0]
    mats = [synth.uniform_matrix(8, seed=1), np.eye(513), synth.uniform_matrix(20, seed=2), np.zeros((0, 0))]
    mats[2][:, 5] = 0.0  # exactly singular: U(6,6) == 0
    dA = [colmajor_dev(m, torch.float64) if m.size else torch.zeros((0, 0), dtype=torch.float64, device="cuda")
          for m in mats]
    piv = [torch.zeros(max(int(n), 1), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv)
    lu.lu_gesv_batched(batch)
    torch.cuda.synchronize()
    info = batch.info.cpu().numpy()
    _, _, info_o, _ = oracle.getrf(mats[2])
    assert info[0] == 0
    assert info[1] == lu.LU_ERR_UNSUPPORTED
    assert info[2] == info_o == 6
    assert info[3] == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_factor_then_solve(lu, dtype):
    """lu_factor_batched followed by lu_solve_batched gives the same bits as the
    fused lu_gesv_batched, and the oracle's backward error bound."""
    count = 40
    sizes, nrhs = synth.batched_sizes(count, seed=11)
    mats = synth.batched_matrices(sizes, seed=11)
    g = synth.rng(11, 9)
    rhs = [g.uniform(-1, 1, size=(int(n), int(r))) for n, r in zip(sizes, nrhs)]
    runs = []
    for split in (False, True):
        dA = [colmajor_dev(m, dtype) for m in mats]
        dB = [colmajor_dev(b, dtype) for b in rhs]
        piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
        batch = lu.Batch(dA, piv, dB)
        if split:
            lu.lu_factor_batched(batch)
            torch.cuda.synchronize()
            assert np.all(batch.info.cpu().numpy() == 0)
            lu.lu_solve_batched(batch)
        else:
            lu.lu_gesv_batched(batch)
        torch.cuda.synchronize()
        assert np.all(batch.info.cpu().numpy() == 0)
        runs.append(([a.cpu() for a in dA], [p.cpu() for p in piv], [b.cpu() for b in dB]))
    u = np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps / 2
    for i in range(count):
        assert torch.equal(runs[0][0][i], runs[1][0][i]) and torch.equal(runs[0][1][i], runs[1][1][i])
        assert torch.equal(runs[0][2][i], runs[1][2][i])
        x = runs[1][2][i].double().numpy()
        src = mats[i] if dtype == torch.float64 else mats[i].astype(np.float32).astype(np.float64)
        b = rhs[i] if dtype == torch.float64 else rhs[i].astype(np.float32).astype(np.float64)
        eta = oracle.backward_error(src, x, b)
        assert eta <= (1e-14 if dtype == torch.float64 else 64 * sizes[i] * u), (i, eta)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_full_size_sampled(lu, dtype):
    """The benchmarked batch at full size (4096 systems, n log-uniform in
    [16, 512], nrhs 1..8, one launch): every info is 0 and a sample of 48
    systems meets the parity criteria against the oracle."""
    count = 4096
    sizes, nrhs = synth.batched_sizes(count, seed=0)
    mats = synth.batched_matrices(sizes, seed=0)
    g = synth.rng(0, 9)
    rhs = [g.uniform(-1, 1, size=(int(n), int(r))) for n, r in zip(sizes, nrhs)]
    if dtype == torch.float32:
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
        rhs = [b.astype(np.float32).astype(np.float64) for b in rhs]
    dA = [colmajor_dev(m, dtype) for m in mats]
    dB = [colmajor_dev(b, dtype) for b in rhs]
    piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv, dB)
    lu.lu_gesv_batched(batch)
    torch.cuda.synchronize()
    assert np.all(batch.info.cpu().numpy() == 0)
    u = np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps / 2
    tau = 1e-8 if dtype == torch.float64 else 1e-3
    pick = synth.rng(5, 5).choice(count, size=48, replace=False)
    pick[:2] = [int(np.argmax(sizes)), int(np.argmin(sizes))]
    for i in pick:
        n = int(sizes[i])
        LU = dA[i].cpu().double().numpy()
        p = piv[i].cpu().numpy()
        _, po, _, gap = oracle.getrf(mats[i])
        sep = gap > tau
        assert np.array_equal(p[sep], po[sep]), i
        fe = oracle.factor_error(mats[i], LU, p)
        eta = oracle.backward_error(mats[i], dB[i].cpu().double().numpy(), rhs[i])
        if dtype == torch.float64:
            assert fe <= 1e-14 and eta <= 1e-14, (i, n, fe, eta)
        else:
            assert fe <= 4 * u * 2 and eta <= 64 * n * u, (i, n, fe, eta)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_designed_pivot_sequences(lu, dtype):
    """The batched kernel composes each panel's interchanges into one gather
    plan; designed sequences (pivot_patterns: none, reversal, one row below
    reached by every step, swaps inside the panel, random and mixed chains) must
    come back exactly, with the factor and solve bounds of the parity test."""
    import pivot_patterns as pp
    cases = [(name, n) for name in pp.PATTERNS for n in (16, 31, 33, 64, 100, 257, 512)]
    built = [pp.patterned_matrix(name, n, seed=5 + n) for name, n in cases]
    mats = [a for a, _ in built]
    pivs = [p for _, p in built]
    g = synth.rng(13, 9)
    rhs = [g.uniform(-1, 1, size=(a.shape[0], 1 + (i % 8))) for i, a in enumerate(mats)]
    if dtype == torch.float32:
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
        rhs = [b.astype(np.float32).astype(np.float64) for b in rhs]
    dA = [colmajor_dev(m, dtype, ld=int(m.shape[0]) + (i % 2)) for i, m in enumerate(mats)]
    dB = [colmajor_dev(b, dtype) for b in rhs]
    piv = [torch.zeros(a.shape[0], dtype=torch.int32, device="cuda") for a in mats]
    batch = lu.Batch(dA, piv, dB)
    lu.lu_gesv_batched(batch)
    torch.cuda.synchronize()
    assert np.all(batch.info.cpu().numpy() == 0)
    u = np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps / 2
    for i, (name, n) in enumerate(cases):
        p = piv[i].cpu().numpy()
        assert np.array_equal(p, pivs[i]), (name, n, np.nonzero(p != pivs[i])[0][:10])
        LU = dA[i].cpu().double().numpy()[:n, :n]
        fe = oracle.factor_error(mats[i], LU, p)
        eta = oracle.backward_error(mats[i], dB[i].cpu().double().numpy(), rhs[i])
        if dtype == torch.float64:
            assert fe <= 1e-14 and eta <= 1e-14, (name, n, fe, eta)
        else:
            assert fe <= 4 * u * 2 and eta <= 64 * n * u, (name, n, fe, eta)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_nan_first_candidate(lu, dtype):
    """A NaN in the first candidate position of column 0 (A(0,0) = NaN) is
    never chosen in the batched kernel either: the NaN row loses every search
    it is the first candidate of and ends as the last row of the factors,
    whole-row NaN, exactly as in the oracle; the other systems of the batch
    are unaffected and meet the usual bounds."""
    sizes = np.array([1, 2, 17, 33, 64, 100, 300, 512, 40, 96])
    mats = [synth.uniform_matrix(int(n), seed=41, stream=int(n)) for n in sizes]
    if dtype == torch.float32:
        mats = [m.astype(np.float32).astype(np.float64) for m in mats]
    poisoned = list(range(0, len(sizes) - 2))
    for i in poisoned:
        mats[i][0, 0] = np.nan
    dA = [colmajor_dev(m, dtype) for m in mats]
    piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv)
    lu.lu_factor_batched(batch)
    torch.cuda.synchronize()
    assert np.all(batch.info.cpu().numpy() == 0)
    tau = 1e-8 if dtype == torch.float64 else 1e-3
    tol = 1e-10 if dtype == torch.float64 else 1e-3
    for i, n in enumerate(int(v) for v in sizes):
        LU = dA[i].cpu().double().numpy()[:n, :n]
        p = piv[i].cpu().numpy()
        LU_o, po, info_o, gap = oracle.getrf(mats[i])
        assert info_o == 0
        nan = np.isnan(LU_o)
        assert np.array_equal(np.isnan(LU), nan), (i, n)
        if i in poisoned:
            assert p[-1] == po[-1] == n and np.all(nan[n - 1]) and not nan[: n - 1].any()
            if n > 1:
                assert po[0] != 1 and p[0] == po[0]
        else:
            assert not nan.any()
        sep = gap > tau
        assert np.array_equal(p[sep], po[sep]), (i, n)
        diff = np.nonzero(p != po)[0]
        d = int(diff[0]) if diff.size else n
        a, b = np.where(nan, 0.0, LU)[:d], np.where(nan, 0.0, LU_o)[:d]
        assert np.abs(a - b).max(initial=0.0) <= tol * max(np.abs(b).max(initial=0.0), 1e-300), (i, n)



@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_tile_cutover_and_tuner(lu, dtype):
    """The batched trailing update's tile shape (32 x 32 below the tuned cut-over,
    64 x 64 above) changes no operation: factors, pivots and solutions are
    bit-identical for every cut-over, and lu_tune_batched stores the fastest
    candidate, which later calls use."""
    count = 60
    sizes, nrhs = synth.batched_sizes(count, seed=17)
    sizes[:3] = [512, 33, 97]
    mats = synth.batched_matrices(sizes, seed=17)
    g = synth.rng(17, 9)
    rhs = [g.uniform(-1, 1, size=(int(n), int(r))) for n, r in zip(sizes, nrhs)]
    code = lu.LU_F64 if dtype == torch.float64 else lu.LU_F32
    kind = lu.LU_TUNE_BATCHED_F64 if dtype == torch.float64 else lu.LU_TUNE_BATCHED_F32
    outs = []
    for cut in (1, 65, 513):
        lu.lu_tune_set(kind, 512, cut)
        dA = [colmajor_dev(m, dtype) for m in mats]
        dB = [colmajor_dev(b, dtype) for b in rhs]
        piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
        batch = lu.Batch(dA, piv, dB)
        lu.lu_gesv_batched(batch)
        torch.cuda.synchronize()
        assert np.all(batch.info.cpu().numpy() == 0)
        outs.append(([a.cpu() for a in dA], [p.cpu() for p in piv], [b.cpu() for b in dB]))
    for o in outs[1:]:
        for i in range(count):
            assert torch.equal(o[0][i], outs[0][0][i]) and torch.equal(o[1][i], outs[0][1][i])
            assert torch.equal(o[2][i], outs[0][2][i])
    lu.lu_tune_clear()
    best, ms = lu.lu_tune_batched(code, sizes, nrhs, [1, 65, 129], reps=2)
    assert best in (1, 65, 129) and min(t for t in ms if t > 0) == ms[[1, 65, 129].index(best)]
    assert lu.lu_tune_get(kind, 512) == best
    lu.lu_tune_clear()
