"""GPU parity of the Householder QR (lu_geqrf_ex) against the CPU oracle
(oracle.geqr2, the unblocked LAPACK-convention reflectors), through the C ABI.

Criteria: R, the reflector vectors and tau agree with the oracle's entry by
entry (FP64 within 1e-12 of max|.|, FP32 within 1e-3); ||A - Q R|| / (n ||A||)
<= 1e-14 in FP64 (8 u32 in FP32) and ||Q^T Q - I|| <= 50 max(m, n) u, with Q
rebuilt from the GPU's reflectors by the oracle; look-ahead on and off give
bit-identical results (the same operations per element); an upper triangular
input needs no reflector (tau = 0) and comes back unchanged, bit for bit.
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


def dev(a, dtype):
    from paper_1804_07017_gb300.api import colmajor
    t = colmajor(a.shape[0], a.shape[1], dtype=dtype)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def qr_gpu(lu, A0, dtype, **opts):
    m, n = A0.shape
    A = dev(A0, dtype)
    tau = torch.zeros(max(min(m, n), 1), dtype=dtype, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    lu.lu_geqrf_ex(A, tau, info, lu.default_opts(**opts))
    torch.cuda.synchronize()
    return A.cpu().double().numpy(), tau[:min(m, n)].cpu().double().numpy(), int(info.item())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,nb", [(700, 700, 64), (1000, 1000, 128), (1200, 500, 96), (300, 700, 32),
                                    (129, 129, 128), (1, 1, 64), (900, 37, 128)])
def test_geqrf_parity(lu, dtype, m, n, nb):
    A0 = synth.uniform_matrix(m, n, seed=80, stream=m + n)
    if dtype == torch.float32:
        A0 = A0.astype(np.float32).astype(np.float64)
    QR, tau, info = qr_gpu(lu, A0, dtype, nb=nb, lookahead=1)
    assert info == 0
    QRo, tauo = oracle.geqr2(A0)
    tol = 1e-12 if dtype == torch.float64 else 1e-3
    scale = max(np.abs(QRo).max(), 1.0)
    assert np.abs(QR - QRo).max() <= tol * scale
    assert np.abs(tau - tauo).max() <= tol * 2
    res, orth = oracle.qr_error(A0, QR, tau)
    u = np.finfo(np.float64 if dtype == torch.float64 else np.float32).eps / 2
    assert res <= (1e-14 if dtype == torch.float64 else 8 * u), res
    assert orth <= 50 * max(m, n) * u, orth


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_geqrf_lookahead_bit_identical(lu, dtype):
    A0 = synth.normal_matrix(1500, seed=81)
    outs = [qr_gpu(lu, A0, dtype, nb=128, lookahead=la) for la in (0, 1, 1)]
    for QR, tau, info in outs:
        assert info == 0
        assert np.array_equal(QR, outs[0][0]) and np.array_equal(tau, outs[0][1])
    # a per-step schedule of widths
    QR, tau, info = qr_gpu(lu, A0, dtype, nb=0, sched=[128, 64, 96, 32], lookahead=1)
    res, _ = oracle.qr_error(A0, QR, tau)
    assert info == 0 and res <= (1e-14 if dtype == torch.float64 else 1e-6)


def test_geqrf_upper_triangular_unchanged(lu):
    g = synth.rng(82, 0)
    U = np.triu(g.uniform(-1, 1, size=(400, 400)))
    QR, tau, info = qr_gpu(lu, U, torch.float64, nb=64)
    assert info == 0 and np.all(tau == 0.0) and np.array_equal(QR, U)


def test_geqrf_tall_panel_rows(lu):
    """A tall matrix (20000 x 256): the panel leaf spreads its rows over the most
    CTAs; compared with the oracle on the reflectors and through the residual."""
    m, n = 20000, 256
    A0 = synth.normal_matrix(m, n, seed=83)
    QR, tau, info = qr_gpu(lu, A0, torch.float64, nb=128)
    assert info == 0
    QRo, tauo = oracle.geqr2(A0)
    assert np.abs(QR - QRo).max() <= 1e-11 * np.abs(QRo).max()
    assert np.abs(tau - tauo).max() <= 1e-12
    R = np.triu(QR[:n])
    # ||A^T A - R^T R|| small: Q has orthonormal columns
    G = A0.T @ A0
    assert np.abs(G - R.T @ R).max() <= 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("m,n,nb", [(2048, 2048, 128), (3000, 1000, 64), (1500, 1500, 96)])
def test_geqrf_tensor_core_update(lu, m, n, nb):
    """FP32 QR with the update's last product on the tensor cores (split-bf16 x6,
    FP32-level accuracy): the FP32 residual and orthogonality bounds against the
    oracle, reflectors within the FP32 tolerance, look-ahead off/on
    bit-identical; with LU_TU_F32 it equals lu_geqrf_ex bit for bit."""
    from paper_1804_07017_gb300.api import colmajor
    A0 = synth.uniform_matrix(m, n, seed=84, stream=nb).astype(np.float32).astype(np.float64)

    def run(prec, la):
        A = colmajor(m, n, dtype=torch.float32)
        A.copy_(torch.from_numpy(A0).float())
        tau = torch.zeros(min(m, n), dtype=torch.float32, device="cuda")
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_geqrf_mixed_ex(A, tau, info, prec, lu.default_opts(nb=nb, lookahead=la))
        torch.cuda.synchronize()
        return A.cpu().double().numpy(), tau.cpu().double().numpy(), int(info.item())

    QR0, t0, i0 = run(lu.LU_TU_BF16X6, 0)
    QR1, t1, i1 = run(lu.LU_TU_BF16X6, 1)
    assert i0 == i1 == 0 and np.array_equal(QR0, QR1) and np.array_equal(t0, t1)
    u = np.finfo(np.float32).eps / 2
    res, orth = oracle.qr_error(A0, QR1, t1)
    assert res <= 8 * u and orth <= 50 * max(m, n) * u, (res, orth)
    QRo, tauo = oracle.geqr2(A0)
    assert np.abs(QR1 - QRo).max() <= 1e-3 * max(np.abs(QRo).max(), 1.0)
    QRs, ts, _ = run(lu.LU_TU_F32, 1)
    QRg, tg, _ = qr_gpu(lu, A0, torch.float32, nb=nb, lookahead=1)
    assert np.array_equal(QRs, QRg) and np.array_equal(ts, tg)
