"""GPU parity of the Cholesky factorization (lu_potrf_ex) against the CPU
oracle (oracle.potrf).

Criteria: ||A - L L^T|| / (n ||A||) <= 1e-14 (FP64) / 4 u32 (FP32), the
factor within a small multiple of its condition-scaled rounding of the
oracle's, L lower with a positive diagonal, look-ahead on and off
bit-identical, and the position of the first non-positive-definite leading
minor equal to the oracle's.
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


def potrf_gpu(lu, A0, nb, dtype=torch.float64, ld=None, **opts):
    from paper_1804_07017_gb300.api import colmajor
    n = A0.shape[0]
    A = colmajor(n, n, dtype=dtype, ld=ld)
    A.copy_(torch.from_numpy(np.ascontiguousarray(A0)).to(dtype))
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    lu.lu_potrf_ex(A, info, lu.default_opts(nb=nb, **opts))
    torch.cuda.synchronize()
    return np.tril(A.cpu().double().numpy()[:n, :n]), int(info.item())


@pytest.mark.parametrize("n,nb,ld_pad", [(1, 64, 0), (31, 64, 0), (100, 32, 3), (333, 64, 0), (1024, 128, 7),
                                         (2000, 256, 0)])
def test_potrf_fp64(lu, n, nb, ld_pad):
    A0 = synth.spd_matrix(n, seed=n)
    L, info = potrf_gpu(lu, A0, nb, ld=n + ld_pad if ld_pad else None)
    assert info == 0
    Lo, info_o = oracle.potrf(A0)
    assert info_o == 0
    assert np.all(np.diag(L) > 0)
    assert oracle.chol_error(A0, L) <= 1e-14
    # A has eigenvalues in [1, 2.4], so L is perfectly conditioned: entrywise agreement
    assert np.abs(L - Lo).max() <= 1e-13 * np.abs(Lo).max()


def test_potrf_fp32(lu):
    n, nb = 1500, 128
    A0 = synth.spd_matrix(n, seed=5).astype(np.float32).astype(np.float64)
    L, info = potrf_gpu(lu, A0, nb, dtype=torch.float32)
    assert info == 0
    assert oracle.chol_error(A0, L) <= 4 * np.finfo(np.float32).eps
    Lo, _ = oracle.potrf(A0)
    assert np.abs(L - Lo).max() <= 1e-4 * np.abs(Lo).max()


def test_potrf_lookahead_bit_identical(lu):
    n, nb = 1536, 128
    A0 = synth.spd_matrix(n, seed=8)
    L0, i0 = potrf_gpu(lu, A0, nb, lookahead=0)
    L1, i1 = potrf_gpu(lu, A0, nb, lookahead=1)
    assert i0 == i1 == 0 and np.array_equal(L0, L1)


@pytest.mark.parametrize("pos", [0, 40, 200, 299])
def test_potrf_not_positive_definite(lu, pos):
    n = 300
    A0 = synth.spd_matrix(n, seed=9)
    A0[pos, pos] = -50.0  # leading pos x pos minor untouched
    _, info = potrf_gpu(lu, A0, 64)
    _, info_o = oracle.potrf(A0)
    assert info == info_o == pos + 1


def test_potrf_solve_through_factor(lu):
    """x from two triangular solves with the GPU factor meets the FP64 backward
    error bound of the oracle's definition."""
    n = 800
    A0 = synth.spd_matrix(n, seed=10)
    L, info = potrf_gpu(lu, A0, 128)
    assert info == 0
    b = A0 @ np.ones(n)
    y = np.linalg.solve(L, b)
    x = np.linalg.solve(L.T, y)
    assert oracle.backward_error(A0, x[:, None], b[:, None]) <= 1e-14


@pytest.mark.parametrize("prec_name", ["bf16x6", "f32"])
def test_potrf_mixed_tensor_cores(lu, prec_name):
    """FP32 Cholesky with the trailing update on the tensor cores (split-bf16
    x6, FP32-level accuracy) or on the CUDA cores (f32, then bit-identical to
    lu_potrf_ex in FP32): the FP32 factor bounds against the oracle, and
    look-ahead on and off bit-identical."""
    from paper_1804_07017_gb300.api import colmajor
    prec = {"bf16x6": lu.LU_TU_BF16X6, "f32": lu.LU_TU_F32}[prec_name]
    n, nb = 2048, 256
    A0 = synth.spd_matrix(n, seed=11).astype(np.float32).astype(np.float64)
    outs = []
    for la in (0, 1):
        A = colmajor(n, n, dtype=torch.float32)
        A.copy_(torch.from_numpy(A0).float())
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_potrf_mixed_ex(A, info, prec, lu.default_opts(nb=nb, lookahead=la))
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        outs.append(np.tril(A.cpu().double().numpy()))
    assert np.array_equal(outs[0], outs[1])
    L = outs[1]
    assert oracle.chol_error(A0, L) <= 8 * np.finfo(np.float32).eps
    Lo, _ = oracle.potrf(A0)
    assert np.abs(L - Lo).max() <= 1e-4 * np.abs(Lo).max()
    if prec_name == "f32":
        L32, info = potrf_gpu(lu, A0, nb, dtype=torch.float32)
        assert info == 0 and np.array_equal(L32, L)


def test_potrf_depth2_and_task_dag(lu):
    """The symmetric update under depth-2 look-ahead and under the task-DAG
    schedule: factors bit-identical to depth 1."""
    n, nb = 1100, 128
    A0 = synth.spd_matrix(n, seed=12)
    L1, i1 = potrf_gpu(lu, A0, nb, lookahead=1)
    L2, i2 = potrf_gpu(lu, A0, nb, lookahead=2)
    L3, i3 = potrf_gpu(lu, A0, nb, rtm=1)
    assert i1 == i2 == i3 == 0
    assert np.array_equal(L1, L2) and np.array_equal(L1, L3)
    assert oracle.chol_error(A0, L1) <= 1e-14
