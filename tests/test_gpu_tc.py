"""GPU parity of the tensor-core trailing update (tcgen05 + TMA), through the C ABI.

Reference: the oracle's RL3 update C - A B evaluated in FP64 on the operands
rounded to the tensor-core operand type by the oracle's own ties-to-even
rounding.  The kernel accumulates in FP32, so the stated tolerance is the
FP32 accumulation bound (k + 2) u32 (|A||B| + |C|) elementwise.
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


def dev32(a):
    from paper_1804_07017_gb300.api import colmajor
    t = colmajor(a.shape[0], a.shape[1], dtype=torch.float32)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).float())
    return t


def split_parts(X):
    p0 = oracle.round_bf16(X)
    p1 = oracle.round_bf16(X - p0)
    p2 = oracle.round_bf16(X - p0 - p1)
    return p0, p1, p2


def split6_product(A, B):
    """The six-product three-part split-bf16 product, exact in FP64."""
    a, b = split_parts(A), split_parts(B)
    pairs = ((0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0))
    prod = sum(a[i] @ b[j] for i, j in pairs)
    aprod = sum(np.abs(a[i]) @ np.abs(b[j]) for i, j in pairs)
    return prod, aprod


def split_product(A, B):
    """hi_A hi_B + hi_A lo_B + lo_A hi_B with hi = bf16(x), lo = bf16(x - hi): the
    split-bf16 product, formed exactly in FP64 from the oracle's rounding."""
    Ah, Bh = oracle.round_bf16(A), oracle.round_bf16(B)
    Al, Bl = oracle.round_bf16(A - Ah), oracle.round_bf16(B - Bh)
    return Ah @ Bh + Ah @ Bl + Al @ Bh, np.abs(Ah) @ np.abs(Bh) + np.abs(Ah) @ np.abs(Bl) + np.abs(Al) @ np.abs(Bh)


@pytest.mark.parametrize("prec_name", ["bf16", "fp16", "bf16x3", "bf16x6", "fp8"])
@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (256, 256, 64), (1000, 700, 256), (300, 5000, 64),
                                   (4097, 129, 512), (1, 1, 64), (129, 257, 128)])
def test_tc_update(lu, prec_name, m, n, k):
    prec = {"bf16": lu.LU_TU_BF16, "fp16": lu.LU_TU_FP16, "bf16x3": lu.LU_TU_BF16X3,
            "bf16x6": lu.LU_TU_BF16X6, "fp8": lu.LU_TU_FP8}[prec_name]
    if prec_name == "fp8" and k % 128:
        pytest.skip("the e4m3 path takes k in multiples of 128")
    rnd = oracle.round_bf16 if prec_name == "bf16" else oracle.round_fp16
    g = synth.rng(31, m + n + k)
    C0, A0, B0 = (g.standard_normal(size=s).astype(np.float32).astype(np.float64)
                  for s in ((m, n), (m, k), (k, n)))
    C = dev32(C0)
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    lu.lu_gemm_update_tc_ex(C, dev32(A0), dev32(B0), prec, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    got = C.cpu().double().numpy()
    u32 = np.finfo(np.float32).eps / 2
    if prec_name == "fp8":
        # power-of-two block scales (per row of A, per column of B), e4m3 values, FP32
        # accumulation; the oracle's quantiser decides the same exponents exactly
        Qa, sa = oracle.quant_e4m3_rows(A0)
        Qb, tb = oracle.quant_e4m3_cols(B0)
        Ad, Bd = Qa * sa[:, None], Qb * tb[None, :]
        ref = C0 - Ad @ Bd
        scale = np.abs(Ad) @ np.abs(Bd) + np.abs(C0)
        err = np.abs(got - ref)
        assert np.all(err <= (k + 2) * u32 * scale), (err / scale).max()
        return
    if prec_name == "bf16x6":
        prod, aprod = split6_product(A0, B0)
        ref = C0 - prod
        scale = aprod + np.abs(C0)
        assert np.all(np.abs(got - ref) <= (6 * k + 2) * u32 * scale)
        # only products of weight <= 2^-24 are dropped: FP32-accurate
        exact = oracle.gemm_update(C0, A0, B0)
        assert np.all(np.abs(got - exact) <= (2.0 ** -21 + (6 * k + 2) * u32) * (np.abs(A0) @ np.abs(B0) + np.abs(C0)))
        return
    if prec_name == "bf16x3":
        prod, aprod = split_product(A0, B0)
        ref = C0 - prod
        scale = aprod + np.abs(C0)
        err = np.abs(got - ref)
        assert np.all(err <= (3 * k + 2) * u32 * scale), (err / scale).max()
        # and it is close to the exact FP64 product: only lo*lo (~2^-16 relative) is missing
        exact = oracle.gemm_update(C0, A0, B0)
        assert np.all(np.abs(got - exact) <= (2.0 ** -15 + (3 * k + 2) * u32) * (np.abs(A0) @ np.abs(B0) + np.abs(C0)))
        return
    Ar, Br = rnd(A0), rnd(B0)
    ref = oracle.gemm_update(C0, Ar, Br)
    scale = np.abs(Ar) @ np.abs(Br) + np.abs(C0)
    err = np.abs(got - ref)
    assert np.all(err <= (k + 2) * u32 * scale), (err / scale).max()
    # the rounding actually happened: against the unrounded operands some entries
    # differ by more than the accumulation bound
    if m * n > 1000:
        ref_unrounded = oracle.gemm_update(C0, A0, B0)
        assert np.any(np.abs(got - ref_unrounded) > (k + 2) * u32 * scale)


def test_tc_update_repeatable(lu):
    m, n, k = 2000, 1500, 256
    g = synth.rng(32, 0)
    C0, A0, B0 = (g.standard_normal(size=s) for s in ((m, n), (m, k), (k, n)))
    outs = []
    for _ in range(3):
        C = dev32(C0)
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        lu.lu_gemm_update_tc_ex(C, dev32(A0), dev32(B0), lu.LU_TU_BF16, info)
        torch.cuda.synchronize()
        outs.append(C.cpu().numpy())
    # the dynamic tile schedule changes which CTA computes a tile, not the arithmetic
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
