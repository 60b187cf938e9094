"""lu_panel_factor_noalloc: the panel factorization for callers that cannot
allocate device memory (code running where cudaMalloc is unavailable or not
allowed).  Its scratch is a static device array inside the library instead of
a handle's workspace.  The test calls it through the C ABI twice in a row (the
array keeps the previous call's contents, so the second call checks that
everything that must start at zero is cleared) and compares each result with
the allocating entry point lu_panel_factor_ex on the same panel: the two run
the same kernels with the same options, so pivots and factors must be
bit-identical.  Each result is also checked against the CPU oracle directly
(pivots at separated steps, factors entry by entry).  The cases cover both
leaf kinds: panels that fit one thread-block cluster, and panels too tall for
one (40000 FP64 rows), which take the grid-barrier leaf and the in-panel
interchange plan, the two largest regions of the static array.  This file is
collected last.
"""
import ctypes

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


@pytest.mark.parametrize("dtype,m,w,tau,tol", [(torch.float64, 3000, 128, 1e-8, 1e-12),
                                               (torch.float32, 5000, 256, 1e-3, 2e-4),
                                               (torch.float64, 700, 37, 1e-8, 1e-12),
                                               (torch.float64, 40000, 64, 1e-8, 1e-12)])
def test_noalloc_matches_allocating_entry_point(lu, dtype, m, w, tau, tol):
    for call in range(2):
        P0 = synth.uniform_matrix(m, w, seed=61, stream=100 * call + w)
        if dtype == torch.float32:
            P0 = P0.astype(np.float32).astype(np.float64)
        ref = dev(P0, dtype)
        piv_ref = torch.zeros(w, dtype=torch.int32, device="cuda")
        info_ref = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_panel_factor_ex(ref, piv_ref, info_ref)
        got = dev(P0, dtype)
        piv = torch.zeros(w, dtype=torch.int32, device="cuda")
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_panel_factor_noalloc(got, piv, info)
        torch.cuda.synchronize()
        assert int(info.item()) == 0 and int(info_ref.item()) == 0
        p = piv.cpu().numpy()
        assert np.array_equal(p, piv_ref.cpu().numpy())
        a = got.cpu().double().numpy()
        assert np.array_equal(a, ref.cpu().double().numpy())
        # and directly against the oracle (RL1 of Sec. 3, LU_unb)
        LU_o, p_o, info_o, gap = oracle.getrf(P0)
        assert info_o == 0
        sep = gap > tau
        assert np.array_equal(p[sep], p_o[sep])
        diff = np.nonzero(p != p_o)[0]
        d = int(diff[0]) if diff.size else w
        assert np.abs(a[:d] - LU_o[:d]).max(initial=0.0) <= tol * np.abs(LU_o).max()
        if d == w:
            assert np.abs(a - LU_o).max() <= tol * np.abs(LU_o).max()


def test_noalloc_zero_pivot_and_limits(lu):
    # an exactly zero column: info must report it on this call even though the
    # previous calls left their own state in the shared array
    m, w = 400, 64
    P0 = synth.uniform_matrix(m, w, seed=62)
    P0[:, 10] = 0.0
    got = dev(P0, torch.float64)
    piv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu.lu_panel_factor_noalloc(got, piv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 11
    # sizes beyond the static array's plan are rejected before any work
    L = lu.lib()
    o = lu.default_opts()
    rc = L.lu_panel_factor_noalloc(0, 4096, 1025, ctypes.c_void_p(got.data_ptr()), 4096,
                                   ctypes.c_void_p(piv.data_ptr()), ctypes.byref(o),
                                   ctypes.c_void_p(info.data_ptr()), None)
    assert rc == lu.LU_ERR_UNSUPPORTED
    assert L.lu_noalloc_scratch_bytes() < 256 * 1024
