"""Failure handling without a GPU fault: a bounded device-side wait that can
never be satisfied gives up after a short limit, reports LU_ERR_TIMEOUT to the
host, and leaves the device usable for the next call."""
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


def test_bounded_wait_reports_timeout_and_device_stays_usable(lu):
    h = lu.Handle()
    h.set_stream()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lu.lib().lu_selftest_wait_timeout(h.ptr, 50_000_000, ctypes.c_void_p(status.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == lu.LU_ERR_TIMEOUT
    # invalid limits are rejected on the host
    assert lu.lib().lu_selftest_wait_timeout(h.ptr, 0, ctypes.c_void_p(status.data_ptr())) == -2
    # the same handle and device factor correctly afterwards
    from paper_1804_07017_gb300.api import colmajor
    n = 300
    A0 = synth.uniform_matrix(n, seed=71)
    A = colmajor(n, n)
    A.copy_(torch.from_numpy(A0))
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    lu.lu_factor_ex(A, ipiv, info, lu.default_opts(nb=64), handle=h)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert oracle.factor_error(A0, A.cpu().numpy(), ipiv.cpu().numpy()) <= 1e-14
    h.close()
