"""GPU checks of the block-size autotuner (lu_tune_nb) and of nb = 0, which
takes the tuned value: the chosen nb is the candidate of least measured time,
rejected candidates are reported as -1, and a factorization called with nb = 0
is bit-identical to one called with the tuned nb."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1804_07017_gb300 as pkg
    pkg.lib()
    pkg.lu_tune_clear()
    yield pkg
    pkg.lu_tune_clear()


def dev(a, dtype):
    from paper_1804_07017_gb300.api import colmajor
    t = colmajor(a.shape[0], a.shape[1], dtype=dtype)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def test_tune_mixed_and_nb_zero(lu):
    n = 2048
    best, ms = lu.lu_tune_nb(lu.LU_TU_BF16X6, n, [128, 256, 2000], reps=3)
    assert ms[2] == -1.0 and ms[0] > 0 and ms[1] > 0
    assert best == (128 if ms[0] <= ms[1] else 256)
    assert lu.lu_tune_get(lu.LU_TU_BF16X6, n) == best
    assert lu.lu_tune_get(lu.LU_TU_BF16X6, n // 2) == 0
    A0 = synth.normal_matrix(n, seed=50)
    outs = []
    for nb in (0, best):
        A = dev(A0, torch.float32)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_factor_mixed_ex(A, ipiv, info, lu.LU_TU_BF16X6, lu.default_opts(nb=nb))
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        outs.append((A.cpu(), ipiv.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_tune_fp64_and_plain_lu_factor(lu):
    n = 1024
    best, ms = lu.lu_tune_nb(lu.LU_TUNE_F64, n, [64, 128], reps=2)
    assert best in (64, 128) and min(ms) > 0
    A0 = synth.uniform_matrix(n, seed=51)
    outs = []
    for nb in (0, best):
        A = dev(A0, torch.float64)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        assert lu.lu_factor(A, ipiv, nb) == 0
        outs.append((A.cpu(), ipiv.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_tune_fp8_skips_invalid_nb(lu):
    best, ms = lu.lu_tune_nb(lu.LU_TU_FP8, 1024, [192, 128], reps=1)
    assert ms[0] == -1.0 and ms[1] > 0 and best == 128


def test_tune_file_round_trip_on_device(lu, tmp_path):
    name = torch.cuda.get_device_name(0)
    lu.lu_tune_set(lu.LU_TUNE_F32, 3000, 192)
    assert lu.lu_tune_get(lu.LU_TUNE_F32, 3000, device=name) == 192
    p = str(tmp_path / "t.txt")
    lu.lu_tune_save(p)
    lu.lu_tune_clear()
    lu.lu_tune_load(p)
    assert lu.lu_tune_get(lu.LU_TUNE_F32, 2049) == 192
