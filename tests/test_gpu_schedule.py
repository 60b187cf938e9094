"""GPU checks of the schedule options of the blocked factorization: per-step
block sizes (the GPU form of the paper's early termination, Sec. 4.2: b
changed from step to step), depth-2 look-ahead, the SMs the right update
leaves to the panel path, the per-step trace and the plan tuner.

Pass criteria (as the other parity tests): against the CPU oracle, pivots
bit-exact at separated steps, factorization backward error <= 1e-14 (FP64) or
4 u32 (FP32), designed interchange sequences returned exactly, solve eta <=
1e-14 after refinement; and, since depth, reserve and stealing only change
which stream or CTA does an update and never an element's operations, the
factors of one schedule are bit-identical across depths 0, 1, 2 and across
reserves.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TAU = {torch.float64: 1e-8, torch.float32: 1e-3}
BOUND = {torch.float64: 1e-14, torch.float32: 4 * np.finfo(np.float32).eps}


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
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    t = colmajor(a.shape[0], a.shape[1], dtype=dtype)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def factor(lu, A0, dtype, mixed=None, **opts):
    n = A0.shape[0]
    A = dev(A0, dtype)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    o = lu.default_opts(**opts)
    if mixed is None:
        lu.lu_factor_ex(A, ipiv, info, o)
    else:
        lu.lu_factor_mixed_ex(A, ipiv, info, mixed, o)
    torch.cuda.synchronize()
    return A.cpu().double().numpy()[:n, :n], ipiv.cpu().numpy(), int(info.item())


SCHEDULES = [[64, 128, 96, 37, 256], [256, 192, 128, 64], [32], [300, 20, 512]]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("sched", SCHEDULES)
def test_schedule_parity_and_depths_identical(lu, dtype, sched):
    n = 1100
    A0 = synth.uniform_matrix(n, seed=71, stream=len(sched))
    if dtype == torch.float32:
        A0 = A0.astype(np.float32).astype(np.float64)
    LU_o, piv_o, _, gap = oracle.getrf(A0)
    runs = []
    for depth, reserve in ((0, 0), (1, 0), (2, 0), (1, 40), (2, 8)):
        LU, piv, info = factor(lu, A0, dtype, nb=0, sched=sched, lookahead=depth, tu_reserve=reserve)
        assert info == 0
        runs.append((LU, piv))
    LU, piv = runs[0]
    sep = gap > TAU[dtype]
    assert np.array_equal(piv[sep], piv_o[sep])
    assert oracle.factor_error(A0, LU, piv) <= BOUND[dtype]
    for LUd, pivd in runs[1:]:
        assert np.array_equal(pivd, piv) and np.array_equal(LUd, LU)


@pytest.mark.parametrize("name", ["last_row", "in_panel", "mixed", "reverse"])
def test_schedule_designed_pivot_sequences(lu, name):
    """Designed interchange sequences through panels of changing width (the
    interchange plans, the leaves and the updates between them must return the
    sequence exactly), FP64 with depth 2 and the tensor-core path (bf16x6)."""
    import pivot_patterns as pp
    n = 900
    A0, piv_expect = pp.patterned_matrix(name, n, seed=19, panel=64)
    LU, piv, info = factor(lu, A0, torch.float64, nb=0, sched=[128, 64, 192, 37], lookahead=2)
    assert info == 0 and np.array_equal(piv, piv_expect)
    assert oracle.factor_error(A0, LU, piv) <= 1e-14
    A32 = A0.astype(np.float32).astype(np.float64)
    LU, piv, info = factor(lu, A32, torch.float32, mixed=lu.LU_TU_BF16X6, nb=0, sched=[128, 64, 192, 256],
                           lookahead=2)
    assert info == 0 and np.array_equal(piv, piv_expect)


def test_mixed_schedule_depth2_solve(lu):
    """lu_gesv_mixed with a per-step schedule and depth-2 look-ahead: the
    refined solution's eta <= 1e-14 (recomputed by the oracle), and the mixed
    factors are bit-identical across depths 1 and 2 and across reserves."""
    n = 2048
    A0 = synth.normal_matrix(n, seed=72)
    b0 = synth.ones_rhs(A0)
    sched = [384, 256, 256, 192, 128, 64]
    A, B, X = dev(A0, torch.float64), dev(b0, torch.float64), dev(np.zeros_like(b0), torch.float64)
    for depth in (1, 2):
        st, it, eta = lu.lu_gesv_mixed(A, B, X, lu.LU_TU_BF16X6, opts=lu.default_opts(nb=0, sched=sched,
                                                                                          lookahead=depth))
        torch.cuda.synchronize()
        x = X.cpu().numpy()
        assert st == 0 and oracle.backward_error(A0, x, b0) <= 1e-14, (depth, it, eta)
    A32 = A0.astype(np.float32).astype(np.float64)
    outs = [factor(lu, A32, torch.float32, mixed=lu.LU_TU_BF16X6, nb=0, sched=sched, lookahead=d, tu_reserve=r)
            for d, r in ((1, 0), (2, 0), (2, 50), (1, 12))]
    for LU, piv, info in outs:
        assert info == 0
        assert np.array_equal(piv, outs[0][1]) and np.array_equal(LU, outs[0][0])


def test_step_trace(lu):
    """The per-step trace covers every column once, in order, with positive
    panel-path and update times."""
    n, nb = 2048, 256
    A0 = synth.normal_matrix(n, seed=73).astype(np.float32).astype(np.float64)
    h = lu.lu_step_trace(True)
    try:
        factor(lu, A0, torch.float32, mixed=lu.LU_TU_BF16X6, nb=nb)
        steps = lu.lu_step_trace_read(h)
    finally:
        lu.lu_step_trace(False)
    assert len(steps) == n // nb
    assert [s["k0"] for s in steps] == list(range(0, n, nb)) and all(s["kb"] == nb for s in steps)
    assert all(s["span_ms"] > 0 and s["tu_ms"] >= 0 for s in steps)
    assert all(s["pu_ms"] > 0 for s in steps[:-1])
    print("\n[trace n=2048 nb=256] step span / PU(k+1) / TU_right(k) ms: " +
          ", ".join(f"{s['span_ms']:.2f}/{s['pu_ms']:.2f}/{s['tu_ms']:.2f}" for s in steps))


def test_tune_plan_and_nb_zero(lu):
    """lu_tune_plan returns a plan no slower than the best fixed plan it
    measured, stores it, and a factorization with nb = 0 applies it: its factors
    are bit-identical to those of the returned options and pass the parity
    criteria."""
    n = 2048
    best, sched, ms, fixed = lu.lu_tune_plan(lu.LU_TU_BF16X6, n, reps=3)
    assert 0 < ms <= fixed
    plan = lu.lu_tune_plan_get(lu.LU_TU_BF16X6, n)
    assert plan is not None and plan[0] == best.nb and plan[3] == sched
    assert best.lookahead in (1, 2) and (best.tu_reserve == 0 or best.tu_reserve >= 4)  # 0: automatic
    assert plan[4] == best.pf_sms
    print(f"\n[tune plan n={n} bf16x6] nb={best.nb} reserve={best.tu_reserve} depth={best.lookahead} "
          f"pf_sms={best.pf_sms} schedule={sched} best {ms:.2f} ms, fixed {fixed:.2f} ms")
    A0 = synth.normal_matrix(n, seed=74).astype(np.float32).astype(np.float64)
    LU0, p0, i0 = factor(lu, A0, torch.float32, mixed=lu.LU_TU_BF16X6, nb=0)
    LU1, p1, i1 = factor(lu, A0, torch.float32, mixed=lu.LU_TU_BF16X6, nb=best.nb, sched=sched,
                         lookahead=best.lookahead, tu_reserve=best.tu_reserve, pf_sms=best.pf_sms)
    assert i0 == i1 == 0 and np.array_equal(p0, p1) and np.array_equal(LU0, LU1)
    assert oracle.factor_error(A0, LU0, p0) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("opts", [dict(nb=64), dict(nb=0, sched=[128, 64, 37, 256]), dict(nb=256)])
def test_rtm_dag_identical_to_lookahead(lu, dtype, opts):
    """The runtime-task schedule (a dependency DAG of PF(k), TU(k, j) and the
    left interchanges, replayed as a CUDA graph) gives factors bit-identical
    to the static look-ahead ones -- the same operations per element -- on the
    first call (capture) and on a repeated call (replay), and meets the
    oracle's criteria."""
    n = 1300
    A0 = synth.uniform_matrix(n, seed=75)
    if dtype == torch.float32:
        A0 = A0.astype(np.float32).astype(np.float64)
    LU1, p1, i1 = factor(lu, A0, dtype, lookahead=1, **opts)
    for _ in range(2):
        LUr, pr, ir = factor(lu, A0, dtype, rtm=1, **opts)
        assert ir == i1 == 0
        assert np.array_equal(pr, p1) and np.array_equal(LUr, LU1)
    _, piv_o, _, gap = oracle.getrf(A0)
    sep = gap > TAU[dtype]
    assert np.array_equal(pr[sep], piv_o[sep])
    assert oracle.factor_error(A0, LUr, pr) <= BOUND[dtype]


def test_rtm_designed_pivots_and_cholesky(lu):
    """Designed interchange sequences come back exactly through the DAG
    schedule, and the Cholesky factorization (elimination without
    interchanges) under the DAG schedule equals its look-ahead result."""
    import pivot_patterns as pp
    for name in ("last_row", "mixed"):
        A0, piv_expect = pp.patterned_matrix(name, 800, seed=23, panel=64)
        LU, piv, info = factor(lu, A0, torch.float64, nb=64, rtm=1)
        assert info == 0 and np.array_equal(piv, piv_expect), name
        assert oracle.factor_error(A0, LU, piv) <= 1e-14
    n = 900
    S0 = synth.spd_matrix(n, seed=24)
    outs = []
    for o in (dict(nb=128), dict(nb=128, rtm=1)):
        A = dev(S0, torch.float64)
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        lu.lu_potrf_ex(A, info, lu.default_opts(**o))
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        outs.append(np.tril(A.cpu().numpy()))
    assert np.array_equal(outs[0], outs[1])
    assert oracle.chol_error(S0, outs[1]) <= 1e-14


def test_rtm_rejected_on_tensor_core_path(lu):
    n = 512
    A = dev(synth.normal_matrix(n, seed=76), torch.float32)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(lu.LuError) as e:
        lu.lu_factor_mixed_ex(A, ipiv, info, lu.LU_TU_BF16X6, lu.default_opts(nb=128, rtm=1))
    assert e.value.code == lu.LU_ERR_UNSUPPORTED


@pytest.mark.parametrize("pf_sms", [16, 24])
def test_leaf_sm_partition_identical(lu, pf_sms):
    """An SM partition for the panel leaves (green contexts; the right update on
    the other SMs) moves work between SMs; at n = 2048 the leaves keep their
    shapes, so the mixed and the FP64 factorizations are bit-identical to the
    unpartitioned ones, and the refined solve meets eta <= 1e-14."""
    n = 2048
    A0 = synth.normal_matrix(n, seed=77)
    A32 = A0.astype(np.float32).astype(np.float64)
    ref = factor(lu, A32, torch.float32, mixed=lu.LU_TU_BF16X6, nb=256)
    from paper_1804_07017_gb300.api import colmajor
    A = colmajor(n, n, dtype=torch.float32)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    o = lu.default_opts(nb=256, pf_sms=pf_sms)
    for _ in range(3):  # eager, captured as a graph, replayed
        A.copy_(torch.from_numpy(A32).float())
        lu.lu_factor_mixed_ex(A, ipiv, info, lu.LU_TU_BF16X6, o)
        torch.cuda.synchronize()
        got = (A.cpu().double().numpy(), ipiv.cpu().numpy(), int(info.item()))
        assert ref[2] == got[2] == 0 and np.array_equal(ref[1], got[1]) and np.array_equal(ref[0], got[0])
    r64 = factor(lu, A0, torch.float64, nb=128)
    g64 = factor(lu, A0, torch.float64, nb=128, pf_sms=pf_sms)
    assert np.array_equal(r64[1], g64[1]) and np.array_equal(r64[0], g64[0])
    b0 = synth.ones_rhs(A0)
    A, B, X = dev(A0, torch.float64), dev(b0, torch.float64), dev(np.zeros_like(b0), torch.float64)
    st, it, eta = lu.lu_gesv_mixed(A, B, X, lu.LU_TU_BF16X6, opts=lu.default_opts(nb=256, pf_sms=pf_sms))
    torch.cuda.synchronize()
    assert st == 0 and oracle.backward_error(A0, X.cpu().numpy(), b0) <= 1e-14


def sampled_residual(A0, LU, piv, rows):
    """max over the sampled rows i of ||(PA - LU)(i, :)||_1 / (n ||A||_inf), each
    row of L U formed on the host from row i of L and the rows of U it touches."""
    n = A0.shape[0]
    order = np.arange(n)
    for k in range(n):
        p = piv[k] - 1
        order[k], order[p] = order[p], order[k]
    anorm = np.abs(A0).sum(axis=1).max()
    worst = 0.0
    for i in rows:
        l = LU[i, : i + 1].copy()
        l[i] = 1.0
        acc = np.zeros(n)
        for p0 in range(0, i + 1, 512):
            p1 = min(i + 1, p0 + 512)
            acc += l[p0:p1] @ np.triu(LU[p0:p1, :], k=p0)
        worst = max(worst, np.abs(A0[order[i], :] - acc).sum() / (n * anorm))
    return worst


@pytest.mark.parametrize("name", ["random", "in_panel"])
def test_leaf_partition_wide_leaves(lu, name):
    """On an SM partition of their own the panel leaves may take more shared
    memory, so a panel taller than 8192 rows is factored by 32-column leaves
    instead of pairs of 16-column ones: another rounding order inside the panel,
    the same partial pivoting.  n = 9216 (the first panels take the wide leaves):
    a designed interchange sequence comes back exactly; on N(0,1) the FP32
    factorization's residual on sampled rows stays within 4 u32 and the refined
    solve reaches eta <= 1e-14."""
    import pivot_patterns as pp
    n = 9216
    A0, piv_expect = pp.patterned_matrix(name, n, seed=23, panel=256)
    A32 = A0.astype(np.float32).astype(np.float64)
    LU, piv, info = factor(lu, A32, torch.float32, mixed=lu.LU_TU_BF16X6, nb=256, pf_sms=24)
    assert info == 0 and np.array_equal(piv, piv_expect)
    del LU
    A0 = synth.normal_matrix(n, seed=24)
    A32 = A0.astype(np.float32).astype(np.float64)
    LU, piv, info = factor(lu, A32, torch.float32, mixed=lu.LU_TU_BF16X6, nb=256, pf_sms=24)
    assert info == 0
    rows = np.concatenate([[0, 1, n // 2, n - 1], synth.rng(25, 0).integers(0, n, size=12)])
    assert sampled_residual(A32, LU, piv, rows) <= BOUND[torch.float32]
    del LU
    b0 = synth.ones_rhs(A0)
    A, B, X = dev(A0, torch.float64), dev(b0, torch.float64), dev(np.zeros_like(b0), torch.float64)
    st, it, eta = lu.lu_gesv_mixed(A, B, X, lu.LU_TU_BF16X6, opts=lu.default_opts(nb=256, pf_sms=24))
    torch.cuda.synchronize()
    assert st == 0 and oracle.backward_error(A0, X.cpu().numpy(), b0) <= 1e-14
