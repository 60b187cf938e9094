"""Single-kernel cases for profilers (ncu) and quick timing on one GPU.

    python -m paper_1804_07017_gb300.profile_cases leaf --m 16384 --w 16
        one FP32 panel factorization of an m x w N(0,1) panel through
        lu_panel_factor_ex (for w <= 32 this is a single cluster-leaf launch)
    python -m paper_1804_07017_gb300.profile_cases tc --m 8192 --n 8192 --k 256 --prec 6
        one tensor-core trailing update C := C - A B (FP32 C of m x n; prec as
        lu_prec, 6 = split-bf16 x6) through lu_gemm_update_tc_ex
    python -m paper_1804_07017_gb300.profile_cases trsv --n 16384
        one FP32 LU of order n (mixed path), then its unit-lower and upper
        triangular solves through lu_solve_ex
    python -m paper_1804_07017_gb300.profile_cases batched --count 4096 --prec 32
        one persistent batched factor + solve of count systems, n_i log-uniform
        in [16, 512], nrhs_i in 1..8, iid U[-1,1) (--prec 32 or 64 selects FP32
        or FP64) through lu_gesv_batched

Each case runs --reps times (default 2) and prints the event-timed duration of
the last repetition.  Inputs are seeded and synthetic.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import api as lu  # noqa: E402


def _timed(fn, reps):
    ms = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    return ms


def case_leaf(a):
    P0 = torch.from_numpy(synth.normal_matrix(a.m, a.w, seed=3)).float()
    P = lu.colmajor(a.m, a.w, dtype=torch.float32)
    ipiv = torch.zeros(a.w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run():
        P.copy_(P0)
        lu.lu_panel_factor_ex(P, ipiv, info, lu.default_opts(leaf=a.w))

    ms = _timed(run, a.reps)
    print(f"leaf m={a.m} w={a.w}: {ms * 1e3:.1f} us (with the panel copy), info={int(info.item())}")


def case_tc(a):
    g = synth.rng(5, 0)
    C0 = torch.from_numpy(g.standard_normal((a.m, a.n))).float()
    A = lu.colmajor(a.m, a.k, dtype=torch.float32)
    B = lu.colmajor(a.k, a.n, dtype=torch.float32)
    A.copy_(torch.from_numpy(g.standard_normal((a.m, a.k))).float())
    B.copy_(torch.from_numpy(g.standard_normal((a.k, a.n))).float())
    C = lu.colmajor(a.m, a.n, dtype=torch.float32)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run():
        C.copy_(C0)
        lu.lu_gemm_update_tc_ex(C, A, B, a.prec, info)

    ms = _timed(run, a.reps)
    print(f"tc m={a.m} n={a.n} k={a.k} prec={a.prec}: {ms * 1e3:.1f} us (with the C copy), info={int(info.item())}")


def case_trsv(a):
    n = a.n
    A0 = synth.normal_matrix(n, seed=0)
    A = lu.colmajor(n, n, dtype=torch.float32)
    A.copy_(torch.from_numpy(A0).float())
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu.lu_factor_mixed_ex(A, ipiv, info, 6, lu.default_opts(nb=256))
    torch.cuda.synchronize()
    B0 = torch.from_numpy(np.ones((n, 1))).float()
    B = lu.colmajor(n, 1, dtype=torch.float32)

    def run():
        B.copy_(B0)
        lu.lu_solve_ex(A, ipiv, B)

    ms = _timed(run, a.reps)
    print(f"trsv n={n}: solve {ms * 1e3:.1f} us, info={int(info.item())}")


def case_batched(a):
    sizes, nrhs = synth.batched_sizes(a.count, seed=0)
    mats = synth.batched_matrices(sizes, seed=0)
    g = synth.rng(0, 9)
    dt = torch.float64 if a.prec == 64 else torch.float32
    A0 = [torch.from_numpy(m).to(dt) for m in mats]
    B0 = [torch.from_numpy(g.uniform(-1, 1, size=(int(n), int(r)))).to(dt) for n, r in zip(sizes, nrhs)]
    dA = [lu.colmajor(x.shape[0], x.shape[1], dtype=dt) for x in A0]
    dB = [lu.colmajor(x.shape[0], x.shape[1], dtype=dt) for x in B0]
    piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv, dB)
    for d, x in zip(dA + dB, A0 + B0):
        d.copy_(x)
    ms = 0.0
    for _ in range(a.reps):
        for d, x in zip(dA + dB, A0 + B0):
            d.copy_(x)
        ms = _timed(lambda: lu.lu_gesv_batched(batch), 1)
    ok = bool((batch.info == 0).all().item())
    print(f"batched count={a.count} prec={a.prec}: {ms * 1e3:.1f} us, all info zero: {ok}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["leaf", "tc", "trsv", "batched"])
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--w", type=int, default=16)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--prec", type=int, default=6)
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    {"leaf": case_leaf, "tc": case_tc, "trsv": case_trsv, "batched": case_batched}[a.case](a)


if __name__ == "__main__":
    main()
