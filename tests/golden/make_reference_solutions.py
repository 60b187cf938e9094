"""Write the CPU oracle's FP64 solutions of the large mixed-precision
configurations, against which the GPU solver's forward error is reported.

For each configuration the script rebuilds the seeded input with `synth`
exactly as `bench.py --workload configs` does, factors it with the oracle's
unblocked right-looking LU with partial pivoting (oracle.getrf, FP64, RL1 of
Sec. 3 run to completion) and solves with oracle.getrs.  It stores, per
configuration, `x_oracle_<name>.npy` (the solution, n x 1) and one entry of
`reference_solutions.json`: n, seed, ||A||_inf, ||x||_inf, the oracle's
backward error of that solution, and a fingerprint of the matrix (sha256 of a
strided sample of its column-major entries), which the bench compares before
using a stored solution.  Nothing here comes from the GPU path.

    python tests/golden/make_reference_solutions.py [name ...]

Runtime: tens of minutes for n = 16384 and over an hour for n = 32768 on a
few host cores (the oracle is unblocked and memory-bound).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

STRIDE = 4099  # fingerprint sample stride (prime, so it walks every row and column)


def fingerprint(A: np.ndarray) -> str:
    flat = np.asfortranarray(A).ravel(order="F")
    return hashlib.sha256(np.ascontiguousarray(flat[::STRIDE]).tobytes()).hexdigest()


def build(name: str):
    if name == "c2_normal_n16384":
        A = synth.normal_matrix(16384, seed=0)
    elif name == "c3_diag_scaled_n32768":
        A = synth.diag_scaled_normal(32768, seed=0)
    else:
        raise SystemExit(f"unknown configuration {name}")
    return A, synth.ones_rhs(A)


CONFIGS = ["c2_normal_n16384", "c3_diag_scaled_n32768"]


def main(names):
    meta_path = os.path.join(HERE, "reference_solutions.json")
    meta = json.load(open(meta_path)) if os.path.exists(meta_path) else {}
    for name in names:
        A, b = build(name)
        n = A.shape[0]
        fp = fingerprint(A)
        anorm = float(oracle.norm_inf(A))
        t0 = time.time()
        LU, ipiv, info, _ = oracle.getrf(A)
        x = oracle.getrs(LU, ipiv, b)
        dt = time.time() - t0
        del LU
        eta = float(oracle.backward_error(A, x, b))
        np.save(os.path.join(HERE, f"x_oracle_{name}.npy"), np.asarray(x, dtype=np.float64))
        meta[name] = {"n": n, "seed": 0, "rhs": "b = A * ones(n)", "fingerprint": fp, "fingerprint_stride": STRIDE,
                      "anorm_inf": anorm, "xnorm_inf": float(np.abs(x).max()), "oracle_bwd_err": eta,
                      "oracle_info": int(info), "oracle_seconds": round(dt, 1), "oracle_threads": oracle.num_threads()}
        with open(meta_path, "w") as f:
            json.dump(meta, f, indent=1, sort_keys=True)
        print(f"{name}: n={n} eta={eta:.2e} in {dt:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or CONFIGS)
