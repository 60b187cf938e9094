"""Benchmark: LU + solve GFLOP/s (2 n^3 / 3 per solve) on one GB300.

Workload (default): the mixed-precision solver at n = 16384 -- A with iid
N(0,1) entries (seed 0), one right-hand side b = A * ones, FP32 panel
factorization, split-bf16 (bf16x6: three bf16 parts, six products) tensor-core
trailing update with FP32 accumulation,
depth-1 look-ahead, FP64 iterative refinement to a normwise backward error
<= 1e-14 (at most 30 corrections).  One step = one lu_gesv_mixed call (the
factorization, the solve and every refinement iteration), with A and b
resident in HBM (2 GiB, larger than L2).  The plain FP64 look-ahead LU + solve
(+ FP64 refinement to the same 1e-14) is timed beside it on the same GPU.

JSON line keys follow the harness contract: value / ms_per_step are the
mixed solver's; "fp64_path" holds the FP64 comparison; "roofline" the
dominant kernel measured with the library's per-launch CUDA events over the
timed region; "cpu_baseline" the CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 16384
NB_DEFAULT = 256
PROF_STRIDE = 7  # one dominant-class launch in 7 carries events (7: no common period with the panel recursion)
TOL = 1e-14
MAX_ITER = 30


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lu_gb300_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
        except Exception:
            rows = []
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) > 8:
                for nm, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist_mod) -> float:
    """The maximum of x over all ranks (x itself without a process group).  The
    tensor lives where the backend wants it: CUDA for NCCL, host for gloo."""
    if dist_mod is None:
        return float(x)
    import torch
    dev = "cuda" if dist_mod.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job GFLOP/s: every rank solves its own system (replicas, weak
    scaling), the step time is the slowest rank's."""
    return world * flops_per_rank / (ms_per_step * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(n: int, nrhs: int, seed: int = 0):
    import synth
    A = synth.normal_matrix(n, seed=seed)
    B = synth.ones_rhs(A, nrhs) if nrhs == 1 else synth.random_rhs(A, nrhs, seed=seed)[0]
    return A, B


def cpu_oracle_sample(n: int, seed: int, budget_s: float = 15.0):
    """The CPU oracle (unblocked FP64 GEPP, OpenMP over columns of each rank-1
    update) on the leading elimination steps of the same n x n matrix: time a
    growing number of steps until ~budget_s of CPU work, report the flops those
    steps perform (sum over steps j of 2 (n-j-1)^2 + (n-j-1)) per second."""
    import numpy as np
    import oracle
    import synth
    A = np.asfortranarray(synth.normal_matrix(n, seed=seed))
    steps = 8
    while True:
        W = A.copy(order="F")
        t0 = time.perf_counter()
        oracle.getrf_steps_inplace(W, steps)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or steps >= n:
            break
        steps = min(n, int(steps * max(2.0, (budget_s / 3) / max(dt, 1e-3))))
    j = np.arange(steps, dtype=np.float64)
    flops = float(np.sum(2.0 * (n - j - 1) ** 2 + (n - j - 1)))
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {steps} of {n} elimination steps of the unblocked FP64 oracle on the same "
                      f"N(0,1) n={n} matrix ({dt:.1f} s, {flops:.3e} flops)", "seconds": dt}


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, timed on the host cores on a
    bounded sample of the same workload (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n = args.n
    budget = float(os.environ.get("LU_BENCH_REF_BUDGET_S", "6"))
    vals = []
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_sample(n, 0, budget_s=budget / 4)
    sample = None
    for _ in range(args.steps):
        sample = cpu_oracle_sample(n, 0, budget_s=budget)
        vals.append(sample["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "LU+solve GFLOP/s (2n^3/3), mixed+IR vs FP64 on same GB300 at bwd err <=1e-14",
            "value": v, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": sample["cores"], "kind": "oracle",
                             "sample": sample["sample"]},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args):
    return {"workload": f"mixed-precision LU+solve+FP64 IR, n={args.n}, nb={args.nb}, N(0,1) seed 0, "
                        f"{args.nrhs} rhs b=A*ones, FP32 panels, {args.prec} tensor-core TU, depth-1 look-ahead",
            "n": args.n, "nb": args.nb, "nrhs": args.nrhs, "tu": args.prec, "lookahead": 1,
            "pf_sms": getattr(args, "pf_sms", 0),
            "tol": TOL, "max_iter": MAX_ITER, "l2": "inputs larger than L2 (A is 2 GiB FP64)"}


def main():
    return main_with_args(None)


def main_with_args(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--nb", type=int, default=NB_DEFAULT)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--pf-sms", type=int, default=24,
                    help="SMs reserved for the panel leaves (a green-context partition; 0 = none); 24 measured "
                         "best at n = 16384 among 0, 16, 24, 32")
    ap.add_argument("--prec", default="bf16x6", choices=["bf16x6", "bf16x3", "bf16", "fp16", "f32"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--workload", default="mixed",
                    choices=["mixed", "batched", "configs", "tune", "chol", "profile", "qr"],
                    help="mixed: the n=16384 solver (default); batched: 4096 uneven systems; "
                         "configs: the configuration comparisons; tune: the block-size sweeps; "
                         "chol: the Cholesky factorization; qr: the Householder QR; profile: one kernel case (--case) for "
                         "profilers and event timing")
    ap.add_argument("--case", default="leaf", choices=sorted(PROFILE_CASES),
                    help="profile case: " + "; ".join(f"{k}: {v[1]}" for k, v in sorted(PROFILE_CASES.items())))
    ap.add_argument("--shape", default="", help="profile case sizes, comma-separated (see --case)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"], help="profile case storage type")
    ap.add_argument("--reps", type=int, default=3, help="profile case repetitions (the median is reported)")
    ap.add_argument("--summarize-launches", metavar="CSV", default=None,
                    help="print per-kernel launches, total time and share from an ncu CSV launch list "
                         "(--metrics gpu__time_duration.sum --csv) and exit; needs no GPU")
    args = ap.parse_args(argv)
    if args.summarize_launches:
        return summarize_launches(args.summarize_launches)
    if args.workload == "profile":
        return run_profile(args)
    if args.workload == "qr":
        return run_qr(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "configs":
        return run_configs(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "tune":
        return run_tune(args)
    if args.workload == "chol":
        return run_chol(args)

    import numpy as np
    import torch

    import paper_1804_07017_gb300 as lu
    from paper_1804_07017_gb300 import _lib
    from paper_1804_07017_gb300.api import colmajor

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    L = lu.lib()
    n, nrhs = args.n, args.nrhs
    prec = {"bf16": lu.LU_TU_BF16, "fp16": lu.LU_TU_FP16, "f32": lu.LU_TU_F32, "bf16x3": lu.LU_TU_BF16X3,
            "bf16x6": lu.LU_TU_BF16X6}[args.prec]
    opts = lu.default_opts(nb=args.nb, pf_sms=args.pf_sms)
    A0, B0 = make_inputs(n, nrhs)
    A = colmajor(n, n)
    A.copy_(torch.from_numpy(A0))
    B = colmajor(n, nrhs)
    B.copy_(torch.from_numpy(B0))
    X = colmajor(n, nrhs)
    flops = 2.0 * n ** 3 / 3.0

    def step():
        return lu.lu_gesv_mixed(A, B, X, prec, TOL, MAX_ITER, opts)

    import ctypes

    def read_prof():
        out = {}
        for i, name in enumerate(_lib.KERNEL_CLASSES):
            c_cnt, c_ms, c_by, c_fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            L.lu_profile_read(i, ctypes.byref(c_cnt), ctypes.byref(c_ms), ctypes.byref(c_by), ctypes.byref(c_fl))
            out[name] = {"launches": c_cnt.value, "ms": c_ms.value, "bytes": c_by.value, "flops": c_fl.value}
        return out

    for _ in range(args.warmup):
        step()
    barrier()
    # one untimed step with every launch bracketed by events: per-class kernel time shares
    L.lu_profile_reset()
    L.lu_profile_enable(-1)
    step()
    L.lu_profile_enable(0)
    prof_all = read_prof()
    L.lu_profile_reset()
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    dom_idx = _lib.KERNEL_CLASSES.index(dom)
    total_kernel_ms = sum(v["ms"] for v in prof_all.values())
    shares = {k: round(v["ms"] / total_kernel_ms, 4) for k, v in prof_all.items() if v["launches"]}
    barrier()
    # timed region: the K steps behind `value` (a repeated factorization is replayed as one
    # CUDA graph, which per-launch events would bypass, so none are recorded here)
    barrier()
    launches0 = lu.lu_launch_count()
    results = []
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            results.append(step())
        ev1.record(stream)
        barrier()
    launches = lu.lu_launch_count() - launches0
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), dist)
    ms_step = ms_total / args.steps
    value = job_throughput(flops, world, ms_step)
    statuses = [r[0] for r in results]
    iters = [r[1] for r in results]
    etas = [r[2] for r in results]
    # roofline region: K more timed steps of the same workload in which one launch in
    # PROF_STRIDE of the dominant class is bracketed by CUDA events on its own stream
    L.lu_profile_reset()
    L.lu_profile_stride(PROF_STRIDE)
    L.lu_profile_enable(1 << dom_idx)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev2.record(stream)
    for _ in range(args.steps):
        step()
    ev3.record(stream)
    barrier()
    L.lu_profile_enable(0)
    L.lu_profile_stride(1)
    roof_ms_step = ev2.elapsed_time(ev3) / args.steps
    prof = read_prof()
    clocks = clk.summary()

    hbm, bf16_burst, bf16_sust, peak_src = load_peaks()
    d = prof[dom]
    avg_ms = d["ms"] / max(d["launches"], 1)
    avg_bytes = d["bytes"] / max(d["launches"], 1)
    avg_flops = d["flops"] / max(d["launches"], 1)
    ach = avg_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": (ach / hbm) if ach else None, "peak_source": peak_src, "traffic": None,
            "bytes_per_launch": avg_bytes, "avg_launch_ms": avg_ms, "launches": d["launches"],
            "flops_per_launch": avg_flops}
    if dom == "tc_update":
        roof["note"] = "HBM-bound at nb=256: 8 B of FP32 C per element vs 2*nb*segments MMA flops"
    elif dom == "panel":
        roof["note"] = ("panel-factorization leaf (thread-block cluster, pushed candidate messages): bound by the "
                        "per-column exchange latency, not by HBM; bytes = read+write of the leaf block plus its "
                        "interchanges on the other panel columns")
    if dom == "panel":
        # latency view: the leaves' time per eliminated column (every column passes one leaf)
        roof["latency"] = {"us_per_column": d["ms"] * PROF_STRIDE / args.steps / n * 1e3,
                           "columns_per_step": n,
                           "note": "pipelined: the leaves run on their own SMs (--pf-sms) or beside the "
                                   "tensor-core update (--pf-sms 0); a 32-column leaf at m = 16384 takes 1.9 us "
                                   "per column of kernel time alone (ncu), 2.6 us per column event-timed with "
                                   "its launch (--workload profile --case leaf --shape 16384,32)"}
    roof["sampled"] = (f"1 launch in {PROF_STRIDE} of the class carries events, over {args.steps} timed steps "
                       f"of the same workload run after the value's timed region ({roof_ms_step:.1f} ms per step "
                       f"there: launches that carry events are not replayed as a graph)")
    roof["launches_sampled"] = d["launches"]
    roof["launches"] = d["launches"] * PROF_STRIDE

    # end to end through the C ABI with host buffers: H2D of A and b, solve, D2H of x
    e2e = None
    if rank == 0 or world > 1:
        A_h = torch.from_numpy(np.asfortranarray(A0).T.copy()).pin_memory()  # row-major view of column-major data
        B_h = torch.from_numpy(np.asfortranarray(B0).T.copy()).pin_memory()
        X_h = torch.empty((nrhs, n), dtype=torch.float64).pin_memory()
        At = A.t()  # (n, n) row-major view of the column-major device buffer
        Bt = B.t()
        Xt = X.t()
        e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(e_steps):
            At.copy_(A_h, non_blocking=True)
            Bt.copy_(B_h, non_blocking=True)
            step()
            X_h.copy_(Xt, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(t0.elapsed_time(t1) / e_steps, dist)
        e2e = {"value": job_throughput(flops, world, e_ms), "unit": "GFLOP/s",
               "h2d_bytes_per_step": 8 * n * n + 8 * n * nrhs, "d2h_bytes_per_step": 8 * n * nrhs,
               "ms_per_step": e_ms}

    # plain FP64 look-ahead LU + solve (+ FP64 refinement to the same tolerance) on the same GPU
    fp64 = None
    if not args.no_fp64 and rank == 0:
        fp64 = fp64_path(lu, A0, B0, n, nrhs, args.nb)

    cpu = None
    if not args.no_cpu and rank == 0:
        cpu = cpu_oracle_sample(n, 0, budget_s=float(os.environ.get("LU_BENCH_CPU_BUDGET_S", "15")))
        cpu.pop("seconds", None)

    if rank == 0:
        ok = all(s == 0 for s in statuses) and max(etas) <= TOL
        line = {
            "metric": "LU+solve GFLOP/s (2n^3/3), mixed+IR vs FP64 on same GB300 at bwd err <=1e-14",
            "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "f32+bf16", "bf16x3": "f32+bf16x3", "bf16x6": "f32+bf16x6", "fp16": "f32+fp16",
                      "f32": "f32"}[args.prec] + "+f64-ir",
            "data": "synthetic", "config": workload_config(args) | {"parallelism": f"replicas{world}"},
            "converged": ok, "refinements": iters, "bwd_err": max(etas),
            "gpu_launches": launches, "kernel_time_share": shares,
            "roofline": roof, "clocks": clocks, "e2e": e2e, "fp64_path": fp64, "cpu_baseline": cpu,
        }
        if fp64 and fp64.get("value"):
            line["speedup_vs_fp64_path"] = value / fp64["value"]
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Single-kernel cases (--workload profile): one launch of one step of the path
# on seeded synthetic inputs, for ncu captures and event timing.  Each prints
# one JSON line: the case, its sizes, the median event-timed duration over
# --reps runs, and the algorithmic bytes and flops of one launch with the
# achieved rates.

def _shape(args, defaults):
    vals = [int(v) for v in args.shape.split(",") if v.strip()] if args.shape else []
    return vals + list(defaults[len(vals):])


def _median_ms(fn, reps, before=None):
    import torch
    out = []
    stream = torch.cuda.current_stream()
    for _ in range(max(1, reps)):
        if before is not None:
            before()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def _prof_line(case, sizes, ms, nbytes, flops, **extra):
    line = {"workload": "profile", "case": case, "sizes": sizes, "ms": ms,
            "bytes": nbytes, "flops": flops,
            "GB/s": nbytes / (ms * 1e-3) / 1e9 if ms > 0 else None,
            "GFLOP/s": flops / (ms * 1e-3) / 1e9 if ms > 0 else None}
    line.update(extra)
    print(json.dumps(line), flush=True)


def prof_leaf(args, lu, torch, dt):
    """panel factorization of an m x w N(0,1) panel with leaves of `leaf` columns
    (default w; w <= 32 and leaf = w: one cluster-leaf launch) on clusters of at
    most pf_ctas CTAs (0: the widest that fits)"""
    import synth
    m, w, leaf, ctas = _shape(args, (16384, 16, 0, 0))
    P0 = torch.from_numpy(synth.normal_matrix(m, w, seed=3)).to(dt)
    P = lu.api.colmajor(m, w, dtype=dt)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    o = lu.default_opts(leaf=leaf or w, pf_ctas=ctas)
    ms = _median_ms(lambda: lu.lu_panel_factor_ex(P, ipiv, info, o), args.reps, before=lambda: P.copy_(P0))
    es = P.element_size()
    _prof_line("leaf", {"m": m, "w": w, "leaf": leaf or w, "pf_ctas": ctas}, ms, 2.0 * m * w * es, float(m) * w * w,
               us_per_column=ms * 1e3 / w, info=int(info.item()))


def prof_tc(args, lu, torch, dt):
    """tensor-core trailing update C := C - A B, FP32 C (m x n), k = nb; --shape m,n,k,prec"""
    import synth
    m, n, k, prec = _shape(args, (8192, 8192, 256, 6))
    g = synth.rng(5, 0)
    C0 = torch.from_numpy(g.standard_normal((m, n))).float()
    A = lu.api.colmajor(m, k, dtype=torch.float32)
    B = lu.api.colmajor(k, n, dtype=torch.float32)
    A.copy_(torch.from_numpy(g.standard_normal((m, k))).float())
    B.copy_(torch.from_numpy(g.standard_normal((k, n))).float())
    C = lu.api.colmajor(m, n, dtype=torch.float32)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ms = _median_ms(lambda: lu.lu_gemm_update_tc_ex(C, A, B, prec, info), args.reps, before=lambda: C.copy_(C0))
    parts = {6: 6, 3: 3}.get(prec, 1)
    _prof_line("tc", {"m": m, "n": n, "k": k, "prec": prec}, ms, 8.0 * m * n + 4.0 * k * (m + n),
               2.0 * m * n * k, products=parts, info=int(info.item()))


def prof_trsm(args, lu, torch, dt):
    """RL2 A12 := L11^-1 A12 with unit-lower L11 (m x m) and A12 (m x n)"""
    import synth
    m, n = _shape(args, (256, 16128))
    g = synth.rng(12, m)
    L0 = np.tril(g.uniform(-1, 1, size=(m, m)), -1) + np.eye(m)
    Lt = lu.api.colmajor(m, m, dtype=dt)
    Lt.copy_(torch.from_numpy(L0).to(dt))
    B0 = torch.from_numpy(g.uniform(-1, 1, size=(m, n))).to(dt)
    B = lu.api.colmajor(m, n, dtype=dt)
    ms = _median_ms(lambda: lu.lu_trsm_ex(Lt, B), args.reps, before=lambda: B.copy_(B0))
    es = B.element_size()
    _prof_line("trsm", {"m": m, "n": n}, ms, es * (2.0 * m * n + 0.5 * m * m), float(m) * m * n)


def prof_laswp(args, lu, torch, dt):
    """the interchanges of one nb-step applied to the other columns: rows
    [k1, k1 + K) of an n x ncols matrix, targets drawn from [j, n)"""
    import synth
    n, ncols, K = _shape(args, (16384, 16128, 256))
    g = synth.rng(11, 0)
    ipiv = np.arange(1, n + 1, dtype=np.int32)
    for j in range(K):
        ipiv[j] = int(g.integers(j, n)) + 1
    A = lu.api.colmajor(n, ncols, dtype=dt)
    A.copy_(torch.from_numpy(g.uniform(-1, 1, size=(n, ncols))).to(dt))
    piv = torch.from_numpy(ipiv).cuda()
    moved = len({int(p) - 1 for p in ipiv[:K]} | set(range(K)))
    ms = _median_ms(lambda: lu.lu_laswp_ex(A, 0, K, piv), args.reps)
    es = A.element_size()
    _prof_line("laswp", {"n": n, "ncols": ncols, "K": K}, ms, 2.0 * moved * ncols * es, 0.0,
               rows_moved=moved, bytes_rule="each moved row read once and written once per column")


def prof_gemm(args, lu, torch, dt):
    """RL3 on the CUDA cores, C := C - A B (m x n, inner k)"""
    import synth
    m, n, k = _shape(args, (8192, 8192, 256))
    g = synth.rng(13, 0)
    C0 = torch.from_numpy(g.uniform(-1, 1, size=(m, n))).to(dt)
    A = lu.api.colmajor(m, k, dtype=dt)
    B = lu.api.colmajor(k, n, dtype=dt)
    A.copy_(torch.from_numpy(g.uniform(-1, 1, size=(m, k))).to(dt))
    B.copy_(torch.from_numpy(g.uniform(-1, 1, size=(k, n))).to(dt))
    C = lu.api.colmajor(m, n, dtype=dt)
    ms = _median_ms(lambda: lu.lu_gemm_update_ex(C, A, B), args.reps, before=lambda: C.copy_(C0))
    es = C.element_size()
    _prof_line("gemm", {"m": m, "n": n, "k": k}, ms, es * (2.0 * m * n + (m + n) * k), 2.0 * m * n * k)


def prof_trsv(args, lu, torch, dt):
    """solve with the factors of an FP32 mixed factorization of order n (N(0,1))"""
    import synth
    (n,) = _shape(args, (16384,))
    A = lu.api.colmajor(n, n, dtype=torch.float32)
    A.copy_(torch.from_numpy(synth.normal_matrix(n, seed=0)).float())
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu.lu_factor_mixed_ex(A, ipiv, info, 6, lu.default_opts(nb=256))
    torch.cuda.synchronize()
    B0 = torch.ones((n, 1), dtype=torch.float32)
    B = lu.api.colmajor(n, 1, dtype=torch.float32)
    ms = _median_ms(lambda: lu.lu_solve_ex(A, ipiv, B), args.reps, before=lambda: B.copy_(B0))
    _prof_line("trsv", {"n": n}, ms, 4.0 * n * n, 2.0 * n * n, info=int(info.item()))


def prof_batched(args, lu, torch, dt):
    """persistent batched factor + solve of count systems (n_i log-uniform in [16, 512], nrhs_i in 1..8)"""
    import synth
    (count,) = _shape(args, (4096,))
    sizes, nrhs = synth.batched_sizes(count, seed=0)
    mats = synth.batched_matrices(sizes, seed=0)
    g = synth.rng(0, 9)
    A0 = [torch.from_numpy(m).to(dt) for m in mats]
    B0 = [torch.from_numpy(g.uniform(-1, 1, size=(int(n), int(r)))).to(dt) for n, r in zip(sizes, nrhs)]
    dA = [lu.api.colmajor(x.shape[0], x.shape[1], dtype=dt) for x in A0]
    dB = [lu.api.colmajor(x.shape[0], x.shape[1], dtype=dt) for x in B0]
    piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
    batch = lu.Batch(dA, piv, dB)

    def restore():
        for d, x in zip(dA + dB, A0 + B0):
            d.copy_(x)

    ms = _median_ms(lambda: lu.lu_gesv_batched(batch), args.reps, before=restore)
    fl = float(sum(2.0 * int(n) ** 3 / 3 + 2.0 * int(n) ** 2 * int(r) for n, r in zip(sizes, nrhs)))
    es = dA[0].element_size()
    nb_ = float(sum(es * (2.0 * int(n) ** 2 + 2.0 * int(n) * int(r)) for n, r in zip(sizes, nrhs)))
    _prof_line("batched", {"count": count}, ms, nb_, fl, all_info_zero=bool((batch.info == 0).all().item()))


def prof_peak(args, lu, torch, dt):
    """CUDA-core FMA throughput (lu_peak_fma): blocks = SMs x 8 of 256 threads, 16 chains each"""
    L = lu.lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {}
    for name, code, tdt, iters in (("f64", 0, torch.float64, 20000), ("f32", 1, torch.float32, 400000)):
        blocks, threads = sms * 8, 256
        sink = torch.empty(blocks * threads, dtype=tdt, device="cuda")
        stream = torch.cuda.current_stream()

        def run():
            rc = L.lu_peak_fma(code, blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()),
                               ctypes.c_void_p(stream.cuda_stream))
            if rc != 0:
                raise RuntimeError(f"lu_peak_fma returned {rc}")

        run()
        with ClockSampler(torch.cuda.current_device()) as clk:
            ms = _median_ms(run, max(args.reps, 5))
        flops = 2.0 * L.lu_peak_fma_chains() * iters * blocks * threads
        res[name] = {"GFLOP/s": flops / (ms * 1e-3) / 1e9, "ms": ms, "clocks": clk.summary()}
    line = {"workload": "profile", "case": "peak", "fma_peak": res,
            "how": "lu_peak_fma: SMs x 8 CTAs of 256 threads, 16 independent FMA chains per thread, "
                   "median of CUDA-event-timed launches; no clock setting changed"}
    print(json.dumps(line), flush=True)


def prof_qr(args, lu, torch, dt):
    """Householder QR (lu_geqrf_ex) of an n x n U[-1,1) matrix, nb columns per panel, look-ahead on"""
    import synth
    n, nb = _shape(args, (4096, 128))
    A0 = torch.from_numpy(synth.uniform_matrix(n, seed=0)).to(dt)
    A = lu.api.colmajor(n, n, dtype=dt)
    tau = torch.zeros(n, dtype=dt, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    o = lu.default_opts(nb=nb)
    ms = _median_ms(lambda: lu.lu_geqrf_ex(A, tau, info, o), args.reps, before=lambda: A.copy_(A0))
    _prof_line("qr", {"n": n, "nb": nb}, ms, float(A.element_size()) * 2 * n * n, 4.0 * n ** 3 / 3,
               info=int(info.item()))


PROFILE_CASES = {
    "qr": (prof_qr, "Householder QR, --shape n,nb (4096,128)"),
    "leaf": (prof_leaf, "panel leaf, --shape m,w,leaf,pf_ctas (16384,16,w,0)"),
    "tc": (prof_tc, "tensor-core update, --shape m,n,k,prec (8192,8192,256,6)"),
    "trsm": (prof_trsm, "RL2 solve, --shape m,n (256,16128)"),
    "laswp": (prof_laswp, "row interchanges, --shape n,ncols,K (16384,16128,256)"),
    "gemm": (prof_gemm, "RL3 on CUDA cores, --shape m,n,k (8192,8192,256)"),
    "trsv": (prof_trsv, "triangular solves of an FP32 factorization, --shape n (16384)"),
    "batched": (prof_batched, "batched factor + solve, --shape count (4096)"),
    "peak": (prof_peak, "CUDA-core FMA throughput, FP64 and FP32"),
}


def summarize_launches(path):
    """Per-kernel launches, device time and share of an ncu launch list."""
    import collections
    import csv
    import re
    with open(path) as f:
        rows = [ln for ln in f if not ln.startswith("==")]
    unit_ms = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in csv.DictReader(rows):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = re.sub(r"^void\s+", "", re.sub(r"\(.*$", "", r["Kernel Name"]).replace("<unnamed>::", "")).strip()
        agg[name][0] += 1
        agg[name][1] += float(r["Metric Value"].replace(",", "")) * unit_ms.get(r["Metric Unit"], 1e-6)
    total = sum(v[1] for v in agg.values())
    print("| kernel | launches | total ms | share |\n|---|---:|---:|---:|")
    for name, (cnt, ms) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"| {name} | {cnt} | {ms:.3f} | {100 * ms / total if total else 0:.1f}% |")
    print(f"| total | {sum(v[0] for v in agg.values())} | {total:.3f} | |")
    return 0


def run_profile(args):
    import torch

    import paper_1804_07017_gb300 as lu
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required")
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    PROFILE_CASES[args.case][0](args, lu, torch, dt)
    return 0


def run_qr(args):
    """Householder QR (lu_geqrf_ex) on the look-ahead skeleton: FP64 n = 8192
    and FP32 n = 16384 on the CUDA cores, FP32 n = 16384 with the update's last
    product on the tensor cores (lu_geqrf_mixed_ex, split-bf16 x6); iid
    U[-1,1) (seed 0), look-ahead off and on, nb 64 and
    128; the matrix is restored from a device copy before each run (outside the
    timed region); median of three event-timed runs after one untimed run.
    GFLOP/s of 4n^3/3.  One JSON object."""
    import torch

    import paper_1804_07017_gb300 as lu
    import synth
    torch.cuda.set_device(0)
    out = {"metric": "QR GFLOP/s (4n^3/3)", "unit": "GFLOP/s", "data": "synthetic"}
    for name, dt, n, prec in (("fp64_n8192", torch.float64, 8192, None), ("fp32_n16384", torch.float32, 16384, None),
                              ("fp32_n16384_tc_bf16x6", torch.float32, 16384, lu.LU_TU_BF16X6)):
        if args.shape and str(n) not in args.shape.split(","):
            continue
        A0 = torch.from_numpy(synth.uniform_matrix(n, seed=0)).to(dt).cuda()
        A = lu.api.colmajor(n, n, dtype=dt)
        tau = torch.zeros(n, dtype=dt, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        res = {}
        for nb in (64, 128):
            for la in (0, 1):
                o = lu.default_opts(nb=nb, lookahead=la)
                if prec is None:
                    fn = (lambda: lu.lu_geqrf_ex(A, tau, info, o))
                else:
                    fn = (lambda: lu.lu_geqrf_mixed_ex(A, tau, info, prec, o))
                ms = _median_ms(fn, 4, before=lambda: A.copy_(A0))
                res[f"nb{nb}_lookahead{la}"] = {"ms": round(ms, 3), "gflops": round(4.0 * n ** 3 / 3 / ms / 1e6, 1),
                                                "info": int(info.item())}
        out[name] = res
        del A, A0
        torch.cuda.empty_cache()
    print(json.dumps(out))
    return 0


def run_chol(args):
    """Cholesky factorization (lu_potrf_ex, nb = 256, depth-1 look-ahead, the
    lower block triangle updated) of A = G G^T / n + I, G iid U[-1,1) from a
    seeded torch generator (formed on the device, outside the timed region):
    FP64 at n = 8192 and FP32 at n = 16384 on the CUDA cores, and FP32 at
    n = 16384 with the split-bf16 x6 tensor-core update (lu_potrf_mixed_ex).
    GFLOP/s of n^3/3 (the Cholesky count); two untimed runs, then the median of
    three event-timed runs, A restored from a device copy before each."""
    import statistics as st_
    import torch

    import paper_1804_07017_gb300 as lu
    from paper_1804_07017_gb300.api import colmajor

    torch.cuda.set_device(0)
    out = {"metric": "Cholesky GFLOP/s (n^3/3)", "unit": "GFLOP/s", "data": "synthetic"}
    for name, dt, n, prec in (("f64_n8192", torch.float64, 8192, None), ("f32_n16384", torch.float32, 16384, None),
                              ("f32_n16384_tc_bf16x6", torch.float32, 16384, "bf16x6")):
        g = torch.Generator(device="cuda")
        g.manual_seed(0)
        G = torch.rand((n, n), generator=g, device="cuda", dtype=dt) * 2 - 1
        S = (G @ G.t()) / n
        S = 0.5 * (S + S.t()) + torch.eye(n, device="cuda", dtype=dt)
        del G
        A = colmajor(n, n, dtype=dt)
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        o = lu.default_opts(nb=256)
        times = []
        for it in range(5):
            A.copy_(S)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if prec is None:
                lu.lu_potrf_ex(A, info, o)
            else:
                lu.lu_potrf_mixed_ex(A, info, lu.LU_TU_BF16X6, o)
            e1.record()
            torch.cuda.synchronize()
            if it >= 2:
                times.append(e0.elapsed_time(e1))
        ms = st_.median(times)
        out[name] = {"n": n, "ms": round(ms, 3), "gflops": round(n ** 3 / 3.0 / (ms * 1e-3) / 1e9, 1),
                     "info": int(info.item())}
        del S, A
        torch.cuda.empty_cache()
    print(json.dumps(out))
    return 0


def run_tune(args):
    """Block-size sweeps through the library's autotuner (lu_tune_nb): the mixed
    factorization with the split-bf16 x6 update at n = 16384 and the FP64
    factorization at n = 8192, each candidate timed three times on a seeded
    U[-1,1) matrix (least time counts); then whole plans (lu_tune_plan) at
    n = 16384 and 32768 (mixed) and 8192 (FP64), with the traced steps of the
    chosen plan.  --shape filters the plan sizes.  One JSON object."""
    import torch

    import paper_1804_07017_gb300 as lu

    torch.cuda.set_device(0)
    out = {"metric": "factorization ms per block size nb (least of 3 runs)", "unit": "ms", "data": "synthetic"}
    sweeps = [("mixed_bf16x6_n16384", lu.LU_TU_BF16X6, 16384, [128, 192, 256, 320, 384, 512, 768, 1024]),
              ("fp64_n8192", lu.LU_TUNE_F64, 8192, [128, 192, 256, 384, 512])]
    for name, kind, n, cand in sweeps:
        best, ms = lu.lu_tune_nb(kind, n, cand, reps=3)
        out[name] = {"n": n, "best_nb": best,
                     "ms": {str(c): (round(t, 3) if t >= 0 else None) for c, t in zip(cand, ms)},
                     "gflops_at_best": round(2.0 * n ** 3 / 3.0 / (min(t for t in ms if t >= 0) * 1e-3) / 1e9, 1)}
    # whole plans (lu_tune_plan): nb, the right update's SM reserve, look-ahead depth and
    # a per-step schedule built from traced steps; fixed = the best plan without a schedule
    plans = [("plan_mixed_bf16x6_n16384", lu.LU_TU_BF16X6, 16384),
             ("plan_mixed_bf16x6_n32768", lu.LU_TU_BF16X6, 32768),
             ("plan_fp64_n8192", lu.LU_TUNE_F64, 8192)]
    if args.shape:
        plans = [p for p in plans if str(p[2]) in args.shape.split(",")]
    for name, kind, n in plans:
        best, sched, ms, fixed = lu.lu_tune_plan(kind, n, reps=3)
        h = lu.lu_step_trace(True)
        A = torch.empty(0)
        try:
            import synth
            A0 = synth.uniform_matrix(n, seed=0)
            dt = torch.float64 if kind == lu.LU_TUNE_F64 else torch.float32
            A = lu.api.colmajor(n, n, dtype=dt)
            A.copy_(torch.from_numpy(A0).to(dt))
            ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
            info = torch.zeros(1, dtype=torch.int32, device="cuda")
            if kind == lu.LU_TUNE_F64:
                lu.lu_factor_ex(A, ipiv, info, best)
            else:
                lu.lu_factor_mixed_ex(A, ipiv, info, kind, best)
            steps = lu.lu_step_trace_read(h)
        finally:
            lu.lu_step_trace(False)
        del A
        torch.cuda.empty_cache()
        out[name] = {"n": n, "nb": best.nb, "tu_reserve": best.tu_reserve, "depth": best.lookahead,
                     "pf_sms": best.pf_sms,
                     "schedule": sched, "ms_best": round(ms, 3), "ms_fixed_plan": round(fixed, 3),
                     "gflops_best": round(2.0 * n ** 3 / 3.0 / (ms * 1e-3) / 1e9, 1),
                     "trace_of_chosen_plan": {
                         "steps": len(steps),
                         "pu_ms_sum": round(sum(x["pu_ms"] for x in steps), 2),
                         "tu_right_ms_sum": round(sum(x["tu_ms"] for x in steps), 2),
                         "span_ms_sum": round(sum(x["span_ms"] for x in steps), 2),
                         "steps_panel_bound": sum(1 for x in steps if x["pu_ms"] >= x["tu_ms"]),
                         "note": "traced run, no graph replay"}}
    print(json.dumps(out))
    return 0


def reference_solution(name, A0):
    """The CPU oracle's FP64 solution of configuration `name`, stored by
    tests/golden/make_reference_solutions.py, if its matrix fingerprint matches
    A0 (same generator, same bits); else (None, reason)."""
    import hashlib
    golden = os.path.join(ROOT, "tests", "golden")
    try:
        meta = json.load(open(os.path.join(golden, "reference_solutions.json")))[name]
        x = np.load(os.path.join(golden, f"x_oracle_{name}.npy"))
    except Exception:
        return None, "no stored oracle solution"
    flat = np.asfortranarray(A0).ravel(order="F")
    fp = hashlib.sha256(np.ascontiguousarray(flat[::meta["fingerprint_stride"]]).tobytes()).hexdigest()
    if fp != meta["fingerprint"]:
        return None, "matrix fingerprint differs from the stored solution's"
    return x, None


def run_configs(args):
    """The comparisons of the hot-path configurations, one JSON object:
    c1  FP64, n = 8192, nb = 256, N(0,1): look-ahead off / depth 1 / depth 1 with
        stealing / depth 2 / the runtime-task DAG schedule (factorization +
        solve, GFLOP/s of 2n^3/3);
    c2  n = 16384, nb = 256: the mixed solver with each trailing-update precision
        (N(0,1), one rhs), then bf16x6 on the row-scaled matrix and with 16 rhs;
    c3  n = 32768, nb = 256, A = diag(10^u) G: bf16x6 and e4m3 updates.
    The tensor-core variants of c2 and c3 run with the panel leaves on an SM
    partition of --pf-sms SMs, as the default bench does (FP32 and FP64 updates
    on the CUDA cores keep every SM).  For c2 (N(0,1), one rhs) and c3 each variant also reports
    ||x - x_oracle||_inf / ||x_oracle||_inf against the CPU oracle's FP64
    solution stored by tests/golden/make_reference_solutions.py.
    Each configuration runs twice untimed, then once timed with CUDA events."""
    import numpy as np
    import torch

    import paper_1804_07017_gb300 as lu
    import synth
    from paper_1804_07017_gb300.api import colmajor

    torch.cuda.set_device(0)
    out = {"metric": "LU+solve GFLOP/s (2n^3/3) per configuration", "unit": "GFLOP/s", "data": "synthetic"}

    def timed(fn):
        # two untimed runs: the second captures the factorization's launch graph
        fn()
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # c1: FP64 look-ahead comparison
    n = 8192
    A0 = synth.normal_matrix(n, seed=0)
    b0 = synth.ones_rhs(A0)
    A = colmajor(n, n)
    B = colmajor(n, 1)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    Ah = torch.from_numpy(A0).cuda()
    bh = torch.from_numpy(b0).cuda()
    c1 = {}
    for name, la, steal, rtm in (("lookahead_off", 0, 0, 0), ("lookahead_1", 1, 0, 0),
                                 ("lookahead_1_steal", 1, 1, 0), ("lookahead_2_steal", 2, 1, 0),
                                 ("rtm_task_dag", 1, 0, 1)):
        o = lu.default_opts(nb=256, lookahead=la, steal=steal, rtm=rtm)

        def run():
            A.copy_(Ah)
            B.copy_(bh)
            lu.lu_factor_ex(A, ipiv, info, o)
            lu.lu_solve_ex(A, ipiv, B)

        ms, _ = timed(run)
        c1[name] = {"ms": ms, "gflops": 2 * n ** 3 / 3 / ms / 1e6, "info": int(info.item())}
    out["c1_fp64_n8192"] = c1
    del A, B, Ah, bh

    def mixed(n, A0, B0, precs, tag, ref=None):
        A = colmajor(n, n)
        A.copy_(torch.from_numpy(A0))
        B = colmajor(n, B0.shape[1])
        B.copy_(torch.from_numpy(B0))
        X = colmajor(n, B0.shape[1])
        res = {}
        for name in precs:
            code = {"bf16": 0, "fp16": 1, "fp8": 2, "f32": 3, "bf16x3": 4, "f64": 5, "bf16x6": 6}[name]
            # the leaf partition pays off beside the fast tensor-core update; a CUDA-core
            # update (FP32, FP64) needs every SM
            pf = 0 if name in ("f32", "f64") else args.pf_sms
            ms, (st, it, eta) = timed(lambda: lu.lu_gesv_mixed(A, B, X, code, TOL, MAX_ITER,
                                                                 lu.default_opts(nb=256, pf_sms=pf)))
            res[f"{tag}{name}"] = {"ms": ms, "gflops": 2 * n ** 3 / 3 / ms / 1e6, "status": int(st),
                                   "refinements": int(it), "bwd_err": float(eta),
                                   "converged": int(st) == 0, "pf_sms": pf}
            if ref is not None:
                x_or, why = ref
                if x_or is None:
                    res[f"{tag}{name}"]["fwd_err_vs_oracle"] = None
                    res[f"{tag}{name}"]["fwd_err_note"] = why
                else:
                    x = X.cpu().numpy()
                    res[f"{tag}{name}"]["fwd_err_vs_oracle"] = float(np.abs(x - x_or).max() / np.abs(x_or).max())
        return res

    n = 16384
    A0 = synth.normal_matrix(n, seed=0)
    c2 = mixed(n, A0, synth.ones_rhs(A0), ["bf16x6", "bf16x3", "bf16", "fp16", "f32", "f64"], "",
               ref=reference_solution("c2_normal_n16384", A0))
    B16, _ = synth.random_rhs(A0, 16, seed=1)
    c2.update(mixed(n, A0, B16, ["bf16x6"], "rhs16_"))
    R0 = synth.row_scaled(A0, seed=3)
    c2.update(mixed(n, R0, synth.ones_rhs(R0), ["bf16x6"], "rowscaled_"))
    out["c2_mixed_n16384"] = c2
    del A0, R0, B16
    n = 32768
    D0 = synth.diag_scaled_normal(n, seed=0)
    out["c3_n32768_diag_scaled"] = mixed(n, D0, synth.ones_rhs(D0), ["bf16x6", "fp8"], "",
                                         ref=reference_solution("c3_diag_scaled_n32768", D0))
    print(json.dumps(out))
    return 0


def run_batched(args):
    """4096 independent systems, n_i log-uniform in [16, 512], nrhs_i in 1..8,
    iid U[-1,1): one graph-captured persistent launch (factor + solve) versus a
    per-matrix loop of plain launches (lu_factor_ex + lu_solve_ex), FP64 and FP32."""
    import numpy as np
    import torch

    import paper_1804_07017_gb300 as lu
    import synth
    from paper_1804_07017_gb300.api import colmajor

    torch.cuda.set_device(0)
    count = 4096
    sizes, nrhs = synth.batched_sizes(count, seed=0)
    mats = synth.batched_matrices(sizes, seed=0)
    g = synth.rng(0, 9)
    rhs = [g.uniform(-1, 1, size=(int(n), int(r))) for n, r in zip(sizes, nrhs)]
    flops = float(np.sum(2.0 * sizes.astype(np.float64) ** 3 / 3.0))
    out = {"metric": "batched LU+solve GFLOP/s (sum 2n^3/3)", "unit": "GFLOP/s", "workload":
           f"{count} systems, n log-uniform [16,512] (sum n^3 = {float(np.sum(sizes.astype(np.float64)**3)):.3e}), "
           f"nrhs 1..8, iid U[-1,1), seed 0", "flops": flops}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        # the batched update's tile cut-over, measured on this batch (lu_tune_batched) and
        # kept in the table, so the timed launches below use it
        cuts = [1, 33, 65, 97, 129, 193]
        best_cut, cut_ms = lu.lu_tune_batched(lu.LU_F64 if dt == torch.float64 else lu.LU_F32, sizes, nrhs, cuts,
                                              reps=3)
        out[f"tile_cutover_{name}"] = {"best": best_cut,
                                       "ms": {str(c): round(t, 3) for c, t in zip(cuts, cut_ms)},
                                       "note": "32 x 32 update tiles below the cut-over, 64 x 64 above; "
                                               "1 = always 64 x 64"}
        dA = []
        for m in mats:
            t = colmajor(m.shape[0], m.shape[1], dtype=dt)
            t.copy_(torch.from_numpy(m).to(dt))
            dA.append(t)
        pristine = [a.clone() for a in dA]
        dB = []
        for b in rhs:
            t = colmajor(b.shape[0], b.shape[1], dtype=dt)
            t.copy_(torch.from_numpy(b).to(dt))
            dB.append(t)
        pB = [b.clone() for b in dB]
        piv = [torch.zeros(int(n), dtype=torch.int32, device="cuda") for n in sizes]
        batch = lu.Batch(dA, piv, dB)

        def restore():
            for a, p in zip(dA, pristine):
                a.copy_(p)
            for b, p in zip(dB, pB):
                b.copy_(p)

        stream = torch.cuda.Stream()
        h = lu.Handle()
        with torch.cuda.stream(stream):
            h.set_stream(stream)
            lu.lu_gesv_batched(batch, handle=h)  # first call allocates the workspace
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                h.set_stream(torch.cuda.current_stream())
                lu.lu_gesv_batched(batch, handle=h)
            h.set_stream(stream)
        times = []
        for it in range(args.warmup + args.steps):
            restore()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                graph.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
        ok = bool((batch.info == 0).all().item())
        ms = statistics.median(times)
        # per-matrix plain-launch loop (same kernels of the blocked path, one matrix at a time)
        restore()
        torch.cuda.synchronize()
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for a, p, b in zip(dA, piv, dB):
            lu.lu_factor_ex(a, p, info, lu.default_opts(nb=32, lookahead=0))
            lu.lu_solve_ex(a, p, b)
        e1.record()
        torch.cuda.synchronize()
        loop_ms = e0.elapsed_time(e1)
        out[name] = {"value": flops / (ms * 1e-3) / 1e9, "ms": ms, "all_info_zero": ok,
                     "per_matrix_loop_ms": loop_ms, "per_matrix_loop_gflops": flops / (loop_ms * 1e-3) / 1e9,
                     "speedup_vs_loop": loop_ms / ms}
        h.close()
    print(json.dumps(out), flush=True)
    return 0


def fp64_path(lu, A0, B0, n, nrhs, nb):
    """FP64 look-ahead LU + solve; FP64 refinement (FP64 solves) until eta <= 1e-14."""
    import torch

    from paper_1804_07017_gb300.api import colmajor
    Ad = colmajor(n, n)
    Ad.copy_(torch.from_numpy(A0))
    Bd = colmajor(n, nrhs)
    Bd.copy_(torch.from_numpy(B0))
    X = colmajor(n, nrhs)
    status, iters, eta = None, None, None
    try:
        status, iters, eta = lu.lu_gesv_mixed(Ad, Bd, X, lu.LU_FULL_F64, TOL, MAX_ITER, lu.default_opts(nb=nb))
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        status, iters, eta = lu.lu_gesv_mixed(Ad, Bd, X, lu.LU_FULL_F64, TOL, MAX_ITER, lu.default_opts(nb=nb))
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
    except Exception as e:  # reported, not fatal for the headline
        return {"error": str(e)}
    return {"value": 2.0 * n ** 3 / 3.0 / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms, "steps": 1,
            "warmup": 1, "refinements": iters, "bwd_err": eta, "status": status,
            "what": "FP64 factorization (same look-ahead schedule, SIMT DFMA trailing update) + FP64 solve + FP64 refinement"}


if __name__ == "__main__":
    sys.exit(main())
