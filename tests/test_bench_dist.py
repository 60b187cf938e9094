"""The multi-process host logic of bench.py on CPU (gloo, world size 2): the
max-over-ranks step time, the whole-job throughput of replicas, and the
reference arm printing one line on rank 0 only.  No GPU involved."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank), "LU_BENCH_REF_BUDGET_S": "0.2"})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist)
        value = bench.job_throughput(2.0 * 64 ** 3 / 3.0, world, ms)
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.main_with_args(["--impl", "reference", "--n", "64", "--steps", "1", "--warmup", "0",
                                       "--gpus", str(world)])
        q.put((rank, ms, value, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_rank_bench_logic():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, ms, value, rc, text = q.get(timeout=180)
        out[rank] = (ms, value, rc, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the slowest rank's time (20 ms) on every rank; whole-job value over both replicas
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == pytest.approx(2 * (2.0 * 64 ** 3 / 3.0) / 0.020 / 1e9)
    # reference arm: rank 0 prints exactly one JSON line, rank 1 prints nothing
    assert out[0][2] == 0 and out[1][2] == 0
    assert out[1][3].strip() == ""
    lines = [ln for ln in out[0][3].splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
