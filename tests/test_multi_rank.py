"""The benchmark's N > 1 path on the CPU: world-size-2 process groups over
gloo. Each rank solves its own scan (replicas, no data-path collective); the
only exchange is the max-reduction of the timings, and rank 0 alone prints."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from paper_1601_08201_gb300 import synth
        seed = bench.replica_seed("tiny_16x16x32", rank)
        P = synth.preset("tiny_16x16x32", seed=seed)
        my_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(my_ms, ws, "cpu")
        rate = bench.whole_job_rate(ws, 10, ms)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"seed": seed, "ms": ms, "rate": rate, "y_sum": float(np.sum(P.y))}, fh)
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_the_slowest_time_over_gloo(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(ws)]
    assert r[0]["ms"] == r[1]["ms"] == 150.0  # every rank sees the slowest rank's time
    assert r[0]["rate"] == pytest.approx(2 * 10 / 0.150)  # whole-job iterations per second
    assert r[0]["seed"] != r[1]["seed"] and r[0]["y_sum"] != r[1]["y_sum"]  # independent scans


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(1, 100, 50.0) == pytest.approx(2000.0)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "tiny_16x16x32", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
