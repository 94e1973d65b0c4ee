"""The multi-process side of bench.py on the CPU (world_size 2, gloo backend).

The hot path does not shard: under torchrun every rank runs an independent replica of
the workload on its own GPU, and the only collectives are the barrier around the timed
region and the all-reduce MAX of the step time.  These tests run that host logic with
two gloo ranks: every rank gets the slowest rank's time, the whole-job value counts the
work of all replicas over that time, and the reference arm does its work on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t_max = bench.max_over_ranks(times[rank], world, "cpu")
        value = bench.job_value(1.0e12, world, t_max)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"t_max": t_max, "value": value}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo(tmp_path):
    import torch.multiprocessing as mp
    times = [0.25, 0.5]
    mp.spawn(_rank_main, args=(2, _free_port(), times, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["t_max"] == 0.5
        # two replicas of 1 TFLOP each in the slowest rank's 0.5 s
        assert g["value"] == pytest.approx(4.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.125, 1, "cpu") == 0.125
    assert bench.job_value(2.0e12, 1, 0.5) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints its line on rank 0; other ranks exit 0
    without work or output."""
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
            "--workload", "corr4-small", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    env1 = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r1 = subprocess.run(base, env=env1, capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    env0 = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r0 = subprocess.run(base, env=env0, capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0, r0.stderr
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
