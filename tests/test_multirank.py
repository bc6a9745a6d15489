"""Replica path of the benchmark on CPU: two gloo ranks, the max-over-ranks
timing and the whole-job rate (each rank solves independently; the only
collectives are the barrier and this reduction)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 + 37.0 * rank
    mx = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
    rate = bench.job_rate(10, world, mx)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(f"{mx} {rate}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_rate(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    vals = [tuple(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(world)]
    for mx, rate in vals:
        assert mx == 137.0                       # the slowest rank's time on every rank
        assert abs(rate - world * 10 / 0.137) < 1e-9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_rate(4, 1, 500.0) == 8.0


def test_reference_arm_runs_on_rank0_only(tmp_path):
    """Under torchrun the reference arm's other ranks exit without work."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""
