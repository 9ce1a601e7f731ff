"""The N>1 path of the benchmark on CPU: two gloo ranks, one independent
system each (replicas, no data-path collective).  Checks that the job's time
is the slowest rank's, that the whole-job throughput counts every replica, and
that the reference arm runs on rank 0 only."""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, per_rank_ms, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        worst = bench.max_over_ranks(per_rank_ms[rank], world, device="cpu")
        value = bench.job_ns_per_day(worst, world, 1.0)
        dist.barrier()
        out_q.put((rank, worst, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    per_rank_ms = [0.61, 0.74]       # ms per step of each rank's replica
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, per_rank_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench

    for rank, worst, value in results:
        assert worst == pytest.approx(0.74)
        # 2 replicas of 1 fs each per 0.74 ms
        assert value == pytest.approx(2 * 86400.0 / 0.74e-3 * 1e-6)
        assert value == pytest.approx(2 * bench.ns_per_day(0.74e-3, 1.0))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_ns_per_day(1.0, 1, 1.0) == pytest.approx(86.4)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
