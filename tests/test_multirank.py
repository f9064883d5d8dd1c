"""The multi-rank host logic of bench.py, on CPU with two gloo ranks.

With N GPUs the bench runs N replicas: every rank merges its own burst and no data moves
between ranks (the method has no exchange step).  What ties the ranks together is the
timing: a step of the whole job lasts as long as its slowest rank, and the job's
throughput counts every rank's burst.  The reference arm (the CPU oracle) runs on rank 0
only; the other ranks exit at once.
"""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, step_ms, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench as b

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = b.max_over_ranks(step_ms[rank], world)
        queue.put((rank, ms, b.whole_job_mps(97.5, world, ms), b.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def _run_ranks(world: int, step_ms):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, step_ms, queue)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        out = sorted(queue.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    return out


def test_two_ranks_time_the_slowest_and_count_both_bursts():
    out = _run_ranks(2, [3.0, 5.0])
    assert [ms for _, ms, _, _ in out] == [5.0, 5.0]  # both ranks report the slowest step
    for _, _, value, _ in out:
        assert value == pytest.approx(2 * 97.5 / 5e-3)  # two bursts per 5 ms step
    assert out[0][3] != out[1][3]  # each rank merges its own burst


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(4.25, 1) == 4.25
    assert bench.whole_job_mps(97.5, 1, 2.0) == pytest.approx(97.5 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only():
    env = {**os.environ, "RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
