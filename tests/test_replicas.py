"""The multi-process path of bench.py (replicas only): barrier, slowest-replica time and the
whole-job throughput, as two gloo ranks on the CPU; and the reference arm's non-zero ranks."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        import bench
        bench.rank_barrier()
        slowest = bench.max_over_ranks(1.5 + rank)          # rank r "took" 1.5 + r seconds
        q.put((rank, slowest, bench.job_throughput(world, 4, slowest)))
        bench.rank_barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    assert [r[1] for r in res] == [2.5, 2.5]                 # max over ranks, on every rank
    assert [r[2] for r in res] == [2 * 4 / 2.5] * 2          # both replicas' solves in the slowest time


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    bench.rank_barrier()
    assert bench.job_throughput(1, 5, 2.0) == 2.5


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
