"""The multi-process path of bench.py on the CPU (gloo, world size 2): each rank times its own
replica instance (no data-path collective), and the job's time is the maximum over ranks."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + rank, dist, device="cpu")
        p = bench.rank_workload(20, rank)
        out.put((rank, t, p["seed"], p["m"], p["n"]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_own_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [11.0, 11.0]          # both ranks see the slowest rank's time
    assert got[0][2] != got[1][2]                        # distinct replica instances
    assert got[0][3:] == got[1][3:] == (2 ** 21, 2 ** 20)  # of the same recipe


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
