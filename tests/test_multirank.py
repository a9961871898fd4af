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


def _bench(args, env_extra, timeout):
    import subprocess
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_runs_on_rank_zero_only():
    """--impl reference under torchrun: ranks other than 0 exit 0 without work or output."""
    r = _bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
               {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, 60)
    assert r.returncode == 0 and r.stdout == ""


def test_reference_arm_json_line():
    """Rank 0 prints one JSON line carrying the contract's keys, with the oracle as the arm."""
    import json
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "0", "WORLD_SIZE": "1"}, 600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
