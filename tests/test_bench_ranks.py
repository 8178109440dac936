"""The multi-rank paths of bench.py on CPU: world_size-2 gloo process groups.

bench.py --gpus N runs one replica of the workload per rank (one process per
GPU); the timed region is the slowest rank's, the value counts every rank's
points, and only rank 0 prints.  These tests exercise that host logic with
gloo ranks (no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 95.5][rank]            # rank 0 is the slow one here
    total = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_value(world, 1_000_000, 1, total / 10)
    dist.barrier()
    with open(out + ".%d" % rank, "w") as f:
        json.dump({"total": total, "value": value}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r")
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    res = [json.load(open(out + ".%d" % r)) for r in range(2)]
    for r in res:
        assert r["total"] == 120.0                       # the slowest rank's time, on every rank
        assert abs(r["value"] - 2 * 1e6 / 12e-3 / 1e6) < 1e-9   # both replicas' points / (120 ms / 10 steps)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5               # one process: identity


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
