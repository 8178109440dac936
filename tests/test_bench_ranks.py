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


def _shard_worker(rank, world, port, out, full_sorted, starts):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    R = full_sorted.shape[0]
    ld = max(starts[s + 1] - starts[s] for s in range(world))
    mine = np.zeros((R, ld), dtype=full_sorted.dtype)      # a shard's slice: its sorted targets, padded to ld
    mine[:, :starts[rank + 1] - starts[rank]] = full_sorted[:, starts[rank]:starts[rank + 1]]
    gathered = torch.zeros((world, R, ld), dtype=torch.complex64)
    bench.gather_slices(torch.from_numpy(mine), gathered, dist)
    np.save(out + ".%d.npy" % rank, gathered.numpy())
    dist.destroy_process_group()


def test_sharded_exchange_with_gloo(tmp_path):
    """The exchange of the sharded apply: every rank holds its shard's potentials in
    sorted order (a slice padded to the longest shard); after the all-gather every rank
    holds every slice, and putting them back in the caller's order (the permutation
    defmm_assemble_slices applies) gives the whole result, bit for bit."""
    import numpy as np
    import torch.multiprocessing as mp
    from paper_2202_04894_gb300 import defmm, workloads as W
    X = W.points("sphere", 2000, 91)
    pl = defmm.Plan(X, kappa=10.0, order=4, leaf_size=24, flags=defmm.PLAN_HOST_ONLY)
    ranges = [pl.shard_range(2, s) for s in range(2)]
    starts = [f for f, _ in ranges] + [2000]
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and sum(n for _, n in ranges) == 2000
    perm = pl.table("perm_t")                         # sorted target j -> caller's index
    rng = np.random.default_rng(3)
    full = (rng.standard_normal((3, 2000)) + 1j * rng.standard_normal((3, 2000))).astype(np.complex64)
    full_sorted = full[:, perm]
    out = str(tmp_path / "s")
    port = 31500 + (os.getpid() % 2000)
    mp.spawn(_shard_worker, args=(2, port, out, full_sorted, starts), nprocs=2, join=True)
    for r in range(2):
        g = np.load(out + ".%d.npy" % r)
        p = np.zeros_like(full)
        for s in range(2):
            n = starts[s + 1] - starts[s]
            p[:, perm[starts[s]:starts[s + 1]]] = g[s, :, :n]
        assert np.array_equal(p, full)
