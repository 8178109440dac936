"""GPU tests of the sharded apply (multi-GPU split of one geometry, run here as
shards one after another on one GPU): each shard writes its targets and zeros
elsewhere, and the shards' outputs sum to the whole apply bit for bit."""
import numpy as np
import pytest
import torch

from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


def _apply(plan, q, dtype):
    return plan.apply(torch.from_numpy(np.ascontiguousarray(q)).to("cuda").to(dtype)).cpu().numpy()


@pytest.mark.parametrize("kind,n,kd,order,nrhs,dtype", [
    ("sphere", 20000, 48.0, 4, 1, torch.complex64),
    ("box", 12000, 32.0, 5, 3, torch.complex64),
    ("ellipsoid", 8000, 24.0, 6, 2, torch.complex64),
    ("sphere", 6000, 20.0, 4, 2, torch.complex128),
])
def test_shards_sum_to_the_whole(kind, n, kd, order, nrhs, dtype):
    X = W.points(kind, n, 101)
    D = float(np.max(X.max(0) - X.min(0)))
    q = W.charges(n, 102, nrhs=nrhs)
    plan = defmm.Plan(X, kappa=kd / D, order=order, leaf_size=32)
    whole = _apply(plan, q, dtype)
    perm = plan.table("perm_t")
    for S in (2, 3):
        acc = np.zeros_like(whole)
        for s in range(S):
            plan.set_shard(S, s)
            part = _apply(plan, q, dtype)
            first, count = plan.shard_range(S, s)
            mine = np.zeros(n, dtype=bool)
            mine[perm[first:first + count]] = True
            assert np.all(part[~mine] == 0)                   # zeros outside the shard
            assert np.array_equal(part[mine], whole[mine])    # the shard's rows, bit for bit
            acc += part
        assert np.array_equal(acc, whole)
        assert plan.info()["device_error"] == 0
    plan.set_shard(1, 0)
    assert np.array_equal(_apply(plan, q, dtype), whole)
    # M2L blocks split by group size (two launches over per-shard lists): the same bits
    plan.set_tuning(m2l_members_per_block=12)
    assert np.array_equal(_apply(plan, q, dtype), whole)
    acc = np.zeros_like(whole)
    for s in range(3):
        plan.set_shard(3, s)
        acc += _apply(plan, q, dtype)
    assert np.array_equal(acc, whole)


def test_shard_with_host_buffers_and_more_shards_than_leaves():
    X = W.points("sphere", 300, 103)
    q = W.charges(300, 104)[:, 0]
    plan = defmm.Plan(X, kappa=5.0, order=4, leaf_size=64)
    whole = plan.apply_host(q.astype(np.complex64)).numpy()
    S = 64                                                  # more shards than leaves: some are empty
    acc = np.zeros_like(whole)
    for s in range(S):
        plan.set_shard(S, s)
        acc += plan.apply_host(q.astype(np.complex64)).numpy()
    assert np.array_equal(acc, whole)


@pytest.mark.parametrize("kind,n,order,nrhs,dtype,S", [
    ("sphere", 20000, 4, 1, torch.complex64, 2),
    ("box", 12000, 5, 3, torch.complex64, 3),
    ("sphere", 6000, 4, 2, torch.complex128, 4),
    ("sphere", 300, 4, 1, torch.complex64, 64),      # more shards than leaves: empty slices
])
def test_slices_assemble_to_the_whole(kind, n, order, nrhs, dtype, S):
    """The all-gather exchange: each shard's sorted-order slice (defmm_apply_slice),
    stacked in shard order with padding and put back in the caller's order
    (defmm_assemble_slices), equals the whole apply bit for bit; padding past a
    shard's count is left untouched."""
    X = W.points(kind, n, 105)
    D = float(np.max(X.max(0) - X.min(0)))
    q = torch.from_numpy(np.ascontiguousarray(W.charges(n, 106, nrhs=nrhs))).to("cuda").to(dtype)
    plan = defmm.Plan(X, kappa=24.0 / D, order=order, leaf_size=32)
    whole = plan.apply(q).cpu().numpy()
    perm = plan.table("perm_t")
    ranges = [plan.shard_range(S, s) for s in range(S)]
    starts = [f for f, _ in ranges] + [n]
    ld = max(c for _, c in ranges) + 3
    sentinel = complex(7.0, -7.0)
    gathered = torch.full((S, nrhs, ld), sentinel, dtype=dtype, device="cuda")
    for s in range(S):
        plan.set_shard(S, s)
        out = plan.apply_slice(q, out=gathered[s])
        first, count = ranges[s]
        got = out.cpu().numpy()
        w2 = whole.reshape(n, nrhs)
        assert np.array_equal(got[:, :count], w2[perm[first:first + count]].T)   # sorted order, same bits
        assert np.all(got[:, count:] == sentinel)                               # padding untouched
    p = plan.assemble_slices(starts, gathered).cpu().numpy()
    assert np.array_equal(p.reshape(whole.shape), whole)
    plan.set_shard(1, 0)
    one = plan.apply_slice(q).cpu().numpy()                  # unsharded: every target, sorted order
    assert np.array_equal(one, whole.reshape(n, nrhs)[perm].T)
    with pytest.raises(defmm.DefmmError):
        plan.assemble_slices([0, n - 1], gathered[:1, :, :])    # starts must end at nx
    assert plan.info()["device_error"] == 0
