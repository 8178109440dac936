"""GPU tests of union plans (several geometries in one plan, one launch per
phase): each geometry's block of the union apply equals its own plan's apply
bit for bit, in both precisions, for one and several right-hand sides."""
import numpy as np
import pytest
import torch

from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


def _geos():
    g = [W.points("sphere", 6000, 121), 0.8 * W.points("box", 9000, 122), W.points("ellipsoid", 3000, 123),
         W.points("sphere", 400, 124) + 3.0]
    kd = [60.0, 24.0, 90.0, 8.0]
    return g, [k / float(np.max(X.max(0) - X.min(0))) for X, k in zip(g, kd)]


@pytest.mark.parametrize("order,nrhs,dtype", [(4, 1, torch.complex64), (4, 3, torch.complex64),
                                              (5, 2, torch.complex64), (4, 2, torch.complex128)])
def test_union_equals_individual_plans(order, nrhs, dtype):
    geos, kappas = _geos()
    uni = defmm.union_plan(geos, kappas, order=order, leaf_size=32)
    q = [W.charges(len(X), 130 + i, nrhs=nrhs) for i, X in enumerate(geos)]
    qu = torch.from_numpy(np.concatenate(q, axis=0)).to("cuda").to(dtype)
    pu = uni.apply(qu).cpu().numpy()
    off = 0
    for X, k, qi in zip(geos, kappas, q):
        single = defmm.Plan(X, kappa=k, order=order, leaf_size=32)
        ps = single.apply(torch.from_numpy(qi).to("cuda").to(dtype)).cpu().numpy()
        assert np.array_equal(pu[off:off + len(X)], ps)
        off += len(X)
    assert uni.info()["device_error"] == 0


def test_union_with_damping_and_shards():
    geos, kappas = _geos()
    uni = defmm.union_plan(geos, kappas, order=4, leaf_size=32, damping=2.0)
    q = torch.from_numpy(np.concatenate([W.charges(len(X), 140 + i) for i, X in enumerate(geos)])[:, 0]).to("cuda")
    whole = uni.apply(q.to(torch.complex64)).cpu().numpy()
    acc = np.zeros_like(whole)
    for s in range(3):
        uni.set_shard(3, s)
        acc += uni.apply(q.to(torch.complex64)).cpu().numpy()
    assert np.array_equal(acc, whole)
    off = 0
    for i, (X, k) in enumerate(zip(geos, kappas)):
        single = defmm.Plan(X, kappa=k, order=4, leaf_size=32, damping=2.0)
        ps = single.apply(q[off:off + len(X)].to(torch.complex64)).cpu().numpy()
        assert np.array_equal(whole[off:off + len(X)], ps)
        off += len(X)


def test_union_in_a_captured_graph():
    """A union plan in a graph batch: one captured CUDA graph replays the whole
    multi-geometry apply (the fused launches), bit for bit the plain apply."""
    from paper_2202_04894_gb300 import serve
    geos, kappas = _geos()
    uni = defmm.union_plan(geos, kappas, order=4, leaf_size=32)
    q = np.concatenate([W.charges(len(X), 150 + i, nrhs=2) for i, X in enumerate(geos)])
    qd = torch.from_numpy(q).to("cuda").to(torch.complex64)
    direct = uni.apply(qd).cpu().numpy()
    b = serve.Batch([uni], [2], torch.complex64)
    b.inputs()[0].copy_(qd.t())
    for _ in range(2):
        b.run()
        torch.cuda.synchronize()
        assert np.array_equal(b.outputs()[0].t().cpu().numpy(), direct)
    assert b.info()["kernel_launches"] > 0
