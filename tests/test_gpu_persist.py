"""GPU tests of plan files: a plan read back from a file applies the operator
bit for bit as the plan that wrote it (one tree, two trees, a union of
geometries), in both precisions."""
import numpy as np
import pytest
import torch

from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("two_trees,dtype", [(False, torch.complex64), (True, torch.complex64),
                                             (False, torch.complex128)])
def test_loaded_plan_applies_bitwise(tmp_path, two_trees, dtype):
    X = W.points("sphere", 20000, 151)
    Y = 0.9 * W.points("box", 15000, 152) if two_trees else None
    pl = defmm.Plan(X, Y, kappa=40.0, order=4, leaf_size=48)
    pl.save(tmp_path / "p.plan")
    back = defmm.Plan.load(tmp_path / "p.plan")
    q = torch.from_numpy(W.charges(pl.ny, 153, nrhs=2)).to("cuda").to(dtype)
    assert np.array_equal(pl.apply(q).cpu().numpy(), back.apply(q).cpu().numpy())
    assert back.info()["device_error"] == 0


def test_loaded_union_plan_applies_bitwise(tmp_path):
    geos = [W.points("sphere", 5000, 161), 0.7 * W.points("box", 7000, 162)]
    uni = defmm.union_plan(geos, [30.0, 12.0], order=5, leaf_size=32, damping=1.0)
    uni.save(tmp_path / "u.plan")
    back = defmm.Plan.load(tmp_path / "u.plan")
    q = torch.from_numpy(W.charges(uni.nx, 163)[:, 0]).to("cuda").to(torch.complex64)
    assert np.array_equal(uni.apply(q).cpu().numpy(), back.apply(q).cpu().numpy())
