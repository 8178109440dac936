"""GPU tests of defmm_gmres: restarted GMRES for (sigma I + A) x = b with every
product a defmm_apply.  The solution is checked against its own residual (the
operator applied again) and against a dense solve with the exact kernel
matrix, which it matches to the FMM's approximation error."""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


def _dense(X, kappa):
    d = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2)
    eps = direct.eps_self(X)
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.where(d > eps, np.exp(1j * kappa * d) / (4 * np.pi * d), 0.0)
    return G


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-10), (torch.complex64, 1e-5)])
def test_gmres_shifted_single_layer(dtype, tol):
    n = 2000
    X = W.points("sphere", n, 51)
    kappa = 6.0
    sigma = 20.0 + 10.0j          # the operator's eigenvalues spread over about [-44, 44]
    plan = defmm.Plan(X, kappa=kappa, order=6, leaf_size=32)
    b = torch.from_numpy(W.charges(n, 52)[:, 0]).to("cuda").to(dtype)
    x, info = plan.gmres(b, shift=sigma, tol=tol, restart=20, max_iter=300)
    assert info["converged"] == 1, info
    assert 0 < info["iterations"] <= 300
    # residual from a fresh apply
    Ax = plan.apply(x)
    r = b - (sigma * x + Ax)
    rel = float(torch.linalg.norm(r.to(torch.complex128)) / torch.linalg.norm(b.to(torch.complex128)))
    assert rel <= 3 * tol, rel
    assert abs(rel - info["rel_residual"]) <= 3 * tol
    # dense solve with the exact kernel: differs by the FMM approximation error
    G = _dense(X, kappa)
    xd = np.linalg.solve(sigma * np.eye(n) + G, b.cpu().numpy().astype(np.complex128))
    err = np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd)
    assert err <= 1e-3, err


def test_gmres_zero_rhs_and_iteration_cap():
    X = W.points("box", 1500, 53)
    plan = defmm.Plan(X, kappa=3.0, order=4, leaf_size=24)
    zero = torch.zeros(1500, dtype=torch.complex128, device="cuda")
    x, info = plan.gmres(zero, x0=torch.ones_like(zero))
    assert info["converged"] == 1 and info["iterations"] == 0
    assert torch.count_nonzero(x).item() == 0
    b = torch.from_numpy(W.charges(1500, 54)[:, 0]).to("cuda")
    x, info = plan.gmres(b, shift=0.01, tol=1e-14, restart=5, max_iter=7)
    assert info["iterations"] == 7 and info["converged"] == 0 and info["rel_residual"] < 1.0


def test_gmres_refuses_a_sharded_plan():
    X = W.points("sphere", 800, 55)
    plan = defmm.Plan(X, kappa=2.0, order=4, leaf_size=32)
    plan.set_shard(2, 1)
    b = torch.ones(800, dtype=torch.complex64, device="cuda")
    with pytest.raises(defmm.DefmmError) as e:
        plan.gmres(b)
    assert e.value.status == 5
    plan.set_shard(1, 0)
    _, info = plan.gmres(b, shift=20.0, tol=1e-4)
    assert info["converged"] == 1
