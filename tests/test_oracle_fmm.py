"""Pins of the oracle's full FMM apply against the direct sum and invariants."""
import numpy as np
import pytest

from oracle import direct, fmm
from paper_2202_04894_gb300 import workloads as W


def _case(kind, n, kd, seed=5, nrhs=1):
    X = W.points(kind, n, seed)
    kappa = kd / float(np.max(X.max(0) - X.min(0)))
    return X, W.charges(n, seed, nrhs), kappa


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_all_p2p_equals_direct_sum():
    """Every MAC false: the FMM reduces to the direct sum."""
    X, q, kappa = _case("box", 900, 20.0)
    plan = fmm.make_plan(X, kappa=kappa, order=4, leaf=30, force_p2p=True)
    assert len(plan.m2l_pairs) == 0
    got = fmm.apply(plan, X, q)
    want = direct.direct_sum(X, X, q, kappa, plan.eps_self)
    assert _rel(got, want) < 1e-14


def test_sphere2k_accuracy_and_geometric_convergence():
    """Sec. 3 / Sec. 6.1: error decreases geometrically with the order."""
    X, q, kappa, order, leaf, _ = W.make("sphere2k_kD8_p4")
    want = direct.direct_sum(X, X, q, kappa, direct.eps_self(X))
    errs = []
    for p in range(2, 8):
        errs.append(_rel(fmm.fmm(X, q, kappa, order=p, leaf=leaf), want))
    assert errs[2] < 1e-3                                      # order 4 on this case
    for a, b in zip(errs, errs[1:]):
        assert b < a / 4
    assert errs[-1] < 1e-6


def test_operator_symmetry():
    """With u(-k) = -u(k) the approximate operator stays symmetric: r^T A q = q^T A r."""
    X, _, kappa = _case("ellipsoid", 2500, 24.0)
    plan = fmm.make_plan(X, kappa=kappa, order=4, leaf=24)
    assert plan.levels.l_hf >= 1 and len(plan.m2l_pairs) > 100
    q = W.charges(2500, 1)[:, 0]
    r = W.charges(2500, 2)[:, 0]
    a = r @ fmm.apply(plan, X, q)
    b = q @ fmm.apply(plan, X, r)
    assert abs(a - b) < 1e-12 * abs(a)


def test_dense_and_explicit_m2l_variants_agree():
    X, q, kappa = _case("sphere", 1500, 12.0, nrhs=2)
    base = fmm.fmm(X, q, kappa, order=3, leaf=20)
    dense = fmm.fmm(X, q, kappa, order=3, leaf=20, dense_m2l=True)
    expl = fmm.fmm(X, q, kappa, order=3, leaf=20, explicit_spectra=True)
    bigN = fmm.fmm(X, q, kappa, order=3, leaf=20, fft_n=8)
    for other in (dense, expl, bigN):
        assert _rel(other, base) < 1e-13


def test_two_trees_and_low_frequency():
    X, _, _ = _case("sphere", 1200, 1.0)
    Y = W.points("box", 1500, 7) * 0.8
    q = W.charges(1500, 7)[:, 0]
    for kappa in (0.0, 9.0):
        plan = fmm.make_plan(X, Y, kappa=kappa, order=5, leaf=25)
        got = fmm.apply(plan, X, q, Y)
        want = direct.direct_sum(X, Y, q, kappa, plan.eps_self)
        assert _rel(got, want) < 2e-4
        assert plan.tt is not plan.ts


@pytest.mark.parametrize("kd,damping_d", [(0.0, 8.0), (16.0, 4.0)])
def test_damped_kernel_against_direct_sum(kd, damping_d):
    """Yukawa (kappa = 0) and damped Helmholtz: the FMM with the damped kernel
    converges to the direct sum with it (order 5 below 1e-4, order 3 above)."""
    X = W.points("sphere", 1500, 12)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa, lam = kd / D, damping_d / D
    q = W.charges(1500, 13)[:, 0]
    want = direct.direct_sum(X, X, q, kappa, direct.eps_self(X), damping=lam)
    e3 = _rel(fmm.fmm(X, q, kappa, order=3, leaf=20, damping=lam), want)
    e5 = _rel(fmm.fmm(X, q, kappa, order=5, leaf=20, damping=lam), want)
    assert e5 < 1e-4 and e5 < e3 / 5
    # the damping changes the result (the kernel is really used everywhere)
    undamped = direct.direct_sum(X, X, q, kappa, direct.eps_self(X))
    assert _rel(undamped, want) > 0.1


@pytest.mark.parametrize("kd", [0.0, 16.0])
def test_power_two_kernel_against_direct_sum(kd):
    """exp(i kappa r)/(4 pi r^2), a kernel outside the Helmholtz family: the FMM
    with it converges to the direct sum with it, and it is really used (the
    power-1 sum differs)."""
    X = W.points("sphere", 1500, 12)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa = kd / D
    q = W.charges(1500, 13)[:, 0]
    want = direct.direct_sum(X, X, q, kappa, direct.eps_self(X), power=2)
    e3 = _rel(fmm.fmm(X, q, kappa, order=3, leaf=20, power=2), want)
    e5 = _rel(fmm.fmm(X, q, kappa, order=5, leaf=20, power=2), want)
    assert e5 < 1e-4 and e5 < e3 / 5
    assert _rel(direct.direct_sum(X, X, q, kappa, direct.eps_self(X)), want) > 0.1
