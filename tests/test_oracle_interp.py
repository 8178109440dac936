"""Pins of the oracle's interpolation operators (Sec. 2.2, 2.3, 5.2)."""
import numpy as np
import pytest

from oracle import interp
from oracle.directions import directions

RNG = np.random.default_rng(99)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_lagrange_cardinal_partition_and_reproduction(p):
    t = RNG.random(50)
    L = interp.lagrange(p, t)
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(interp.lagrange(p, interp.nodes1d(p)), np.eye(p), atol=1e-14)
    for deg in range(p):
        coef = RNG.standard_normal(deg + 1)
        f = lambda x: np.polyval(coef, x)
        assert np.allclose(L @ f(interp.nodes1d(p)), f(t), atol=1e-12)
    xh = RNG.random((20, 3))
    Sv = interp.S(p, xh)
    mi = interp.multi_index(p) / (p - 1)
    poly = lambda y: (1 + y[..., 0] - 2 * y[..., 1] * y[..., 0]) * (0.5 + y[..., 2])
    assert np.allclose(Sv @ poly(mi), poly(xh), atol=1e-12)


def _parent_child(p):
    corner, side = np.array([0.2, -0.1, 0.4]), 0.5
    octant = 5
    bits = np.array([(octant >> a) & 1 for a in range(3)])
    child = corner + bits * side / 2
    return corner, side, child, octant


@pytest.mark.parametrize("p", [3, 4, 5])
def test_lf_m2m_and_l2l_are_exact(p):
    """Non-directional M2M o P2M(son) == P2M(father); L2P(son) o L2L == L2P(father)."""
    corner, side, child, _ = _parent_child(p)
    Y = child + RNG.random((30, 3)) * side / 2
    q = RNG.standard_normal((30, 2)) + 1j * RNG.standard_normal((30, 2))
    Mc = interp.p2m(0.0, p, child, side / 2, Y, q, None)
    T = interp.m2m_matrix(0.0, p, corner, side, child, None)
    Mp = interp.p2m(0.0, p, corner, side, Y, q, None)
    assert np.max(np.abs(T @ Mc - Mp)) <= 1e-12 * np.max(np.abs(Mp))
    L = RNG.standard_normal((p ** 3, 1)) + 0j
    U = interp.l2l_matrix(0.0, p, corner, side, child, None)
    a = interp.l2p(0.0, p, child, side / 2, Y, U @ L, None)
    b = interp.l2p(0.0, p, corner, side, Y, L, None)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("p", [3, 4])
def test_directional_m2m_exact_for_same_direction(p):
    """With the son expanded in the father's own direction v the plane-wave
    factors cancel: M2M^v o P2M^v(son) == P2M^v(father) exactly.  Pins the
    signs of both exponentials and the L2L transpose."""
    kappa = 30.0
    corner, side, child, _ = _parent_child(p)
    v = directions(1)[7]
    Y = child + RNG.random((25, 3)) * side / 2
    q = RNG.standard_normal((25, 1)) + 0j
    Mc = interp.p2m(kappa, p, child, side / 2, Y, q, v)
    T = interp.m2m_matrix(kappa, p, corner, side, child, v)
    Mp = interp.p2m(kappa, p, corner, side, Y, q, v)
    assert np.max(np.abs(T @ Mc - Mp)) <= 1e-11 * np.max(np.abs(Mp))
    L = RNG.standard_normal((p ** 3, 1)) + 1j
    U = interp.l2l_matrix(kappa, p, corner, side, child, v)
    a = interp.l2p(kappa, p, child, side / 2, Y, U @ L, v)
    b = interp.l2p(kappa, p, corner, side, Y, L, v)
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b))
    # L2L(v) is the transpose of M2M(-v) on the same geometry
    assert np.allclose(interp.l2l_matrix(kappa, p, corner, side, child, -v),
                       T.T, atol=1e-14)


@pytest.mark.parametrize("p", [3, 4, 5])
def test_tensorised_equals_dense(p):
    """Sec. 5.2: D0 (x)M^(p) D1 (t), stacked over directions (t+s), real split (t+s+r)."""
    kappa = 12.0
    corner, side, child, octant = _parent_child(p)
    us = [directions(1)[i] for i in (0, 5, 13, 22)]
    V = RNG.standard_normal((p ** 3, len(us))) + 1j * RNG.standard_normal((p ** 3, len(us)))
    dense = np.stack([interp.m2m_matrix(kappa, p, corner, side, child, u) @ V[:, j]
                      for j, u in enumerate(us)], axis=1)
    for real in (False, True):
        t = interp.tensorised_m2m(kappa, p, corner, side, child, octant, us, V, real_split=real)
        assert np.max(np.abs(t - dense)) <= 1e-13 * np.max(np.abs(dense))
