"""Pins of the oracle's direct sum (Eq. 1.1) against closed forms and invariants."""
import numpy as np
import pytest

from oracle import direct
from paper_2202_04894_gb300 import workloads as W


def _sphere_quadrature(nt, nphi, radius):
    """Gauss-Legendre in cos(theta) x trapezoid in phi; weights sum to 1."""
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    pts = radius * np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    wts = (np.repeat(w, nphi) / 2.0 / nphi)
    return pts, wts


@pytest.mark.parametrize("kappa", [0.0, 1.3, 4.0])
def test_shell_mean_value(kappa):
    """Mean of G over a sphere of radius a seen from distance R > a:
    sin(kappa a)/(kappa a) * exp(i kappa R)/(4 pi R)  (spherical mean value
    of outgoing Helmholtz waves)."""
    a, R = 0.5, 1.7
    Y, w = _sphere_quadrature(48, 96, a)
    x = np.array([[0.3 * R, -0.4 * R, np.sqrt(1 - 0.25) * R]])
    got = direct.direct_sum(x, Y, w, kappa, 1e-12)[0]
    j0 = 1.0 if kappa == 0 else np.sin(kappa * a) / (kappa * a)
    want = j0 * np.exp(1j * kappa * R) / (4 * np.pi * R)
    assert abs(got - want) <= 1e-12 * abs(want)


def test_unit_sphere_to_centre():
    """Charges 1/N on the unit sphere, target at the origin: exp(i kappa)/(4 pi)."""
    Y = W.sphere(777, 3)
    q = np.full(len(Y), 1.0 / len(Y))
    for kappa in (0.7, 5.0):
        got = direct.direct_sum(np.zeros((1, 3)), Y, q, kappa, 1e-12)[0]
        assert abs(got - np.exp(1j * kappa) / (4 * np.pi)) < 1e-14


def test_single_charge_translation_and_self_mask():
    X = W.sphere(50, 4)
    q = np.zeros(50, dtype=complex)
    q[7] = 2.0 - 1.0j
    p = direct.direct_sum(X, X, q, 3.0, 1e-10)
    assert p[7] == 0                       # self interaction removed
    r = np.linalg.norm(X[11] - X[7])
    assert abs(p[11] - (2 - 1j) * np.exp(3j * r) / (4 * np.pi * r)) < 1e-15 * abs(p[11]) * 10


def test_reciprocity():
    """G(x,y) = G(y,x): r^T (A q) = q^T (A r)."""
    X = W.points("box", 300, 5)
    q = W.charges(300, 5)[:, 0]
    r = W.charges(300, 6)[:, 0]
    A_q = direct.direct_sum(X, X, q, 7.0, 1e-10)
    A_r = direct.direct_sum(X, X, r, 7.0, 1e-10)
    assert abs(r @ A_q - q @ A_r) < 1e-13 * abs(r @ A_q)


def test_c_direct_matches_numpy():
    X = W.points("ellipsoid", 400, 8)
    q = W.charges(400, 8, nrhs=3)
    tg = np.array([0, 5, 399, 123])
    a = direct.direct_sum(X, X, q, 5.0, 1e-10, targets=tg)
    b = direct.direct_sum_c(X, X, q, 5.0, 1e-10, targets=tg)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
    Y, w = _sphere_quadrature(40, 80, 0.5)
    got = direct.direct_sum_c(np.array([[0, 0, 1.5]]), Y, w, 2.0, 1e-12)[0]
    want = np.sin(1.0) / 1.0 * np.exp(3j) / (4 * np.pi * 1.5)
    assert abs(got - want) < 1e-12 * abs(want)


@pytest.mark.parametrize("kappa,damping", [(0.0, 2.0), (3.0, 1.5), (0.0, 0.0)])
def test_shell_mean_value_damped(kappa, damping):
    """The damped kernel is the Helmholtz kernel of the complex wavenumber
    k = kappa + i*damping, so the spherical mean value over a sphere of radius a
    seen from R > a is sin(k a)/(k a) * exp(i k R)/(4 pi R); for kappa = 0 that
    is sinh(damping a)/(damping a) * exp(-damping R)/(4 pi R) (Yukawa)."""
    a, R = 0.5, 1.7
    Y, w = _sphere_quadrature(48, 96, a)
    x = np.array([[0.3 * R, -0.4 * R, np.sqrt(1 - 0.25) * R]])
    got = direct.direct_sum(x, Y, w, kappa, 1e-12, damping=damping)[0]
    k = kappa + 1j * damping
    j0 = 1.0 if k == 0 else np.sin(k * a) / (k * a)
    want = j0 * np.exp(1j * k * R) / (4 * np.pi * R)
    assert abs(got - want) <= 1e-12 * abs(want)
    if kappa == 0 and damping > 0:
        yukawa = np.sinh(damping * a) / (damping * a) * np.exp(-damping * R) / (4 * np.pi * R)
        assert abs(got - yukawa) <= 1e-12 * yukawa


def test_c_direct_matches_numpy_damped():
    X = W.points("box", 300, 9)
    q = W.charges(300, 9, nrhs=2)
    tg = np.array([3, 77, 299])
    a = direct.direct_sum(X, X, q, 4.0, 1e-10, targets=tg, damping=2.5)
    b = direct.direct_sum_c(X, X, q, 4.0, 1e-10, targets=tg, damping=2.5)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("kappa", [0.0, 2.5, 7.0])
def test_shell_mean_value_power_two(kappa):
    """Radial power 2: with r^2 = R^2 + a^2 - 2aR cos(theta) the spherical mean of
    exp(i kappa r)/(4 pi r^2) over a sphere of radius a seen from R > a is
    (1/(8 pi a R)) * integral_{R-a}^{R+a} exp(i kappa r)/r dr
    = [Ci(kappa r) + i Si(kappa r)]_{R-a}^{R+a} / (8 pi a R), and ln((R+a)/(R-a))/(8 pi a R)
    at kappa = 0."""
    sici = pytest.importorskip("scipy.special").sici
    a, R = 0.5, 1.7
    Y, w = _sphere_quadrature(64, 128, a)
    x = np.array([[0.3 * R, -0.4 * R, np.sqrt(1 - 0.25) * R]])
    got = direct.direct_sum(x, Y, w, kappa, 1e-12, power=2)[0]
    if kappa == 0:
        want = np.log((R + a) / (R - a)) / (8 * np.pi * a * R)
    else:
        (s1, c1), (s0, c0) = sici(kappa * (R + a)), sici(kappa * (R - a))
        want = ((c1 - c0) + 1j * (s1 - s0)) / (8 * np.pi * a * R)
    assert abs(got - want) <= 1e-12 * abs(want)
    # a different kernel: the power-1 mean differs
    assert abs(direct.direct_sum(x, Y, w, kappa, 1e-12)[0] - want) > 1e-3 * abs(want)


def test_c_direct_matches_numpy_power_two():
    X = W.points("box", 300, 9)
    q = W.charges(300, 9, nrhs=2)
    tg = np.array([3, 77, 299])
    a = direct.direct_sum(X, X, q, 4.0, 1e-10, targets=tg, damping=1.5, power=2)
    b = direct.direct_sum_c(X, X, q, 4.0, 1e-10, targets=tg, damping=1.5, power=2)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
