"""Pins of the oracle's Fourier-domain M2L (Sec. 2.3) and symmetries (Sec. 4.3)."""
import itertools

import numpy as np
import pytest

from oracle import m2l

RNG = np.random.default_rng(1234)


def _rand(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7])
def test_fft_m2l_equals_dense(p):
    """chi^T F^-1 diag(F g_k) F chi == the dense matrix sum_b G(x_a - y_b)."""
    kappa, side = 9.0, 0.25
    N = 2 * p - 1
    for k in [(2, 0, 0), (3, -1, 2), (-4, 4, 1), (0, -2, 5)]:
        M = _rand((p ** 3, 2))
        dense = m2l.dense_m2l(kappa, side, p, k, M)
        g = m2l.spectrum(kappa, side, p, N, k)
        fft = m2l.f2l(g[None] * m2l.m2f(M, p, N), p)
        assert np.max(np.abs(fft - dense)) <= 1e-13 * np.max(np.abs(dense))


@pytest.mark.parametrize("kappa,damping,power", [(0.0, 6.0, 1), (9.0, 3.0, 1), (0.0, 0.0, 2), (9.0, 3.0, 2)])
def test_fft_m2l_equals_dense_damped(kappa, damping, power):
    """The same identity for the damped kernel (Yukawa; damped Helmholtz) and the
    radial power 2 kernel exp((i kappa - lambda) r) / (4 pi r^2)."""
    side, p = 0.25, 4
    N = 2 * p - 1
    for k in [(2, 0, 0), (3, -1, 2), (-4, 4, 1)]:
        M = _rand((p ** 3, 2))
        dense = m2l.dense_m2l(kappa, side, p, k, M, damping, power)
        g = m2l.spectrum(kappa, side, p, N, k, damping, power)
        fft = m2l.f2l(g[None] * m2l.m2f(M, p, N), p)
        assert np.max(np.abs(fft - dense)) <= 1e-13 * np.max(np.abs(dense))


@pytest.mark.parametrize("p,extra", [(3, 1), (4, 1), (4, 3), (5, 2)])
def test_fft_length_does_not_matter(p, extra):
    kappa, side, k = 3.0, 0.5, (1, -3, 2)
    M = _rand((p ** 3, 1))
    outs = []
    for N in (2 * p - 1, 2 * p - 1 + extra):
        g = m2l.spectrum(kappa, side, p, N, k)
        outs.append(m2l.f2l(g[None] * m2l.m2f(M, p, N), p))
    assert np.max(np.abs(outs[0] - outs[1])) <= 1e-13 * np.max(np.abs(outs[0]))


def _signed_permutations():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            yield perm, signs


@pytest.mark.parametrize("p", [3, 4])
def test_permuted_spectra_equal_explicit(p):
    """All 48 elements of the hyperoctahedral group act on the symbol by
    xi'_{sigma(i)} = s_i xi_i (Eq. permuteM2L)."""
    kappa, side = 6.0, 0.125
    N = 2 * p - 1
    for kbar in [(3, 2, 0), (4, 1, 1), (2, 2, 2), (5, 0, 0)]:
        gbar = m2l.spectrum(kappa, side, p, N, kbar)
        for perm, signs in _signed_permutations():
            k = [0, 0, 0]
            for i in range(3):
                k[i] = signs[i] * kbar[perm[i]]
            kb2, sigma, s = m2l.canonical(k)
            assert kb2 == tuple(sorted(kbar, reverse=True))
            explicit = m2l.spectrum(kappa, side, p, N, k)
            permuted = m2l.permute_spectrum(gbar, sigma, s, N)
            assert np.max(np.abs(explicit - permuted)) <= 1e-13 * np.max(np.abs(explicit))


def test_spectrum_of_opposite_offset():
    """G(x - y) = G(y - x): g_{-k}(delta) = g_k(-delta), so F(g_{-k})(xi) = F(g_k)(-xi)."""
    N, p = 9, 4
    g = m2l.spectrum(2.0, 0.3, p, N, (3, 1, 0))
    gm = m2l.spectrum(2.0, 0.3, p, N, (-3, -1, 0))
    neg = (-np.arange(N)) % N
    assert np.max(np.abs(gm - g[np.ix_(neg, neg, neg)])) <= 1e-13 * np.max(np.abs(g))


def test_m2f_f2l_roundtrip_and_canonical_form():
    p, N = 4, 7
    M = _rand((p ** 3, 3))
    assert np.allclose(m2l.f2l(m2l.m2f(M, p, N), p), M, atol=1e-14)
    assert m2l.canonical((0, -3, 3)) == ((3, 3, 0), (2, 0, 1), (1, -1, 1))
    assert m2l.canonical((-1, 0, 0)) == ((1, 0, 0), (0, 1, 2), (-1, 1, 1))
