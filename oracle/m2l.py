"""M2L on equispaced grids: difference grid, circulant embedding, DFT, symmetries.

Sec. 2.3 (Eq. NormalizedKernel, CirculantKernel, FactorizedM2LMatrix1,
DFTformula, FourierDiagonal) and Sec. 4.3 (Eq. PermutationRepresentation,
permuteM2L).

For two cells of the same level with integer offset k = coords(t) - coords(s),
side beta and node spacing h = beta/(p-1), the M2L matrix is

    L[a] = sum_b G(x_a - y_b) M[b] = sum_b g_k(a - b) M[b],
    g_k(delta) = G(beta k + h delta),   delta in {-(p-1) .. p-1}^3,

a linear convolution.  Embedding M (zero padding, chi) and g_k (at delta mod N)
in Z_N^3 with N >= 2p - 1 turns it into a circular convolution, diagonalised by
the DFT:  L = chi^T F^-1 diag(F g_k) F chi M.  We use the unnormalised forward
DFT for data and kernel and 1/N^3 in the inverse (the paper's unitary F with
a T^{d/2}-scaled symbol gives the same operator; its T = 2L+1 is our N for
the minimal choice).  Any N >= 2p-1 gives the same result.

Symmetries (Sec. 4.3): G is radial, so for a signed permutation R of the
axes, with k = R kbar (k_i = s_i kbar_{sigma(i)}),
    F(g_k)(xi) = F(g_kbar)(xi'),   xi'_{sigma(i)} = s_i xi_i  (mod N),
the Fourier-domain permutation of Eq. (permuteM2L).  Only the canonical
kbar = (|k| sorted decreasing) spectra are formed.  Canonical order: axes
sorted by (-|k_i|, i); s_i = sign(k_i) with sign(0) = +1.

Arrays over the grid are indexed [z, y, x] (x fastest, as Def. 1).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .direct import helmholtz


def kernel_samples(kappa: float, side: float, p: int, k, damping: float = 0.0, power: int = 1) -> np.ndarray:
    """g_k(delta) on the difference grid, array [dz, dy, dx] of shape (2p-1)^3."""
    h = side / (p - 1)
    d = np.arange(-(p - 1), p, dtype=np.float64)
    dz, dy, dx = np.meshgrid(d, d, d, indexing="ij")
    vx = side * k[0] + h * dx
    vy = side * k[1] + h * dy
    vz = side * k[2] + h * dz
    return helmholtz(np.sqrt(vx * vx + vy * vy + vz * vz), kappa, damping, power)


def embed_kernel(g: np.ndarray, p: int, N: int) -> np.ndarray:
    """First column of the circulant matrix: g(delta) placed at delta mod N."""
    out = np.zeros((N, N, N), dtype=np.complex128)
    idx = np.arange(-(p - 1), p) % N
    out[np.ix_(idx, idx, idx)] = g
    return out


def spectrum(kappa: float, side: float, p: int, N: int, k, damping: float = 0.0, power: int = 1) -> np.ndarray:
    """F(g_k): diagonal of the Fourier-domain M2L operator (Eq. FourierDiagonal)."""
    return np.fft.fftn(embed_kernel(kernel_samples(kappa, side, p, k, damping, power), p, N))


def canonical(k):
    """(kbar, sigma, s): kbar canonical offset, sigma[i] = position of axis i, s[i] = sign."""
    k = [int(v) for v in k]
    order = sorted(range(3), key=lambda i: (-abs(k[i]), i))
    kbar = tuple(abs(k[order[j]]) for j in range(3))
    sigma = [0, 0, 0]
    for j, i in enumerate(order):
        sigma[i] = j
    s = tuple(1 if v >= 0 else -1 for v in k)
    return kbar, tuple(sigma), s


def permute_spectrum(ghat_bar: np.ndarray, sigma, s, N: int) -> np.ndarray:
    """F(g_k)(xi) = F(g_kbar)(xi') with xi'_{sigma(i)} = s_i xi_i mod N (Sec. 4.3.1)."""
    xi = np.arange(N)
    Z, Y, X = np.meshgrid(xi, xi, xi, indexing="ij")
    comp = [X, Y, Z]                              # xi_0 = x, xi_1 = y, xi_2 = z
    prime = [None, None, None]
    for i in range(3):
        prime[sigma[i]] = (s[i] * comp[i]) % N
    return ghat_bar[prime[2], prime[1], prime[0]]


def m2f(M: np.ndarray, p: int, N: int) -> np.ndarray:
    """M2F = F chi: zero-pad the p^3 grid (per column) into N^3 and DFT it."""
    R = M.shape[1]
    out = np.zeros((R, N, N, N), dtype=np.complex128)
    for r in range(R):
        out[r, :p, :p, :p] = M[:, r].reshape(p, p, p)
    return np.fft.fftn(out, axes=(1, 2, 3))


def f2l(Lhat: np.ndarray, p: int) -> np.ndarray:
    """F2L = chi^T F^-1: inverse DFT (1/N^3 included) and crop to the p^3 grid."""
    full = np.fft.ifftn(Lhat, axes=(1, 2, 3))
    R = Lhat.shape[0]
    return np.stack([full[r, :p, :p, :p].reshape(p ** 3) for r in range(R)], axis=1)


def dense_m2l(kappa: float, side: float, p: int, k, M: np.ndarray, damping: float = 0.0,
              power: int = 1) -> np.ndarray:
    """The definition: L[a] = sum_b G(x_a - y_b) M[b] (no FFT)."""
    from .interp import multi_index
    h = side / (p - 1)
    mi = multi_index(p).astype(np.float64)
    diff = side * np.asarray(k, dtype=np.float64)[None, None, :] + h * (mi[:, None, :] - mi[None, :, :])
    G = helmholtz(np.sqrt(np.sum(diff * diff, axis=2)), kappa, damping, power)
    return G @ M
