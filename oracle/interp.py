"""Equispaced Lagrange interpolation and the interpolation operators.

Sec. 2.2 (Eq. interpapprox and the operator list) with the equispaced grids
of Sec. 2.3.  The order p is the number of interpolation points per
dimension (the paper's "order L": L equispaced points, Lemma 1, and the
(2L-1)^d Hadamard size of Sec. 2.3).  The grid of a cell with lower corner
alpha and side beta is  alpha + beta * {0, 1/(p-1), ..., 1}^3, node index
a = a_x + p a_y + p^2 a_z (Def. 1, Sec. 5.2.1).

Directional operators carry plane-wave factors (Sec. 2.2, grey terms):

  S_a^u[c](y) = exp(i kappa <y_a - y, u>) S_a[c](y)

(the paper writes exp(i k <y_a,u>) ... exp(-i k <y,u>); the product is the same
and only the difference is ever formed).  With u = None the factor is 1
(low-frequency, non-directional operators).

  P2M  M_c^u[a]  = sum_{y in c} S_a^u[c](y) q(y)
  M2M  M_c^v[a] += sum_b S_a^v[c](y'_b) M_{c'}^{u}[b]      (y'_b nodes of son c')
  L2L  L_{c'}^u[b] += sum_a S_a^v[c](x'_b)^~ L_c^v[a]     with the conjugate
                      phase exp(i kappa <x'_b - x_a, v>)  (transpose, Sec. 2.2)
  L2P  p(x) += sum_a exp(i kappa <x - x_a, u>) S_a[c](x) L_c^u[a]

where u = Father(v) if the son is high-frequency and None otherwise.  The
paper's L2L line reads L_{t'}^v on its right-hand side; the transpose of M2M
it describes reads L_t^v (a typo).

Dense operators are the definition; ``tensorised_m2m`` is Sec. 5.2.1-5.2.3
(D0 (x) M^(p) D1, stacked over directions, real/imaginary split) and is
pinned against the dense form.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def nodes1d(p: int) -> np.ndarray:
    return np.arange(p, dtype=np.float64) / (p - 1)


def lagrange(p: int, t: np.ndarray) -> np.ndarray:
    """l_j(t) = prod_{m != j} (t - t_m) / (t_j - t_m), shape t.shape + (p,)."""
    tm = nodes1d(p)
    t = np.asarray(t, dtype=np.float64)
    out = np.ones(t.shape + (p,), dtype=np.float64)
    for j in range(p):
        for m in range(p):
            if m != j:
                out[..., j] *= (t - tm[m]) / (tm[j] - tm[m])
    return out


def multi_index(p: int) -> np.ndarray:
    """(p^3, 3) array of (a_x, a_y, a_z) for a = a_x + p a_y + p^2 a_z."""
    a = np.arange(p ** 3)
    return np.stack([a % p, (a // p) % p, a // (p * p)], axis=1)


def S(p: int, xhat: np.ndarray) -> np.ndarray:
    """Tensor Lagrange basis S_a at normalised points xhat (n,3) -> (n, p^3)."""
    lx = lagrange(p, xhat[:, 0])
    ly = lagrange(p, xhat[:, 1])
    lz = lagrange(p, xhat[:, 2])
    mi = multi_index(p)
    return lx[:, mi[:, 0]] * ly[:, mi[:, 1]] * lz[:, mi[:, 2]]


def grid(corner: np.ndarray, side: float, p: int) -> np.ndarray:
    """(p^3, 3) interpolation nodes of the cell alpha + side [0,1]^3."""
    return corner[None, :] + side * multi_index(p) / (p - 1)


def _phase(kappa, diff, u):
    if u is None:
        return np.ones(diff.shape[:-1], dtype=np.complex128)
    return np.exp(1j * kappa * (diff @ np.asarray(u, dtype=np.float64)))


def p2m(kappa, p, corner, side, Y, q, u):
    """M[a] = sum_y exp(i kappa <y_a - y, u>) S_a(y_hat) q(y);  q (n, R) -> (p^3, R)."""
    nodes = grid(corner, side, p)
    A = S(p, (Y - corner) / side) * _phase(kappa, nodes[None, :, :] - Y[:, None, :], u)
    return A.T @ q


def m2m_matrix(kappa, p, corner, side, child_corner, u):
    """T[a, b] = exp(i kappa <y_a - y'_b, u>) S_a[c](y'_b), the M2M matrix."""
    nodes = grid(corner, side, p)
    cnodes = grid(child_corner, side / 2, p)
    Sb = S(p, (cnodes - corner) / side)                  # [b, a]
    ph = _phase(kappa, nodes[:, None, :] - cnodes[None, :, :], u)   # [a, b]
    return Sb.T * ph


def l2l_matrix(kappa, p, corner, side, child_corner, v):
    """U[b, a] = exp(i kappa <x'_b - x_a, v>) S_a[c](x'_b), the L2L matrix."""
    nodes = grid(corner, side, p)
    cnodes = grid(child_corner, side / 2, p)
    Sb = S(p, (cnodes - corner) / side)                  # [b, a]
    ph = _phase(kappa, cnodes[:, None, :] - nodes[None, :, :], v)   # [b, a]
    return Sb * ph


def l2p(kappa, p, corner, side, X, L, u):
    """p(x) = sum_a exp(i kappa <x - x_a, u>) S_a(x_hat) L[a];  L (p^3, R) -> (n, R)."""
    nodes = grid(corner, side, p)
    A = S(p, (X - corner) / side) * _phase(kappa, X[:, None, :] - nodes[None, :, :], u)
    return A @ L


# ---------------------------------------------------------------------------
# Sec. 5.2: tensorised (t), stacked (t+s) and real (t+s+r) M2M evaluation.

def m2m_1d(p: int, octant_bit: int) -> np.ndarray:
    """M^(p)[a, b] = l_a(t'_b), t'_b = (bit + b/(p-1))/2: 1-D son-to-father matrix."""
    tb = (octant_bit + nodes1d(p)) / 2.0
    return lagrange(p, tb).T


def m2m_diagonals(kappa, p, corner, side, child_corner, u):
    """D0(u) = diag(exp(i kappa <y_a - c, u>)), D1(u) = diag(exp(-i kappa <y'_b - c, u>))."""
    c = corner + side / 2.0
    nodes = grid(corner, side, p)
    cnodes = grid(child_corner, side / 2, p)
    return _phase(kappa, nodes - c, u), _phase(kappa, c - cnodes, u)


def tensorised_m2m(kappa, p, corner, side, child_corner, octant, us, V, real_split=False):
    """Applies the M2M of every direction in ``us`` to the stacked columns V.

    V is (p^3, len(us)) with column j the son's expansion for direction us[j];
    the d one-dimensional products of Def. 1 act on all columns at once
    (t+s); with ``real_split`` the real and imaginary parts are stacked as
    separate real columns (t+s+r).
    """
    D1 = np.stack([m2m_diagonals(kappa, p, corner, side, child_corner, u)[1] for u in us], 1)
    D0 = np.stack([m2m_diagonals(kappa, p, corner, side, child_corner, u)[0] for u in us], 1)
    W = D1 * V
    if real_split:
        W = np.concatenate([W.real, W.imag], axis=1)
    ncol = W.shape[1]
    X = W.reshape(p, p, p, ncol)                  # [b_z, b_y, b_x, col]
    bits = [(octant >> a) & 1 for a in range(3)]
    X = np.einsum("ij,zyjc->zyic", m2m_1d(p, bits[0]), X)   # x pass
    X = np.einsum("ij,zjxc->zixc", m2m_1d(p, bits[1]), X)   # y pass
    X = np.einsum("ij,jyxc->iyxc", m2m_1d(p, bits[2]), X)   # z pass
    X = X.reshape(p ** 3, ncol)
    if real_split:
        h = ncol // 2
        X = X[:, :h] + 1j * X[:, h:]
    return D0 * X
