"""O(N^2) direct evaluation of the N-body sum, Eq. (1.1) of Sec. 1.

    p(x) = sum_{y in Y} G(x, y) q(y),   G(x, y) = exp(i kappa |x-y|) / (4 pi |x-y|)

With a damping lambda >= 0 the kernel is exp((i kappa - lambda) |x-y|) / (4 pi |x-y|),
the Helmholtz kernel of the complex wavenumber kappa + i lambda: lambda = 0 is the
paper's kernel, kappa = lambda = 0 the Laplace kernel, kappa = 0 < lambda the
Yukawa (modified Helmholtz) kernel.  The method applies to asymptotically smooth
kernels in general (Sec. 1); kappa alone sets the oscillation the directional
machinery follows.  A radial power P = 2 gives exp((i kappa - lambda) r) / (4 pi r^2),
an oscillatory asymptotically smooth kernel outside the Helmholtz family.

Pairs closer than ``eps_self`` are skipped: the paper resolves coincident
particles by zeroing the interaction when the distance is "too small"
(Sec. 5.3); we read "too small" as |x - y| <= 1e-10 * D, D the side of the
smallest box holding X and Y (the same rule is used by every other path).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

EPS_SELF_REL = 1e-10


def helmholtz(r: np.ndarray, kappa: float, damping: float = 0.0, power: int = 1) -> np.ndarray:
    """G as a function of r = |x - y| (Sec. 1), with the damping lambda and the radial power P above."""
    return np.exp((1j * kappa - damping) * r) / (4.0 * np.pi * r ** power)


def eps_self(X: np.ndarray, Y: np.ndarray | None = None) -> float:
    P = X if Y is None else np.vstack([X, Y])
    return EPS_SELF_REL * float(np.max(P.max(axis=0) - P.min(axis=0)))


def direct_sum(X, Y, q, kappa, eps, targets=None, chunk=256, damping=0.0, power=1):
    """p at X[targets] (all of X by default) for charges q (ny,) or (ny, R)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    q = np.asarray(q, dtype=np.complex128)
    squeeze = q.ndim == 1
    if squeeze:
        q = q[:, None]
    idx = np.arange(len(X)) if targets is None else np.asarray(targets)
    out = np.zeros((len(idx), q.shape[1]), dtype=np.complex128)
    for c0 in range(0, len(idx), chunk):
        xs = X[idx[c0:c0 + chunk]]
        d = xs[:, None, :] - Y[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=2))
        far = r > eps
        G = np.zeros(r.shape, dtype=np.complex128)
        G[far] = helmholtz(r[far], kappa, damping, power)
        out[c0:c0 + chunk] = G @ q
    return out[:, 0] if squeeze else out


# ---------------------------------------------------------------------------
# The same sum as plain C (oracle/direct.c), for sampled targets of large
# clouds.  It is pinned against ``direct_sum`` above in the CPU tests.

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(__file__), "_direct.so")
        if not os.path.exists(path):
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(path)
        lib.oracle_direct_sum.restype = None
        lib.oracle_direct_sum.argtypes = [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        _LIB = lib
    return _LIB


def direct_sum_c(X, Y, q, kappa, eps, targets=None, damping=0.0, power=1):
    """Same as ``direct_sum`` but in C with OpenMP over targets."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    q = np.asarray(q, dtype=np.complex128)
    squeeze = q.ndim == 1
    if squeeze:
        q = q[:, None]
    qf = np.asfortranarray(q)
    idx = np.ascontiguousarray(np.arange(len(X)) if targets is None else targets,
                               dtype=np.int64)
    out = np.zeros((q.shape[1], len(idx)), dtype=np.complex128)
    _lib().oracle_direct_sum(X.ctypes.data, len(X), Y.ctypes.data, len(Y),
                             qf.ctypes.data, q.shape[1], float(kappa), float(damping), float(eps),
                             int(power), idx.ctypes.data, out.ctypes.data, len(idx))
    out = out.T
    return out[:, 0] if squeeze else out
