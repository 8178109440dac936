"""Seeded synthetic point clouds and charge vectors.

This module holds no arithmetic of the FMM: it only draws inputs. Both the
CUDA path (through the tests and the benchmark) and the CPU oracle receive
the arrays it returns, so neither side generates its own data.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used here as a counter-based
generator: the i-th draw of a stream with seed s is mix(s + (i+1)*gamma).

The distributions stand in for the paper's four 10^7-point test cases of
Sec. 6.2 (uniform cube, quasi-uniform sphere, edge/corner-refined cube,
pole-concentrated ellipse); the paper gives no samplers, so these are our
own recipes with the same character:

* ``sphere``     -- Gaussian triples normalised onto the unit sphere (D = 2);
* ``box``        -- surface of an axis-aligned box, face chosen by area, each
                    face coordinate warped by t -> (1 - cos(pi t))/2 so that
                    points crowd edges and corners;
* ``ellipsoid``  -- surface with semi-axes (1, 0.5, 0.2) parametrised by
                    uniform (theta, phi), which crowds the two poles;
* ``cube``       -- uniform in the volume of [-1, 1]^3 (Sec. 6.1 accuracy case).

Charges are complex and uniform in the unit disk (r = sqrt(U1), arg = 2 pi U2).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHARGE_SALT = 0x5851F42D4C957F2D


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _gaussian(seed: int, n: int, offset: int) -> np.ndarray:
    # Box-Muller on pairs of uniforms; 1 - u keeps the logarithm finite.
    u = uniform(seed, 2 * n, offset)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def sphere(n: int, seed: int) -> np.ndarray:
    g = np.stack([_gaussian(seed, n, 2 * n * a) for a in range(3)], axis=1)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def box_surface(n: int, seed: int, dims=(1.0, 1.0, 0.25)) -> np.ndarray:
    a, b, c = (float(v) for v in dims)
    areas = np.array([b * c, b * c, a * c, a * c, a * b, a * b])
    u = uniform(seed, 3 * n).reshape(n, 3)
    face = np.searchsorted(np.cumsum(areas) / areas.sum(), u[:, 0], side="right")
    face = np.minimum(face, 5)
    s = 0.5 * (1.0 - np.cos(np.pi * u[:, 1]))
    t = 0.5 * (1.0 - np.cos(np.pi * u[:, 2]))
    half = np.array([a, b, c]) / 2.0
    pts = np.empty((n, 3))
    for f in range(6):
        m = face == f
        axis, sign = f // 2, (1.0 if f % 2 == 0 else -1.0)
        o1, o2 = [ax for ax in range(3) if ax != axis]
        pts[m, axis] = sign * half[axis]
        pts[m, o1] = (2.0 * s[m] - 1.0) * half[o1]
        pts[m, o2] = (2.0 * t[m] - 1.0) * half[o2]
    return pts


def ellipsoid(n: int, seed: int, axes=(1.0, 0.5, 0.2)) -> np.ndarray:
    u = uniform(seed, 2 * n).reshape(n, 2)
    theta = np.pi * u[:, 0]
    phi = 2.0 * np.pi * u[:, 1]
    return np.stack([axes[0] * np.cos(theta),
                     axes[1] * np.sin(theta) * np.cos(phi),
                     axes[2] * np.sin(theta) * np.sin(phi)], axis=1)


def uniform_cube(n: int, seed: int) -> np.ndarray:
    return 2.0 * uniform(seed, 3 * n).reshape(n, 3) - 1.0


def charges(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Complex charges uniform in the unit disk, shape (n, nrhs), column-major."""
    u = uniform(seed ^ _CHARGE_SALT, 2 * n * nrhs).reshape(nrhs, n, 2)
    r = np.sqrt(u[..., 0])
    th = 2.0 * np.pi * u[..., 1]
    q = r * np.exp(1j * th)
    return np.asfortranarray(q.T)


DISTRIBUTIONS = {
    "sphere": sphere,
    "box": box_surface,
    "ellipsoid": ellipsoid,
    "cube": uniform_cube,
}


def points(kind: str, n: int, seed: int) -> np.ndarray:
    """(n, 3) float64 point cloud of the named distribution."""
    return np.ascontiguousarray(DISTRIBUTIONS[kind](n, seed), dtype=np.float64)


# The workloads the benchmark and the parity tests are quoted on.
# kappa is chosen from the stated kappa*D with D the bounding-cube side.
WORKLOADS = {
    # 2,000 points on the unit sphere, kappa*D = 8, order 4, leaf <= 64, complex128
    "sphere2k_kD8_p4": dict(kind="sphere", n=2000, seed=1, kappa_d=8.0, order=4,
                            leaf=64, nrhs=1, dtype="c128"),
    # 10^6 points on the unit sphere, kappa*D = 128, order 4, leaf <= 64, complex64
    "sphere1M_kD128_p4": dict(kind="sphere", n=1_000_000, seed=2, kappa_d=128.0,
                              order=4, leaf=64, nrhs=1, dtype="c64"),
    # 5*10^5 points on a 1 x 1 x 0.25 box surface, kappa*D = 64, order 5, 32 RHS
    "box500k_kD64_p5_r32": dict(kind="box", n=500_000, seed=3, kappa_d=64.0,
                                order=5, leaf=64, nrhs=32, dtype="c64"),
    # 5*10^5 points uniform in a cube, kappa*D = 64, order 4, leaf <= 64, complex64:
    # the volumetric distribution, whose M2L lists are the densest
    "cube500k_kD64_p4": dict(kind="cube", n=500_000, seed=4, kappa_d=64.0,
                             order=4, leaf=64, nrhs=1, dtype="c64"),
}


def make(name: str, n: int | None = None):
    """Returns (X, q, kappa, order, leaf, dtype) for a named workload.

    ``n`` overrides the point count (same distribution, seed and kappa*D),
    which is how bounded samples of a workload are drawn.
    """
    w = WORKLOADS[name]
    npts = w["n"] if n is None else int(n)
    X = points(w["kind"], npts, w["seed"])
    D = float(np.max(X.max(axis=0) - X.min(axis=0)))
    kappa = w["kappa_d"] / D
    q = charges(npts, w["seed"], w["nrhs"])
    return X, q, kappa, w["order"], w["leaf"], w["dtype"]


def _log_uniform(u: float, lo: float, hi: float) -> float:
    return float(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))))


def geometry_set(count: int, seed0: int, n_range, kd_range, orders=(4,)):
    """Uneven geometries for batched and served applies.

    Geometry i (seed seed0 + i) cycles through sphere, ellipsoid (axes
    1 : 0.5 : 0.2) and box surface; its point count and kappa*D are drawn
    log-uniform from n_range and kd_range, its order from ``orders``.
    Returns dicts (kind, n, seed, kappa_d, order).
    """
    kinds = ("sphere", "ellipsoid", "box")
    out = []
    for i in range(count):
        u = uniform(seed0 + i, 3)
        out.append(dict(kind=kinds[i % 3], n=int(round(_log_uniform(u[0], *n_range))), seed=seed0 + i,
                        kappa_d=_log_uniform(u[1], *kd_range),
                        order=int(orders[min(len(orders) - 1, int(u[2] * len(orders)))])))
    return out


def make_geometry(g: dict):
    """(X, kappa) of a geometry_set entry; kappa = kappa*D / D with D the extent."""
    X = points(g["kind"], g["n"], g["seed"])
    D = float(np.max(X.max(axis=0) - X.min(axis=0)))
    return X, g["kappa_d"] / D


# 48 uneven geometries applied together: N log-uniform in [2*10^4, 8*10^5],
# kappa*D log-uniform in [16, 256], order 4, one complex64 right-hand side each.
BATCH48 = dict(count=48, seed0=100, n_range=(2e4, 8e5), kd_range=(16.0, 256.0), orders=(4,))
# the same recipe with small geometries (2*10^4 to 5*10^4 points), where launch gaps weigh most
BATCH48_SMALL = dict(count=48, seed0=100, n_range=(2e4, 5e4), kd_range=(16.0, 64.0), orders=(4,))
# 16 resident geometries for the request server: N log-uniform in
# [5*10^4, 2*10^6], kappa*D log-uniform in [32, 256], order 4, 5 or 6.
SERVE16 = dict(count=16, seed0=200, n_range=(5e4, 2e6), kd_range=(32.0, 256.0), orders=(4, 5, 6))


def request_stream(count: int, seed: int, mean_gap_ms: float, ngeom: int, max_rhs: int = 8):
    """Poisson arrivals: (arrival_ms, geometry, nrhs) with exponential gaps of the
    given mean, geometry uniform over ngeom and nrhs uniform in 1..max_rhs."""
    u = uniform(seed, 3 * count).reshape(count, 3)
    gaps = -mean_gap_ms * np.log(1.0 - u[:, 0])
    t = np.cumsum(gaps)
    g = np.minimum((u[:, 1] * ngeom).astype(np.int64), ngeom - 1)
    r = 1 + np.minimum((u[:, 2] * max_rhs).astype(np.int64), max_rhs - 1)
    return [(float(t[i]), int(g[i]), int(r[i])) for i in range(count)]
