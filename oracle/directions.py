"""Direction sets and the direction tree (Sec. 2.1, Sec. 4.1.2).

At the E-th high-frequency level (E = 0 at the deepest high-frequency level,
E growing toward the root), the directions are the centres of the faces of
the cube [-1,1]^3, each face cut into a 2^E x 2^E grid of sub-squares,
projected on the unit sphere: 6 * 4^E directions (Sec. 4.1.2; the paper's
"d! faces" is 2d = 6 faces for d = 3).  Each direction at level E is the son
of the direction of the enclosing sub-square at level E - 1, i.e. of the
next deeper octree level (Sec. 2.1); ``father`` returns it.

Indexing (ours): face f in order +x, -x, +y, -y, +z, -z; on a face normal to
axis m the two other axes m1 < m2 carry the sub-square indices (i, j);
index = f * 4^E + i * 2^E + j.  The unnormalised integer vector of a
direction has 2^E * sign on axis m and 2i + 1 - 2^E, 2j + 1 - 2^E on m1, m2.

The best direction of an M2L pair (Alg. 2) is
    u = argmin_{v in D(l)} | v - k/|k| |  =  argmax_v <v, k> / |v|,
k the integer offset between target and source cells.  Ties (common for
axis-aligned k) are resolved exactly with integer arithmetic: among the
maximisers we take the lowest index when k is "positive" (first non-zero
component > 0), and the negation of the choice for -k otherwise, so that
u(-k) = -u(k).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import functools

import numpy as np


def face_axes(f: int):
    m = f // 2
    sign = 1 if f % 2 == 0 else -1
    m1, m2 = [a for a in range(3) if a != m]
    return m, sign, m1, m2


@functools.lru_cache(maxsize=None)
def integer_vectors(E: int) -> np.ndarray:
    """(6*4^E, 3) int64 unnormalised direction vectors at level E."""
    n = 1 << E
    out = np.zeros((6 * n * n, 3), dtype=np.int64)
    idx = 0
    for f in range(6):
        m, sign, m1, m2 = face_axes(f)
        for i in range(n):
            for j in range(n):
                out[idx, m] = sign * n
                out[idx, m1] = 2 * i + 1 - n
                out[idx, m2] = 2 * j + 1 - n
                idx += 1
    return out


@functools.lru_cache(maxsize=None)
def directions(E: int) -> np.ndarray:
    w = integer_vectors(E).astype(np.float64)
    return w / np.linalg.norm(w, axis=1, keepdims=True)


def father(E: int, d: int) -> int:
    """Direction at level E-1 (one octree level deeper) whose son is d."""
    n = 1 << E
    f, rem = divmod(d, n * n)
    i, j = divmod(rem, n)
    h = n // 2
    return f * h * h + (i // 2) * h + (j // 2)


def negate(E: int, d: int) -> int:
    n = 1 << E
    f, rem = divmod(d, n * n)
    i, j = divmod(rem, n)
    return (f ^ 1) * n * n + (n - 1 - i) * n + (n - 1 - j)


@functools.lru_cache(maxsize=None)
def _best_positive(E: int, k) -> int:
    w = integer_vectors(E)
    k = np.asarray(k, dtype=np.int64)
    dots = w @ k                         # exact integers
    norms2 = np.sum(w * w, axis=1)       # exact integers
    cand = np.nonzero(dots > 0)[0]
    # exact comparison of dots[a]/sqrt(norms2[a]) between positive candidates:
    # a beats b  iff  dots[a]^2 * norms2[b] > dots[b]^2 * norms2[a]
    best = int(cand[0])
    for a in cand[1:]:
        a = int(a)
        lhs = int(dots[a]) ** 2 * int(norms2[best])
        rhs = int(dots[best]) ** 2 * int(norms2[a])
        if lhs > rhs:
            best = a
    return best


def best_direction(E: int, k) -> int:
    k = [int(v) for v in k]
    first = next(v for v in k if v != 0)
    if first > 0:
        return _best_positive(E, tuple(k))
    return negate(E, _best_positive(E, tuple(-v for v in k)))
