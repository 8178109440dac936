"""Bounding cube, Morton ordering and the Ncrit 2^d-tree of Sec. 4.2.1.

* The computational box B is the smallest axis-aligned cube holding X and Y
  (side D, Sec. 1), enlarged by a factor 1 + 2^-20 so that every particle is
  inside; quantised coordinates are clamped to the cube as well.
* Particles are sorted in Morton order (21 bits per axis, x in the lowest
  interleaved bit), ties kept in input order (stable sort), so that every cell
  owns a contiguous range of the sorted particles (Sec. 4.2.1).
* A cell is split into its 2^d sons while it holds more than Ncrit particles;
  empty sons are not stored (Sec. 4.2.1); 21 is the deepest level.
* A cell at level l is  alpha_c + beta_c * [0,1]^3  with beta_c = side/2^l
  (Eq. CellCorrespondance, Sec. 2.3).

Cells are numbered level by level, in Morton order inside a level, so the
sons of a cell are consecutive and in octant order (octant o = ox + 2 oy + 4 oz).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAXLEVEL = 21
ENLARGE = 1.0 + 2.0 ** -20


def bounding_cube(X: np.ndarray, Y: np.ndarray | None = None):
    """(corner, side, d_aabb): lower corner and side of the enlarged cube B."""
    P = X if Y is None else np.vstack([X, Y])
    lo = P.min(axis=0)
    hi = P.max(axis=0)
    d_aabb = float(np.max(hi - lo))
    if d_aabb == 0.0:
        d_aabb = 1.0
    side = d_aabb * ENLARGE
    corner = (lo + hi) / 2.0 - side / 2.0
    return corner, side, d_aabb


def quantise(P: np.ndarray, corner: np.ndarray, side: float) -> np.ndarray:
    """Integer coordinates on the 2^21 grid of B, clamped into the cube."""
    g = np.floor((P - corner) / side * float(1 << MAXLEVEL)).astype(np.int64)
    return np.clip(g, 0, (1 << MAXLEVEL) - 1)


def morton_keys(P: np.ndarray, corner: np.ndarray, side: float) -> np.ndarray:
    g = quantise(P, corner, side)
    key = np.zeros(len(P), dtype=np.int64)
    for b in range(MAXLEVEL):
        for a in range(3):
            key |= ((g[:, a] >> b) & 1) << (3 * b + a)
    return key


@dataclass
class Tree:
    corner: np.ndarray
    side: float
    ncrit: int
    perm: np.ndarray               # sorted position -> input index
    keys: np.ndarray               # Morton keys in sorted order
    level: np.ndarray = field(default=None)
    coords: np.ndarray = field(default=None)   # (ncell, 3) integer cell coords
    begin: np.ndarray = field(default=None)
    end: np.ndarray = field(default=None)
    parent: np.ndarray = field(default=None)
    first_child: np.ndarray = field(default=None)
    nchild: np.ndarray = field(default=None)
    level_range: list = field(default=None)    # [(first cell, last+1)] per level

    @property
    def ncell(self) -> int:
        return len(self.level)

    @property
    def nlevel(self) -> int:
        return len(self.level_range)

    def is_leaf(self, c: int) -> bool:
        return self.nchild[c] == 0

    def children(self, c: int) -> range:
        return range(self.first_child[c], self.first_child[c] + self.nchild[c])

    def cell_side(self, lev: int) -> float:
        return self.side / float(1 << lev)

    def cell_corner(self, c: int) -> np.ndarray:
        return self.corner + self.coords[c] * self.cell_side(int(self.level[c]))

    def octant(self, c: int) -> int:
        o = self.coords[c] & 1
        return int(o[0] + 2 * o[1] + 4 * o[2])


def build_tree(P: np.ndarray, corner: np.ndarray, side: float, ncrit: int) -> Tree:
    """Ncrit 2^d-tree on the Morton-sorted particles (Sec. 4.2.1)."""
    keys = morton_keys(P, corner, side)
    perm = np.argsort(keys, kind="stable")
    skeys = keys[perm]
    level, coords, begin, end, parent = [0], [(0, 0, 0)], [0], [len(P)], [-1]
    first_child, nchild = [], []
    level_range = []
    start = 0
    lev = 0
    while start < len(level):
        stop = len(level)
        level_range.append((start, stop))
        for c in range(start, stop):
            b, e = begin[c], end[c]
            if e - b > ncrit and lev < MAXLEVEL:
                shift = 3 * (MAXLEVEL - lev - 1)
                prefix = skeys[b:e] >> shift
                base = prefix[0] >> 3 << 3
                cuts = np.searchsorted(prefix, base + np.arange(9), side="left") + b
                first_child.append(len(level))
                n = 0
                for o in range(8):
                    if cuts[o + 1] > cuts[o]:
                        cx, cy, cz = coords[c]
                        level.append(lev + 1)
                        coords.append((2 * cx + (o & 1), 2 * cy + ((o >> 1) & 1),
                                       2 * cz + ((o >> 2) & 1)))
                        begin.append(int(cuts[o]))
                        end.append(int(cuts[o + 1]))
                        parent.append(c)
                        n += 1
                nchild.append(n)
            else:
                first_child.append(-1)
                nchild.append(0)
        start = stop
        lev += 1
    t = Tree(corner=np.asarray(corner, dtype=np.float64), side=float(side), ncrit=ncrit,
             perm=perm, keys=skeys)
    t.level = np.array(level, dtype=np.int64)
    t.coords = np.array(coords, dtype=np.int64)
    t.begin = np.array(begin, dtype=np.int64)
    t.end = np.array(end, dtype=np.int64)
    t.parent = np.array(parent, dtype=np.int64)
    t.first_child = np.array(first_child, dtype=np.int64)
    t.nchild = np.array(nchild, dtype=np.int64)
    t.level_range = level_range
    return t
