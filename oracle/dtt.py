"""Multipole acceptance criteria, the Dual Tree Traversal and the blank passes.

* Regime of a level (Sec. 4.1.1, Fig. of operators): the paper does not fix
  the boundary between low and high frequency; we call level l
  high-frequency iff kappa * w_l > hf_kw (default 1), w_l = sqrt(3)/2 * side_l
  the cell radius.  The deepest high-frequency level has E = 0.
* Strict MAC (low frequency, footnote of Sec. 3.2): two same-level cells are
  well separated iff their distance is at least their side, i.e. max|k_i| >= 2
  for the integer offset k.
* Directional MAC, Eq. (macdirref) of Sec. 4.2.2:  max(kappa w^2, 2 w) <= eta dist,
  with dist = side * sqrt(S), S = sum_i max(0, |k_i| - 1)^2, evaluated as
  max(kappa w^2, 2w)^2 <= eta^2 side^2 S.
* Dual Tree Traversal, Alg. 1 (Sec. 4.2.2): MAC -> M2L pair; else a leaf on
  either side -> P2P pair; else recurse on every pair of sons.
* Blank DTT, Alg. 2, and blank downward pass, Alg. 3 (Sec. 4.2.3): every
  high-frequency M2L pair marks its target and its source with the best
  direction u; then marks move down the trees, a son receiving Father(u).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import math

import numpy as np

from . import directions as dirs


class Levels:
    """Per-level geometry and regime shared by both trees (same cube B)."""

    def __init__(self, side: float, kappa: float, hf_kw: float = 1.0, eta: float = 1.0,
                 nlevel: int = 22):
        self.side0 = side
        self.kappa = kappa
        self.eta = eta
        self.hf_kw = hf_kw
        self.nlevel = nlevel
        self.hf = [self.kappa * self.radius(l) > hf_kw for l in range(nlevel)]
        hf_levels = [l for l in range(nlevel) if self.hf[l]]
        self.l_hf = max(hf_levels) if hf_levels else -1

    def side(self, l: int) -> float:
        return self.side0 / float(1 << l)

    def radius(self, l: int) -> float:
        return math.sqrt(3.0) / 2 * self.side(l)

    def E(self, l: int) -> int:
        """Direction-tree level of a high-frequency octree level."""
        return self.l_hf - l

    def mac(self, l: int, k) -> bool:
        if self.hf[l]:
            S = sum(max(0, abs(int(v)) - 1) ** 2 for v in k)
            w = self.radius(l)
            A = max(self.kappa * w * w, 2 * w)
            return A * A <= self.eta * self.eta * self.side(l) * self.side(l) * float(S)
        return max(abs(int(v)) for v in k) >= 2


def dual_tree_traversal(tt, ts, lv: Levels, force_p2p: bool = False):
    """Alg. 1 from (root, root).  Returns (m2l, p2p) lists of (t, s) cell pairs.

    ``force_p2p`` makes every MAC false (all interactions become P2P).
    """
    m2l, p2p = [], []

    def visit(t, s):
        l = int(tt.level[t])
        k = tt.coords[t] - ts.coords[s]
        if not force_p2p and lv.mac(l, k):
            m2l.append((t, s))
            return
        if tt.is_leaf(t) or ts.is_leaf(s):
            p2p.append((t, s))
            return
        for t2 in tt.children(t):
            for s2 in ts.children(s):
                visit(t2, s2)

    visit(0, 0)
    return m2l, p2p


def pair_direction(tt, ts, lv: Levels, t: int, s: int) -> int:
    """Best direction of a high-frequency M2L pair (Alg. 2); -1 in low frequency."""
    l = int(tt.level[t])
    if not lv.hf[l]:
        return -1
    k = tt.coords[t] - ts.coords[s]
    return dirs.best_direction(lv.E(l), k)


def blank_passes(tt, ts, lv: Levels, m2l):
    """Alg. 2 marks followed by Alg. 3 on both trees.

    Returns (marks_t, marks_s): per cell, the sorted list of directions of its
    effective local (target tree) or multipole (source tree) expansions; a
    low-frequency cell has the single non-directional expansion, written -1.
    """
    mt = [set() for _ in range(tt.ncell)]
    ms = [set() for _ in range(ts.ncell)]
    for (t, s) in m2l:
        u = pair_direction(tt, ts, lv, t, s)
        if u >= 0:
            mt[t].add(u)
            ms[s].add(u)

    def downward(tree, marks):
        for c in range(tree.ncell):          # level order: fathers first
            l = int(tree.level[c])
            if not lv.hf[l]:
                continue
            for u in marks[c]:
                for c2 in tree.children(c):
                    if lv.hf[l + 1]:
                        marks[c2].add(dirs.father(lv.E(l), u))

    downward(tt, mt)
    downward(ts, ms)

    def finish(tree, marks):
        out = []
        for c in range(tree.ncell):
            if lv.hf[int(tree.level[c])]:
                out.append(sorted(marks[c]))
            else:
                out.append([-1])
        return out

    return finish(tt, mt), finish(ts, ms)
