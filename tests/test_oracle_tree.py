"""Pins of the oracle's tree, directions, MACs and traversals (Sec. 4.1-4.2)."""
import itertools

import numpy as np
import pytest

from oracle import directions as dirs
from oracle import dtt, fmm
from oracle.tree import MAXLEVEL, bounding_cube, build_tree
from paper_2202_04894_gb300 import workloads as W


@pytest.mark.parametrize("kind,n,leaf", [("sphere", 3000, 40), ("box", 2000, 8), ("cube", 1500, 1)])
def test_tree_structure(kind, n, leaf):
    X = W.points(kind, n, 11)
    corner, side, _ = bounding_cube(X)
    t = build_tree(X, corner, side, leaf)
    Xs = X[t.perm]
    assert sorted(t.perm.tolist()) == list(range(n))
    for c in range(t.ncell):
        lo = t.cell_corner(c)
        cs = t.cell_side(int(t.level[c]))
        pts = Xs[t.begin[c]:t.end[c]]
        assert t.end[c] > t.begin[c]                          # no empty cells stored
        assert np.all(pts >= lo - 1e-12) and np.all(pts <= lo + cs + 1e-12)
        if t.is_leaf(c):
            assert t.end[c] - t.begin[c] <= leaf or t.level[c] == MAXLEVEL
        else:
            assert t.end[c] - t.begin[c] > leaf
            ch = list(t.children(c))
            assert t.begin[ch[0]] == t.begin[c] and t.end[ch[-1]] == t.end[c]
            for a, b in zip(ch, ch[1:]):
                assert t.end[a] == t.begin[b] and t.octant(a) < t.octant(b)
            assert all(t.parent[x] == c for x in ch)
    # leaves partition the particles
    leaves = [c for c in range(t.ncell) if t.is_leaf(c)]
    assert sum(t.end[c] - t.begin[c] for c in leaves) == n


def test_duplicate_points_terminate():
    X = np.zeros((10, 3))
    X[5:] = 1.0
    corner, side, _ = bounding_cube(X)
    t = build_tree(X, corner, side, 2)
    assert t.nlevel == MAXLEVEL + 1


@pytest.mark.parametrize("E", [0, 1, 2, 3])
def test_direction_sets(E):
    d = dirs.directions(E)
    assert len(d) == 6 * 4 ** E
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert len({tuple(np.round(v, 12)) for v in d}) == len(d)
    w = dirs.integer_vectors(E)
    for i in range(len(d)):
        assert np.array_equal(w[dirs.negate(E, i)], -w[i])
        if E > 0:
            f = dirs.father(E, i)
            wf = dirs.integer_vectors(E - 1)[f]
            # the son's sub-square lies inside the father's: same face, and the
            # son's centre is within half a father square of the father's centre
            m = np.argmax(np.abs(wf))
            assert w[i][m] * wf[m] > 0 and np.abs(w[i][m]) == 2 * np.abs(wf[m])
            assert np.all(np.abs(w[i] - 2 * wf) <= (1 << E) // 2 * np.ones(3) + 0)
            assert dirs.father(E, dirs.negate(E, i)) == dirs.negate(E - 1, f)


def test_best_direction_argmin_and_symmetry():
    rng = np.random.default_rng(3)
    for E in (0, 1, 2):
        d = dirs.directions(E)
        for _ in range(200):
            k = rng.integers(-9, 10, size=3)
            if not k.any():
                continue
            u = dirs.best_direction(E, k)
            dist = np.linalg.norm(d - k / np.linalg.norm(k), axis=1)
            assert dist[u] <= dist.min() + 1e-12
            assert dirs.best_direction(E, -k) == dirs.negate(E, u)
    # ties: k = e_x is equidistant to the four +x sub-squares at E=1 -> lowest index
    assert dirs.best_direction(1, (1, 0, 0)) == 0
    assert dirs.best_direction(1, (-1, 0, 0)) == dirs.negate(1, 0)


def _box_distance_brute(k):
    g = np.linspace(0, 1, 5)
    P = np.array(list(itertools.product(g, g, g)))
    Q = P + np.asarray(k, dtype=float)
    return np.min(np.linalg.norm(P[:, None] - Q[None], axis=2))


def test_macs_against_brute_force_distance():
    side0, kappa = 2.0, 40.0
    lv = dtt.Levels(side0, kappa)
    rng = np.random.default_rng(5)
    for l in range(lv.l_hf + 3):
        side = lv.side(l)
        w = np.sqrt(3) / 2 * side
        for _ in range(40):
            k = rng.integers(-6, 7, size=3)
            dist = side * _box_distance_brute(k)
            if lv.hf[l]:
                want = max(kappa * w * w, 2 * w) <= dist * (1 + 1e-12)
                if abs(max(kappa * w * w, 2 * w) - dist) > 1e-9 * dist:
                    assert lv.mac(l, k) == want
            else:
                assert lv.mac(l, k) == (dist >= side * (1 - 1e-12))


@pytest.mark.parametrize("case", [("sphere", 700, 20, 8.0, None), ("box", 600, 10, 30.0, None),
                                  ("sphere", 400, 15, 6.0, ("ellipsoid", 350))])
def test_dtt_covers_every_pair_once(case):
    """Every (x, y) is handled by exactly one P2P pair or one M2L pair."""
    kind, n, leaf, kd, other = case
    X = W.points(kind, n, 2)
    Y = None if other is None else W.points(other[0], other[1], 3)
    plan = fmm.make_plan(X, Y, kappa=kd / 2.0, order=3, leaf=leaf)
    ny = n if Y is None else len(Y)
    cnt = np.zeros((n, ny), dtype=np.int32)
    for (t, s) in plan.m2l_pairs + plan.p2p_pairs:
        cnt[plan.tt.begin[t]:plan.tt.end[t], plan.ts.begin[s]:plan.ts.end[s]] += 1
    assert np.all(cnt == 1)
    assert len(plan.m2l_pairs) > 0


def test_blank_passes_supply_every_needed_expansion():
    X = W.points("sphere", 3000, 4)
    plan = fmm.make_plan(X, kappa=24.0, order=3, leaf=16)
    lv, t = plan.levels, plan.tt
    assert lv.l_hf >= 2
    for (a, b), u in zip(plan.m2l_pairs, plan.pair_dir):
        assert u in plan.marks_t[a] and u in plan.marks_s[b]
    for c in range(t.ncell):
        l = int(t.level[c])
        for c2 in t.children(c):
            for v in plan.marks_s[c]:
                want = -1 if (v < 0 or not lv.hf[l + 1]) else dirs.father(lv.E(l), v)
                assert want in plan.marks_s[c2]


@pytest.mark.parametrize("other", [None, ("ellipsoid", 2500)])
def test_blank_passes_on_both_trees_exact(other):
    """Alg. 2 and Alg. 3 on the target tree as well as the source tree, with one tree
    and with two different trees: every HF cell's marks are exactly the directions of
    its own M2L pairs plus Father(u) of its father's marks (nothing missing, nothing
    extra), and every LF cell has the single non-directional expansion."""
    X = W.points("sphere", 3000, 4)
    Y = None if other is None else 0.9 * W.points(other[0], other[1], 5)
    plan = fmm.make_plan(X, Y, kappa=24.0, order=3, leaf=16)
    lv = plan.levels
    assert lv.l_hf >= 2
    for tree, marks, side in ((plan.tt, plan.marks_t, 0), (plan.ts, plan.marks_s, 1)):
        own = [set() for _ in range(tree.ncell)]
        for pair, u in zip(plan.m2l_pairs, plan.pair_dir):
            if u >= 0:
                own[pair[side]].add(u)
        parent_of = {}
        for c in range(tree.ncell):
            for c2 in tree.children(c):
                parent_of[c2] = c
        for c in range(tree.ncell):
            l = int(tree.level[c])
            if not lv.hf[l]:
                assert marks[c] == [-1]
                continue
            want = set(own[c])
            f = parent_of.get(c)
            if f is not None and lv.hf[l - 1]:
                want |= {dirs.father(lv.E(l - 1), v) for v in marks[f]}
            assert set(marks[c]) == want, (side, c)
            assert marks[c] == sorted(marks[c])
