"""The plan and the application phase of the directional equispaced FMM.

Follows the paper's design, step by step, in the order of Sec. 4:

plan
  1. cube, Morton sort and Ncrit trees (Sec. 4.2.1);      ``tree``
  2. per-level regime and direction sets (Sec. 4.1.2);    ``dtt.Levels``
  3. Dual Tree Traversal (Alg. 1) -> M2L and P2P pairs;   ``dtt``
  4. blank DTT (Alg. 2) + blank downward pass (Alg. 3) -> effective expansions;
  5. canonical transfer spectra of every M2L offset, with symmetries (Sec. 4.3).

apply (Sec. 2.2 operators, Sec. 4.1.1 M2F / F2L)
  P2M at source leaves -> M2M bottom-up -> M2F -> Hadamard M2L over the pairs
  -> F2L -> L2L top-down -> L2P at target leaves, plus P2P over the near pairs.

Sums run over pairs in DTT order and over sons in octant order, in float64.

Options kept for the pins: ``force_p2p`` (every MAC false), ``dense_m2l``
(matrix M2L without FFT), ``explicit_spectra`` (no symmetry reuse),
``fft_n`` (any N >= 2p-1).

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import directions as dirs
from . import dtt, interp, m2l
from .direct import EPS_SELF_REL, helmholtz
from .tree import bounding_cube, build_tree


@dataclass
class Plan:
    kappa: float
    order: int
    fft_n: int
    tt: object
    ts: object
    same: bool
    levels: dtt.Levels
    m2l_pairs: list
    p2p_pairs: list
    pair_dir: list
    marks_t: list
    marks_s: list
    eps_self: float
    d_aabb: float
    spectra: dict          # (level, kbar) -> canonical spectrum
    dense_m2l: bool = False
    explicit_spectra: bool = False
    damping: float = 0.0   # kernel exp((i kappa - damping) r) / (4 pi r^power)
    power: int = 1


def make_plan(X, Y=None, kappa=1.0, order=4, leaf=64, eta=1.0, hf_kw=1.0, fft_n=None,
              force_p2p=False, dense_m2l=False, explicit_spectra=False, damping=0.0, power=1) -> Plan:
    X = np.asarray(X, dtype=np.float64)
    same = Y is None
    Ys = X if same else np.asarray(Y, dtype=np.float64)
    corner, side, d_aabb = bounding_cube(X, None if same else Ys)
    tt = build_tree(X, corner, side, leaf)
    ts = tt if same else build_tree(Ys, corner, side, leaf)
    lv = dtt.Levels(side, kappa, hf_kw=hf_kw, eta=eta)
    m2l_pairs, p2p_pairs = dtt.dual_tree_traversal(tt, ts, lv, force_p2p=force_p2p)
    pair_dir = [dtt.pair_direction(tt, ts, lv, t, s) for (t, s) in m2l_pairs]
    marks_t, marks_s = dtt.blank_passes(tt, ts, lv, m2l_pairs)
    N = fft_n if fft_n is not None else 2 * order - 1
    assert N >= 2 * order - 1
    spectra = {}
    for (t, s) in m2l_pairs:
        l = int(tt.level[t])
        kbar, _, _ = m2l.canonical(tt.coords[t] - ts.coords[s])
        if (l, kbar) not in spectra:
            spectra[(l, kbar)] = m2l.spectrum(kappa, lv.side(l), order, N, kbar, damping, power)
    return Plan(kappa=kappa, order=order, fft_n=N, tt=tt, ts=ts, same=same, levels=lv,
                m2l_pairs=m2l_pairs, p2p_pairs=p2p_pairs, pair_dir=pair_dir,
                marks_t=marks_t, marks_s=marks_s, eps_self=EPS_SELF_REL * d_aabb,
                d_aabb=d_aabb, spectra=spectra, dense_m2l=dense_m2l,
                explicit_spectra=explicit_spectra, damping=damping, power=power)


def _dir_vec(lv, l, u):
    return None if u < 0 else dirs.directions(lv.E(l))[u]


def _child_dir(lv, l, v):
    """Direction of the son's expansion feeding (or fed by) direction v at level l."""
    if v < 0 or not lv.hf[l + 1]:
        return -1
    return dirs.father(lv.E(l), v)


def upward(plan: Plan, qs: np.ndarray) -> dict:
    """P2M and M2M: multipole expansions {(cell, dir): (p^3, R)} on the source tree."""
    ts, lv, p, kappa = plan.ts, plan.levels, plan.order, plan.kappa
    Ys = plan.Ys_sorted
    M = {}
    for l in reversed(range(ts.nlevel)):
        c0, c1 = ts.level_range[l]
        side = lv.side(l)
        for c in range(c0, c1):
            corner = ts.cell_corner(c)
            for u in plan.marks_s[c]:
                uvec = _dir_vec(lv, l, u)
                if ts.is_leaf(c):
                    b, e = ts.begin[c], ts.end[c]
                    M[(c, u)] = interp.p2m(kappa, p, corner, side, Ys[b:e], qs[b:e], uvec)
                else:
                    acc = np.zeros((p ** 3, qs.shape[1]), dtype=np.complex128)
                    for c2 in ts.children(c):
                        u2 = _child_dir(lv, l, u)
                        T = interp.m2m_matrix(kappa, p, corner, side, ts.cell_corner(c2), uvec)
                        acc += T @ M[(c2, u2)]
                    M[(c, u)] = acc
    return M


def transfer(plan: Plan, M: dict) -> dict:
    """M2F, Hadamard products over the M2L pairs, F2L: {(cell, dir): L} on the target tree."""
    tt, ts, lv, p, N = plan.tt, plan.ts, plan.levels, plan.order, plan.fft_n
    R = next(iter(M.values())).shape[1] if M else 1
    L = {}
    if plan.dense_m2l:
        for (t, s), u in zip(plan.m2l_pairs, plan.pair_dir):
            l = int(tt.level[t])
            k = tt.coords[t] - ts.coords[s]
            contrib = m2l.dense_m2l(plan.kappa, lv.side(l), p, k, M[(s, u)], plan.damping, plan.power)
            L[(t, u)] = L.get((t, u), 0) + contrib
        return L
    Mhat = {}
    for (t, s), u in zip(plan.m2l_pairs, plan.pair_dir):
        if (s, u) not in Mhat:
            Mhat[(s, u)] = m2l.m2f(M[(s, u)], p, N)
    Lhat = {}
    for (t, s), u in zip(plan.m2l_pairs, plan.pair_dir):
        l = int(tt.level[t])
        k = tt.coords[t] - ts.coords[s]
        if plan.explicit_spectra:
            g = m2l.spectrum(plan.kappa, lv.side(l), p, N, k, plan.damping, plan.power)
        else:
            kbar, sigma, sg = m2l.canonical(k)
            g = m2l.permute_spectrum(plan.spectra[(l, kbar)], sigma, sg, N)
        if (t, u) not in Lhat:
            Lhat[(t, u)] = np.zeros((R, N, N, N), dtype=np.complex128)
        Lhat[(t, u)] += g[None] * Mhat[(s, u)]
    for key, val in Lhat.items():
        L[key] = m2l.f2l(val, p)
    return L


def downward(plan: Plan, L: dict, R: int) -> np.ndarray:
    """L2L top-down then L2P: far-field potentials in target sorted order."""
    tt, lv, p, kappa = plan.tt, plan.levels, plan.order, plan.kappa
    Xs = plan.Xs_sorted
    pot = np.zeros((len(Xs), R), dtype=np.complex128)
    zero = np.zeros((p ** 3, R), dtype=np.complex128)
    for l in range(tt.nlevel):
        c0, c1 = tt.level_range[l]
        side = lv.side(l)
        for c in range(c0, c1):
            corner = tt.cell_corner(c)
            for v in plan.marks_t[c]:
                Lc = L.get((c, v), zero)
                vvec = _dir_vec(lv, l, v)
                if tt.is_leaf(c):
                    b, e = tt.begin[c], tt.end[c]
                    pot[b:e] += interp.l2p(kappa, p, corner, side, Xs[b:e], Lc, vvec)
                else:
                    for c2 in tt.children(c):
                        u2 = _child_dir(lv, l, v)
                        U = interp.l2l_matrix(kappa, p, corner, side, tt.cell_corner(c2), vvec)
                        L[(c2, u2)] = L.get((c2, u2), zero) + U @ Lc
    return pot


def near_field(plan: Plan, qs: np.ndarray) -> np.ndarray:
    """P2P over the near pairs of Alg. 1 (Sec. 2.2), masking |x-y| <= eps_self."""
    tt, ts = plan.tt, plan.ts
    Xs, Ys = plan.Xs_sorted, plan.Ys_sorted
    pot = np.zeros((len(Xs), qs.shape[1]), dtype=np.complex128)
    for (t, s) in plan.p2p_pairs:
        bt, et, bs, es = tt.begin[t], tt.end[t], ts.begin[s], ts.end[s]
        d = Xs[bt:et, None, :] - Ys[None, bs:es, :]
        r = np.sqrt(np.sum(d * d, axis=2))
        G = np.zeros(r.shape, dtype=np.complex128)
        far = r > plan.eps_self
        G[far] = helmholtz(r[far], plan.kappa, plan.damping, plan.power)
        pot[bt:et] += G @ qs[bs:es]
    return pot


def apply(plan: Plan, X, q, Y=None, parts=False):
    """Potentials p(x) for charges q (ny,) or (ny, R), in input order.

    With ``parts`` returns (near, far) separately (sorted order) as well.
    """
    X = np.asarray(X, dtype=np.float64)
    Ys = X if Y is None else np.asarray(Y, dtype=np.float64)
    q = np.asarray(q, dtype=np.complex128)
    squeeze = q.ndim == 1
    if squeeze:
        q = q[:, None]
    plan.Xs_sorted = X[plan.tt.perm]
    plan.Ys_sorted = Ys[plan.ts.perm]
    qs = q[plan.ts.perm]
    M = upward(plan, qs)
    L = transfer(plan, M)
    far = downward(plan, L, q.shape[1])
    near = near_field(plan, qs)
    out = np.zeros((len(X), q.shape[1]), dtype=np.complex128)
    out[plan.tt.perm] = far + near
    res = out[:, 0] if squeeze else out
    if parts:
        return res, near, far
    return res


def fmm(X, q, kappa, order=4, leaf=64, Y=None, **kw):
    """Plan + apply in one call."""
    plan = make_plan(X, Y, kappa=kappa, order=order, leaf=leaf, **kw)
    return apply(plan, X, q, Y)
