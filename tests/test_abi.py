"""CPU tests of the C ABI: the library loads, exports what include/defmm.h
declares, validates arguments, and its host plan tables equal the oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import fmm as oracle_fmm
from paper_2202_04894_gb300 import build as pkg_build
from paper_2202_04894_gb300 import defmm, serve, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg_build.build()


def _declared(header="defmm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(defmm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    L = defmm.lib()
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["defmm.h", "defmm_serve.h"]
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(L, n), n
    assert set(defmm.EXPORTED) <= set(names)
    served = _declared("defmm_serve.h")
    for n in served:
        assert hasattr(L, n), n
    assert set(serve.SERVE_EXPORTED) == set(served)


def test_serving_argument_errors():
    """The serving entry points reject bad arguments before touching a GPU."""
    import ctypes
    L = serve.slib()
    X = W.points("sphere", 200, 1)
    pl = _host_plan(X, kappa=1.0, order=4, leaf_size=8)
    h = ctypes.c_void_p()
    assert L.defmm_workspace_create(pl.handle, 1, defmm.C64, ctypes.byref(h)) == 5       # host-only plan
    assert L.defmm_workspace_create(None, 1, defmm.C64, ctypes.byref(h)) == 1
    b = ctypes.c_size_t()
    assert L.defmm_workspace_bytes(pl.handle, 0, defmm.C64, ctypes.byref(b)) == 1
    assert L.defmm_workspace_bytes(pl.handle, 3, defmm.C64, ctypes.byref(b)) == 0
    b64, b128 = b.value, ctypes.c_size_t()
    assert L.defmm_workspace_bytes(pl.handle, 3, defmm.C128, ctypes.byref(b128)) == 0
    assert b64 % 256 == 0 and b128.value > b64 and b64 >= 3 * 8 * 2 * 200
    arr = (ctypes.c_void_p * 1)(pl.handle.value)
    rr = (ctypes.c_int * 1)(1)
    assert L.defmm_batch_create(arr, rr, 1, defmm.C64, 0, ctypes.byref(h)) == 5
    assert L.defmm_batch_create(arr, rr, 0, defmm.C64, 0, ctypes.byref(h)) == 1
    o = serve.ServerOptions()
    L.defmm_server_default_options(ctypes.byref(o))
    assert (o.streams, o.max_batch_rhs, o.hbm_budget) == (4, 16, 4 << 30)
    assert L.defmm_server_create(arr, 1, defmm.C64, ctypes.byref(o), ctypes.byref(h)) == 5
    assert L.defmm_apply_ws(None, None, None, None, 1, defmm.C64, None) == 1


def _host_plan(X, Y=None, **kw):
    return defmm.Plan(X, Y, flags=defmm.PLAN_HOST_ONLY, **kw)


def test_argument_errors():
    X = W.points("sphere", 100, 1)
    for kw, frag in [(dict(order=1), "order"), (dict(order=9), "order"), (dict(leaf_size=0), "leaf"),
                     (dict(kappa=-1.0), "kappa"), (dict(fft_n=5, order=4), "fft_n"),
                     (dict(damping=-0.5), "damping"), (dict(damping=float("inf")), "damping"),
                     (dict(m2l_chunk_blocks=1), "m2l_chunk_blocks"), (dict(m2l_chunk_blocks=-2), "m2l_chunk_blocks")]:
        args = dict(kappa=1.0, order=4, leaf_size=8)
        args.update(kw)
        with pytest.raises(defmm.DefmmError) as e:
            _host_plan(X, **args)
        assert e.value.status == 1 and frag in str(e.value)
    bad = X.copy()
    bad[3, 1] = np.nan
    with pytest.raises(defmm.DefmmError):
        _host_plan(bad, kappa=1.0, order=4, leaf_size=8)
    pl = _host_plan(X, kappa=1.0, order=4, leaf_size=8)
    with pytest.raises(defmm.DefmmError) as e:
        pl.apply_raw(1, 1, 1, defmm.C64)
    assert e.value.status == 5


def test_tuning_values():
    """Apply-time tuning takes 0, 1, 2, 4 right-hand sides per M2L pass and rejects others."""
    pl = _host_plan(W.points("sphere", 300, 2), kappa=2.0, order=4, leaf_size=16)
    assert pl.tuning() == {"m2l_rhs_block": 0, "p2p_tc_min_rhs": 0, "m2l_members_per_block": 0,
                           "p2p_reduce_phase": 0}
    for v in (1, 2, 4, 0):
        pl.set_tuning(m2l_rhs_block=v, p2p_tc_min_rhs=v, m2l_members_per_block=v if v in (0, 4) else 8,
                      p2p_reduce_phase=v % 2)
        assert pl.tuning() == {"m2l_rhs_block": v, "p2p_tc_min_rhs": v,
                               "m2l_members_per_block": v if v in (0, 4) else 8, "p2p_reduce_phase": v % 2}
    with pytest.raises(defmm.DefmmError) as e:
        pl.set_tuning(p2p_reduce_phase=2)
    assert e.value.status == 1
    for v in (12, 14):
        pl.set_tuning(m2l_members_per_block=v)
        assert pl.tuning()["m2l_members_per_block"] == v
    for v in (2, 6, -4, 16):
        with pytest.raises(defmm.DefmmError) as e:
            pl.set_tuning(m2l_members_per_block=v)
        assert e.value.status == 1
    for v in (3, -1, 8):
        with pytest.raises(defmm.DefmmError) as e:
            pl.set_tuning(m2l_rhs_block=v)
        assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        pl.set_tuning(p2p_tc_min_rhs=-1)
    assert e.value.status == 1
    assert pl.tuning()["m2l_rhs_block"] == 0


def _oracle_tables(op):
    cells = np.stack([op.tt.level, op.tt.coords[:, 0], op.tt.coords[:, 1], op.tt.coords[:, 2],
                      op.tt.begin, op.tt.end, op.tt.parent], 1)
    m2l = sorted((t, s, u) for (t, s), u in zip(op.m2l_pairs, op.pair_dir))
    mult = [(c, u) for c in range(op.ts.ncell) for u in op.marks_s[c]]
    loc = [(c, u) for c in range(op.tt.ncell) for u in op.marks_t[c]]
    return cells, m2l, sorted(op.p2p_pairs), mult, loc


CASES = [
    ("sphere", 2000, None, 4.0, 4, 64),
    ("box", 4000, None, 16.0, 4, 20),
    ("ellipsoid", 3000, ("sphere", 2500), 30.0, 3, 16),
    ("cube", 2500, None, 0.0, 5, 10),
    ("sphere", 1500, None, 60.0, 6, 8),
]


@pytest.mark.parametrize("case", CASES)
def test_plan_tables_equal_oracle(case):
    """Tree, DTT pairs with best directions, and effective expansions are bit-identical."""
    kind, n, other, kappa, order, leaf = case
    X = W.points(kind, n, 3)
    Y = None if other is None else 0.5 * W.points(other[0], other[1], 4)
    pl = _host_plan(X, Y, kappa=kappa, order=order, leaf_size=leaf)
    op = oracle_fmm.make_plan(X, Y, kappa=kappa, order=order, leaf=leaf)
    cells, m2l, p2p, mult, loc = _oracle_tables(op)
    assert np.array_equal(pl.table("perm_t"), op.tt.perm)
    assert np.array_equal(pl.table("perm_s"), op.ts.perm)
    assert np.array_equal(pl.table("cells_t").reshape(-1, 7), cells)
    assert sorted(map(tuple, pl.table("m2l").reshape(-1, 3).tolist())) == [tuple(map(int, r)) for r in m2l]
    assert sorted(map(tuple, pl.table("p2p").reshape(-1, 2).tolist())) == [tuple(map(int, r)) for r in p2p]
    assert list(map(tuple, pl.table("mult").reshape(-1, 2).tolist())) == mult
    assert list(map(tuple, pl.table("local").reshape(-1, 2).tolist())) == loc
    info = pl.info()
    assert info["n_m2l_pairs"] == len(m2l) and info["n_p2p_pairs"] == len(p2p)
    assert info["deepest_hf"] == op.levels.l_hf
    assert info["n_spectra"] == len(op.spectra)


def _rows(a):
    """Rows of a 2-D integer array in lexicographic order."""
    a = np.asarray(a, dtype=np.int64)
    return a[np.lexsort(a.T[::-1])]


def test_plan_tables_equal_oracle_above_2_20_pairs(monkeypatch):
    """A plan of more than 2^20 M2L pairs (its chunks built by several threads): tree, DTT
    pairs with directions and effective expansions equal the oracle's (Sec. 4.2.1, Alg. 1-3)
    bit for bit, and the schedule and near-field tables are the same whether one, eight or
    sixteen threads build them."""
    X = W.points("sphere", 60000, 7)
    D = float(np.max(X.max(0) - X.min(0)))
    kw = dict(kappa=60.0 / D, order=4, leaf_size=32)
    monkeypatch.setenv("DEFMM_PLAN_THREADS", "8")
    pl = _host_plan(X, **kw)
    op = oracle_fmm.make_plan(X, None, kappa=kw["kappa"], order=4, leaf=32)
    m2l = np.array([(t, s, u) for (t, s), u in zip(op.m2l_pairs, op.pair_dir)], dtype=np.int64)
    assert len(m2l) > 1 << 20
    cells = np.stack([op.tt.level, op.tt.coords[:, 0], op.tt.coords[:, 1], op.tt.coords[:, 2],
                      op.tt.begin, op.tt.end, op.tt.parent], 1)
    assert np.array_equal(pl.table("perm_t"), op.tt.perm)
    assert np.array_equal(pl.table("cells_t").reshape(-1, 7), cells)
    assert np.array_equal(_rows(pl.table("m2l").reshape(-1, 3)), _rows(m2l))
    assert np.array_equal(_rows(pl.table("p2p").reshape(-1, 2)), _rows(np.array(op.p2p_pairs)))
    mult = np.array([(c, u) for c in range(op.ts.ncell) for u in op.marks_s[c]])
    loc = np.array([(c, u) for c in range(op.tt.ncell) for u in op.marks_t[c]])
    assert np.array_equal(pl.table("mult").reshape(-1, 2), mult)
    assert np.array_equal(pl.table("local").reshape(-1, 2), loc)
    names = ("grp_member_off", "grp_members", "grp_chunk_off", "chk_blk_off", "chk_nspec", "chk_blk",
             "chk_op_off", "chk_op", "mult", "local", "p2p_unit_leaf", "p2p_unit_off", "p2p_unit_ranges")
    threaded = {k: pl.table(k) for k in names}
    for nth in ("1", "16"):
        monkeypatch.setenv("DEFMM_PLAN_THREADS", nth)
        other = _host_plan(X, **kw)
        for k in names:
            assert np.array_equal(other.table(k), threaded[k]), (nth, k)


def test_degenerate_inputs_host_plan():
    one = np.array([[0.1, 0.2, 0.3]])
    pl = _host_plan(one, kappa=3.0, order=4, leaf_size=4)
    assert pl.info()["ncells_t"] == 1 and pl.info()["n_p2p_pairs"] == 1
    dup = np.repeat(np.array([[1.0, 2.0, 3.0]]), 10, axis=0)
    pl = _host_plan(dup, kappa=3.0, order=4, leaf_size=3)
    assert pl.info()["nlevels"] == 22


def test_autotune_argument_errors():
    """defmm_plan_autotune validates its arguments before touching a GPU."""
    X = W.points("sphere", 100, 1)
    for kw in (dict(leaf_range=(0, 64)), dict(leaf_range=(64, 32)), dict(nrhs=0), dict(reps=0)):
        with pytest.raises(defmm.DefmmError) as e:
            defmm.autotune(X, kappa=1.0, order=4, **kw)
        assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        defmm.autotune(X, kappa=1.0, order=1)
    assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        defmm.autotune(X, kappa=1.0, order=4, flags=defmm.PLAN_HOST_ONLY)
    assert e.value.status == 5


def test_gmres_argument_errors():
    """defmm_gmres validates its arguments before touching a GPU."""
    import ctypes
    L = defmm.lib()
    pl = _host_plan(W.points("sphere", 200, 1), kappa=1.0, order=4, leaf_size=8)
    o = defmm.GmresOptions()
    L.defmm_default_gmres_options(ctypes.byref(o))
    assert (o.shift_re, o.shift_im, o.tol, o.restart, o.max_iter) == (1.0, 0.0, 1e-6, 30, 200)
    dummy = ctypes.c_void_p(16)
    assert L.defmm_gmres(None, dummy, dummy, defmm.C64, ctypes.byref(o), None, None) == 1
    assert L.defmm_gmres(pl.handle, None, dummy, defmm.C64, ctypes.byref(o), None, None) == 1
    assert L.defmm_gmres(pl.handle, dummy, dummy, 7, ctypes.byref(o), None, None) == 5
    for field, bad in (("restart", 0), ("max_iter", -1), ("tol", -1.0)):
        b = defmm.GmresOptions()
        L.defmm_default_gmres_options(ctypes.byref(b))
        setattr(b, field, bad)
        assert L.defmm_gmres(pl.handle, dummy, dummy, defmm.C64, ctypes.byref(b), None, None) == 1
    assert L.defmm_gmres(pl.handle, dummy, dummy, defmm.C64, ctypes.byref(o), None, None) == 5   # host-only
    two = _host_plan(W.points("sphere", 200, 1), W.points("sphere", 150, 2), kappa=1.0, order=4, leaf_size=8)
    # a non-square operator is refused (checked after the host-only test)
    assert L.defmm_gmres(two.handle, dummy, dummy, defmm.C64, ctypes.byref(o), None, None) == 5


def test_bench_finds_the_row_kernel_source():
    """bench.py keys the recorded M2L DRAM traffic to the row kernel's source text."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    h = bench.m2l_rows_source_sha()
    assert len(h) == 16 and int(h, 16) >= 0


@pytest.mark.parametrize("kind,n,order", [("sphere", 3000, 4), ("box", 4000, 5)])
def test_shard_ranges_partition_the_targets(kind, n, order):
    """Shard ranges are contiguous, cover every target once, start on leaf boundaries,
    and hold comparable work (here: no shard of 2 or 3 is empty or above 2/3 of the points)."""
    X = W.points(kind, n, 81)
    pl = _host_plan(X, kappa=30.0, order=order, leaf_size=24)
    cells = pl.table("cells_t").reshape(-1, 7)            # level, ix, iy, iz, begin, end, parent
    parents = set(cells[:, 6].tolist())
    leaf_begins = {int(c[4]) for i, c in enumerate(cells) if i not in parents}
    for S in (1, 2, 3, 5):
        ranges = [pl.shard_range(S, s) for s in range(S)]
        pos = 0
        for first, count in ranges:
            assert first == pos and count >= 0
            assert first in leaf_begins or first == n
            pos += count
        assert pos == n
        if S in (2, 3):
            assert all(0 < c < 2 * n / 3 for _, c in ranges)
    for bad in ((0, 0), (2, 2), (2, -1)):
        with pytest.raises(defmm.DefmmError) as e:
            pl.shard_range(*bad)
        assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        pl.set_shard(2, 0)
    assert e.value.status == 5


def test_union_plan_tables_are_the_concatenation():
    """A union of three geometries: its host tables are each geometry's own, offset
    (points, cells, global levels), and its counts are the sums."""
    geos = [W.points("sphere", 1500, 111), W.points("box", 2200, 112) * 0.7, W.points("ellipsoid", 900, 113)]
    kappas = [12.0, 30.0, 5.0]
    singles = [_host_plan(X, kappa=k, order=4, leaf_size=24) for X, k in zip(geos, kappas)]
    uni = defmm.union_plan(geos, kappas, order=4, leaf_size=24, flags=defmm.PLAN_HOST_ONLY)
    assert uni.nx == sum(len(X) for X in geos)
    perm, cells = uni.table("perm_t"), uni.table("cells_t").reshape(-1, 7)
    m2l, p2p = uni.table("m2l").reshape(-1, 3), uni.table("p2p").reshape(-1, 2)
    pb = cb = lb = mb = pp = 0
    for X, sp in zip(geos, singles):
        sperm, scells = sp.table("perm_t"), sp.table("cells_t").reshape(-1, 7)
        assert np.array_equal(perm[pb:pb + len(X)], sperm + pb)
        uc = cells[cb:cb + len(scells)]
        assert np.array_equal(uc[:, 0], scells[:, 0] + lb)                       # global level ids
        assert np.array_equal(uc[:, 1:4], scells[:, 1:4])
        assert np.array_equal(uc[:, 4:6], scells[:, 4:6] + pb)
        assert np.array_equal(uc[:, 6], np.where(scells[:, 6] >= 0, scells[:, 6] + cb, scells[:, 6]))
        sm = sp.table("m2l").reshape(-1, 3)
        assert np.array_equal(m2l[mb:mb + len(sm)], sm + np.array([cb, cb, 0]))
        s2 = sp.table("p2p").reshape(-1, 2)
        assert np.array_equal(p2p[pp:pp + len(s2)], s2 + cb)
        pb += len(X); cb += len(scells); mb += len(sm); pp += len(s2)
        lb += int(scells[:, 0].max()) + 1
    iu = uni.info()
    for key in ("n_m2l_pairs", "n_p2p_pairs", "n_multipole", "n_local", "n_fourier", "n_spectra", "p2p_interactions"):
        assert iu[key] == sum(sp.info()[key] for sp in singles), key
    with pytest.raises(defmm.DefmmError) as e:
        defmm.union_plan(geos, [1.0, -2.0, 1.0], flags=defmm.PLAN_HOST_ONLY)
    assert e.value.status == 1


def test_plan_file_round_trip(tmp_path):
    """A plan written by save() and read by load() has the same tables and counts;
    truncated, foreign and missing files are argument errors."""
    X = W.points("sphere", 1800, 121)
    Y = W.points("box", 1300, 122) * 0.8
    for src in (None, Y):
        pl = _host_plan(X, src, kappa=9.0, order=5, leaf_size=20, damping=0.25)
        path = tmp_path / ("same.plan" if src is None else "xy.plan")
        pl.save(path)
        back = defmm.Plan.load(path, flags=defmm.PLAN_HOST_ONLY)
        a, b = pl.info(), back.info()
        for key in a:
            if key not in ("plan_bytes", "workspace_bytes") and not key.startswith("plan_"):
                assert a[key] == b[key], key
        for name in ("perm_t", "perm_s", "cells_t", "cells_s", "m2l", "p2p", "mult", "local"):
            assert np.array_equal(pl.table(name), back.table(name)), name
        # the same plan always gives the same bytes (no padding or other indeterminate bytes)
        again = _host_plan(X, src, kappa=9.0, order=5, leaf_size=20, damping=0.25)
        again.save(tmp_path / "again.plan")
        back.save(tmp_path / "back.plan")
        assert path.read_bytes() == (tmp_path / "again.plan").read_bytes() == (tmp_path / "back.plan").read_bytes()
    geos = [W.points("sphere", 700, 123), W.points("ellipsoid", 500, 124)]
    uni = defmm.union_plan(geos, [4.0, 7.0], order=4, leaf_size=24, flags=defmm.PLAN_HOST_ONLY)
    uni.save(tmp_path / "u.plan")
    ub = defmm.Plan.load(tmp_path / "u.plan", flags=defmm.PLAN_HOST_ONLY)
    assert ub.nx == ub.ny == 1200
    for name in ("perm_t", "cells_t", "m2l", "p2p"):
        assert np.array_equal(uni.table(name), ub.table(name)), name
    raw = (tmp_path / "xy.plan").read_bytes()
    flipped = bytearray(raw)
    flipped[len(raw) // 3] ^= 0x10
    huge = bytearray(raw)
    ylen = len(raw) - 8 - 3 * len(Y) * 8 - 8            # Y's length field, before Y and the checksum
    assert int.from_bytes(raw[ylen:ylen + 8], "little") == 3 * len(Y)
    huge[ylen:ylen + 8] = (1 << 62).to_bytes(8, "little")
    for bad, content in (("short.plan", raw[: len(raw) // 2]), ("foreign.plan", b"NOTAPLAN" + raw[8:]),
                         ("empty.plan", b""), ("flipped.plan", bytes(flipped)), ("huge.plan", bytes(huge)),
                         ("long.plan", raw + b"\0")):
        (tmp_path / bad).write_bytes(content)
        with pytest.raises(defmm.DefmmError) as e:
            defmm.Plan.load(tmp_path / bad, flags=defmm.PLAN_HOST_ONLY)
        assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        defmm.Plan.load(tmp_path / "missing.plan", flags=defmm.PLAN_HOST_ONLY)
    assert e.value.status == 1
    with pytest.raises(defmm.DefmmError) as e:
        pl.save(tmp_path / "no_such_dir" / "x.plan")
    assert e.value.status == 1
    # saving over an existing plan file replaces it whole; no temporary file stays behind
    uni.save(tmp_path / "xy.plan")
    assert defmm.Plan.load(tmp_path / "xy.plan", flags=defmm.PLAN_HOST_ONLY).nx == 1200
    assert not [f for f in tmp_path.iterdir() if ".tmp" in f.name]


@pytest.mark.parametrize("kind,n,kd,order", [("sphere", 4000, 40.0, 4), ("box", 4000, 8.0, 5), ("ellipsoid", 3000, 0.0, 4)])
def test_m2l_schedule_covers_every_pair_once(kind, n, kd, order):
    """The M2L work schedule (groups of sibling targets, chunks of staged blocks, pair
    ops) names every M2L pair of the traversal exactly once: the op's member is the
    pair's target expansion, its staged multipole the source's expansion in the same
    direction, and its staged spectrum the canonical one of the same level whose
    offset is the pair's offset t - s under the op's symmetry (Sec. 4.3)."""
    X = W.points(kind, n, 131)
    D = float(np.max(X.max(0) - X.min(0)))
    pl = _host_plan(X, kappa=kd / D, order=order, leaf_size=24)
    t = {k: pl.table(k) for k in ("m2l", "mult", "local", "m2f_list", "spectra", "grp_member_off", "grp_members",
                                  "grp_chunk_off", "chk_blk_off", "chk_nspec", "chk_blk", "chk_op_off", "chk_op",
                                  "cells_t")}
    m2l, mult, loc = t["m2l"].reshape(-1, 3), t["mult"].reshape(-1, 2), t["local"].reshape(-1, 2)
    cells, spec = t["cells_t"].reshape(-1, 7), t["spectra"].reshape(-1, 4)
    goff, gch, boff, ooff = t["grp_member_off"], t["grp_chunk_off"], t["chk_blk_off"], t["chk_op_off"].reshape(-1, 9)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]     # sigma of each code >> 3
    assert len(t["chk_op"]) == len(m2l) == pl.info()["n_m2l_pairs"] > 0
    seen = {}
    for g in range(len(goff) - 1):
        nm = goff[g + 1] - goff[g]
        assert 1 <= nm <= 8
        for ch in range(gch[g], gch[g + 1]):
            assert np.all(np.diff(ooff[ch]) >= 0) and np.all(ooff[ch][nm:] == ooff[ch][nm])
            nb, ns = boff[ch + 1] - boff[ch], t["chk_nspec"][ch]
            for m in range(nm):
                tc, td = loc[t["grp_members"][goff[g] + m]]
                for op in t["chk_op"][ooff[ch][m]:ooff[ch][m + 1]]:
                    bs, bm, code = op & 255, (op >> 8) & 255, op >> 16
                    assert bs < ns <= bm < nb
                    sc, sd = mult[t["m2f_list"][t["chk_blk"][boff[ch] + bm]]]
                    lev, kbar = spec[t["chk_blk"][boff[ch] + bs], 0], spec[t["chk_blk"][boff[ch] + bs], 1:]
                    k = cells[tc, 1:4] - cells[sc, 1:4]
                    sigma = perms[code >> 3]
                    for a in range(3):
                        assert kbar[sigma[a]] == (-k[a] if (code >> a) & 1 else k[a])
                    assert lev == cells[tc, 0] and sd == td
                    assert (tc, sc) not in seen
                    seen[(int(tc), int(sc))] = int(td)
    assert seen == {(int(a), int(b)): int(d) for a, b, d in m2l}     # every pair once, in its direction


def test_m2l_schedule_of_a_large_plan():
    """The same schedule checks, vectorised, on a plan of more than 2^20 M2L pairs (whose
    chunks are built by several threads over slices of the group order, then concatenated):
    op ranges are contiguous, every op names blocks of its own chunk, and the ops cover
    every M2L pair once with the right expansions, level and symmetry."""
    X = W.points("sphere", 100000, 7)
    D = float(np.max(X.max(0) - X.min(0)))
    pl = _host_plan(X, kappa=60.0 / D, order=4, leaf_size=32)
    t = {k: pl.table(k) for k in ("m2l", "mult", "local", "m2f_list", "spectra", "grp_member_off", "grp_members",
                                  "grp_chunk_off", "chk_blk_off", "chk_nspec", "chk_blk", "chk_op_off", "chk_op",
                                  "cells_t")}
    m2l, mult, loc = t["m2l"].reshape(-1, 3), t["mult"].reshape(-1, 2), t["local"].reshape(-1, 2)
    cells, spec = t["cells_t"].reshape(-1, 7), t["spectra"].reshape(-1, 4)
    goff, gch, boff, nspec = t["grp_member_off"], t["grp_chunk_off"], t["chk_blk_off"], t["chk_nspec"]
    ooff, ops = t["chk_op_off"].reshape(-1, 9), t["chk_op"]
    assert len(m2l) > 1 << 20
    nch = len(nspec)
    assert gch[0] == 0 and gch[-1] == nch and len(boff) == nch + 1 and len(ooff) == nch
    assert ooff[0, 0] == 0 and ooff[-1, 8] == len(ops) and np.all(ooff[1:, 0] == ooff[:-1, 8])
    counts = np.diff(ooff, axis=1)
    assert np.all(counts >= 0)
    chunk = np.repeat(np.arange(nch), ooff[:, 8] - ooff[:, 0])
    member = np.repeat(np.tile(np.arange(8), nch), counts.ravel())
    group = np.repeat(np.arange(len(goff) - 1), np.diff(gch))[chunk]
    assert np.all(member < (goff[group + 1] - goff[group]))
    te = t["grp_members"][goff[group] + member]
    bs, bm, code = ops & 255, (ops >> 8) & 255, ops >> 16
    assert np.all(bs < nspec[chunk]) and np.all(nspec[chunk] <= bm) and np.all(bm < (boff[chunk + 1] - boff[chunk]))
    sid, slot = t["chk_blk"][boff[chunk] + bs], t["chk_blk"][boff[chunk] + bm]
    tc, td = loc[te, 0], loc[te, 1]
    sc, sd = mult[t["m2f_list"][slot], 0], mult[t["m2f_list"][slot], 1]
    assert np.all(td == sd) and np.all(spec[sid, 0] == cells[tc, 0])
    k = cells[tc, 1:4] - cells[sc, 1:4]
    perms = np.array([(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)])
    sigma = perms[code >> 3]
    for a in range(3):
        sign = np.where((code >> a) & 1, -1, 1)
        assert np.all(spec[sid, 1 + sigma[:, a]] == sign * k[:, a])
    got = np.lexsort((td, sc, tc))
    want = np.lexsort((m2l[:, 2], m2l[:, 1], m2l[:, 0]))
    assert np.array_equal(np.stack([tc, sc, td], 1)[got], m2l[want])


def test_radial_power_option():
    """radial_power selects the kernel exp((i kappa - lambda) r)/(4 pi r^P), P = 1 or 2."""
    X = W.points("sphere", 300, 2)
    assert defmm.default_options().radial_power == 1
    _host_plan(X, kappa=2.0, order=4, leaf_size=16, radial_power=2)
    for bad in (0, 3, -1):
        with pytest.raises(defmm.DefmmError) as e:
            _host_plan(X, kappa=2.0, order=4, leaf_size=16, radial_power=bad)
        assert e.value.status == 1


def test_slice_exchange_argument_checks():
    """defmm_apply_slice / defmm_assemble_slices on the host: NULL pointers and
    nrhs < 1 are argument errors, starts must run from 0 to nx without decreasing
    and fit ld, and a host-only plan cannot apply (no GPU involved)."""
    import ctypes
    X = W.points("sphere", 400, 7)
    pl = _host_plan(X, kappa=3.0, order=4, leaf_size=16)
    L = defmm.lib()
    h = pl._h
    i64 = ctypes.c_int64

    def starts(*v):
        return (i64 * len(v))(*v)

    assert L.defmm_apply_slice(h, None, None, 10, 1, defmm.C64, None) == 1
    assert L.defmm_apply_slice(h, ctypes.c_void_p(8), ctypes.c_void_p(8), 400, 0, defmm.C64, None) == 1
    assert L.defmm_apply_slice(h, ctypes.c_void_p(8), ctypes.c_void_p(8), 400, 1, 7, None) == 5
    assert L.defmm_apply_slice(h, ctypes.c_void_p(8), ctypes.c_void_p(8), 400, 1, defmm.C64, None) == 5
    dummy = ctypes.c_void_p(8)
    assert L.defmm_assemble_slices(h, 2, None, dummy, 400, dummy, 1, defmm.C64, None) == 1
    assert L.defmm_assemble_slices(h, 2, starts(0, 200, 400), None, 400, dummy, 1, defmm.C64, None) == 1
    assert L.defmm_assemble_slices(h, 0, starts(0, 400), dummy, 400, dummy, 1, defmm.C64, None) == 1
    assert L.defmm_assemble_slices(h, 2, starts(0, 200, 400), dummy, 400, dummy, 1, defmm.C128, None) == 5
