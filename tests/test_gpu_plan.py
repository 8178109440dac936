"""The plan's front end built on the device (Morton keys and their radix sort,
the Ncrit octree level by level, the breadth-first dual tree traversal, the
best directions and the marks of Alg. 2) against the host construction, table
for table: the host construction is itself checked against the oracle's tree,
traversal and blank passes (tests/test_abi.py), so equal tables tie the device
path to the oracle too."""
import numpy as np
import pytest

from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu

TABLES = ("perm_t", "perm_s", "cells_t", "cells_s", "m2l", "p2p", "mult", "local", "m2f_list", "spectra",
          "grp_member_off", "grp_members", "grp_chunk_off", "chk_blk_off", "chk_nspec", "chk_blk", "chk_op_off",
          "chk_op", "p2p_leaf", "p2p_unit_leaf", "p2p_unit_off", "p2p_unit_ranges")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _same_tables(dev, host):
    for name in TABLES:
        assert np.array_equal(dev.table(name), host.table(name)), name
    a, b = dev.info(), host.info()
    for key in ("nlevels", "deepest_hf", "ncells_t", "ncells_s", "n_m2l_pairs", "n_p2p_pairs", "n_multipole",
                "n_local", "n_fourier", "n_spectra", "p2p_interactions"):
        assert a[key] == b[key], key
    assert a["plan_front_device_ms"] > 0 and b["plan_front_device_ms"] == 0


CASES = [
    # kind, n, sources, kappa*D, order, leaf
    ("sphere", 2000, None, 8.0, 4, 64),
    ("box", 4000, None, 16.0, 4, 20),
    ("ellipsoid", 3000, ("sphere", 2500), 30.0, 3, 16),
    ("cube", 2500, None, 0.0, 5, 10),
    ("sphere", 1500, None, 60.0, 6, 8),
    ("sphere", 6000, None, 200.0, 4, 32),
    ("box", 30000, None, 64.0, 5, 64),
]


@pytest.mark.parametrize("case", CASES)
def test_device_front_equals_host(case):
    kind, n, other, kd, order, leaf = case
    X = W.points(kind, n, 3)
    Y = None if other is None else 0.5 * W.points(other[0], other[1], 4)
    P = X if Y is None else np.vstack([X, Y])
    kappa = kd / float(np.max(P.max(0) - P.min(0)))
    dev = defmm.Plan(X, Y, kappa=kappa, order=order, leaf_size=leaf)
    host = defmm.Plan(X, Y, kappa=kappa, order=order, leaf_size=leaf, flags=defmm.PLAN_HOST_ONLY)
    _same_tables(dev, host)
    dev.close()


def test_device_front_degenerate_and_deep():
    """One point; coincident points (the tree goes down to level 21); a tight
    cluster beside a far point (a long chain of one-child cells)."""
    one = np.array([[0.1, 0.2, 0.3]])
    dup = np.repeat(np.array([[1.0, 2.0, 3.0]]), 40, axis=0)
    rng = np.random.default_rng(5)
    cluster = np.vstack([1e-9 * rng.standard_normal((300, 3)), [[1.0, 1.0, 1.0]]])
    for X, kappa, leaf in ((one, 3.0, 4), (dup, 3.0, 3), (cluster, 2.0, 8)):
        dev = defmm.Plan(X, kappa=kappa, order=4, leaf_size=leaf)
        host = defmm.Plan(X, kappa=kappa, order=4, leaf_size=leaf, flags=defmm.PLAN_HOST_ONLY)
        _same_tables(dev, host)


def test_device_front_union_and_large():
    """A union of geometries, and a plan above 2^20 M2L pairs."""
    geos = [W.points("sphere", 7000, 123), W.points("ellipsoid", 5000, 124), W.points("box", 6000, 125)]
    dev = defmm.union_plan(geos, [20.0, 35.0, 50.0], order=4, leaf_size=24)
    host = defmm.union_plan(geos, [20.0, 35.0, 50.0], order=4, leaf_size=24, flags=defmm.PLAN_HOST_ONLY)
    for name in TABLES:
        assert np.array_equal(dev.table(name), host.table(name)), name
    X = W.points("sphere", 60000, 7)
    D = float(np.max(X.max(0) - X.min(0)))
    dev = defmm.Plan(X, kappa=60.0 / D, order=4, leaf_size=32)
    host = defmm.Plan(X, kappa=60.0 / D, order=4, leaf_size=32, flags=defmm.PLAN_HOST_ONLY)
    assert dev.info()["n_m2l_pairs"] > 1 << 20
    _same_tables(dev, host)
