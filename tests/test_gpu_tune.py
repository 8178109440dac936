"""GPU tests of the autotuner (defmm_plan_autotune): the tuned plan is one of
the candidates, equals an untuned plan built with the same choice bit for bit,
stays within the order's accuracy against the direct sum, and a second call
with the same tune cache rebuilds the same choice without timing."""
import numpy as np
import pytest
import torch

from oracle import direct
from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_choice_cache_and_results(tmp_path):
    n, R = 20000, 4
    X = W.points("sphere", n, 41)
    kappa = 32.0 / 2.0
    q = W.charges(n, 42, nrhs=R)
    qd = torch.from_numpy(q).to("cuda").to(torch.complex64)
    cache = tmp_path / "tune.txt"
    plan, choice = defmm.autotune(X, kappa=kappa, order=4, nrhs=R, leaf_range=(24, 64), reps=3,
                                  cache_path=str(cache))
    assert choice["from_cache"] == 0
    assert choice["leaf_size"] in (24, 32, 48, 64)
    assert choice["fft_n"] in (0, 8)
    assert choice["m2l_rhs_block"] in (1, 2, 4)
    # per leaf: N = 7 times 1 column per pass with 4 block splits, 2 and 4 columns with 2;
    # N = 8 times 3 column counts with 2
    assert choice["candidates"] == 4 * ((4 + 2 + 2) + 3 * 2)
    assert choice["m2l_members_per_block"] in (4, 8, 12, 14)
    assert choice["ms"] > 0
    assert plan.tuning()["m2l_rhs_block"] == choice["m2l_rhs_block"]
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("defmm-tune ")

    tuned = plan.apply(qd).cpu().numpy()
    ref_plan = defmm.Plan(X, kappa=kappa, order=4, leaf_size=choice["leaf_size"], fft_n=choice["fft_n"])
    assert np.array_equal(ref_plan.apply(qd).cpu().numpy(), tuned)

    idx = np.random.default_rng(5).choice(n, 300, replace=False)
    exact = direct.direct_sum(X[idx], X, q, kappa, direct.eps_self(X))
    err = np.linalg.norm(tuned[idx] - exact) / np.linalg.norm(exact)
    assert err <= 3e-3, err

    again, c2 = defmm.autotune(X, kappa=kappa, order=4, nrhs=R, leaf_range=(24, 64), reps=3,
                               cache_path=str(cache))
    assert c2["from_cache"] == 1 and c2["candidates"] == 0
    for k in ("leaf_size", "fft_n", "m2l_rhs_block", "m2l_members_per_block"):
        assert c2[k] == choice[k]
    assert np.array_equal(again.apply(qd).cpu().numpy(), tuned)
    assert len(cache.read_text().splitlines()) == 1

    # another nrhs is another key: tuned again, a second line appended
    _, c3 = defmm.autotune(X, kappa=kappa, order=4, nrhs=1, leaf_range=(48, 64), reps=2,
                           tune_fft_n=False, cache_path=str(cache))
    assert c3["from_cache"] == 0 and c3["candidates"] == 2 * 4 and c3["m2l_rhs_block"] == 0
    assert c3["p2p_tensor_cores"] == 0
    assert len(cache.read_text().splitlines()) == 2

    # 8 columns: the tensor-core near field is a candidate too
    p8, c4 = defmm.autotune(X, kappa=kappa, order=4, nrhs=8, leaf_range=(64, 64), reps=2,
                            tune_fft_n=False, cache_path=str(cache))
    assert c4["candidates"] == 2 * (4 + 2 + 2) and c4["p2p_tensor_cores"] in (0, 1)
    assert p8.tuning()["p2p_tc_min_rhs"] == (1 if c4["p2p_tensor_cores"] else 0)


def test_autotune_union_plan(tmp_path):
    """A union of uneven geometries tuned as one plan: the choice is a candidate,
    the tuned union equals an untuned union with that choice bit for bit, and the
    cache rebuilds it without timing."""
    geos = [W.points("sphere", 9000, 141), W.points("ellipsoid", 4000, 142), W.points("box", 6000, 143)]
    kappas = [12.0, 30.0, 20.0]
    total = sum(len(g) for g in geos)
    q = torch.from_numpy(W.charges(total, 144)[:, 0]).to("cuda").to(torch.complex64)
    cache = tmp_path / "tune_u.txt"
    plan, choice = defmm.autotune_union(geos, kappas, order=4, leaf_range=(32, 64), reps=3, cache_path=str(cache))
    assert choice["from_cache"] == 0 and choice["candidates"] > 0
    assert choice["leaf_size"] in (32, 48, 64) and choice["fft_n"] in (0, 8)
    assert plan.nx == total
    tuned = plan.apply(q).cpu().numpy()
    ref = defmm.union_plan(geos, kappas, order=4, leaf_size=choice["leaf_size"], fft_n=choice["fft_n"])
    ref.set_tuning(m2l_members_per_block=choice["m2l_members_per_block"])
    assert np.array_equal(ref.apply(q).cpu().numpy(), tuned)
    again, c2 = defmm.autotune_union(geos, kappas, order=4, leaf_range=(32, 64), reps=3, cache_path=str(cache))
    assert c2["from_cache"] == 1 and c2["leaf_size"] == choice["leaf_size"]
    assert np.array_equal(again.apply(q).cpu().numpy(), tuned)
