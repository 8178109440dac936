"""GPU tests of the serving layer (include/defmm_serve.h): caller workspaces,
graph-replayed batches over uneven geometries, and the request server with
continuous batching.  Every path runs the kernels of defmm_apply, so results
are compared with defmm_apply (bit for bit where the same kernels run with the
same right-hand-side blocking) and, on small cases, with the oracle."""
import threading

import numpy as np
import pytest

from oracle import fmm as oracle_fmm
from paper_2202_04894_gb300 import defmm, serve, workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL64 = 1e-5
MIX_TOL = 1e-6       # a request's result alone vs inside a batch with other requests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _geometries(n, seed, nmin=3000, nmax=20000):
    """Uneven geometries: spheres, ellipsoids, box surfaces; log-uniform sizes and kappa*D."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = ("sphere", "ellipsoid", "box")[i % 3]
        npts = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        kd = float(np.exp(rng.uniform(np.log(16), np.log(64))))
        X = W.points(kind, npts, 100 + i)
        kappa = kd / float(np.max(X.max(0) - X.min(0)))
        out.append((X, kappa))
    return out


@pytest.fixture(scope="module")
def plans():
    return [defmm.Plan(X, kappa=k, order=4, leaf_size=64) for X, k in _geometries(6, 5)]


def _dev(q, dtype):
    return torch.from_numpy(np.ascontiguousarray(q)).to("cuda").to(dtype)


def test_workspace_apply_equals_apply(plans):
    plan = plans[0]
    q = W.charges(plan.ny, 7, nrhs=3)
    for dt in (torch.complex64, torch.complex128):
        ref = plan.apply(_dev(q, dt)).cpu().numpy()
        ws = serve.Workspace(plan, 3, dt)
        got = ws.apply(_dev(q, dt)).cpu().numpy()
        assert np.array_equal(got, ref)
        one = ws.apply(_dev(q[:, 1], dt)).cpu().numpy()          # fewer columns than the capacity
        assert np.array_equal(one, plan.apply(_dev(q[:, 1], dt)).cpu().numpy())
        ws.close()
    assert serve.workspace_bytes(plan, 3, torch.complex64) < serve.workspace_bytes(plan, 3, torch.complex128)


def test_workspaces_run_concurrently_on_one_plan(plans):
    """Two workspaces, two streams, two threads, one plan: both results exact."""
    plan = plans[1]
    qa, qb = W.charges(plan.ny, 8), W.charges(plan.ny, 9)
    ra = plan.apply(_dev(qa, torch.complex64)).cpu().numpy()
    rb = plan.apply(_dev(qb, torch.complex64)).cpu().numpy()
    out = {}

    def run(name, q):
        s = torch.cuda.Stream()
        ws = serve.Workspace(plan, 1, torch.complex64)
        with torch.cuda.stream(s):
            qd = _dev(q, torch.complex64)
            res = [ws.apply(qd, stream=s) for _ in range(5)]
        s.synchronize()
        out[name] = [r.cpu().numpy() for r in res]
        ws.close()

    ts = [threading.Thread(target=run, args=("a", qa)), threading.Thread(target=run, args=("b", qb))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert all(np.array_equal(r, ra) for r in out["a"])
    assert all(np.array_equal(r, rb) for r in out["b"])


def test_batch_graph_equals_individual_applies(plans):
    """Six uneven geometries with 1-3 right-hand sides each, replayed as one CUDA graph."""
    nrhs = [1, 2, 1, 3, 1, 2]
    for dt in (torch.complex64, torch.complex128):
        b = serve.Batch(plans, nrhs, dt, branches=3)
        for rep in range(2):
            qs = [W.charges(p.ny, 40 + 7 * rep + i, nrhs=r) for i, (p, r) in enumerate(zip(plans, nrhs))]
            got = b.apply([_dev(q, dt) for q in qs])
            torch.cuda.synchronize()
            for p, q, g in zip(plans, qs, got):
                ref = p.apply(_dev(q, dt))
                assert torch.equal(g, ref)
        info = b.info()
        per = sum(p.info()["launches_per_apply"] for p in plans)
        assert info["kernel_launches"] == per and info["graph_nodes"] >= per
        b.close()


def test_batch_against_oracle():
    geos = _geometries(3, 11, nmin=1500, nmax=2500)
    plans = [defmm.Plan(X, kappa=k, order=4, leaf_size=32) for X, k in geos]
    b = serve.Batch(plans, [1, 2, 1], torch.complex64)
    qs = [W.charges(len(X), 60 + i, nrhs=r) for i, ((X, _), r) in enumerate(zip(geos, [1, 2, 1]))]
    got = b.apply([_dev(q, torch.complex64) for q in qs])
    for (X, k), q, g in zip(geos, qs, got):
        ref = oracle_fmm.fmm(X, q, k, order=4, leaf=32)
        assert _rel(g.cpu().numpy().reshape(ref.shape), ref) <= TOL64


def _requests(plans, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        g = int(rng.integers(len(plans)))
        R = int(rng.integers(1, 5))
        reqs.append((g, W.charges(plans[g].ny, 1000 + i, nrhs=R).astype(np.complex64)))
    return reqs


def test_server_results_alone_equal_results_in_the_mix(plans):
    """Each request served alone (one at a time) equals the same request served
    while others are in flight and merged into its batch."""
    reqs = _requests(plans, 40, 3)
    alone = []
    with_one = serve.Server(plans, torch.complex64, streams=1, max_batch_rhs=16)
    for g, q in reqs:
        t = with_one.submit(g, q)
        p, _ = with_one.wait(t)
        alone.append(p.numpy().copy())
    st1 = with_one.stats()
    with_one.close()
    assert st1["batches"] == len(reqs) and st1["max_batch_requests"] == 1

    srv = serve.Server(plans, torch.complex64, streams=4, max_batch_rhs=16)
    tickets = [srv.submit(g, q) for g, q in reqs]
    mixed, lat = [], []
    for t in tickets:
        p, l = srv.wait(t)
        mixed.append(p.numpy().copy())
        lat.append(l)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["batches"] < len(reqs)      # requests were merged
    assert st["max_batch_requests"] >= 2 and st["peak_arena_bytes"] <= st["arena_bytes"]
    worst, exact = 0.0, 0
    for (g, q), a, m in zip(reqs, alone, mixed):
        worst = max(worst, _rel(m, a))
        exact += int(np.array_equal(m, a))
        ref = plans[g].apply(_dev(q, torch.complex64)).cpu().numpy().reshape(a.shape)
        assert np.array_equal(a, ref)                 # alone = defmm_apply of that request
    print("server: %d requests in %d batches, worst alone-vs-mix rel %.2e, %d bitwise equal, p50 %.2f ms"
          % (len(reqs), st["batches"], worst, exact, float(np.median(lat))))
    assert worst <= MIX_TOL
    assert all(l > 0 for l in lat)


def test_server_against_oracle():
    geos = _geometries(2, 13, nmin=1500, nmax=2500)
    plans = [defmm.Plan(X, kappa=k, order=4, leaf_size=32) for X, k in geos]
    srv = serve.Server(plans, torch.complex128, streams=2)
    qs = [W.charges(len(X), 70 + i, nrhs=2) for i, (X, _) in enumerate(geos)]
    ts = [srv.submit(i, q) for i, q in enumerate(qs)]
    for (X, k), q, t in zip(geos, qs, ts):
        p, _ = srv.wait(t)
        ref = oracle_fmm.fmm(X, q, k, order=4, leaf=32)
        assert _rel(p.numpy(), ref) <= 1e-12
    srv.close()


def test_server_admission_by_memory_budget(plans):
    """An arena that holds one batch at a time still completes every request, in
    order of admission; a request that can never fit is refused at submit."""
    need = max(serve.workspace_bytes(p, 4, torch.complex64) + 8 * 4 * (p.nx + p.ny) for p in plans)
    srv = serve.Server(plans, torch.complex64, streams=4, max_batch_rhs=4, hbm_budget=need + 4096)
    reqs = _requests(plans, 12, 4)
    ts = [srv.submit(g, q) for g, q in reqs]
    for (g, q), t in zip(reqs, ts):
        p, _ = srv.wait(t)
        ref = plans[g].apply(_dev(q, torch.complex64)).cpu().numpy().reshape(p.shape)
        assert _rel(p.numpy(), ref) <= MIX_TOL
    st = srv.stats()
    assert st["completed"] == 12 and st["peak_arena_bytes"] <= st["arena_bytes"]
    with pytest.raises(defmm.DefmmError) as e:
        srv.submit(0, W.charges(plans[0].ny, 1, nrhs=64).astype(np.complex64))
    assert e.value.status == 5
    srv.close()


def test_server_wait_timeout_and_unknown_ticket(plans):
    srv = serve.Server(plans[:1], torch.complex64, streams=1)
    with pytest.raises(defmm.DefmmError) as e:
        srv.wait(12345, timeout_ms=10)
    assert e.value.status == 1
    t = srv.submit(0, W.charges(plans[0].ny, 2).astype(np.complex64))
    p, lat = srv.wait(t, timeout_ms=60000)
    assert lat > 0 and p.shape == (plans[0].nx, 1)
    srv.close()
