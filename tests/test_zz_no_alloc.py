"""defmm_apply_noalloc: the application phase for callers that cannot allocate
device memory when they apply the operator (inside a CUDA graph capture, or
when a pool owned by another component holds the device memory).

Its scratch lives in a fixed 64 MiB array inside the library, so its results
must equal defmm_apply's on problems that fit, stay equal on a second call
that finds the previous call's data in that array, and problems that do not
fit must be refused with a clear message.  This file is collected last so a
failure here does not hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest

from paper_2202_04894_gb300 import defmm, workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _noalloc(plan, q, p, nrhs, dtype):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return defmm.lib().defmm_apply_noalloc(plan.handle, ctypes.c_void_p(q.data_ptr()),
                                           ctypes.c_void_p(p.data_ptr()), nrhs, dtype, stream)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_matches_apply_twice(dtype):
    X, q, kappa, order, leaf, _ = W.make("sphere2k_kD8_p4")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    R = 2
    qq = np.asfortranarray(W.charges(len(X), 5, nrhs=R))
    qd = torch.from_numpy(np.ascontiguousarray(qq.T)).to("cuda").to(dtype)   # (R, n): column-major (n, R)
    ref = plan.apply(qd.t()).t().contiguous()
    torch.cuda.synchronize()
    code = defmm.C64 if dtype == torch.complex64 else defmm.C128
    for call in range(2):
        out = torch.full_like(qd, float("nan"))
        status = _noalloc(plan, qd, out, R, code)
        assert status == 0, defmm.lib().defmm_last_error()
        torch.cuda.synchronize()
        # the same kernels in the same order on the same tables: the same bits
        assert torch.equal(out, ref), call
    plan.close()


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_noalloc_on_a_sharded_plan(dtype):
    """A plan set to one shard of its targets: the no-allocation apply computes
    that shard (zeros elsewhere), like defmm_apply, and the shards sum to the
    whole operator."""
    X = W.points("sphere", 6000, 111)
    q = W.charges(len(X), 112, nrhs=1)[:, 0]
    D = float(np.max(X.max(0) - X.min(0)))
    plan = defmm.Plan(X, kappa=24.0 / D, order=4, leaf_size=32)
    qd = torch.from_numpy(q).to("cuda").to(dtype)
    code = defmm.C64 if dtype == torch.complex64 else defmm.C128
    whole = plan.apply(qd)
    acc = torch.zeros_like(whole)
    for s in range(3):
        plan.set_shard(3, s)
        ref = plan.apply(qd)
        out = torch.full_like(qd, float("nan"))
        status = _noalloc(plan, qd, out, 1, code)
        assert status == 0, defmm.lib().defmm_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref), s
        acc += out
    assert torch.equal(acc, whole)
    plan.close()


def test_noalloc_rejects_oversized_problem():
    X, q, kappa, order, leaf, _ = W.make("sphere2k_kD8_p4")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    qd = torch.zeros((1, len(X)), dtype=torch.complex128, device="cuda")
    status = _noalloc(plan, qd, qd.clone(), 100000, defmm.C128)
    assert status == 5                                   # DEFMM_ERR_UNSUPPORTED
    msg = defmm.lib().defmm_last_error().decode()
    assert "scratch" in msg and "67108864" in msg
    plan.close()
