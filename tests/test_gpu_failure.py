"""Failure detection without a GPU fault: a device-side wait that nothing
completes gives up after its bound, the host reads DEFMM_ERR_TIMEOUT, and the
context stays usable (an apply afterwards is exact)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_04894_gb300 import defmm, workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    L = defmm.lib()
    assert L.defmm_selftest_bounded_wait(1 << 12, None) == 4            # DEFMM_ERR_TIMEOUT
    assert b"gave up" in L.defmm_last_error()
    assert L.defmm_selftest_bounded_wait(0, None) == 1                  # DEFMM_ERR_ARG
    # the context is still usable: an apply afterwards equals one before
    X = W.points("sphere", 3000, 161)
    plan = defmm.Plan(X, kappa=10.0, order=4, leaf_size=32)
    q = torch.from_numpy(W.charges(3000, 162)[:, 0]).to("cuda").to(torch.complex64)
    a = plan.apply(q).cpu().numpy()
    assert L.defmm_selftest_bounded_wait(1 << 12, None) == 4
    b = plan.apply(q).cpu().numpy()
    assert np.array_equal(a, b)
    assert plan.info()["device_error"] == 0
