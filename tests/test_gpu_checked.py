"""The bounds-checked build (every CUDA unit compiled with DEFMM_CHECKED: the
kernels test each table index they follow and raise the plan's error flag,
value 2, instead of reading outside a table) on the parity cases: no index is
out of range, and the results still equal the oracle's.  The checked library
runs in a child process (DEFMM_LIBRARY=checked), apart from the tests'
regular library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
from oracle import fmm as oracle_fmm
from paper_2202_04894_gb300 import defmm, workloads as W
assert defmm.lib()._name.endswith("libdefmm_checked.so")

def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

def gpu(plan, q, dt):
    out = plan.apply(torch.from_numpy(np.ascontiguousarray(q)).to("cuda").to(dt))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)

cases = [("sphere", 2000, None, 8.0, 4, 64), ("box", 5000, None, 16.0, 4, 20),
         ("ellipsoid", 3000, ("sphere", 2500), 30.0, 3, 16), ("sphere", 1500, None, 60.0, 6, 8),
         ("sphere", 1500, None, 10.0, 3, 30)]
for kind, n, other, kd, order, leaf in cases:
    X = W.points(kind, n, 21)
    Y = None if other is None else 0.5 * W.points(other[0], other[1], 22)
    P = X if Y is None else np.vstack([X, Y])
    kappa = kd / float(np.max(P.max(0) - P.min(0)))
    q = W.charges(len(X) if Y is None else len(Y), 23, nrhs=2)
    plan = defmm.Plan(X, Y, kappa=kappa, order=order, leaf_size=leaf)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=leaf, Y=Y)
    for dt in (np.complex128, np.complex64):   # the host-buffer apply names a failed index
        try:
            plan.apply_host(np.ascontiguousarray(q.astype(dt)))
        except defmm.DefmmError as ex:
            print("checked %s %d: %s" % (kind, n, ex))
            raise
    e128, e64 = rel(gpu(plan, q, torch.complex128), ref), rel(gpu(plan, q, torch.complex64), ref)
    plan.set_tuning(p2p_tc_min_rhs=1, m2l_members_per_block=4)
    etc = rel(gpu(plan, q, torch.complex64), ref)
    if Y is None:
        plan.set_shard(3, 1)
        gpu(plan, q, torch.complex64)
        plan.set_shard(1, 0)
    err = plan.info()["device_error"]
    print("checked %s %d: c128 %.2e c64 %.2e tc/blocks of 4 %.2e flag %d" % (kind, n, e128, e64, etc, err))
    assert err == 0 and e128 <= 1e-12 and e64 <= 1e-5 and etc <= 1e-5
geos = [W.points("sphere", 3000, 123), W.points("ellipsoid", 2000, 124)]
uni = defmm.union_plan(geos, [10.0, 20.0], order=4, leaf_size=24)
qu = W.charges(5000, 125)[:, 0]
got = gpu(uni, qu, torch.complex64)
for g, (Xg, kg, a, b) in enumerate([(geos[0], 10.0, 0, 3000), (geos[1], 20.0, 3000, 5000)]):
    assert rel(got[a:b], oracle_fmm.fmm(Xg, qu[a:b], kg, order=4, leaf=24)) <= 1e-5
assert uni.info()["device_error"] == 0
print("checked union ok")
'''


def test_checked_build_on_parity_cases():
    from paper_2202_04894_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, DEFMM_LIBRARY="checked")
    out = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                         text=True, timeout=1200)
    print(out.stdout[-3000:])
    assert out.returncode == 0, out.stderr[-3000:]
    assert "checked union ok" in out.stdout
