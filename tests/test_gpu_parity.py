"""GPU parity: the CUDA application phase (through the C ABI) against the CPU oracle.

Tolerances (relative L2 over all targets and right-hand sides):
  complex128 path vs oracle FMM   <= 1e-12  (same method, different summation order)
  complex64  path vs oracle FMM   <= 1e-5   (single-precision arithmetic)
  FMM vs direct sum               <= the order-p approximation error
"""
import numpy as np
import pytest

from oracle import direct, fmm as oracle_fmm
from paper_2202_04894_gb300 import defmm, workloads as W

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
TOL64 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(plan, q, dtype):
    qd = torch.from_numpy(np.ascontiguousarray(q)).to("cuda").to(dtype)
    out = plan.apply(qd)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def test_sphere2k_against_oracle_and_direct():
    """2,000 sphere points, kappa*D = 8, order 4, leaf 64: directional M2L at level 2."""
    X, q, kappa, order, leaf, _ = W.make("sphere2k_kD8_p4")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=leaf)
    p128 = _gpu(plan, q, torch.complex128)
    p64 = _gpu(plan, q, torch.complex64)
    assert _rel(p128, ref) <= TOL128
    assert _rel(p64, ref) <= TOL64
    assert np.max(np.abs(p128 - ref)) <= 1e-11 * np.max(np.abs(ref))
    exact = direct.direct_sum(X, X, q, kappa, direct.eps_self(X))
    assert _rel(p128, exact) <= 1e-3          # order-4 accuracy on this case (oracle: 3.1e-4)
    info = plan.info()
    assert info["deepest_hf"] == 2 and info["n_m2l_pairs"] > 0


CASES = [
    # kind, n, sources, kappa*D, order, leaf, fft_n
    ("box", 5000, None, 16.0, 4, 20, 0),
    ("ellipsoid", 3000, ("sphere", 2500), 30.0, 3, 16, 0),
    ("cube", 2500, None, 0.0, 5, 10, 0),
    ("sphere", 1500, None, 60.0, 6, 8, 0),
    ("sphere", 3000, None, 24.0, 3, 150, 8),      # leaves of >64 targets, >128 sources, N > 2p-1
    ("box", 1200, None, 40.0, 2, 12, 0),
    ("ellipsoid", 4000, None, 64.0, 4, 40, 0),
    ("sphere", 1500, None, 10.0, 3, 30, 13),       # N^3 = 2197 samples: four per M2L thread
    ("box", 2500, None, 20.0, 4, 200, 0),          # leaves of 129..200 targets: two P2P passes
]


@pytest.mark.parametrize("case", CASES)
def test_against_oracle(case):
    kind, n, other, kd, order, leaf, fft_n = case
    X = W.points(kind, n, 21)
    Y = None if other is None else 0.5 * W.points(other[0], other[1], 22)
    P = X if Y is None else np.vstack([X, Y])
    kappa = kd / float(np.max(P.max(0) - P.min(0)))
    q = W.charges(len(X) if Y is None else len(Y), 23, nrhs=2)
    plan = defmm.Plan(X, Y, kappa=kappa, order=order, leaf_size=leaf, fft_n=fft_n)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=leaf, Y=Y,
                         fft_n=fft_n if fft_n else None)
    p128 = _gpu(plan, q, torch.complex128)
    p64 = _gpu(plan, q, torch.complex64)
    assert _rel(p128, ref) <= TOL128, _rel(p128, ref)
    assert _rel(p64, ref) <= TOL64, _rel(p64, ref)
    for r in range(q.shape[1]):
        assert _rel(p64[:, r], ref[:, r]) <= TOL64


TC_CASES = [CASES[0], CASES[1], CASES[3], CASES[4], CASES[8]]


@pytest.mark.parametrize("case", TC_CASES)
def test_tensor_core_near_field_against_oracle(case):
    """The tcgen05 near field (forced on for 2 columns) against the oracle: leaves
    of up to 200 targets (several target tiles), two trees, orders 3-6."""
    kind, n, other, kd, order, leaf, fft_n = case
    X = W.points(kind, n, 21)
    Y = None if other is None else 0.5 * W.points(other[0], other[1], 22)
    P = X if Y is None else np.vstack([X, Y])
    kappa = kd / float(np.max(P.max(0) - P.min(0)))
    q = W.charges(len(X) if Y is None else len(Y), 23, nrhs=2)
    plan = defmm.Plan(X, Y, kappa=kappa, order=order, leaf_size=leaf, fft_n=fft_n)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=leaf, Y=Y,
                         fft_n=fft_n if fft_n else None)
    cuda_cores = _gpu(plan, q, torch.complex64)
    plan.set_tuning(p2p_tc_min_rhs=1)
    tensor = _gpu(plan, q, torch.complex64)
    assert plan.info()["device_error"] == 0
    for r in range(q.shape[1]):
        assert _rel(tensor[:, r], ref[:, r]) <= TOL64, _rel(tensor[:, r], ref[:, r])
    assert _rel(tensor, cuda_cores) <= TOL64
    assert np.array_equal(tensor, _gpu(plan, q, torch.complex64))    # deterministic


def test_tensor_core_near_field_many_columns():
    """40 columns: one full 32-column tensor-core pass and a ragged one of 8; every
    column against the complex128 path, and a column alone equals it in the block."""
    X = W.points("box", 6000, 33)
    kappa = 24.0
    q = W.charges(6000, 34, nrhs=40)
    plan = defmm.Plan(X, kappa=kappa, order=4, leaf_size=48)
    p128 = _gpu(plan, q, torch.complex128)
    plan.set_tuning(p2p_tc_min_rhs=32)
    p64 = _gpu(plan, q, torch.complex64)          # 40 >= 32: tensor-core near field
    for r in range(40):
        assert _rel(p64[:, r], p128[:, r]) <= TOL64
    plan.set_tuning(p2p_tc_min_rhs=1)
    one = _gpu(plan, q[:, 37], torch.complex64)
    assert _rel(one, p64[:, 37]) <= 1e-6


@pytest.mark.parametrize("order", [4, 5, 6])
def test_m2l_rhs_blocks_are_bitwise_identical(order):
    """1, 2 and 4 right-hand sides per M2L pass (with a ragged last pass: 5 columns),
    blocks of 8 or 4 members or split by group size and a smaller chunk budget give the same bits, and equal
    the oracle; N = 7, 9 (blocks of at most 2 columns) and 11 (one column per pass)."""
    X = W.points("sphere", 3000, 61)
    q = W.charges(3000, 62, nrhs=5)
    kappa = 30.0
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=24)
    outs = []
    for rb in (1, 2, 4, 0):
        for members in (8, 4, 12, 14):
            plan.set_tuning(m2l_rhs_block=rb, m2l_members_per_block=members)
            outs.append(_gpu(plan, q, torch.complex64))
            outs.append(_gpu(plan, q[:, 3], torch.complex64)[:, None])   # one column alone
    for o in outs[1:]:
        assert np.array_equal(o, outs[o.shape[1] == 1])
    # smaller chunks stage fewer blocks at a time: same bits
    small = defmm.Plan(X, kappa=kappa, order=order, leaf_size=24, m2l_chunk_blocks=3)
    small.set_tuning(m2l_members_per_block=4)
    assert np.array_equal(_gpu(small, q, torch.complex64), outs[0])
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=24)
    assert _rel(outs[0], ref) <= TOL64


@pytest.mark.parametrize("kind,kd,damping_d,order", [("sphere", 0.0, 8.0, 5), ("box", 24.0, 6.0, 4),
                                                     ("ellipsoid", 48.0, 2.0, 4)])
def test_damped_kernel_against_oracle(kind, kd, damping_d, order):
    """Yukawa (kappa = 0) and damped Helmholtz kernels exp((i kappa - lambda) r)/(4 pi r):
    complex128 and complex64 (CUDA-core and tensor-core near field) against the oracle."""
    X = W.points(kind, 2500, 71)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa, lam = kd / D, damping_d / D
    q = W.charges(2500, 72, nrhs=2)
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=20, damping=lam)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=20, damping=lam)
    assert _rel(_gpu(plan, q, torch.complex128), ref) <= TOL128
    assert _rel(_gpu(plan, q, torch.complex64), ref) <= TOL64
    plan.set_tuning(p2p_tc_min_rhs=1)
    assert _rel(_gpu(plan, q, torch.complex64), ref) <= TOL64
    undamped = oracle_fmm.fmm(X, q, kappa, order=order, leaf=20)
    assert _rel(undamped, ref) > 0.05


@pytest.mark.parametrize("kind,kd,damping_d,order", [("sphere", 24.0, 0.0, 4), ("cube", 0.0, 0.0, 5),
                                                    ("box", 16.0, 4.0, 4)])
def test_power_two_kernel_against_oracle(kind, kd, damping_d, order):
    """exp((i kappa - lambda) r)/(4 pi r^2), outside the Helmholtz family (the plan
    option radial_power = 2 reaches the transfer spectra and every near-field kernel):
    complex128 and complex64 (one column, several columns, tensor-core near field,
    both phase forms) against the oracle, element by element."""
    X = W.points(kind, 2500, 73)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa, lam = kd / D, damping_d / D
    q = W.charges(2500, 74, nrhs=2)
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=20, damping=lam, radial_power=2)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=20, damping=lam, power=2)
    _check_close(_gpu(plan, q, torch.complex128), ref, TOL128, 1e-11, "r^-2 %s c128" % kind)
    _check_close(_gpu(plan, q, torch.complex64), ref, TOL64, 1e-4, "r^-2 %s c64" % kind)
    _check_close(_gpu(plan, q[:, 0], torch.complex64), ref[:, 0], TOL64, 1e-4, "r^-2 %s c64 one column" % kind)
    plan.set_tuning(p2p_reduce_phase=1)
    _check_close(_gpu(plan, q[:, 0], torch.complex64), ref[:, 0], TOL64, 1e-4, "r^-2 %s c64 reduced" % kind)
    plan.set_tuning(p2p_tc_min_rhs=1)
    _check_close(_gpu(plan, q, torch.complex64), ref, TOL64, 1e-4, "r^-2 %s c64 tensor cores" % kind)
    assert _rel(oracle_fmm.fmm(X, q, kappa, order=order, leaf=20, damping=lam), ref) > 0.05


def test_multi_rhs_columns_and_determinism():
    X = W.points("sphere", 4000, 31)
    kappa = 20.0
    q = W.charges(4000, 32, nrhs=6)
    plan = defmm.Plan(X, kappa=kappa, order=4, leaf_size=32)
    ref = oracle_fmm.fmm(X, q, kappa, order=4, leaf=32)
    for dt, tol in ((torch.complex128, TOL128), (torch.complex64, TOL64)):
        a = _gpu(plan, q, dt)
        b = _gpu(plan, q, dt)
        assert np.array_equal(a, b)                      # deterministic
        assert _rel(a, ref) <= tol
        one = _gpu(plan, q[:, 4], dt)
        assert _rel(one, a[:, 4]) <= tol
        if dt == torch.complex64:
            # one column (packed-FP32 near field) equals its column in the block (scalar kernel)
            assert np.array_equal(one, a[:, 4])


def test_apply_host_matches_device():
    X, q, kappa, order, leaf, _ = W.make("sphere2k_kD8_p4")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    dev = _gpu(plan, q, torch.complex64)
    qh = torch.from_numpy(q.astype(np.complex64)).pin_memory()
    host = plan.apply_host(qh).numpy()
    assert np.array_equal(host, dev.astype(np.complex64))


def test_degenerate_geometries():
    one = np.array([[0.3, -0.2, 0.1]])
    plan = defmm.Plan(one, kappa=2.0, order=4, leaf_size=8)
    assert np.all(_gpu(plan, np.array([1.0 + 1j]), torch.complex128) == 0)
    two = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    plan = defmm.Plan(two, kappa=1.5, order=4, leaf_size=1)
    got = _gpu(plan, np.array([1.0, 2.0 + 0j]), torch.complex128)
    g = np.exp(1.5j * 2.0) / (4 * np.pi * 2.0)
    assert np.allclose(got, [2.0 * g, 1.0 * g], rtol=1e-13, atol=0)
    dup = np.repeat(np.array([[1.0, 2.0, 3.0]]), 40, axis=0)
    plan = defmm.Plan(dup, kappa=3.0, order=4, leaf_size=3)
    assert np.all(_gpu(plan, np.ones(40, dtype=complex), torch.complex128) == 0)


@pytest.mark.slow
def test_sphere1M_sampled_against_direct():
    """10^6 sphere points, kappa*D = 128, order 4, leaf 64, complex64: the
    benchmarked workload.  2,000 seeded targets are checked against the direct
    sum, and the complex64 result against the complex128 one everywhere."""
    X, q, kappa, order, leaf, _ = W.make("sphere1M_kD128_p4")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    p64 = _gpu(plan, q, torch.complex64)
    p128 = _gpu(plan, q, torch.complex128)
    assert _rel(p64, p128) <= TOL64
    idx = np.sort(np.random.default_rng(7).choice(len(X), 2000, replace=False))
    exact = direct.direct_sum_c(X, X, q, kappa, direct.eps_self(X), targets=idx)
    err = _rel(p64[idx], exact)
    print("sphere1M: rel-L2 vs direct on 2000 targets %.3e, c64 vs c128 %.3e" % (err, _rel(p64, p128)))
    assert err <= 5e-3


@pytest.mark.slow
def test_box500k_order5_32rhs_sampled_against_direct():
    """5*10^5 points on a 1 x 1 x 0.25 box surface (edge-refined), kappa*D = 64,
    order 5, 32 complex64 right-hand sides in one apply: every column against
    the direct sum on 400 sampled targets (order-5 accuracy)."""
    X, q, kappa, order, leaf, _ = W.make("box500k_kD64_p5_r32")
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    p64 = _gpu(plan, q, torch.complex64)
    idx = np.sort(np.random.default_rng(11).choice(len(X), 400, replace=False))
    exact = direct.direct_sum_c(X, X, q, kappa, direct.eps_self(X), targets=idx)
    errs = [_rel(p64[idx, r], exact[:, r]) for r in range(q.shape[1])]
    print("box500k p5 x32: rel-L2 vs direct, worst column %.3e, mean %.3e" % (max(errs), np.mean(errs)))
    assert max(errs) <= 2e-3
    one = _gpu(plan, q[:, 17], torch.complex64)
    assert _rel(one, p64[:, 17]) <= TOL64          # a column alone equals the column in the batch


def _check_close(got, ref, rel_tol, max_tol, what):
    rel = _rel(got, ref)
    worst = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print("%s: rel-L2 %.3e, max|d|/max|ref| %.3e" % (what, rel, worst))
    assert rel <= rel_tol, (what, rel)
    assert worst <= max_tol, (what, worst)


SCALE_CASES = [
    # kind, n, order, leaf: the benchmark's recipe (kappa*D scaled by sqrt(n / 10^6), so the
    # points per wavelength^2 are the 10^6-point workload's)
    ("sphere", 40000, 4, 64),
    ("cube", 12000, 4, 32),
]


@pytest.mark.parametrize("case", SCALE_CASES)
def test_oracle_parity_at_scale(case):
    """Tens of thousands of points against the oracle FMM, element by element, on plans
    large enough to take the paths small cases miss: near-field work units cut at 4,096
    sources, M2L groups with more chunks than the ring has stages, and M2L blocks of all
    three size classes (groups of <= 4, 5-7 and 8 siblings)."""
    kind, n, order, leaf = case
    X = W.points(kind, n, 2)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa = 128.0 * (n / 1e6) ** 0.5 / D
    q = W.charges(n, 2, nrhs=1)[:, 0]
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    ref = oracle_fmm.fmm(X, q, kappa, order=order, leaf=leaf)
    # the paths this case is there for
    ul, uo = plan.table("p2p_unit_leaf"), plan.table("p2p_unit_off")
    rr = plan.table("p2p_unit_ranges").reshape(-1, 2)
    per_unit = np.add.reduceat(rr[:, 1] - rr[:, 0], uo[:-1])
    sizes = np.diff(plan.table("grp_member_off"))
    chunks = np.diff(plan.table("grp_chunk_off"))
    assert chunks.max() > 3                                  # longer than any ring
    if kind == "sphere":
        assert len(ul) > len(np.unique(ul)) and per_unit.max() == 4096   # leaves split into units
        assert np.any(sizes <= 4) and np.any((sizes >= 5) & (sizes <= 7))
    else:
        assert np.any(sizes == 8) and np.any(sizes <= 4)
    p128 = _gpu(plan, q, torch.complex128)
    _check_close(p128, ref, TOL128, 1e-11, "%s %d c128" % (kind, n))
    p64 = _gpu(plan, q, torch.complex64)
    _check_close(p64, ref, TOL64, 1e-4, "%s %d c64" % (kind, n))
    # two columns (right-hand-side blocks in M2L, several columns per near-field pass):
    # the second column is (1 + 2i) q, whose exact image is (1 + 2i) ref
    q2 = np.stack([q, (1 + 2j) * q], 1)
    p2 = _gpu(plan, q2, torch.complex64)
    _check_close(p2[:, 0], ref, TOL64, 1e-4, "%s %d c64 column 0 of 2" % (kind, n))
    _check_close(p2[:, 1], (1 + 2j) * ref, TOL64, 1e-4, "%s %d c64 column 1 of 2" % (kind, n))
    assert plan.info()["device_error"] == 0
    plan.close()


@pytest.mark.parametrize("kd", [120.0, 200.0])
def test_near_field_phase_forms(kd):
    """The complex64 near field with the phase given to the hardware sine and cosine
    directly (every near-field phase below 90 pi: kappa*D = 120 here, up to ~208 rad)
    and with the exact reduction to [-1/2, 1/2] turns (kappa*D = 200: phases up to
    ~346 rad, where the library must reduce), both against the oracle FMM."""
    X = W.points("sphere", 6000, 31)
    D = float(np.max(X.max(0) - X.min(0)))
    kappa = kd / D
    q = W.charges(len(X), 32, nrhs=1)[:, 0]
    plan = defmm.Plan(X, kappa=kappa, order=4, leaf_size=32)
    ref = oracle_fmm.fmm(X, q, kappa, order=4, leaf=32)
    for reduce_phase in (0, 1):
        plan.set_tuning(p2p_reduce_phase=reduce_phase)
        p64 = _gpu(plan, q, torch.complex64)
        _check_close(p64, ref, TOL64, 1e-4, "kD %g reduce %d c64" % (kd, reduce_phase))
    plan.close()
