"""Benchmark of the defmm application phase on GB300.

Default workload: 10^6 points on the unit sphere, kappa*D = 128, order 4,
leaf <= 64, one complex64 right-hand side (the high-frequency configuration
with directional levels active).  A step is one defmm_apply: gather, P2P,
P2M, M2M, M2F, Hadamard M2L + F2L, L2L, L2P, scatter.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line on rank 0.  value = Mpoints*RHS/s over all ranks (replicas:
each rank applies its own copy of the workload; there is no data-path
collective).  With --sharded and N > 1 the ranks split the one workload
instead (defmm_plan_set_shard: each rank computes its Morton range of target
leaves, the upward pass replicated), each writes its targets' potentials in
sorted order (defmm_apply_slice), an all-gather of those slices inside the
timed region gives every rank all of them, and defmm_assemble_slices puts
them in the caller's order: strong scaling.  Inputs are resident in HBM for
`value`; `e2e` times the
host-buffer entry point (defmm_apply_host) with both copies inside.  L2 is
flushed (a 512 MB write) before every timed step, outside the step's events.

Two more workloads, each printing its own JSON line:

  --workload batch48   48 uneven geometries (spheres, ellipsoids, box
                       surfaces; N log-uniform in [2e4, 8e5], kappa*D in
                       [16, 256], order 4, complex64) applied together as one
                       union plan (every phase one launch over all geometries;
                       the JSON value), against one replayed CUDA graph of
                       per-geometry applies and the applies one after another.
  --workload serve16   the request server over 16 resident geometries (N in
                       [5e4, 2e6], kappa*D in [32, 256], order 4-6): Poisson
                       arrivals (mean gap --gap-ms, seed 300) of requests with
                       1-8 right-hand sides on a uniformly drawn geometry,
                       host buffers in and out; p50/p99 latency and throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "sphere1M_kD128_p4"
METRIC = "Mpoints·RHS/s at rel-L2 err≤1e-4 vs FP64 oracle; M2L HBM GB/s; p50/p99 ms"
UNIT = "Mpoints·RHS/s"
# CPU sample of the same workload: same distribution, order and leaf size, and
# kappa*D scaled with sqrt(N) so that the points per wavelength^2 stay those of
# the 10^6-point case.
SAMPLE_N = 16000          # cpu_baseline: ~10-20 s of single-core oracle work
ORACLE_S_PER_POINT = 6e-4  # measured oracle cost on this recipe, used to size samples


# the row M2L kernel and its launch (which blocks serve which groups) in kernels.cu, and the
# plan's M2L schedule (chunks) in plan.cpp
M2L_REGIONS = [("kernels.cu", "// The same group schedule with rows of samples",
                "// Ring depth S and the dynamic shared memory of the per-sample M2L kernel"),
               ("kernels.cu", "// The Hadamard M2L + F2L of one apply", "cudaError_t launch_wait_probe"),
               ("plan.cpp", "    // ---- M2L groups and chunks", "    // ---- M2M per parent level")]


def m2l_rows_source_sha():
    """sha256 (first 16 hex) of the row M2L kernel's, its launch's and the M2L schedule's source text."""
    import hashlib
    h = hashlib.sha256()
    for name, begin, end in M2L_REGIONS:
        src = open(os.path.join(ROOT, "paper_2202_04894_gb300", "csrc", name)).read()
        a = src.index(begin)
        h.update(src[a:src.index(end, a)].encode())
    return h.hexdigest()[:16]


def _recorded_traffic_per_pair():
    """DRAM bytes per M2L pair from the committed ncu summary, or None when the
    row M2L kernel has changed since those counters were taken."""
    import re
    path = os.path.join(ROOT, "profiles", "m2l_rows_sphere300k_kD128_p4.md")
    try:
        text = open(path).read()
        sha = m2l_rows_source_sha()
    except (OSError, ValueError):
        return None
    m = re.search(r"traffic_bytes_per_pair:\s*([0-9.]+)", text)
    h = re.search(r"k_m2l_rows source sha256 \(first 16 hex\):\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != sha:
        return None
    return float(m.group(1))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 10:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r for r in self.rows if not self.bus_id or self.bus_id.endswith(r[1].lower()[-12:])
                or r[1].lower().endswith(self.bus_id[-12:])]
        rows = rows or self.rows
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(total_ms, dist=None, device="cpu"):
    """The timed region's length (ms) as the slowest rank saw it; identity on one process."""
    if dist is None:
        return float(total_ms)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_slices(slice_buf, gathered, dist=None):
    """The exchange step of the sharded apply: rank s holds its targets'
    potentials in sorted order, slice_buf (R, ld); an all-gather leaves every
    rank's slice at gathered[s] (gathered: (world, R, ld)) on every rank.  Each
    rank sends its own targets only, and nothing is summed."""
    import torch
    if dist is None:
        gathered[0].copy_(slice_buf)
        return gathered
    parts = [gathered[s] for s in range(gathered.shape[0])]
    if slice_buf.is_complex():
        dist.all_gather([torch.view_as_real(t) for t in parts], torch.view_as_real(slice_buf))
    else:
        dist.all_gather(parts, slice_buf)
    return gathered


def whole_job_value(world, points, nrhs, ms_per_step):
    """Mpoints*RHS/s of the whole job: every rank applies its own replica of the workload."""
    return world * points * nrhs / (ms_per_step * 1e-3) / 1e6


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_sample(n=SAMPLE_N):
    """The oracle on a bounded sample of the workload (same recipe, n points)."""
    from paper_2202_04894_gb300 import workloads as W
    w = W.WORKLOADS[WORKLOAD]
    kd = w["kappa_d"] * (n / w["n"]) ** 0.5
    X = W.points(w["kind"], n, w["seed"])
    kappa = kd / float(np.max(X.max(0) - X.min(0)))
    q = W.charges(n, w["seed"], w["nrhs"])
    desc = ("sphere, %d points, kappa*D=%.2f (10^6-point density per wavelength^2), order %d, leaf %d, "
            "%d RHS, float64 oracle" % (n, kd, w["order"], w["leaf"], w["nrhs"]))
    return X, q, kappa, w["order"], w["leaf"], desc


def time_oracle(steps, warmup, n=SAMPLE_N, out_path=None, ready_dir=None, nready=0):
    """Times the oracle's apply (plan excluded) on the sample; saves the last result to
    out_path (.npy) if given.  With ready_dir, waits after building the plan until nready
    processes have done so, so that concurrent copies time overlapping applies."""
    from oracle import fmm
    X, q, kappa, order, leaf, desc = cpu_sample(n)
    plan = fmm.make_plan(X, kappa=kappa, order=order, leaf=leaf)
    if ready_dir:
        open(os.path.join(ready_dir, "ready.%d" % os.getpid()), "w").close()
        t_wait = time.perf_counter()
        while len(os.listdir(ready_dir)) < nready and time.perf_counter() - t_wait < 600:
            time.sleep(0.01)
    for _ in range(warmup):
        fmm.apply(plan, X, q)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        p = fmm.apply(plan, X, q)
        ts.append(time.perf_counter() - t0)
    if out_path:
        np.save(out_path, p)
    sec = sum(ts) / len(ts)
    return len(X) * q.shape[1] / sec / 1e6, sec, desc


def _oracle_cmd(steps, warmup, n, out_path=None, ready_dir=None, nready=0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.time_oracle(%d, %d, %d, %r, %r, %d)))"
            % (ROOT, steps, warmup, n, out_path, ready_dir, nready))
    return [sys.executable, "-c", code], env


def oracle_subprocess(steps, warmup, n, timeout=1800, out_path=None):
    """Runs time_oracle in a fresh single-threaded interpreter (BLAS pinned to 1 thread)."""
    cmd, env = _oracle_cmd(steps, warmup, n, out_path)
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-400:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_all_cores(n, timeout=900):
    """One single-threaded oracle process per host core, each applying the same sample at
    the same time (they start timing together); returns (aggregate Mpoints*RHS/s, cores,
    slowest apply in s).  The oracle itself is unchanged: this is nproc copies of it."""
    import tempfile
    cores = os.cpu_count() or 1
    with tempfile.TemporaryDirectory() as ready:
        procs = []
        for _ in range(cores):
            cmd, env = _oracle_cmd(1, 0, n, None, ready, cores)
            procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
        secs = []
        for pr in procs:
            out, err = pr.communicate(timeout=timeout)
            if pr.returncode != 0:
                raise RuntimeError(err[-400:])
            secs.append(json.loads(out.strip().splitlines()[-1])[1])
    slowest = max(secs)
    return cores * n / slowest / 1e6, cores, slowest


def reference_arm(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    # each step is a bounded sample sized so that the whole run takes ~2.5 minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(min(SAMPLE_N, max(1000, budget / ORACLE_S_PER_POINT)))
    value, sec, desc = oracle_subprocess(args.steps, args.warmup, n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="defmm", choices=["defmm", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="point count (same recipe; for profiling)")
    ap.add_argument("--nrhs", type=int, default=None, help="right-hand sides (same charge recipe; for profiling)")
    ap.add_argument("--p2p-tensor-cores", action="store_true",
                    help="tensor-core near field (defmm_tuning.p2p_tc_min_rhs = 1)")
    ap.add_argument("--sharded", action="store_true",
                    help="N > 1: split the one workload across the ranks (strong scaling) instead of replicas")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=10000, help="serve16: number of requests")
    ap.add_argument("--gap-ms", type=float, default=2.0, help="serve16: mean inter-arrival time")
    ap.add_argument("--load-fracs", default="0.5,0.8,0.95",
                    help="serve16: offered loads (fractions of the measured capacity) for the latency curve; '' skips")
    ap.add_argument("--curve-requests", type=int, default=400, help="serve16: requests per load-curve point")
    ap.add_argument("--streams", type=int, default=4, help="serve16: batches in flight")
    ap.add_argument("--branches", type=int, default=8, help="batch48: graph branches")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload in ("batch48", "batch48small", "serve16"):
        (bench_serve if args.workload == "serve16" else bench_batch)(args)
        return

    import torch
    import __graft_entry__
    from paper_2202_04894_gb300 import defmm, workloads as W

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    W_ = W.WORKLOADS[args.workload]
    X, q, kappa, order, leaf, dtype = W.make(args.workload, n=args.n)
    if args.nrhs:
        q = W.charges(len(X), W_["seed"], args.nrhs)
    cdt = torch.complex64 if dtype == "c64" else torch.complex128
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = defmm.Plan(X, kappa=kappa, order=order, leaf_size=leaf)
    plan_s = time.perf_counter() - t0
    if args.p2p_tensor_cores:
        plan.set_tuning(p2p_tc_min_rhs=1)
    sharded = args.sharded and world > 1
    if sharded:   # this rank computes its shard of the targets; an all-gather of the slices assembles p
        plan.set_shard(world, rank)
        ranges = [plan.shard_range(world, s) for s in range(world)]
        shard_starts = [f for f, _ in ranges] + [len(X)]
        ld = max(1, max(n for _, n in ranges))
    info = plan.info()
    R = q.shape[1]
    qd = torch.from_numpy(np.ascontiguousarray(q)).to("cuda").to(cdt)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # accuracy of the timed (complex64) form against the float64 path, and the
    # plain float64 GPU apply (same kernels in double) as the comparison bar
    p_lo = plan.apply(qd)
    q_hi = qd.to(torch.complex128)
    p_hi = plan.apply(q_hi)
    torch.cuda.synchronize()
    rel = float(torch.linalg.norm(p_lo.to(torch.complex128) - p_hi) / torch.linalg.norm(p_hi))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.apply(q_hi)
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    del q_hi, p_hi

    for _ in range(args.warmup):
        plan.apply(qd)
    plan.profile(True)
    phase_sum = {}
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    bus = None
    try:
        props = torch.cuda.get_device_properties(local)
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        pass
    clocks = ClockSampler(bus)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    pbuf = torch.empty((R, len(X)), dtype=cdt, device="cuda") if sharded else None
    if sharded:
        slice_buf = torch.empty((R, ld), dtype=cdt, device="cuda")
        gathered = torch.empty((world, R, ld), dtype=cdt, device="cuda")
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        if sharded:
            plan.apply_slice(qd, out=slice_buf)
            gather_slices(slice_buf, gathered, dist)
            plan.assemble_slices(shard_starts, gathered, out=pbuf)
        else:
            plan.apply(qd, out=pbuf)
        ends[k].record(stream)
        ends[k].synchronize()
        step_ms.append(starts[k].elapsed_time(ends[k]))
        for name, ms in plan.phase_ms().items():
            phase_sum[name] = phase_sum.get(name, 0.0) + ms
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    plan.profile(False)
    launches_per_apply = int(plan.info()["launches_per_apply"])
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_value(1 if sharded else world, len(X), R, ms_per_step)
    units = (1 if sharded else world) * len(X) * R

    # end to end through the host-buffer entry point (pinned host memory)
    qh = torch.from_numpy(np.ascontiguousarray(q.T)).to(cdt).pin_memory()
    ph = torch.empty((R, len(X)), dtype=cdt).pin_memory()
    for _ in range(3):
        plan.apply_host(qh.t(), out=ph)
    e2e_ms = []
    for k in range(max(5, args.steps // 5)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.apply_host(qh.t(), out=ph)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = units / (statistics.mean(e2e_ms) * 1e-3) / 1e6
    csz = 8 if cdt == torch.complex64 else 16

    # dominant phase and its roofline
    phase_avg = {k: v / args.steps for k, v in phase_sum.items()}
    NF = info["fft_n"] ** 3
    P3 = order ** 3
    m2l_bytes = (info["n_m2l_pairs"] * R * csz * NF + info["n_spectra"] * csz * NF)
    m2l_gbs = m2l_bytes / (phase_avg["m2l"] * 1e-3) / 1e9
    peak_gbs, peak_kind = _peaks()
    kernel_phases = {k: v for k, v in phase_avg.items() if k not in ("total", "join_wait")}
    dominant = max(kernel_phases, key=kernel_phases.get)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    # P2P, one right-hand side: 3 SFU operations (rsqrt, sin, cos) per
    # interaction; 16 SFU results per clock per SM (SM count queried).  Several
    # right-hand sides: 4 FP32 FMA per interaction and column (complex
    # multiply-add) against 128 FMA per clock per SM.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    inter = info["p2p_interactions"] * R
    p2p_achieved = inter / (phase_avg["p2p"] * 1e-3) / 1e9
    if R == 1:
        p2p_peak = sms * 16 / 3 * sm_max * 1e6 / 1e9
        p2p_src = "SFU: %d SMs x 16/clk / 3 per interaction at %.0f MHz" % (sms, sm_max)
        p2p_unit = "Ginteractions/s"
    else:
        p2p_peak = sms * 128 / 4 * sm_max * 1e6 / 1e9
        p2p_src = "FP32 FMA: %d SMs x 128/clk / 4 per interaction and column at %.0f MHz" % (sms, sm_max)
        p2p_unit = "Ginteraction-columns/s"
    p2p_roof = {"kernel": "p2p", "bound": "alu", "achieved": p2p_achieved, "peak": p2p_peak,
                "unit": p2p_unit, "frac": p2p_achieved / p2p_peak, "traffic": None, "peak_source": p2p_src}
    per_pair = _recorded_traffic_per_pair()
    m2l_traffic = None if per_pair is None or R != 1 else per_pair * info["n_m2l_pairs"]
    m2l_roof = {"kernel": "m2l", "bound": "hbm", "achieved": m2l_gbs, "peak": peak_gbs, "unit": "GB/s",
                "frac": m2l_gbs / peak_gbs, "traffic": m2l_traffic, "algorithmic_bytes": m2l_bytes,
                "ms": phase_avg["m2l"], "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic_source": "profiles/m2l_rows_sphere300k_kD128_p4.md, DRAM bytes per pair x pairs"}
    roof = p2p_roof if dominant == "p2p" else m2l_roof
    # the M2L phase under three more views: operand reads from shared memory (a gathered
    # spectrum sample and a multipole sample, 16 B per sample-pair and column, against
    # 128 B per clock per SM), the DRAM traffic it really moves, and its compulsory bytes
    # (each Fourier multipole read once, each local expansion written once, the spectra once)
    m2l_s = phase_avg["m2l"] * 1e-3
    smem_bytes = info["n_m2l_pairs"] * NF * 16 * R
    smem_peak = sms * 128 * sm_max * 1e6 / 1e9
    compulsory = (info["n_fourier"] * info["fft_n"] ** 3 + info["n_local"] * P3) * csz * R + info["n_spectra"] * NF * csz
    m2l_views = {
        "smem_operands": {"achieved": smem_bytes / m2l_s / 1e9, "peak": smem_peak, "unit": "GB/s",
                          "frac": smem_bytes / m2l_s / 1e9 / smem_peak,
                          "peak_source": "%d SMs x 128 B/clk at %.0f MHz" % (sms, sm_max)},
        "dram_measured": None if m2l_traffic is None else
        {"achieved": m2l_traffic / m2l_s / 1e9, "peak": peak_gbs, "unit": "GB/s",
         "frac": m2l_traffic / m2l_s / 1e9 / peak_gbs},
        "compulsory": {"achieved": compulsory / m2l_s / 1e9, "peak": peak_gbs, "unit": "GB/s",
                       "frac": compulsory / m2l_s / 1e9 / peak_gbs}}

    cpu, vs_oracle = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD and not args.n:
        import tempfile
        try:
            with tempfile.TemporaryDirectory() as tmp:
                ref_path = os.path.join(tmp, "oracle.npy")
                v1, s1, d = oracle_subprocess(1, 0, SAMPLE_N, out_path=ref_path)
                ref = np.load(ref_path)
            vall, cores, sall = oracle_all_cores(SAMPLE_N)
            cpu = {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": d + "; %d single-threaded oracle processes applying it at once" % cores,
                   "seconds": sall, "value_1core": v1, "seconds_1core": s1}
            # the timed form (complex64, same plan options) on the oracle's own sample
            Xs, qs_, ks, os_, ls, _ = cpu_sample(SAMPLE_N)
            sp = defmm.Plan(Xs, kappa=ks, order=os_, leaf_size=ls)
            got = sp.apply(torch.from_numpy(np.ascontiguousarray(qs_[:, 0])).to("cuda").to(cdt)).cpu().numpy()
            sp.close()
            ref = ref.reshape(got.shape)
            vs_oracle = {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                         "max_rel": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
                         "dtype": dtype, "sample": d}
        except Exception as ex:  # reported, never fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(ex)[:200]}

    if rank == 0:
        srt = sorted(step_ms)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak",
                "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": {"workload": args.workload, "points": len(X), "kappa_d": W_["kappa_d"], "order": order,
                           "leaf": leaf, "nrhs": R, "distribution": W_["kind"], "l2": "flushed (512 MB write) before each step",
                           "p2p": "tensor cores (tcgen05)" if args.p2p_tensor_cores else "cuda cores",
                           "parallelism": ("sharded targets, all-gather of sorted slices" if sharded else "replicas") if world > 1
                           else "single"},
                "roofline": roof, "m2l_roofline": m2l_roof, "m2l_views": m2l_views, "p2p_roofline": p2p_roof,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": len(X) * R * csz,
                        "d2h_bytes_per_step": len(X) * R * csz, "ms_per_step": statistics.mean(e2e_ms)},
                "clocks": clk, "gpu_launches": launches_per_apply * args.steps,
                "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                "rel_l2_c64_vs_c128": rel, "rel_l2_vs_oracle": vs_oracle and vs_oracle["rel_l2"],
                "vs_oracle": vs_oracle, "phase_ms": phase_avg, "plan_s": plan_s,
                "plan_ms": {"front_device": info["plan_front_device_ms"], "front_wall": info["plan_front_ms"],
                            "host_rest": info["plan_host_ms"], "upload_and_spectra": info["plan_upload_ms"]},
                "fp64_gpu_apply": {"ms": fp64_ms, "value": units / (fp64_ms * 1e-3) / 1e6, "unit": UNIT,
                                   "speedup_of_c64": fp64_ms / ms_per_step},
                "plan": {k: info[k] for k in ("n_m2l_pairs", "n_p2p_pairs", "n_multipole", "n_local", "n_fourier",
                                              "n_spectra", "p2p_interactions", "nlevels", "deepest_hf")}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _plans_of(geos, defmm, W, leaf=64):
    plans = []
    t0 = time.perf_counter()
    for g in geos:
        X, kappa = W.make_geometry(g)
        plans.append(defmm.Plan(X, kappa=kappa, order=g["order"], leaf_size=leaf))
    return plans, time.perf_counter() - t0


def _bus(torch):
    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        return "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        return None


def bench_batch(args):
    """48 uneven geometries: one union plan (every phase one launch over all
    geometries), one replayed CUDA graph of per-geometry applies, and the same
    applies in sequence."""
    import torch
    import __graft_entry__
    from paper_2202_04894_gb300 import defmm, serve, workloads as W
    __graft_entry__.build()
    geos = W.geometry_set(**(W.BATCH48_SMALL if args.workload == "batch48small" else W.BATCH48))
    plans, plan_s = _plans_of(geos, defmm, W)
    c64 = torch.complex64
    qs = [torch.from_numpy(np.ascontiguousarray(W.charges(p.ny, g["seed"]))).to("cuda").to(c64)
          for p, g in zip(plans, geos)]
    b = serve.Batch(plans, [1] * len(plans), c64, branches=args.branches)
    for buf, q in zip(b.inputs(), qs):
        buf.copy_(q.t())
    b.run()
    torch.cuda.synchronize()
    worst = 0.0
    for i, (p, q) in enumerate(zip(plans, qs)):
        hi = p.apply(q.to(torch.complex128))
        lo = b.outputs()[i].t().to(torch.complex128)
        worst = max(worst, float(torch.linalg.norm(lo - hi) / torch.linalg.norm(hi)))
        del hi
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    outs = [None] * len(plans)

    def seq():
        for i, (p, q) in enumerate(zip(plans, qs)):
            outs[i] = p.apply(q)

    def timed(fn, steps):
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    # the union plan: one plan over all 48 geometries
    t0 = time.perf_counter()
    pts = [W.make_geometry(g) for g in geos]
    uni = defmm.union_plan([X for X, _ in pts], [k for _, k in pts], order=4, leaf_size=64)
    union_s = time.perf_counter() - t0
    qu = torch.cat([q for q in qs]).contiguous()
    pu = torch.empty((1, qu.shape[0]), dtype=c64, device="cuda")

    def union():
        uni.apply(qu, out=pu)

    union()
    torch.cuda.synchronize()
    ref = torch.cat([b.outputs()[i].reshape(-1) for i in range(len(plans))])
    union_bitwise = bool(torch.equal(pu.reshape(-1), ref))

    for _ in range(args.warmup):
        b.run()
        seq()
        union()
    clocks = ClockSampler(_bus(torch))
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    u_ms = timed(union, args.steps)
    g_ms = timed(b.run, args.steps)
    s_ms = timed(seq, args.steps)
    clk = clocks.stop()
    points = sum(p.nx for p in plans)
    u_avg, g_avg, s_avg = statistics.mean(u_ms), statistics.mean(g_ms), statistics.mean(s_ms)
    info = b.info()
    u_launches = int(uni.info()["launches_per_apply"])
    uni.profile(True)   # phase times of one union apply (events on its stream), after the timed steps
    union()
    torch.cuda.synchronize()
    u_phases = uni.phase_ms()
    uni.profile(False)
    bset = W.BATCH48_SMALL if args.workload == "batch48small" else W.BATCH48
    line = {"metric": METRIC, "value": points / (u_avg * 1e-3) / 1e6, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": u_avg, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": args.workload, "geometries": len(plans), "points": points,
                       "n_range": list(bset["n_range"]), "kappa_d_range": list(bset["kd_range"]),
                       "order": 4, "leaf": 64, "nrhs": 1, "form": "union plan (one launch per phase)",
                       "l2": "flushed (512 MB write) before each step", "parallelism": "single"},
            "union": {"kernel_launches": u_launches, "plan_s": union_s, "bitwise_equal_to_individual": union_bitwise,
                      "phase_ms": u_phases},
            "graph": {"ms_per_step": g_avg, "value": points / (g_avg * 1e-3) / 1e6, "branches": args.branches,
                      "kernel_launches": info["kernel_launches"], "graph_nodes": info["graph_nodes"]},
            "sequential": {"ms_per_step": s_avg, "value": points / (s_avg * 1e-3) / 1e6},
            "gpu_launches": u_launches * args.steps,
            "max_rel_l2_c64_vs_c128": worst, "plan_s": plan_s, "clocks": clk,
            "p50_ms": sorted(u_ms)[len(u_ms) // 2], "p99_ms": sorted(u_ms)[min(len(u_ms) - 1, int(0.99 * len(u_ms)))]}
    print(json.dumps(line), flush=True)


def bench_serve(args):
    """Poisson request stream through the request server."""
    import torch
    import __graft_entry__
    from paper_2202_04894_gb300 import defmm, serve, workloads as W
    __graft_entry__.build()
    geos = W.geometry_set(**W.SERVE16)
    plans, plan_s = _plans_of(geos, defmm, W)
    c64 = torch.complex64
    maxr = 8
    qh = [torch.from_numpy(np.ascontiguousarray(W.charges(p.ny, g["seed"], nrhs=maxr).T)).to(c64).pin_memory()
          for p, g in zip(plans, geos)]
    ph = [torch.empty((maxr, p.nx), dtype=c64).pin_memory() for p in plans]   # results land here (overwritten)
    reqs = W.request_stream(args.requests, 300, args.gap_ms, len(plans), maxr)
    budget = 96 << 30
    srv = serve.Server(plans, c64, streams=args.streams, max_batch_rhs=16, hbm_budget=budget)
    for g in range(len(plans)):                                   # warm-up: every geometry once
        srv.wait_ticket(srv.submit_ptr(g, qh[g].data_ptr(), ph[g].data_ptr(), maxr))
    st0 = srv.stats()
    clocks = ClockSampler(_bus(torch))
    clocks.start()
    time.sleep(0.3)

    def run(stream):
        """Submits the (t_ms, geometry, nrhs) stream on its schedule; returns latencies and wall time."""
        tickets = [None] * len(stream)

        def producer():
            t0 = time.perf_counter()
            for i, (t_ms, g, r) in enumerate(stream):
                delay = t0 + t_ms * 1e-3 - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = srv.submit_ptr(g, qh[g].data_ptr(), ph[g].data_ptr(), r)

        t_start = time.perf_counter()
        th = threading.Thread(target=producer)
        th.start()
        lat = []
        for i in range(len(stream)):
            while tickets[i] is None:
                time.sleep(1e-4)
            lat.append(srv.wait_ticket(tickets[i]))
        th.join()
        return lat, time.perf_counter() - t_start

    def work_of(stream):
        return sum(plans[g].nx * r for _, g, r in stream)

    def pct(v, f):
        srt = sorted(v)
        return srt[min(len(srt) - 1, int(f * len(srt)))]

    # latency at sustainable loads: the capacity from a burst (every request at once),
    # then Poisson streams offering a fraction of it
    curve, capacity = [], None
    if args.load_fracs:
        burst = [(0.0, g, r) for _, g, r in W.request_stream(args.curve_requests, 301, 1.0, len(plans), maxr)]
        _, wall_b = run(burst)
        capacity = work_of(burst) / wall_b / 1e6
        mean_work = work_of(burst) / len(burst)
        for frac in [float(f) for f in args.load_fracs.split(",")]:
            gap = mean_work / (frac * capacity * 1e6) * 1e3
            stream = W.request_stream(args.curve_requests, 302, gap, len(plans), maxr)
            lat_f, wall_f = run(stream)
            curve.append({"load": frac, "mean_gap_ms": gap, "p50_ms": pct(lat_f, 0.5), "p99_ms": pct(lat_f, 0.99),
                          "served": work_of(stream) / wall_f / 1e6, "requests": len(stream)})
    st0 = srv.stats()   # the stated stream alone in the server counters below
    lat, wall = run(reqs)
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    work = work_of(reqs)
    srt = sorted(lat)
    offered = sum(plans[g].nx * r for _, g, r in reqs) / (reqs[-1][0] * 1e-3) / 1e6
    line = {"metric": METRIC, "value": work / wall / 1e6, "unit": UNIT, "n_gpus": 1, "steps": len(reqs),
            "warmup": len(plans), "ms_per_step": wall * 1e3 / len(reqs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "serve16", "geometries": len(plans),
                       "points": [p.nx for p in plans], "orders": [g["order"] for g in geos],
                       "kappa_d": [round(g["kappa_d"], 1) for g in geos], "requests": len(reqs),
                       "mean_gap_ms": args.gap_ms, "rhs_per_request": "uniform 1..8", "streams": args.streams,
                       "max_batch_rhs": 16, "hbm_budget": budget, "parallelism": "single"},
            "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
            "mean_ms": statistics.mean(lat), "max_ms": srt[-1],
            "offered_load": {"value": offered, "unit": UNIT},
            "capacity": {"value": capacity, "unit": UNIT, "from": "%d requests submitted at once" % args.curve_requests}
            if capacity else None,
            "load_curve": curve,
            "e2e": {"value": work / wall / 1e6, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * sum(plans[g].ny * r for _, g, r in reqs) // len(reqs),
                    "d2h_bytes_per_step": 8 * sum(plans[g].nx * r for _, g, r in reqs) // len(reqs)},
            "server": {k: st[k] - st0.get(k, 0) if k in ("submitted", "completed", "batches", "rhs_applied",
                                                          "kernel_launches") else st[k] for k in st},
            "gpu_launches": st["kernel_launches"] - st0["kernel_launches"], "plan_s": plan_s, "clocks": clk}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
