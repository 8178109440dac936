"""Python binding of libdefmm.so (include/defmm.h): argument marshalling only.

Every step of the application phase runs in the library's CUDA kernels; this
module allocates tensors with torch, passes raw pointers and the current CUDA
stream, and converts status codes into exceptions.  There is no fallback:
if the library is missing, importing it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdefmm.so")

C64, C128 = 0, 1
PLAN_HOST_ONLY = 1
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT",
           5: "ERR_UNSUPPORTED", 6: "ERR_BUSY"}

EXPORTED = ["defmm_default_options", "defmm_plan_create", "defmm_apply", "defmm_apply_host",
            "defmm_destroy", "defmm_plan_info", "defmm_plan_table", "defmm_profile_enable",
            "defmm_profile_read", "defmm_apply_noalloc", "defmm_plan_set_tuning",
            "defmm_plan_get_tuning", "defmm_default_tune_options", "defmm_plan_autotune",
            "defmm_plan_autotune_union",
            "defmm_default_gmres_options", "defmm_gmres", "defmm_plan_set_shard", "defmm_plan_shard_range",
            "defmm_apply_slice", "defmm_assemble_slices",
            "defmm_plan_create_union", "defmm_selftest_bounded_wait", "defmm_plan_save", "defmm_plan_load",
            "defmm_last_error"]
PHASES = ["gather", "p2p", "p2m", "m2m", "m2f", "m2l", "l2l", "l2p", "scatter"]


class Options(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("hf_kw", ctypes.c_double), ("fft_n", ctypes.c_int),
                ("flags", ctypes.c_int), ("self_eps", ctypes.c_double),
                ("hbm_budget", ctypes.c_size_t), ("damping", ctypes.c_double),
                ("m2l_chunk_blocks", ctypes.c_int), ("radial_power", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("order", ctypes.c_int32),
                ("fft_n", ctypes.c_int32), ("nlevels", ctypes.c_int32), ("deepest_hf", ctypes.c_int32),
                ("ncells_t", ctypes.c_int64), ("ncells_s", ctypes.c_int64),
                ("n_m2l_pairs", ctypes.c_int64), ("n_p2p_pairs", ctypes.c_int64),
                ("n_multipole", ctypes.c_int64), ("n_local", ctypes.c_int64),
                ("n_fourier", ctypes.c_int64), ("n_spectra", ctypes.c_int64),
                ("p2p_interactions", ctypes.c_int64), ("plan_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("launches_per_apply", ctypes.c_int64),
                ("device_error", ctypes.c_int64),
                ("d_aabb", ctypes.c_double), ("cube_side", ctypes.c_double),
                ("plan_front_device_ms", ctypes.c_double), ("plan_front_ms", ctypes.c_double),
                ("plan_host_ms", ctypes.c_double), ("plan_upload_ms", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("m2l_rhs_block", ctypes.c_int), ("p2p_tc_min_rhs", ctypes.c_int),
                ("m2l_members_per_block", ctypes.c_int), ("p2p_reduce_phase", ctypes.c_int)]


class TuneOptions(ctypes.Structure):
    _fields_ = [("leaf_min", ctypes.c_int), ("leaf_max", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("dtype", ctypes.c_int), ("reps", ctypes.c_int), ("tune_fft_n", ctypes.c_int),
                ("cache_path", ctypes.c_char_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("fft_n", ctypes.c_int), ("m2l_rhs_block", ctypes.c_int),
                ("p2p_tensor_cores", ctypes.c_int), ("m2l_members_per_block", ctypes.c_int),
                ("ms", ctypes.c_double), ("candidates", ctypes.c_int),
                ("from_cache", ctypes.c_int)]


class GmresOptions(ctypes.Structure):
    _fields_ = [("shift_re", ctypes.c_double), ("shift_im", ctypes.c_double), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int)]


class GmresResult(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int)]


class DefmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


_LIB = None


def lib():
    """Loads libdefmm.so (raises if it has not been built).  With the environment
    variable DEFMM_LIBRARY=checked it loads libdefmm_checked.so instead, the
    bounds-checked build (build.build(checked=True))."""
    global _LIB
    if _LIB is None:
        path = LIB_PATH
        if os.environ.get("DEFMM_LIBRARY") == "checked":
            path = os.path.join(os.path.dirname(LIB_PATH), "libdefmm_checked.so")
        if not os.path.exists(path):
            raise RuntimeError("%s is not built; run __graft_entry__.build()" % os.path.basename(path))
        L = ctypes.CDLL(path)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.defmm_default_options.argtypes = [ctypes.POINTER(Options)]
        L.defmm_default_options.restype = None
        L.defmm_plan_create.argtypes = [vp, i64, vp, i64, dbl, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.defmm_plan_create.restype = ctypes.c_int
        L.defmm_apply.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.defmm_apply.restype = ctypes.c_int
        L.defmm_apply_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.defmm_apply_noalloc.restype = ctypes.c_int
        L.defmm_apply_host.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
        L.defmm_apply_host.restype = ctypes.c_int
        L.defmm_destroy.argtypes = [vp]
        L.defmm_destroy.restype = ctypes.c_int
        L.defmm_plan_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.defmm_plan_info.restype = ctypes.c_int
        L.defmm_plan_table.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(i64), i64, ctypes.POINTER(i64)]
        L.defmm_plan_table.restype = ctypes.c_int
        L.defmm_profile_enable.argtypes = [vp, ctypes.c_int]
        L.defmm_profile_enable.restype = ctypes.c_int
        L.defmm_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
        L.defmm_profile_read.restype = ctypes.c_int
        L.defmm_plan_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.defmm_plan_set_tuning.restype = ctypes.c_int
        L.defmm_plan_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.defmm_plan_get_tuning.restype = ctypes.c_int
        L.defmm_default_tune_options.argtypes = [ctypes.POINTER(TuneOptions)]
        L.defmm_default_tune_options.restype = None
        L.defmm_plan_autotune.argtypes = [vp, i64, vp, i64, dbl, ctypes.c_int, ctypes.POINTER(Options),
                                          ctypes.POINTER(TuneOptions), vp, ctypes.POINTER(vp),
                                          ctypes.POINTER(TuneResult)]
        L.defmm_plan_autotune.restype = ctypes.c_int
        L.defmm_plan_autotune_union.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                                ctypes.POINTER(dbl), ctypes.c_int, ctypes.POINTER(Options),
                                                ctypes.POINTER(TuneOptions), vp, ctypes.POINTER(vp),
                                                ctypes.POINTER(TuneResult)]
        L.defmm_plan_autotune_union.restype = ctypes.c_int
        L.defmm_default_gmres_options.argtypes = [ctypes.POINTER(GmresOptions)]
        L.defmm_default_gmres_options.restype = None
        L.defmm_gmres.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(GmresOptions), vp,
                                  ctypes.POINTER(GmresResult)]
        L.defmm_gmres.restype = ctypes.c_int
        L.defmm_plan_set_shard.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.defmm_plan_set_shard.restype = ctypes.c_int
        L.defmm_plan_shard_range.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.defmm_plan_shard_range.restype = ctypes.c_int
        L.defmm_apply_slice.argtypes = [vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp]
        L.defmm_apply_slice.restype = ctypes.c_int
        L.defmm_assemble_slices.argtypes = [vp, ctypes.c_int, ctypes.POINTER(i64), vp, i64, vp, ctypes.c_int,
                                            ctypes.c_int, vp]
        L.defmm_assemble_slices.restype = ctypes.c_int
        L.defmm_plan_create_union.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                              ctypes.POINTER(dbl), ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.defmm_plan_create_union.restype = ctypes.c_int
        L.defmm_selftest_bounded_wait.argtypes = [ctypes.c_int, vp]
        L.defmm_selftest_bounded_wait.restype = ctypes.c_int
        L.defmm_plan_save.argtypes = [vp, ctypes.c_char_p]
        L.defmm_plan_save.restype = ctypes.c_int
        L.defmm_plan_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.defmm_plan_load.restype = ctypes.c_int
        L.defmm_last_error.argtypes = []
        L.defmm_last_error.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def _check(status):
    if status != 0:
        raise DefmmError(status, lib().defmm_last_error().decode(errors="replace"))


def _stream_handle(stream):
    import torch
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    if stream is None and not torch.cuda.is_available():
        return None
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def default_options(**kw) -> Options:
    o = Options()
    lib().defmm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Plan:
    """A defmm plan: geometry, traversal tables and transfer spectra on the GPU.

    X (nx, 3) and Y (ny, 3) are float64 arrays (numpy or torch, host or
    device); Y=None means sources = targets (one tree).
    """

    def __init__(self, X, Y=None, kappa=1.0, order=4, leaf_size=64, stream=None, **options):
        Xh = self._points(X)
        Yh = None if Y is None else self._points(Y)
        opt = default_options(**options)
        h = ctypes.c_void_p()
        self._keep = (Xh, Yh)
        _check(lib().defmm_plan_create(
            ctypes.c_void_p(Xh.data_ptr()), Xh.shape[0],
            None if Yh is None else ctypes.c_void_p(Yh.data_ptr()),
            Xh.shape[0] if Yh is None else Yh.shape[0],
            float(kappa), int(order), int(leaf_size), ctypes.byref(opt),
            None if (opt.flags & PLAN_HOST_ONLY) else _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self._keep = None
        self.nx = Xh.shape[0]
        self.ny = Xh.shape[0] if Yh is None else Yh.shape[0]

    @staticmethod
    def _points(P):
        import torch
        if not isinstance(P, torch.Tensor):
            P = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float64))
        P = P.to(torch.float64).contiguous()
        if P.dim() != 2 or P.shape[1] != 3:
            raise ValueError("points must have shape (n, 3)")
        return P

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().defmm_destroy(h)
            except Exception:
                pass
            self._h = None

    def close(self):
        if self._h is not None and self._h.value:
            _check(lib().defmm_destroy(self._h))
        self._h = None

    def info(self) -> dict:
        i = Info()
        _check(lib().defmm_plan_info(self._h, ctypes.byref(i)))
        return {name: getattr(i, name) for name, _ in Info._fields_}

    def profile(self, enable: bool = True):
        """Turns per-phase event timing of later applies on or off."""
        _check(lib().defmm_profile_enable(self._h, 1 if enable else 0))

    def phase_ms(self) -> dict:
        """Phase durations (ms) of the last profiled apply (waits for it)."""
        buf = (ctypes.c_double * len(PHASES))()
        n = ctypes.c_int()
        _check(lib().defmm_profile_read(self._h, buf, len(PHASES), ctypes.byref(n)))
        return {PHASES[i]: buf[i] for i in range(n.value)}

    def set_tuning(self, m2l_rhs_block: int = 0, p2p_tc_min_rhs: int = 0, m2l_members_per_block: int = 0,
                   p2p_reduce_phase: int = 0):
        """defmm_plan_set_tuning: launch choices of later applies."""
        t = Tuning(int(m2l_rhs_block), int(p2p_tc_min_rhs), int(m2l_members_per_block), int(p2p_reduce_phase))
        _check(lib().defmm_plan_set_tuning(self._h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().defmm_plan_get_tuning(self._h, ctypes.byref(t)))
        return {"m2l_rhs_block": t.m2l_rhs_block, "p2p_tc_min_rhs": t.p2p_tc_min_rhs,
                "m2l_members_per_block": t.m2l_members_per_block, "p2p_reduce_phase": t.p2p_reduce_phase}

    def gmres(self, b, x0=None, shift=1.0, tol=1e-6, restart=30, max_iter=200, stream=None):
        """defmm_gmres: solves (shift I + A) x = b on the GPU.  b: complex64/complex128
        CUDA tensor (n,).  Returns (x, {iterations, rel_residual, converged})."""
        import torch
        if b.dim() != 1 or b.shape[0] != self.nx or self.nx != self.ny:
            raise ValueError("b must have shape (n,) with n = nx = ny")
        if b.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("b must be complex64 or complex128")
        bc = b.contiguous()
        x = torch.zeros_like(bc) if x0 is None else x0.to(bc.dtype).contiguous().clone()
        o = GmresOptions()
        lib().defmm_default_gmres_options(ctypes.byref(o))
        o.shift_re, o.shift_im = float(complex(shift).real), float(complex(shift).imag)
        o.tol, o.restart, o.max_iter = float(tol), int(restart), int(max_iter)
        r = GmresResult()
        _check(lib().defmm_gmres(self._h, ctypes.c_void_p(bc.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                 C64 if bc.dtype == torch.complex64 else C128, ctypes.byref(o),
                                 _stream_handle(stream), ctypes.byref(r)))
        return x, {name: getattr(r, name) for name, _ in GmresResult._fields_}

    def set_shard(self, nshards: int = 1, shard: int = 0, stream=None):
        """defmm_plan_set_shard: later applies compute shard `shard` of `nshards`."""
        _check(lib().defmm_plan_set_shard(self._h, int(nshards), int(shard), _stream_handle(stream)))
        self._shard = (int(nshards), int(shard))

    def shard_range(self, nshards: int, shard: int):
        """defmm_plan_shard_range: (first, count) of the shard's targets in sorted order."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().defmm_plan_shard_range(self._h, int(nshards), int(shard), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def apply_slice(self, q, out=None, stream=None):
        """defmm_apply_slice: the plan's shard of p in sorted target order.

        q: complex64/complex128 CUDA tensor (ny,) or (ny, R).  out: None or a CUDA
        tensor (R, ld) with ld >= the shard's target count, whose columns j < count
        receive the potentials.  Returns that (R, ld) tensor."""
        import torch
        qm = q.reshape(-1, 1) if q.dim() == 1 else q
        if qm.shape[0] != self.ny:
            raise ValueError("q has %d rows, plan has %d sources" % (qm.shape[0], self.ny))
        R = qm.shape[1]
        qc = qm.t().contiguous()
        if out is None:
            out = torch.empty((R, self.shard_range(*getattr(self, "_shard", (1, 0)))[1]), dtype=qm.dtype,
                              device=qm.device)
        if out.dim() != 2 or out.shape[0] != R or not out.is_contiguous():
            raise ValueError("out must be a contiguous (R, ld) tensor")
        _check(lib().defmm_apply_slice(self._h, ctypes.c_void_p(qc.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       out.shape[1], R, C64 if qm.dtype == torch.complex64 else C128,
                                       _stream_handle(stream)))
        self._last_q = qc
        return out

    def assemble_slices(self, starts, slices, out=None, stream=None):
        """defmm_assemble_slices: p (nx, R) from every shard's slice.

        starts: the nshards + 1 sorted-target boundaries; slices: a contiguous CUDA
        tensor (nshards, R, ld) holding shard s's apply_slice output at [s]."""
        import torch
        nsh, R, ld = slices.shape
        st = (ctypes.c_int64 * len(starts))(*[int(v) for v in starts])
        if len(starts) != nsh + 1:
            raise ValueError("starts must have nshards + 1 entries")
        if not slices.is_contiguous():
            raise ValueError("slices must be contiguous")
        pc = out if out is not None else torch.empty((R, self.nx), dtype=slices.dtype, device=slices.device)
        _check(lib().defmm_assemble_slices(self._h, nsh, st, ctypes.c_void_p(slices.data_ptr()), ld,
                                           ctypes.c_void_p(pc.data_ptr()), R,
                                           C64 if slices.dtype == torch.complex64 else C128, _stream_handle(stream)))
        return pc.t()

    def save(self, path):
        """defmm_plan_save: the plan's host tables and coordinates to a file."""
        _check(lib().defmm_plan_save(self._h, os.fsencode(path)))

    @staticmethod
    def load(path, stream=None, **options):
        """defmm_plan_load: a plan from a file written by save()."""
        opt = default_options(**options)
        h = ctypes.c_void_p()
        _check(lib().defmm_plan_load(os.fsencode(path), ctypes.byref(opt),
                                     None if (opt.flags & PLAN_HOST_ONLY) else _stream_handle(stream), ctypes.byref(h)))
        plan = Plan.__new__(Plan)
        plan._h = h
        plan._keep = None
        info = plan.info()
        plan.nx, plan.ny = int(info["nx"]), int(info["ny"])
        return plan

    def table(self, name: str) -> np.ndarray:
        n = ctypes.c_int64()
        _check(lib().defmm_plan_table(self._h, name.encode(), None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.int64)
        _check(lib().defmm_plan_table(self._h, name.encode(),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      n.value, ctypes.byref(n)))
        return out

    def apply(self, q, out=None, stream=None):
        """p = A q on the GPU.  q: complex64/complex128 CUDA tensor (ny,) or (ny, R).

        Returns p with the same shape convention (nx,) or (nx, R).
        """
        import torch
        squeeze = q.dim() == 1
        qm = q.reshape(-1, 1) if squeeze else q
        if qm.shape[0] != self.ny:
            raise ValueError("q has %d rows, plan has %d sources" % (qm.shape[0], self.ny))
        if qm.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("q must be complex64 or complex128")
        R = qm.shape[1]
        qc = qm.t().contiguous()                      # (R, ny): column-major (ny, R)
        if out is None:
            pc = torch.empty((R, self.nx), dtype=qm.dtype, device=qm.device)
        else:
            pc = out
        _check(lib().defmm_apply(self._h, ctypes.c_void_p(qc.data_ptr()), ctypes.c_void_p(pc.data_ptr()),
                                 R, C64 if qm.dtype == torch.complex64 else C128, _stream_handle(stream)))
        self._last_q = qc
        res = pc.t()
        return res[:, 0] if squeeze else res

    def apply_raw(self, q_ptr: int, p_ptr: int, nrhs: int, dtype: int, stream=None):
        """defmm_apply on raw device pointers (column-major (n, nrhs) buffers)."""
        _check(lib().defmm_apply(self._h, ctypes.c_void_p(q_ptr), ctypes.c_void_p(p_ptr), int(nrhs),
                                 int(dtype), _stream_handle(stream)))

    def apply_host(self, q, out=None, stream=None):
        """defmm_apply_host: q and p in host memory (numpy or pinned torch CPU tensors)."""
        import torch
        if isinstance(q, np.ndarray):
            q = torch.from_numpy(q)
        squeeze = q.dim() == 1
        qm = q.reshape(-1, 1) if squeeze else q
        R = qm.shape[1]
        qc = qm.t().contiguous() if not (R == 1 and qm.is_contiguous()) else qm.reshape(1, -1)
        pc = out if out is not None else torch.empty((R, self.nx), dtype=qm.dtype)
        _check(lib().defmm_apply_host(self._h, ctypes.c_void_p(qc.data_ptr()), ctypes.c_void_p(pc.data_ptr()),
                                      R, C64 if qm.dtype == torch.complex64 else C128, _stream_handle(stream)))
        res = pc.t()
        return res[:, 0] if squeeze else res


def autotune(X, Y=None, kappa=1.0, order=4, nrhs=1, dtype=C64, leaf_range=(16, 64), reps=5,
             tune_fft_n=True, cache_path=None, stream=None, **options):
    """defmm_plan_autotune: the fastest of the candidate plans for this geometry.

    Returns (plan, choice) with choice = {leaf_size, fft_n, m2l_rhs_block, ms,
    candidates, from_cache}.  The timing runs in the library (CUDA events on
    ``stream``); this function only marshals arguments.
    """
    Xh = Plan._points(X)
    Yh = None if Y is None else Plan._points(Y)
    opt = default_options(**options)
    t = TuneOptions()
    lib().defmm_default_tune_options(ctypes.byref(t))
    t.leaf_min, t.leaf_max = int(leaf_range[0]), int(leaf_range[1])
    t.nrhs, t.dtype, t.reps, t.tune_fft_n = int(nrhs), int(dtype), int(reps), 1 if tune_fft_n else 0
    t.cache_path = None if cache_path is None else os.fsencode(cache_path)
    h = ctypes.c_void_p()
    r = TuneResult()
    _check(lib().defmm_plan_autotune(
        ctypes.c_void_p(Xh.data_ptr()), Xh.shape[0],
        None if Yh is None else ctypes.c_void_p(Yh.data_ptr()),
        Xh.shape[0] if Yh is None else Yh.shape[0], float(kappa), int(order), ctypes.byref(opt),
        ctypes.byref(t), _stream_handle(stream), ctypes.byref(h), ctypes.byref(r)))
    plan = Plan.__new__(Plan)
    plan._h = h
    plan._keep = None
    plan.nx = Xh.shape[0]
    plan.ny = Xh.shape[0] if Yh is None else Yh.shape[0]
    return plan, {name: getattr(r, name) for name, _ in TuneResult._fields_}


def union_plan(geometries, kappas, order=4, leaf_size=64, stream=None, **options):
    """defmm_plan_create_union: several geometries (sources = targets) in one plan.

    q and p of an apply hold the geometries' points one after another.  Returns
    a Plan whose nx = ny = the total point count.
    """
    pts = [Plan._points(X) for X in geometries]
    n = len(pts)
    opt = default_options(**options)
    xs = (ctypes.c_void_p * n)(*[ctypes.c_void_p(P.data_ptr()) for P in pts])
    ns = (ctypes.c_int64 * n)(*[P.shape[0] for P in pts])
    ks = (ctypes.c_double * n)(*[float(k) for k in kappas])
    if len(kappas) != n:
        raise ValueError("one kappa per geometry")
    h = ctypes.c_void_p()
    _check(lib().defmm_plan_create_union(
        n, ctypes.cast(xs, ctypes.POINTER(ctypes.c_void_p)), ns, ks, int(order), int(leaf_size),
        ctypes.byref(opt), None if (opt.flags & PLAN_HOST_ONLY) else _stream_handle(stream), ctypes.byref(h)))
    plan = Plan.__new__(Plan)
    plan._h = h
    plan._keep = None
    plan.nx = plan.ny = int(sum(P.shape[0] for P in pts))
    return plan


def autotune_union(geometries, kappas, order=4, nrhs=1, dtype=C64, leaf_range=(16, 64), reps=5,
                   tune_fft_n=True, cache_path=None, stream=None, **options):
    """defmm_plan_autotune_union: the fastest candidate union plan of these geometries.

    Returns (plan, choice) like ``autotune``; the plan is a union plan (nx = ny =
    the total point count)."""
    pts = [Plan._points(X) for X in geometries]
    n = len(pts)
    if len(kappas) != n:
        raise ValueError("one kappa per geometry")
    opt = default_options(**options)
    t = TuneOptions()
    lib().defmm_default_tune_options(ctypes.byref(t))
    t.leaf_min, t.leaf_max = int(leaf_range[0]), int(leaf_range[1])
    t.nrhs, t.dtype, t.reps, t.tune_fft_n = int(nrhs), int(dtype), int(reps), 1 if tune_fft_n else 0
    t.cache_path = None if cache_path is None else os.fsencode(cache_path)
    xs = (ctypes.c_void_p * n)(*[ctypes.c_void_p(P.data_ptr()) for P in pts])
    ns = (ctypes.c_int64 * n)(*[P.shape[0] for P in pts])
    ks = (ctypes.c_double * n)(*[float(k) for k in kappas])
    h = ctypes.c_void_p()
    r = TuneResult()
    _check(lib().defmm_plan_autotune_union(n, xs, ns, ks, int(order), ctypes.byref(opt), ctypes.byref(t),
                                           _stream_handle(stream), ctypes.byref(h), ctypes.byref(r)))
    plan = Plan.__new__(Plan)
    plan._h = h
    plan._keep = None
    plan.nx = plan.ny = int(sum(P.shape[0] for P in pts))
    return plan, {name: getattr(r, name) for name, _ in TuneResult._fields_}
