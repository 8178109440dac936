"""Python binding of the serving layer (include/defmm_serve.h): argument marshalling only.

Workspaces, graph batches and the request server are implemented in the
library (C++/CUDA); this module passes tensors' raw pointers and converts
status codes into exceptions.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import defmm
from .defmm import C64, C128, _check, _stream_handle, lib

SERVE_EXPORTED = ["defmm_workspace_bytes", "defmm_workspace_create", "defmm_workspace_wrap",
                  "defmm_workspace_destroy", "defmm_apply_ws", "defmm_batch_create", "defmm_batch_apply",
                  "defmm_batch_info", "defmm_batch_destroy", "defmm_server_default_options",
                  "defmm_server_create", "defmm_server_submit", "defmm_server_wait",
                  "defmm_server_get_stats", "defmm_server_destroy"]


class ServerOptions(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int), ("max_batch_rhs", ctypes.c_int), ("hbm_budget", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("rhs_applied", ctypes.c_int64), ("max_batch_requests", ctypes.c_int64),
                ("max_inflight", ctypes.c_int64), ("arena_bytes", ctypes.c_size_t),
                ("peak_arena_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_int64)]


_READY = False


def slib():
    """The library with the serving entry points' signatures declared."""
    global _READY
    L = lib()
    if not _READY:
        vp, i64, ci, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        sigs = {
            "defmm_workspace_bytes": [vp, ci, ci, ctypes.POINTER(sz)],
            "defmm_workspace_create": [vp, ci, ci, ctypes.POINTER(vp)],
            "defmm_workspace_wrap": [vp, ci, ci, vp, sz, ctypes.POINTER(vp)],
            "defmm_workspace_destroy": [vp],
            "defmm_apply_ws": [vp, vp, vp, vp, ci, ci, vp],
            "defmm_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(ci), ci, ci, ci, ctypes.POINTER(vp)],
            "defmm_batch_apply": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp],
            "defmm_batch_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "defmm_batch_destroy": [vp],
            "defmm_server_create": [ctypes.POINTER(vp), ci, ci, ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)],
            "defmm_server_submit": [vp, ci, vp, vp, ci, ctypes.POINTER(ctypes.c_uint64)],
            "defmm_server_wait": [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
            "defmm_server_get_stats": [vp, ctypes.POINTER(ServerStats)],
            "defmm_server_destroy": [vp],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.defmm_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
        L.defmm_server_default_options.restype = None
        _READY = True
    return L


def _dtype_code(dtype):
    import torch
    if dtype in (torch.complex64, C64, "c64"):
        return C64
    if dtype in (torch.complex128, C128, "c128"):
        return C128
    raise TypeError("dtype must be complex64 or complex128")


def _colmajor(q, n):
    """(n,) or (n, R) tensor -> contiguous (R, n) tensor (column-major (n, R))."""
    qm = q.reshape(-1, 1) if q.dim() == 1 else q
    if qm.shape[0] != n:
        raise ValueError("expected %d rows, got %d" % (n, qm.shape[0]))
    return qm.t().contiguous(), qm.shape[1]


def workspace_bytes(plan: defmm.Plan, nrhs: int, dtype) -> int:
    b = ctypes.c_size_t()
    _check(slib().defmm_workspace_bytes(plan.handle, int(nrhs), _dtype_code(dtype), ctypes.byref(b)))
    return b.value


class Workspace:
    """Caller-owned scratch for applies of up to nrhs right-hand sides on one plan."""

    def __init__(self, plan: defmm.Plan, nrhs: int, dtype):
        self.plan, self.nrhs, self.code = plan, int(nrhs), _dtype_code(dtype)
        h = ctypes.c_void_p()
        _check(slib().defmm_workspace_create(plan.handle, self.nrhs, self.code, ctypes.byref(h)))
        self._h = h

    def apply(self, q, stream=None):
        """p = A q with this workspace (q: CUDA tensor (ny,) or (ny, R), R <= nrhs)."""
        import torch
        qc, R = _colmajor(q, self.plan.ny)
        pc = torch.empty((R, self.plan.nx), dtype=qc.dtype, device=qc.device)
        _check(slib().defmm_apply_ws(self.plan.handle, self._h, ctypes.c_void_p(qc.data_ptr()),
                                     ctypes.c_void_p(pc.data_ptr()), R, _dtype_code(qc.dtype),
                                     _stream_handle(stream)))
        self._keep = qc
        res = pc.t()
        return res[:, 0] if q.dim() == 1 else res

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            slib().defmm_workspace_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Applies of several plans (nrhs[i] right-hand sides each) replayed as one CUDA graph."""

    def __init__(self, plans, nrhs, dtype, branches: int = 0):
        import torch
        self.plans = list(plans)
        self.nrhs = [int(r) for r in nrhs]
        self.code = _dtype_code(dtype)
        self.tdtype = torch.complex64 if self.code == C64 else torch.complex128
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        rr = (ctypes.c_int * n)(*self.nrhs)
        h = ctypes.c_void_p()
        _check(slib().defmm_batch_create(arr, rr, n, self.code, int(branches), ctypes.byref(h)))
        self._h = h
        self._q = [torch.empty((r, p.ny), dtype=self.tdtype, device="cuda") for p, r in zip(self.plans, self.nrhs)]
        self._p = [torch.empty((r, p.nx), dtype=self.tdtype, device="cuda") for p, r in zip(self.plans, self.nrhs)]

    def inputs(self):
        """The batch's resident input buffers, (R_i, ny_i) = column-major (ny_i, R_i)."""
        return self._q

    def outputs(self):
        return self._p

    def run(self, stream=None):
        """Replays the graph on the resident buffers (captured on the first call)."""
        n = len(self.plans)
        qa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self._q])
        pa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in self._p])
        _check(slib().defmm_batch_apply(self._h, qa, pa, _stream_handle(stream)))

    def apply(self, qs, stream=None):
        """Copies qs[i] ((ny_i,) or (ny_i, R_i) CUDA tensors) in, runs, returns copies of the outputs."""
        for buf, q in zip(self._q, qs):
            qc, _ = _colmajor(q, buf.shape[1])
            buf.copy_(qc)
        self.run(stream)
        return [p.t().clone() for p in self._p]

    def info(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(slib().defmm_batch_info(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"kernel_launches": a.value, "graph_nodes": b.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            slib().defmm_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server with continuous batching over resident plans (see defmm_serve.h)."""

    def __init__(self, plans, dtype, streams: int = 4, max_batch_rhs: int = 16, hbm_budget: int = 4 << 30):
        import torch
        self.plans = list(plans)
        self.code = _dtype_code(dtype)
        self.tdtype = torch.complex64 if self.code == C64 else torch.complex128
        o = ServerOptions()
        slib().defmm_server_default_options(ctypes.byref(o))
        o.streams, o.max_batch_rhs, o.hbm_budget = int(streams), int(max_batch_rhs), int(hbm_budget)
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(slib().defmm_server_create(arr, n, self.code, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, geometry: int, q) -> int:
        """Queues plans[geometry] applied to q (host tensor or array (ny,) or (ny, R)); returns a ticket."""
        import torch
        if isinstance(q, np.ndarray):
            q = torch.from_numpy(q)
        plan = self.plans[geometry]
        qc, R = _colmajor(q.to(self.tdtype), plan.ny)
        qc = qc.pin_memory()
        pc = torch.empty((R, plan.nx), dtype=self.tdtype).pin_memory()
        t = ctypes.c_uint64()
        _check(slib().defmm_server_submit(self._h, int(geometry), ctypes.c_void_p(qc.data_ptr()),
                                          ctypes.c_void_p(pc.data_ptr()), R, ctypes.byref(t)))
        self._live[t.value] = (qc, pc, q.dim() == 1)
        return t.value

    def submit_ptr(self, geometry: int, q_ptr: int, p_ptr: int, nrhs: int) -> int:
        """Queues a request on caller-managed host buffers (column-major, kept alive
        by the caller until the ticket completes); wait for it with wait_ticket."""
        t = ctypes.c_uint64()
        _check(slib().defmm_server_submit(self._h, int(geometry), ctypes.c_void_p(q_ptr), ctypes.c_void_p(p_ptr),
                                          int(nrhs), ctypes.byref(t)))
        return t.value

    def wait_ticket(self, ticket: int, timeout_ms: float = -1.0) -> float:
        """Blocks for a ticket of submit_ptr; returns its latency in ms."""
        lat = ctypes.c_double()
        _check(slib().defmm_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_ms), ctypes.byref(lat)))
        return lat.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        """Blocks for a ticket; returns (p, latency_ms), p shaped like the request's q."""
        lat = ctypes.c_double()
        _check(slib().defmm_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout_ms), ctypes.byref(lat)))
        qc, pc, squeeze = self._live.pop(ticket)
        res = pc.t()
        return (res[:, 0] if squeeze else res), lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(slib().defmm_server_get_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(slib().defmm_server_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
