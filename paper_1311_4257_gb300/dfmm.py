"""Thin Python binding of the dfmm C ABI (include/dfmm.h).

Argument marshalling only: every step of the matvec runs in the CUDA library
libdfmm.so.  Device buffers are torch tensors (torch is used for device
memory and streams).  If the library is missing this module raises at import
of the first call; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfmm.so")

OK, ERR_INVALID, ERR_DOMAIN, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_DEVICE = 0, -1, -2, -3, -4, -5, -6, -7
ERR_CANCELLED = -8

EXPORT = {"perm": 0, "keys": 1, "boxes": 2, "hf_pairs": 3, "slots_out": 4, "slots_in": 5, "v_pairs": 6,
          "u_pairs": 7, "w_pairs": 8, "x_pairs": 9, "ranks": 10}
EXPORT_COLS = {0: 1, 1: 1, 2: 5, 3: 5, 4: 3, 5: 3, 6: 3, 7: 4, 8: 4, 9: 4, 10: 3}


class DfmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dfmm error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_int32), ("sample_box", ctypes.c_int32), ("sample_far", ctypes.c_int32),
                ("sketch_rows", ctypes.c_int32), ("eps_op_factor", ctypes.c_double), ("m2l_mode", ctypes.c_int32),
                ("host_threads", ctypes.c_int32), ("cache_dir", ctypes.c_char_p), ("tc_stages", ctypes.c_int32),
                ("wait_test", ctypes.c_int32), ("tile_order", ctypes.c_int32), ("p2p_mode", ctypes.c_int32),
                ("tc_layout", ctypes.c_int32), ("tc_accumulate", ctypes.c_int32), ("tc_precision", ctypes.c_int32),
                ("arith", ctypes.c_int32), ("skeleton_host", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("K", ctypes.c_double), ("W", ctypes.c_double), ("eps", ctypes.c_double),
                ("eps_op", ctypes.c_double), ("n_levels", ctypes.c_int32), ("level_hf_top", ctypes.c_int32),
                ("level_w1", ctypes.c_int32), ("boxes", ctypes.c_int64 * 32), ("leaves", ctypes.c_int64 * 32),
                ("hf_pairs", ctypes.c_int64 * 32), ("hf_offsets", ctypes.c_int64 * 32),
                ("slots_out", ctypes.c_int64 * 32), ("slots_in", ctypes.c_int64 * 32),
                ("rank", ctypes.c_int32 * 32), ("v_pairs", ctypes.c_int64), ("u_pairs", ctypes.c_int64),
                ("w_pairs", ctypes.c_int64), ("x_pairs", ctypes.c_int64), ("p2p_interactions", ctypes.c_int64),
                ("plan_bytes", ctypes.c_int64), ("plan_seconds", ctypes.c_double), ("m2l_flops", ctypes.c_double),
                ("other_translation_flops", ctypes.c_double), ("hf_ops", ctypes.c_int64 * 32),
                ("p2p_close_pairs", ctypes.c_int64), ("arith", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("plan_phase_seconds", ctypes.c_double * 8), ("skeleton_phase_seconds", ctypes.c_double * 4),
                ("skeleton_types", ctypes.c_int64), ("plan_id", ctypes.c_int64)]

    def to_dict(self) -> dict:
        n = self.n_levels
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            # per-level arrays (32 slots) hold n_levels entries
            d[name] = (list(v)[:n] if len(v) == 32 else list(v)) if hasattr(v, "__len__") else v
        return d


class ServerReport(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_int64), ("requests_failed", ctypes.c_int64), ("applies", ctypes.c_int64),
                ("rhs_done", ctypes.c_int64), ("points_rhs_done", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("max_concurrent_applies", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("wall_seconds", ctypes.c_double), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class BatchReport(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("waves", ctypes.c_int64), ("merged_launches", ctypes.c_int64),
                ("merged_stages", ctypes.c_int64), ("order_chosen", ctypes.c_int32 * 3), ("graph", ctypes.c_int32),
                ("tune_ms", ctypes.c_double * 3)]


class Peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("reserved", ctypes.c_int32), ("fp32_fma_tflops", ctypes.c_double),
                ("fp64_fma_tflops", ctypes.c_double), ("sincos_gops", ctypes.c_double),
                ("rsqrt_gops", ctypes.c_double), ("tf32_mma_tflops", ctypes.c_double),
                ("f16_mma_tflops", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libdfmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1311_4257_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.dfmm_plan.argtypes = [vp, i64, dbl, dbl, ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.dfmm_apply.argtypes = [vp, vp, vp, i32, vp]
        L.dfmm_apply_host.argtypes = [vp, vp, vp, i32, vp]
        L.dfmm_sync_status.argtypes = [vp, vp]
        L.dfmm_validate.argtypes = [vp, vp, i32]
        L.dfmm_destroy.argtypes = [vp]
        L.dfmm_plan_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.dfmm_apply_workspace_bytes.argtypes = [vp, i32]
        L.dfmm_apply_workspace_bytes.restype = i64
        L.dfmm_export.argtypes = [vp, i32, vp, ctypes.POINTER(i64)]
        L.dfmm_profile.argtypes = [vp, vp, i32, ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
        L.dfmm_apply_launches.argtypes = [vp, i32]
        L.dfmm_apply_launches.restype = i64
        L.dfmm_representation.argtypes = [dbl, i32, dbl, dbl, i32, i32, i32, ctypes.POINTER(i32), vp, vp, i32]
        L.dfmm_representation_device.argtypes = [dbl, i32, dbl, dbl, i32, i32, i32, ctypes.POINTER(i32), vp, vp, i32]
        L.dfmm_plan_bytes.argtypes = [vp]
        L.dfmm_plan_bytes.restype = i64
        L.dfmm_apply_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(i32), i32, vp]
        L.dfmm_server_create.argtypes = [i32, i64, i32, ctypes.POINTER(vp)]
        L.dfmm_server_submit.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(i64)]
        L.dfmm_server_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(dbl)]
        L.dfmm_server_cancel.argtypes = [vp, i64]
        L.dfmm_server_fail_next.argtypes = [vp, i32]
        L.dfmm_server_stats.argtypes = [vp, ctypes.POINTER(ServerReport)]
        L.dfmm_server_destroy.argtypes = [vp]
        L.dfmm_graph_create.argtypes = [vp, vp, vp, i32, vp, ctypes.POINTER(vp)]
        L.dfmm_graph_launch.argtypes = [vp, vp]
        L.dfmm_graph_destroy.argtypes = [vp]
        L.dfmm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(i32), i32, vp, i32, ctypes.POINTER(vp)]
        L.dfmm_batch_launch.argtypes = [vp, vp]
        L.dfmm_batch_stats.argtypes = [vp, ctypes.POINTER(BatchReport)]
        L.dfmm_batch_destroy.argtypes = [vp]
        L.dfmm_solve.argtypes = [vp, dbl, dbl, dbl, dbl, vp, vp, i32, i32, dbl, vp, ctypes.POINTER(i32),
                                 ctypes.POINTER(dbl)]
        L.dfmm_measure_peaks.argtypes = [ctypes.POINTER(Peaks)]
        L.dfmm_last_error.restype = ctypes.c_char_p
        for f in ("dfmm_plan", "dfmm_apply", "dfmm_apply_host", "dfmm_sync_status", "dfmm_validate", "dfmm_destroy",
                  "dfmm_plan_stats", "dfmm_export", "dfmm_representation", "dfmm_representation_device", "dfmm_profile", "dfmm_apply_batched",
                  "dfmm_server_create", "dfmm_server_submit", "dfmm_server_wait", "dfmm_server_cancel",
                  "dfmm_server_fail_next", "dfmm_server_stats",
                  "dfmm_server_destroy", "dfmm_solve", "dfmm_graph_create", "dfmm_graph_launch",
                  "dfmm_graph_destroy", "dfmm_measure_peaks", "dfmm_batch_create", "dfmm_batch_launch",
                  "dfmm_batch_stats", "dfmm_batch_destroy"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def _check(code: int):
    if code != OK:
        raise DfmmError(code, lib().dfmm_last_error().decode())


def representation(w: float, cell: int, w_top: float, eps_op: float, sample_box: int = 0, sample_far: int = 0,
                   sketch_rows: int = 0, device: bool = False):
    """(rank, b2 [2r,3], a2 [2r,3]) of one representation type; pivot selection on
    host threads, or on the current GPU with device=True."""
    r = ctypes.c_int(0)
    cap = 1024
    b2 = np.zeros((cap, 3))
    a2 = np.zeros((cap, 3))
    fn = lib().dfmm_representation_device if device else lib().dfmm_representation
    _check(fn(w, cell, w_top, eps_op, sample_box, sample_far, sketch_rows,
              ctypes.byref(r), b2.ctypes.data, a2.ctypes.data, cap))
    n = 2 * r.value
    return r.value, b2[:n].copy(), a2[:n].copy()


def measure_peaks() -> dict:
    """dfmm_measure_peaks: probed peak rates of the current GPU."""
    pk = Peaks()
    _check(lib().dfmm_measure_peaks(ctypes.byref(pk)))
    return {name: getattr(pk, name) for name, _ in pk._fields_ if name != "reserved"}


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Plan:
    """A resident plan: dfmm_plan(points, N, K, eps) on the current device."""

    def __init__(self, points, K: float, eps: float, leaf_max: int = 0, sample_box: int = 0, sample_far: int = 0,
                 sketch_rows: int = 0, eps_op_factor: float = 0.0, host_threads: int = 0,
                 cache_dir: str | None = None, m2l_mode: int = 0, tc_stages: int = 0, wait_test: int = 0,
                 tile_order: int = 0, p2p_mode: int = 0, tc_layout: int = 0,
                 tc_accumulate: int = 0, tc_precision: int = 0, arith: int = 0, skeleton_host: int = 0):
        import torch
        if not (isinstance(points, torch.Tensor) and points.is_cuda):
            points = torch.as_tensor(np.ascontiguousarray(points, dtype=np.float64), device="cuda")
        points = points.to(torch.float64).contiguous()
        if points.ndim != 2 or points.shape[1] != 3:
            raise ValueError("points must be [N, 3]")
        self.N = int(points.shape[0])
        self.K = float(K)
        self.eps = float(eps)
        o = Options(leaf_max, sample_box, sample_far, sketch_rows, eps_op_factor, m2l_mode, host_threads,
                    cache_dir.encode() if cache_dir else None, tc_stages, wait_test, tile_order, p2p_mode, tc_layout, tc_accumulate, tc_precision,
                    arith, skeleton_host)
        h = ctypes.c_void_p()
        _check(lib().dfmm_plan(points.data_ptr(), self.N, self.K, self.eps, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        # element type of densities and potentials: complex128 when the plan computes in FP64
        self.arith = int(self.stats()["arith"])
        self.dtype = torch.complex128 if self.arith == 64 else torch.complex64
        self.np_dtype = np.complex128 if self.arith == 64 else np.complex64

    def apply(self, f, u=None, stream=None):
        """u = G f.  f: cuda complex64 [nrhs, N] (or [N]), complex128 for an FP64 plan
        (self.dtype); returns u (same shape)."""
        import torch
        squeeze = f.ndim == 1
        f2 = f.reshape(1, -1) if squeeze else f
        if f2.dtype != self.dtype or not f2.is_cuda:
            raise TypeError(f"f must be a cuda {self.dtype} tensor")
        f2 = f2.contiguous()
        nrhs = int(f2.shape[0])
        if f2.shape[1] != self.N:
            raise ValueError("f has the wrong number of points")
        if u is None:
            u = torch.empty_like(f2)
        _check(lib().dfmm_apply(self._h, f2.data_ptr(), u.data_ptr(), nrhs, _stream_ptr(stream)))
        return u.reshape(-1) if squeeze else u

    def apply_host(self, f: np.ndarray, stream=None) -> np.ndarray:
        """Host-buffer matvec: f numpy complex64 [nrhs, N] -> u numpy complex64
        (complex128 for an FP64 plan)."""
        f2 = np.ascontiguousarray(np.atleast_2d(f), dtype=self.np_dtype)
        u = np.empty_like(f2)
        _check(lib().dfmm_apply_host(self._h, f2.ctypes.data, u.ctypes.data, int(f2.shape[0]),
                                     _stream_ptr(stream)))
        return u

    def apply_host_ptr(self, f_ptr: int, u_ptr: int, nrhs: int, stream=None):
        """Host-buffer matvec on raw host pointers (e.g. pinned torch tensors)."""
        _check(lib().dfmm_apply_host(self._h, f_ptr, u_ptr, nrhs, _stream_ptr(stream)))

    def profile_start(self, stream=None):
        _check(lib().dfmm_profile(self._h, _stream_ptr(stream), 1, None, 0, None))

    def profile_stop(self, stream=None) -> dict:
        """Per kernel family: launches, summed CUDA-event ms, algorithmic flops and bytes."""
        out = (KernelTime * 32)()
        n = ctypes.c_int(0)
        _check(lib().dfmm_profile(self._h, _stream_ptr(stream), 0, out, 32, ctypes.byref(n)))
        return {out[k].name.decode(): dict(launches=out[k].launches, ms=out[k].ms, flops=out[k].flops,
                                           bytes=out[k].bytes) for k in range(n.value)}

    def launches(self, nrhs: int = 1) -> int:
        return int(lib().dfmm_apply_launches(self._h, nrhs))

    def sync_status(self, stream=None) -> int:
        return lib().dfmm_sync_status(self._h, _stream_ptr(stream))

    def validate(self, plant: bool = False, stream=None):
        """dfmm_validate: device-side bounds check of every index table (raises DfmmError)."""
        _check(lib().dfmm_validate(self._h, _stream_ptr(stream), 1 if plant else 0))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().dfmm_plan_stats(self._h, ctypes.byref(s)))
        return s.to_dict()

    def workspace_bytes(self, nrhs: int) -> int:
        return int(lib().dfmm_apply_workspace_bytes(self._h, nrhs))

    def plan_bytes(self) -> int:
        return int(lib().dfmm_plan_bytes(self._h))

    def graph(self, f, u, stream=None) -> "Graph":
        """dfmm_graph_create: capture the apply u = G f on these buffers."""
        import torch
        f2 = f.reshape(1, -1) if f.ndim == 1 else f
        if f2.dtype != self.dtype or not f2.is_cuda or not f2.is_contiguous() or f2.shape[1] != self.N:
            raise TypeError(f"f must be a contiguous cuda {self.dtype} [nrhs, N] tensor")
        if u.shape != f.shape or u.dtype != f.dtype or not u.is_contiguous():
            raise TypeError("u must match f")
        h = ctypes.c_void_p()
        _check(lib().dfmm_graph_create(self._h, f2.data_ptr(), u.data_ptr(), int(f2.shape[0]), _stream_ptr(stream),
                                       ctypes.byref(h)))
        return Graph(h, self, f, u)

    def solve(self, b, alpha=1.0, beta=1.0, x0=None, restart: int = 30, maxit: int = 300, tol: float = 1e-5,
              stream=None):
        """dfmm_solve: restarted GMRES for (alpha I + beta G) x = b.
        b: cuda complex64 [N]; returns (x, matvecs, true relative residual)."""
        import torch
        if b.dtype != torch.complex64 or not b.is_cuda or b.numel() != self.N:
            raise TypeError("b must be a cuda complex64 tensor of N values")
        b = b.reshape(-1).contiguous()
        x = torch.zeros_like(b) if x0 is None else x0.reshape(-1).clone()
        a, c = complex(alpha), complex(beta)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        _check(lib().dfmm_solve(self._h, a.real, a.imag, c.real, c.imag, b.data_ptr(), x.data_ptr(), restart, maxit,
                                tol, _stream_ptr(stream), ctypes.byref(it), ctypes.byref(rr)))
        return x, it.value, rr.value

    def export(self, what) -> np.ndarray:
        wid = EXPORT[what] if isinstance(what, str) else int(what)
        n = ctypes.c_int64(0)
        _check(lib().dfmm_export(self._h, wid, None, ctypes.byref(n)))
        buf = np.zeros(max(1, n.value), dtype=np.int64)
        _check(lib().dfmm_export(self._h, wid, buf.ctypes.data, ctypes.byref(n)))
        return buf[:n.value].reshape(-1, EXPORT_COLS[wid])

    def close(self):
        """dfmm_destroy; refused (DfmmError) while a request server holds the plan."""
        if getattr(self, "_h", None):
            _check(lib().dfmm_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured apply (dfmm_graph_*): launch() recomputes u = G f from the
    current contents of the f tensor it was created with."""

    def __init__(self, h, plan, f, u):
        self._h, self.plan, self.f, self.u = h, plan, f, u

    def launch(self, stream=None):
        _check(lib().dfmm_graph_launch(self._h, _stream_ptr(stream)))
        return self.u

    def close(self):
        if getattr(self, "_h", None):
            lib().dfmm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_batched(plans, fs, us=None, stream=None):
    """dfmm_apply_batched: u[k] = G_k f[k] for several plans in one call.
    fs: cuda complex64 tensors [nrhs_k, N_k]; returns the list of u tensors."""
    import torch
    n = len(plans)
    if len(fs) != n:
        raise ValueError("one density tensor per plan")
    fs = [f.reshape(1, -1) if f.ndim == 1 else f for f in fs]
    for p, f in zip(plans, fs):
        if f.dtype != p.dtype or not f.is_cuda or not f.is_contiguous() or f.shape[1] != p.N:
            raise TypeError("each f must be a contiguous cuda [nrhs, N] tensor of its plan's dtype")
    if us is None:
        us = [torch.empty_like(f) for f in fs]
    vp = ctypes.c_void_p
    P = (vp * n)(*[p._h.value for p in plans])
    F = (vp * n)(*[f.data_ptr() for f in fs])
    U = (vp * n)(*[u.data_ptr() for u in us])
    R = (ctypes.c_int * n)(*[int(f.shape[0]) for f in fs])
    _check(lib().dfmm_apply_batched(P, F, U, R, n, _stream_ptr(stream)))
    return us


BATCH_GRAPH, BATCH_TUNE = 1, 2


class Batch:
    """dfmm_batch_*: the batched form with one merged launch per translation stage
    across the plans, on fixed device buffers (fs[k] read, us[k] written).
    launch() recomputes every u[k] = G_k f[k] from the current contents of f."""

    def __init__(self, plans, fs, us=None, stream=None, graph: bool = True, tune: bool = True):
        import torch
        n = len(plans)
        fs = [f.reshape(1, -1) if f.ndim == 1 else f for f in fs]
        for p, f in zip(plans, fs):
            if f.dtype != p.dtype or not f.is_cuda or not f.is_contiguous() or f.shape[1] != p.N:
                raise TypeError("each f must be a contiguous cuda [nrhs, N] tensor of its plan's dtype")
        self.plans, self.fs = list(plans), fs
        self.us = us if us is not None else [torch.empty_like(f) for f in fs]
        vp = ctypes.c_void_p
        P = (vp * n)(*[p._h.value for p in plans])
        F = (vp * n)(*[f.data_ptr() for f in fs])
        U = (vp * n)(*[u.data_ptr() for u in self.us])
        R = (ctypes.c_int * n)(*[int(f.shape[0]) for f in fs])
        h = ctypes.c_void_p()
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_TUNE if tune else 0)
        _check(lib().dfmm_batch_create(P, F, U, R, n, _stream_ptr(stream), flags, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().dfmm_batch_launch(self._h, _stream_ptr(stream)))
        return self.us

    def stats(self) -> dict:
        r = BatchReport()
        _check(lib().dfmm_batch_stats(self._h, ctypes.byref(r)))
        return {"launches": r.launches, "waves": r.waves, "merged_launches": r.merged_launches,
                "merged_stages": r.merged_stages, "order_chosen": list(r.order_chosen), "graph": r.graph,
                "tune_ms": list(r.tune_ms)}

    def close(self):
        if getattr(self, "_h", None):
            lib().dfmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """dfmm_server_*: continuous batching of matvec requests over resident plans.

    submit() takes host complex64 buffers [nrhs, N] (complex128 for a plan whose
    dtype is complex128; pinned torch tensors keep
    the copies asynchronous); the caller keeps them alive until wait() returns."""

    def __init__(self, streams: int = 4, budget_bytes: int = 8 << 30, max_rhs: int = 16):
        h = ctypes.c_void_p()
        _check(lib().dfmm_server_create(streams, int(budget_bytes), max_rhs, ctypes.byref(h)))
        self._h = h

    def submit(self, plan: Plan, f_ptr: int, u_ptr: int, nrhs: int) -> int:
        t = ctypes.c_int64(0)
        _check(lib().dfmm_server_submit(self._h, plan._h, f_ptr, u_ptr, nrhs, ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout: float = 60.0) -> float:
        """Blocks until the request has finished; returns its latency in ms."""
        lat = ctypes.c_double(0)
        _check(lib().dfmm_server_wait(self._h, ticket, timeout, ctypes.byref(lat)))
        return lat.value

    def cancel(self, ticket: int):
        """dfmm_server_cancel: drop a request that has not started."""
        _check(lib().dfmm_server_cancel(self._h, ticket))

    def fail_next(self, status: int):
        """dfmm_server_fail_next (testing aid): the next group fails on the host with `status`."""
        _check(lib().dfmm_server_fail_next(self._h, status))

    def stats(self) -> dict:
        r = ServerReport()
        _check(lib().dfmm_server_stats(self._h, ctypes.byref(r)))
        return {name: getattr(r, name) for name, _ in r._fields_ if name != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            lib().dfmm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
