"""Python binding of the GB300 fractional Adams-Bashforth-Moulton engine.

Thin ctypes marshalling over ``libfabm.so`` (the C ABI in include/fabm.h):
the functions below carry the C names and only convert arguments.  Every step
of a solve runs in the library's CUDA kernels; there is no CPU fallback, and
``load()`` raises if the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FABM_OK, FABM_EINVAL, FABM_ENOMEM, FABM_ECUDA, FABM_ENONFINITE, FABM_ETIMEOUT, FABM_EBUSY = range(7)
FABM_FP64, FABM_SPLIT, FABM_FP64X2 = 0, 1, 2
FABM_HIST_AUTO, FABM_HIST_FP64, FABM_HIST_TENSOR, FABM_HIST_FP32C = range(4)
FABM_HIST_X2, FABM_HIST_TENSOR_WIDE, FABM_HIST_FP64_PERSIST = 4, 5, 6
HIST = {"auto": 0, "fp64": 1, "tensor": 2, "fp32c": 3, "x2": 4, "tensor-wide": 5,
        "fp64-persist": 6}
RECURRENCE = {"auto": 0, "columns": 1, "targets": 2}
RHS = {"const": 0, "time": 1, "linear": 2, "lorenz": 3, "duffing": 4, "manufactured": 5,
       "lcr": 6}
PRECISION = {"fp64": FABM_FP64, "split": FABM_SPLIT, "fp64x2": FABM_FP64X2}
_EXPORTS = ("fabm_create", "fabm_solve", "fabm_solve_batch", "fabm_destroy",
            "fabm_last_error", "fabm_set_block", "fabm_get_block", "fabm_last_launch_count",
            "fabm_copy_weights", "fabm_set_timing", "fabm_kernel_stats", "fabm_set_graphs",
            "fabm_solve_noalloc", "fabm_set_history_kernel", "fabm_get_history_kernel",
            "fabm_server_create", "fabm_server_submit", "fabm_server_step", "fabm_server_poll",
            "fabm_server_result", "fabm_server_stats", "fabm_server_destroy", "fabm_autotune",
            "fabm_stroboscope", "fabm_server_checkpoint", "fabm_server_resume",
            "fabm_server_cancel", "fabm_server_shape", "fabm_solve_batch_ic",
            "fabm_create_multi", "fabm_server_finished", "fabm_kernel_busy",
            "fabm_set_recurrence_layout", "fabm_get_recurrence_layout", "fabm_weights_x2",
            "fabm_server_wait", "fabm_set_wait_limit", "fabm_inject_alloc_failures",
            "fabm_copy_weights_lo", "fabm_server_submit_ic", "fabm_last_history_kernel",
            "fabm_set_recurrence_warps", "fabm_get_recurrence_warps")
FABM_REQ_WAITING, FABM_REQ_RUNNING, FABM_REQ_DONE, FABM_REQ_FAILED = range(4)


class fabm_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("alpha", ctypes.c_double), ("h", ctypes.c_double),
                ("N", ctypes.c_int64), ("rhs_id", ctypes.c_int),
                ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int),
                ("y0", ctypes.POINTER(ctypes.c_double))]
KERNEL_KINDS = ("weights", "init", "history", "combine", "recurrence", "slice")

_lib = None


class FabmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fabm status {status}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfabm.so (building it first if needed); raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libfabm.so not found at {path}; run paper_1710_01133_gb300.build")
    lib = ctypes.CDLL(path)
    d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    P = ctypes.POINTER
    lib.fabm_create.argtypes = [i, d, d, i64, i, P(d), i, i, P(vp)]
    lib.fabm_create_multi.argtypes = [i, P(d), d, i64, i, P(d), i, i, P(vp)]
    lib.fabm_solve.argtypes = [vp, P(d), P(d)]
    lib.fabm_solve_batch.argtypes = [vp, i64, P(d), P(d), P(i64), vp, i]
    lib.fabm_solve_batch_ic.argtypes = [vp, i64, P(d), P(d), P(d), P(i64), vp, i]
    lib.fabm_destroy.argtypes = [vp]
    lib.fabm_last_error.argtypes = []
    lib.fabm_last_error.restype = ctypes.c_char_p
    lib.fabm_set_block.argtypes = [vp, i]
    lib.fabm_get_block.argtypes = [vp]
    lib.fabm_last_launch_count.argtypes = [vp]
    lib.fabm_last_launch_count.restype = i64
    lib.fabm_copy_weights.argtypes = [vp, i64, P(d), P(d), P(d)]
    lib.fabm_copy_weights_lo.argtypes = [vp, i64, P(d), P(d), P(d)]
    lib.fabm_copy_weights_lo.restype = i
    lib.fabm_set_timing.argtypes = [vp, i]
    lib.fabm_set_graphs.argtypes = [vp, i]
    lib.fabm_server_create.argtypes = [ctypes.c_size_t, i, i, P(vp)]
    lib.fabm_server_submit.argtypes = [vp, P(fabm_request), P(i64)]
    lib.fabm_server_submit_ic.argtypes = [vp, P(fabm_request), P(d), P(i64)]
    lib.fabm_server_step.argtypes = [vp, P(i), P(i)]
    lib.fabm_server_poll.argtypes = [vp, i64, P(i)]
    lib.fabm_server_result.argtypes = [vp, i64, P(d)]
    lib.fabm_server_wait.argtypes = [vp, i64, P(d)]
    lib.fabm_server_stats.argtypes = [vp, P(i64), P(i64), P(ctypes.c_size_t)]
    lib.fabm_server_destroy.argtypes = [vp]
    lib.fabm_server_checkpoint.argtypes = [vp, i64, vp, ctypes.c_size_t, P(ctypes.c_size_t)]
    lib.fabm_server_resume.argtypes = [vp, vp, ctypes.c_size_t, P(i64)]
    lib.fabm_server_cancel.argtypes = [vp, i64]
    lib.fabm_server_shape.argtypes = [vp, i64, P(i64), P(i)]
    lib.fabm_server_finished.argtypes = [vp, P(i64), i, P(i)]
    for f in ("fabm_server_create", "fabm_server_submit", "fabm_server_submit_ic",
              "fabm_server_step", "fabm_server_poll",
              "fabm_server_result", "fabm_server_wait", "fabm_server_stats", "fabm_server_destroy",
              "fabm_server_checkpoint", "fabm_server_resume", "fabm_server_cancel",
              "fabm_server_shape", "fabm_server_finished"):
        getattr(lib, f).restype = i
    lib.fabm_autotune.argtypes = [vp, i64, P(d), P(d), i64, i, P(d), P(i), P(i), P(i)]
    lib.fabm_autotune.restype = i
    lib.fabm_set_history_kernel.argtypes = [vp, i]
    lib.fabm_get_history_kernel.argtypes = [vp]
    lib.fabm_last_history_kernel.argtypes = [vp]
    lib.fabm_set_recurrence_warps.argtypes = [vp, i]
    lib.fabm_get_recurrence_warps.argtypes = [vp]
    lib.fabm_set_recurrence_layout.argtypes = [vp, i]
    lib.fabm_weights_x2.argtypes = [d, i64] + [P(d)] * 6
    lib.fabm_weights_x2.restype = i
    lib.fabm_get_recurrence_layout.argtypes = [vp]
    lib.fabm_solve_noalloc.argtypes = [i, d, d, i64, i, P(d), i, P(d), P(d)]
    lib.fabm_kernel_stats.argtypes = [vp, i, P(i64), P(d), P(d)]
    lib.fabm_kernel_busy.argtypes = [vp, i, P(d)]
    lib.fabm_kernel_busy.restype = i
    lib.fabm_stroboscope.argtypes = [vp, i64, i64, i, vp, d, d, d, i64, i, vp]
    lib.fabm_stroboscope.restype = i
    lib.fabm_set_wait_limit.argtypes = [vp, i64]
    lib.fabm_set_wait_limit.restype = i
    lib.fabm_inject_alloc_failures.argtypes = [i]
    lib.fabm_inject_alloc_failures.restype = i
    for f in ("fabm_create", "fabm_create_multi", "fabm_solve", "fabm_solve_batch",
              "fabm_solve_batch_ic",
              "fabm_destroy", "fabm_set_block",
              "fabm_get_block", "fabm_copy_weights", "fabm_set_timing", "fabm_kernel_stats",
              "fabm_set_graphs", "fabm_solve_noalloc", "fabm_set_history_kernel",
              "fabm_get_history_kernel", "fabm_set_recurrence_layout",
              "fabm_get_recurrence_layout", "fabm_last_history_kernel",
              "fabm_set_recurrence_warps", "fabm_get_recurrence_warps"):
        getattr(lib, f).restype = i
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(st: int):
    if st != FABM_OK:
        raise FabmError(st, fabm_last_error())


# ------------------------------------------------------------- C names ---

def fabm_last_error() -> str:
    return load().fabm_last_error().decode()


def fabm_create(dim, alpha, h, N, rhs_id, params, precision=FABM_FP64):
    """alpha: one order, or a sequence of dim orders (fabm_create_multi)."""
    p = _f64(params if params is not None else []).reshape(-1)
    handle = ctypes.c_void_p()
    if np.ndim(alpha) > 0:
        al = _f64(alpha).reshape(-1)
        _check(load().fabm_create_multi(int(dim), _dp(al), float(h), int(N), int(rhs_id),
                                        _dp(p) if p.size else None, int(p.size), int(precision),
                                        ctypes.byref(handle)))
        return handle
    _check(load().fabm_create(int(dim), float(alpha), float(h), int(N), int(rhs_id),
                              _dp(p) if p.size else None, int(p.size), int(precision),
                              ctypes.byref(handle)))
    return handle


def fabm_stroboscope(Y, N, h, t0, period, n_samples, comp=0, N_each=None):
    """Samples of the device trajectories Y (torch tensor B x (N+1) x dim on the
    GPU) at t0 + j*period, linearly interpolated; returns a device tensor
    B x n_samples.  N_each: optional device int64 tensor of B step counts."""
    import torch
    if not (Y.is_cuda and Y.dtype == torch.float64 and Y.is_contiguous() and Y.dim() == 3):
        raise ValueError("Y must be a contiguous float64 CUDA tensor B x (N+1) x dim")
    B, rows, dim = Y.shape
    if rows != N + 1:
        raise ValueError(f"Y has {rows} rows per trajectory, expected N+1 = {N + 1}")
    out = torch.empty((B, int(n_samples)), dtype=torch.float64, device=Y.device)
    ne = None
    if N_each is not None:
        if not (N_each.is_cuda and N_each.dtype == torch.int64 and N_each.numel() == B):
            raise ValueError("N_each must be a CUDA int64 tensor of B entries")
        ne = ctypes.c_void_p(N_each.data_ptr())
    with torch.cuda.device(Y.device):
        _check(load().fabm_stroboscope(ctypes.c_void_p(Y.data_ptr()), int(B), int(N), int(dim),
                                       ne, float(h), float(t0), float(period), int(n_samples),
                                       int(comp), ctypes.c_void_p(out.data_ptr())))
    return out


def fabm_solve(handle, y0, out):
    _check(load().fabm_solve(handle, _dp(y0), _dp(out)))


def fabm_solve_batch(handle, B, y0, traj_params, N_each, out_ptr, out_on_device):
    ne = None
    if N_each is not None:
        ne = N_each.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(load().fabm_solve_batch(handle, int(B), _dp(y0), _dp(traj_params), ne,
                                   ctypes.c_void_p(out_ptr), int(out_on_device)))


def fabm_solve_batch_ic(handle, B, y0, y1, traj_params, N_each, out_ptr, out_on_device):
    ne = None
    if N_each is not None:
        ne = N_each.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    _check(load().fabm_solve_batch_ic(handle, int(B), _dp(y0), _dp(y1), _dp(traj_params), ne,
                                      ctypes.c_void_p(out_ptr), int(out_on_device)))


def fabm_destroy(handle):
    _check(load().fabm_destroy(handle))


def fabm_set_block(handle, L):
    _check(load().fabm_set_block(handle, int(L)))


def fabm_get_block(handle) -> int:
    return load().fabm_get_block(handle)


def fabm_copy_weights(handle, n):
    """(B, A, D) device weights, n entries each (see include/fabm.h)."""
    B, A, D = np.empty(n), np.empty(n), np.empty(n)
    _check(load().fabm_copy_weights(handle, int(n), _dp(B), _dp(A), _dp(D)))
    return B, A, D


def fabm_copy_weights_lo(handle, n):
    """Low parts (Bl, Al, Dl) of an FP64X2 solver's double-double weights, d < n."""
    Bl, Al, Dl = np.empty(n), np.empty(n), np.empty(n)
    _check(load().fabm_copy_weights_lo(handle, int(n), _dp(Bl), _dp(Al), _dp(Dl)))
    return Bl, Al, Dl


def fabm_weights_x2(alpha: float, n: int):
    """Double-double weights (B_hi, B_lo, A_hi, A_lo, D_hi, D_lo), n+1 entries
    each, computed on the host in binary128 (no GPU needed)."""
    out = [np.empty(int(n) + 1) for _ in range(6)]
    _check(load().fabm_weights_x2(float(alpha), int(n), *[_dp(a) for a in out]))
    return tuple(out)


def fabm_last_launch_count(handle) -> int:
    return load().fabm_last_launch_count(handle)


def fabm_solve_noalloc(dim, alpha, h, N, rhs_id, params, y0, out):
    """One FP64 trajectory without device allocation (see include/fabm.h);
    out: host float64 array of (N+1) x dim entries."""
    p = _f64(params if params is not None else []).reshape(-1)
    y0 = _f64(y0).reshape(-1)
    _check(load().fabm_solve_noalloc(int(dim), float(alpha), float(h), int(N), int(rhs_id),
                                     _dp(p) if p.size else None, int(p.size), _dp(y0),
                                     _dp(out)))


def fabm_set_history_kernel(handle, kernel):
    k = HIST[kernel] if isinstance(kernel, str) else int(kernel)
    _check(load().fabm_set_history_kernel(handle, k))


def fabm_get_history_kernel(handle) -> int:
    return load().fabm_get_history_kernel(handle)


def fabm_set_recurrence_warps(handle, warps: int):
    """Warps per CTA of the lane-per-column recurrence (0: automatic, 1..12)."""
    _check(load().fabm_set_recurrence_warps(handle, int(warps)))


def fabm_get_recurrence_warps(handle) -> int:
    return load().fabm_get_recurrence_warps(handle)


def fabm_last_history_kernel(handle) -> int:
    """FABM_HIST_* that the last solve ran (-1 before the first)."""
    return load().fabm_last_history_kernel(handle)


def fabm_set_recurrence_layout(handle, layout):
    """Recurrence layout of the tensor-history path: "auto", "columns" or "targets"."""
    k = RECURRENCE[layout] if isinstance(layout, str) else int(layout)
    _check(load().fabm_set_recurrence_layout(handle, k))


def fabm_get_recurrence_layout(handle) -> int:
    return load().fabm_get_recurrence_layout(handle)


def fabm_set_graphs(handle, enable: bool):
    _check(load().fabm_set_graphs(handle, int(bool(enable))))


def fabm_set_timing(handle, period):
    _check(load().fabm_set_timing(handle, int(period)))


def fabm_kernel_stats(handle, kind):
    """(launches, total_ms, flops) of one kernel class (name or id)."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    n, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(load().fabm_kernel_stats(handle, k, ctypes.byref(n), ctypes.byref(ms),
                                    ctypes.byref(fl)))
    return n.value, ms.value, fl.value


def fabm_kernel_busy(handle, kind):
    """Milliseconds during which the timed launches of one kind ran (overlaps once)."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ms = ctypes.c_double()
    _check(load().fabm_kernel_busy(handle, k, ctypes.byref(ms)))
    return ms.value


def fabm_set_wait_limit(handle, cycles: int):
    _check(load().fabm_set_wait_limit(handle, int(cycles)))


def fabm_inject_alloc_failures(n: int):
    _check(load().fabm_inject_alloc_failures(int(n)))


# ---------------------------------------------------------- convenience ---

class Solver:
    """Owns one fabm_solver.  ``rhs`` and ``precision`` are names or ids."""

    def __init__(self, rhs, dim, alpha, h, N, params=None, precision="fp64", block=None,
                 history=None, recurrence=None):
        self.rhs = RHS[rhs] if isinstance(rhs, str) else int(rhs)
        self.dim, self.h, self.N = int(dim), float(h), int(N)
        self.alpha = tuple(float(a) for a in alpha) if np.ndim(alpha) > 0 else float(alpha)
        self.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self.params = _f64(params if params is not None else []).reshape(-1)
        self.handle = fabm_create(dim, alpha, h, N, self.rhs, self.params, self.precision)
        if block is not None:
            fabm_set_block(self.handle, block)
        if history is not None:
            fabm_set_history_kernel(self.handle, history)
        if recurrence is not None:
            fabm_set_recurrence_layout(self.handle, recurrence)

    def close(self):
        if self.handle is not None and self.handle.value:
            fabm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def block(self) -> int:
        return fabm_get_block(self.handle)

    @block.setter
    def block(self, L: int):
        fabm_set_block(self.handle, L)

    def weights(self, n=None):
        return fabm_copy_weights(self.handle, self.N + 1 if n is None else n)

    @property
    def last_launch_count(self) -> int:
        return fabm_last_launch_count(self.handle)

    @property
    def last_history_kernel(self) -> str:
        """Name (as in HIST) of the history kernel the last solve ran, or None."""
        k = fabm_last_history_kernel(self.handle)
        return next((n for n, v in HIST.items() if v == k and n != "auto"), None)

    def autotune(self, y0, traj_params=None, n_probe=4096):
        """Time truncated solves of this batch for each candidate setting, keep
        the fastest; returns [(ms, history kernel, CTA target), ...]."""
        y0 = _f64(y0).reshape(-1, self.dim)
        B = y0.shape[0]
        tp = None if traj_params is None else _f64(traj_params).reshape(B, -1)
        ms = np.zeros(8)
        kern = (ctypes.c_int * 8)()
        ctas = (ctypes.c_int * 8)()
        n = ctypes.c_int()
        _check(load().fabm_autotune(self.handle, B, _dp(y0), _dp(tp), int(n_probe), 8, _dp(ms),
                                    kern, ctas, ctypes.byref(n)))
        return [(float(ms[i]), int(kern[i]), int(ctas[i])) for i in range(min(n.value, 8))]

    def set_graphs(self, enable: bool = True):
        fabm_set_graphs(self.handle, enable)

    def set_wait_limit(self, cycles: int = 0):
        """Clock cycles after which the tensor kernel's waits give up (0: default)."""
        fabm_set_wait_limit(self.handle, cycles)

    def set_timing(self, period: int = 1):
        """period > 0: time the launches of every period-th block; 0: off."""
        fabm_set_timing(self.handle, int(period))

    def kernel_stats(self) -> dict:
        """Per kernel class: timed launches, their summed durations (ms), the time
        they ran with overlaps counted once (busy_ms) and their algorithmic flops."""
        out = {}
        for k in KERNEL_KINDS:
            st = dict(zip(("launches", "ms", "flops"), fabm_kernel_stats(self.handle, k)))
            st["busy_ms"] = fabm_kernel_busy(self.handle, k)
            out[k] = st
        return out

    def solve(self, y0, y1=None) -> np.ndarray:
        """One trajectory; y1 = y'(0) for 1 < alpha < 2."""
        y0 = _f64(y0).reshape(-1)
        if y0.size != self.dim:
            raise ValueError("y0 must have dim entries")
        if y1 is not None:
            return self.solve_batch(y0.reshape(1, -1), y1=_f64(y1).reshape(1, -1))[0]
        out = np.empty((self.N + 1, self.dim))
        fabm_solve(self.handle, y0, out)
        return out

    def solve_batch(self, y0, traj_params=None, N_each=None, out=None, y1=None):
        """y0 (and y1 = y'(0), for 1 < alpha < 2): (B, dim).  out: None (a new
        host array), a host float64 array of shape (B, N+1, dim), or a CUDA
        tensor of that shape (written in place on the device).  Returns out."""
        y0 = _f64(y0).reshape(-1, self.dim)
        B = y0.shape[0]
        y1 = None if y1 is None else _f64(y1).reshape(B, self.dim)
        tp = None if traj_params is None else _f64(traj_params).reshape(B, -1)
        ne = None if N_each is None else np.ascontiguousarray(np.asarray(N_each, np.int64))
        if out is None:
            out = np.full((B, self.N + 1, self.dim), np.nan)
        on_dev = 0
        if isinstance(out, np.ndarray):
            if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != B * (self.N + 1) * self.dim:
                raise ValueError("out must be a C-contiguous float64 array of shape (B, N+1, dim)")
            ptr = out.ctypes.data
        else:  # a torch tensor (host or CUDA)
            if not out.is_contiguous() or out.numel() != B * (self.N + 1) * self.dim:
                raise ValueError("out must be contiguous with B*(N+1)*dim elements")
            if str(out.dtype) != "torch.float64":
                raise ValueError("out must be float64")
            ptr = out.data_ptr()
            on_dev = 1 if out.is_cuda else 0
        if y1 is None:
            fabm_solve_batch(self.handle, B, y0, tp, ne, ptr, on_dev)
        else:
            fabm_solve_batch_ic(self.handle, B, y0, y1, tp, ne, ptr, on_dev)
        return out


class Server:
    """Owns one fabm_server (continuous batching of independent solves)."""

    def __init__(self, budget_bytes, precision="fp64", max_slots=4096):
        self.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        _check(load().fabm_server_create(int(budget_bytes), self.precision, int(max_slots),
                                         ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(load().fabm_server_destroy(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, rhs, dim, alpha, h, N, y0, params=None, y1=None) -> int:
        """Queue a request; y1 = y'(0) (dim values) for 1 < alpha < 2."""
        rid = RHS[rhs] if isinstance(rhs, str) else int(rhs)
        p = _f64(params if params is not None else []).reshape(-1)
        y = _f64(y0).reshape(-1)
        req = fabm_request(int(dim), float(alpha), float(h), int(N), rid,
                           _dp(p) if p.size else None, int(p.size), _dp(y))
        t = ctypes.c_int64()
        if y1 is None:
            _check(load().fabm_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        else:
            v = _f64(y1).reshape(-1)
            if v.size != int(dim):
                raise ValueError("y1 needs dim values")
            _check(load().fabm_server_submit_ic(self.handle, ctypes.byref(req), _dp(v),
                                                ctypes.byref(t)))
        return t.value

    def step(self):
        a, w = ctypes.c_int(), ctypes.c_int()
        _check(load().fabm_server_step(self.handle, ctypes.byref(a), ctypes.byref(w)))
        return a.value, w.value

    def poll(self, ticket) -> int:
        st = ctypes.c_int()
        _check(load().fabm_server_poll(self.handle, int(ticket), ctypes.byref(st)))
        return st.value

    def shape(self, ticket):
        """(N, dim) of a known request."""
        n, d = ctypes.c_int64(), ctypes.c_int()
        _check(load().fabm_server_shape(self.handle, int(ticket), ctypes.byref(n), ctypes.byref(d)))
        return n.value, d.value

    def result(self, ticket) -> np.ndarray:
        N, dim = self.shape(ticket)
        out = np.empty((N + 1, dim))
        _check(load().fabm_server_result(self.handle, int(ticket), _dp(out)))
        return out

    def wait(self, ticket) -> np.ndarray:
        """Step the server until the request has finished; its (N+1, dim) result."""
        N, dim = self.shape(ticket)
        out = np.empty((N + 1, dim))
        _check(load().fabm_server_wait(self.handle, int(ticket), _dp(out)))
        return out

    def checkpoint(self, ticket) -> bytes:
        """Serialized state of a waiting or running request (it keeps running)."""
        size = ctypes.c_size_t()
        _check(load().fabm_server_checkpoint(self.handle, int(ticket), None, 0, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        _check(load().fabm_server_checkpoint(self.handle, int(ticket), buf, size.value,
                                             ctypes.byref(size)))
        return buf.raw[: size.value]

    def resume(self, state: bytes) -> int:
        """Queue a request from a checkpoint; returns its ticket."""
        t = ctypes.c_int64()
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(load().fabm_server_resume(self.handle, buf, len(state), ctypes.byref(t)))
        return t.value

    def cancel(self, ticket):
        _check(load().fabm_server_cancel(self.handle, int(ticket)))

    def finished(self, max_n=65536):
        """Tickets that finished since the last call."""
        buf = (ctypes.c_int64 * max_n)()
        n = ctypes.c_int()
        out = []
        while True:
            _check(load().fabm_server_finished(self.handle, buf, max_n, ctypes.byref(n)))
            out.extend(buf[: n.value])
            if n.value < max_n:
                return out

    def stats(self):
        s, l, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(load().fabm_server_stats(self.handle, ctypes.byref(s), ctypes.byref(l),
                                        ctypes.byref(b)))
        return {"steps": s.value, "launches": l.value, "bytes_in_use": b.value}
