"""fabm_solve_noalloc: the solve for callers that cannot allocate device memory.

Those callers (a framework whose caching allocator owns the whole device
budget, code that must not synchronize the device through cudaMalloc/cudaFree,
plug-ins whose host forbids them allocations) get a variant of the FP64 solve
whose buffers live in one fixed device array inside the library.  These tests
call it through the C ABI twice in a row, with different problem sizes so the
second call reuses the array the first one left behind, and compare each
result with fabm_solve on the same inputs at the FP64 bar (1e-12 of the
solution scale).  This file is collected last on purpose: if it fails, a run
that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from fabm_workloads import lorenz_single, ml_scalar

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12


def rel_err(got, ref):
    scale = np.max(np.abs(ref), axis=0, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(got - ref) / scale))


def _noalloc(lib, w, N):
    out = np.full((N + 1, w.dim), np.nan)
    p = np.ascontiguousarray(np.asarray(w.params, dtype=np.float64))
    y0 = np.ascontiguousarray(w.y0[0], dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.fabm_solve_noalloc(w.dim, w.alpha, w.h, N, _rhs_id(w.rhs), p.ctypes.data_as(dp),
                                p.size, y0.ctypes.data_as(dp), out.ctypes.data_as(dp))
    return st, out


def _rhs_id(name):
    import paper_1710_01133_gb300 as fabm
    return fabm.RHS[name]


def test_noalloc_matches_solve_on_two_calls_in_a_row(gpu_lib, parity):
    lib = gpu_lib.load()
    cases = [(lorenz_single(N=20_000), 20_000), (ml_scalar(), 10_000)]
    for w, N in cases:
        st, got = _noalloc(lib, w, N)
        assert st == gpu_lib.FABM_OK, gpu_lib.fabm_last_error()
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, N, w.params) as s:
            ref = s.solve(w.y0[0])
        assert np.all(np.isfinite(got))
        parity(rel_err(got, ref), TOL_FP64, "")


def test_noalloc_rejects_sizes_beyond_its_array(gpu_lib):
    lib = gpu_lib.load()
    w = ml_scalar()
    st, _ = _noalloc(lib, w, 65_537)
    assert st == gpu_lib.FABM_EINVAL
    assert "at most 65536 steps" in gpu_lib.fabm_last_error()
