"""fabm_solve_noalloc: the solve for callers that cannot allocate device memory.

Those callers (a framework whose caching allocator owns the whole device
budget, code that must not synchronize the device through cudaMalloc/cudaFree,
plug-ins whose host forbids them allocations) get a variant of the FP64 solve
whose buffers live in one fixed device array inside the library.  These tests
call it through the C ABI twice in a row, with different problem sizes so the
second call reuses the array the first one left behind, and compare each
result with fabm_solve on the same inputs and with the CPU oracle, both at the
FP64 bar (1e-12 of the solution scale).  The array's limits are reached too:
65,536 steps with four components fill every region of it, and a call in a
process that has already made one must not change the device's free memory.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import concurrent.futures as cf
import ctypes

import numpy as np
import pytest

import oracle
from fabm_workloads import duffing_sweep, lorenz_single, ml_scalar

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


def _oracle(w, N):
    return oracle.solve(w.rhs, w.alpha, w.h, N, w.y0[0], params=w.params)


def test_noalloc_matches_solve_on_two_calls_in_a_row(gpu_lib, parity):
    lib = gpu_lib.load()
    cases = [(lorenz_single(N=20_000), 20_000), (ml_scalar(), 10_000)]
    with cf.ThreadPoolExecutor(2) as ex:
        refs = list(ex.map(lambda c: _oracle(*c), cases))
    for (w, N), orc in zip(cases, refs):
        st, got = _noalloc(lib, w, N)
        assert st == gpu_lib.FABM_OK, gpu_lib.fabm_last_error()
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, N, w.params) as s:
            ref = s.solve(w.y0[0])
        assert np.all(np.isfinite(got))
        parity(rel_err(got, ref), TOL_FP64, f"{w.rhs}-vs-solve")
        parity(rel_err(got, orc), TOL_FP64, f"{w.rhs}-vs-oracle")


def _four_component_linear():
    """D^a y = -p y with four components: the largest dim at the largest N."""
    w = ml_scalar(N=65_536)
    w.dim = 4
    w.y0 = np.array([[1.0, -2.0, 0.5, 3.0]])
    return w


def test_noalloc_at_the_limits_of_its_array(gpu_lib, parity):
    """N = 65536 with dim = 4 (every region of the array full, the last block
    ending on the last rows of the history and the output, the weights at their
    widest) and N = 65535 (a ragged last block), each called twice in a row:
    equal to fabm_solve and to the oracle, and the second call leaves the
    device's free memory unchanged."""
    import torch
    lib = gpu_lib.load()
    w4 = _four_component_linear()
    wd = duffing_sweep(B=1, N=65_535).subset(np.array([0]))
    with cf.ThreadPoolExecutor(5) as ex:
        # the linear components are independent scalar solves: one oracle
        # trajectory per component, in parallel
        f4 = ex.submit(oracle.solve_batch, "linear", w4.alpha, w4.h, w4.N,
                       w4.y0.reshape(4, 1), params=w4.params, threads=4)
        fd = ex.submit(oracle.solve_batch, wd.rhs, wd.alpha, wd.h, wd.N, wd.y0,
                       params=wd.params, traj_params=wd.traj_params)
        orc4 = f4.result()[:, :, 0].T
        orcd = fd.result()[0]
    cases = [(w4, orc4, None), (wd, orcd, tuple(wd.traj_params[0]))]
    for w, orc, p in cases:
        if p is not None:
            w.params = p
        st, got = _noalloc(lib, w, w.N)
        assert st == gpu_lib.FABM_OK, gpu_lib.fabm_last_error()
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
            ref = s.solve(w.y0[0])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st2, again = _noalloc(lib, w, w.N)
        free1 = torch.cuda.mem_get_info()[0]
        assert st2 == gpu_lib.FABM_OK, gpu_lib.fabm_last_error()
        assert free1 == free0, (free0, free1)
        assert np.array_equal(again, got)
        parity(rel_err(got, ref), TOL_FP64, f"{w.rhs}-N{w.N}-vs-solve")
        parity(rel_err(got, orc), TOL_FP64, f"{w.rhs}-N{w.N}-vs-oracle")


def test_noalloc_rejects_sizes_beyond_its_array(gpu_lib):
    lib = gpu_lib.load()
    w = ml_scalar()
    st, _ = _noalloc(lib, w, 65_537)
    assert st == gpu_lib.FABM_EINVAL
    assert "at most 65536 steps" in gpu_lib.fabm_last_error()
