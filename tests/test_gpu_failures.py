"""Failure paths that can be exercised without faulting a GPU (needs a GPU).

* The tensor-core history kernel's bounded waits: with a wait limit of a few
  clock cycles every wait on another warp gives up at once, the CTA records the
  timeout, drains its own copies and MMAs, frees its tensor memory and
  returns; the solve reports FABM_ETIMEOUT, and the next solve on the same
  solver (default limit) is correct against the oracle.
* Device allocations: host-side injected failures (no allocator call) make the
  solve or the server admission that needed the memory fail with FABM_ENOMEM,
  and the solver or server keeps working.
"""
import numpy as np
import pytest

import oracle
from fabm_workloads import duffing_sweep

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


@pytest.mark.parametrize("hist", ["tensor", "tensor-wide"])
def test_tensor_kernel_wait_timeout_is_reported_and_the_solver_recovers(gpu_lib, parity, hist):
    w = duffing_sweep(B=96, N=700)  # 192 columns: two column tiles, 11 blocks
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                        history=hist) as s:
        s.set_wait_limit(16)
        with pytest.raises(gpu_lib.FabmError) as e:
            s.solve_batch(w.y0, traj_params=w.traj_params)
        assert e.value.status == gpu_lib.FABM_ETIMEOUT
        s.set_wait_limit(0)  # back to the default
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
    idx = np.array([0, 50, 95])
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx])
    for j, b in enumerate(idx):
        parity(rel_err(got[b], ref[j]), 1e-6, f"after-timeout-traj{b}")


def test_injected_allocation_failure_in_a_solve(gpu_lib, parity):
    w = duffing_sweep(B=8, N=300)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        gpu_lib.fabm_inject_alloc_failures(1)
        try:
            with pytest.raises(gpu_lib.FabmError) as e:
                s.solve_batch(w.y0, traj_params=w.traj_params)
        finally:
            gpu_lib.fabm_inject_alloc_failures(0)
        assert e.value.status == gpu_lib.FABM_ENOMEM
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params,
                             traj_params=w.traj_params)
    parity(rel_err(got, ref), 1e-12, "after-enomem")


def test_injected_allocation_failure_in_a_solver_creation(gpu_lib):
    gpu_lib.fabm_inject_alloc_failures(1)
    try:
        with pytest.raises(gpu_lib.FabmError) as e:
            gpu_lib.Solver("linear", 1, 0.8, 1e-3, 1000, (1.0,))
    finally:
        gpu_lib.fabm_inject_alloc_failures(0)
    assert e.value.status == gpu_lib.FABM_ENOMEM
    with gpu_lib.Solver("linear", 1, 0.8, 1e-3, 1000, (1.0,)) as s:
        assert np.all(np.isfinite(s.solve([1.0])))


def test_injected_allocation_failure_in_a_server_admission(gpu_lib, parity):
    with gpu_lib.Server(1 << 30) as srv:
        gpu_lib.fabm_inject_alloc_failures(1)
        try:
            lost = srv.submit("linear", 1, 0.8, 1e-3, 500, [1.0], (1.0,))
            srv.step()  # admission: its allocation fails, nothing else is running
        finally:
            gpu_lib.fabm_inject_alloc_failures(0)
        assert srv.poll(lost) == gpu_lib.FABM_REQ_FAILED
        with pytest.raises(gpu_lib.FabmError) as e:
            srv.result(lost)
        assert e.value.status == gpu_lib.FABM_ENOMEM
        ok = srv.submit("linear", 1, 0.8, 1e-3, 500, [1.0], (1.0,))
        got = srv.wait(ok)
    parity(rel_err(got, oracle.solve("linear", 0.8, 1e-3, 500, [1.0], params=[1.0])), 1e-12,
           "after-enomem")


def test_persistent_fp64_wait_timeout_is_reported_and_the_solver_recovers(gpu_lib, parity):
    """The persistent FP64 launch's flag waits: with a 16-cycle limit the first
    wait gives up, every CTA leaves its loop, the solve reports FABM_ETIMEOUT;
    with the default limit the next solve is correct."""
    from fabm_workloads import lorenz_single
    w = lorenz_single(N=3000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, history="fp64-persist") as s:
        s.set_wait_limit(16)
        with pytest.raises(gpu_lib.FabmError) as e:
            s.solve(w.y0[0])
        assert e.value.status == gpu_lib.FABM_ETIMEOUT
        s.set_wait_limit(0)
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), 1e-12, "after-timeout")
