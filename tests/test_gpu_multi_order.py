"""One fractional order per component (needs a GPU): the GPU solver built with
fabm_create_multi against the oracle (FP64: 1e-12, split: 1e-6 of the
solution scale), and its reductions to the single-order solver."""
import numpy as np
import pytest

import oracle
from fabm_workloads import LCR_PARAMS, lcr_sweep, lorenz_single

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_lcr_two_orders_vs_oracle(gpu_lib, parity, precision):
    """The paper's LCR system with alpha1 = 0.9, alpha2 = 0.8 over a small
    amplitude sweep."""
    w = lcr_sweep(B=8, N=3000)
    al = [0.9, 0.8]
    with gpu_lib.Solver(w.rhs, w.dim, al, w.h, w.N, w.params, precision=precision) as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
    ref = oracle.solve_batch(w.rhs, al, w.h, w.N, w.y0, params=w.params,
                             traj_params=w.traj_params)
    parity(rel_err(got, ref), 1e-12 if precision == "fp64" else 1e-6, precision)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_lorenz_three_orders_vs_oracle(gpu_lib, parity, precision):
    w = lorenz_single(N=5000)
    al = [0.97, 0.93, 0.88]
    with gpu_lib.Solver(w.rhs, w.dim, al, w.h, w.N, w.params, precision=precision) as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, al, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), 1e-12 if precision == "fp64" else 1e-6, precision)


def test_orders_above_and_below_one(gpu_lib, parity):
    al = [0.6, 1.5]
    y0, y1 = [[1.0, 0.5], [0.2, -1.0]], [[0.0, 0.7], [0.0, 0.1]]
    with gpu_lib.Solver("linear", 2, al, 2e-3, 2000, [1.0]) as s:
        got = s.solve_batch(y0, y1=y1)
    ref = oracle.solve_batch("linear", al, 2e-3, 2000, y0, params=[1.0], y1=y1)
    parity(rel_err(got, ref), 1e-12)


def test_uncoupled_components_match_scalar_solves_bitwise(gpu_lib):
    al = [0.55, 0.9, 0.75]
    y0 = [1.0, -2.0, 0.5]
    N = 1500
    with gpu_lib.Solver("linear", 3, al, 1e-3, N, [0.8]) as s:
        y = s.solve(y0)
    for i, a in enumerate(al):
        # the same schedule as the multi-order solve (single-order FP64 batches
        # of few trajectories default to the persistent kernel)
        with gpu_lib.Solver("linear", 1, a, 1e-3, N, [0.8], history="fp64") as s1:
            yi = s1.solve([y0[i]])
        assert np.array_equal(y[:, i], yi[:, 0]), i


def test_equal_orders_is_the_single_order_solver(gpu_lib):
    w = lorenz_single(N=2000)
    with gpu_lib.Solver(w.rhs, 3, [w.alpha] * 3, w.h, w.N, w.params) as s:
        a = s.solve(w.y0[0])
    with gpu_lib.Solver(w.rhs, 3, w.alpha, w.h, w.N, w.params) as s:
        b = s.solve(w.y0[0])
    assert np.array_equal(a, b)
