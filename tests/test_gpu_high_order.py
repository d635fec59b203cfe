"""Orders 1 < alpha < 2 (needs a GPU): the same weights, with the Taylor part
y0 + t y'(0) of Sec. 2's formulas; FP64 path against the oracle at 1e-12 of
the solution scale, split path (both history kernels) at 1e-6."""
import math

import numpy as np
import pytest

import oracle
from fabm_workloads import SEED_BASE, duffing_sweep, uniform

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


def test_weights_match_oracle_above_one(gpu_lib):
    for alpha in (1.2, 1.5, 1.9):
        N = 70000
        with gpu_lib.Solver("linear", 1, alpha, 1e-3, N, [1.0]) as s:
            B, A, D = s.weights()
        b, a, c = oracle.weights(alpha, N)
        np.testing.assert_allclose(B[1:], b, rtol=2e-15, atol=0)
        np.testing.assert_allclose(A[1:], a, rtol=2e-15, atol=0)
        np.testing.assert_allclose(D[1:], c - a, rtol=4e-15, atol=0)


@pytest.mark.parametrize("N", [1, 31, 32, 33, 65, 1000])
def test_constant_rhs_closed_form_above_one(gpu_lib, N):
    alpha, h = 1.5, 0.01
    with gpu_lib.Solver("const", 2, alpha, h, N, [1.5]) as s:
        y = s.solve([0.25, -1.0], y1=[-0.7, 2.0])
    t = np.arange(N + 1) * h
    ex = 1.5 * t ** alpha / math.gamma(alpha + 1)
    np.testing.assert_allclose(y[:, 0], 0.25 - 0.7 * t + ex, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(y[:, 1], -1.0 + 2.0 * t + ex, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("precision,hist", [("fp64", None), ("split", "fp32c"),
                                            ("split", "tensor")])
def test_oscillator_vs_oracle(gpu_lib, parity, precision, hist):
    """D^1.5 y = -y with y(0) = (1, 0), y'(0) = (0, 1): both Mittag-Leffler
    solutions of the damped fractional oscillator, 3000 steps."""
    alpha, h, N = 1.5, 2e-3, 3000
    y0, y1 = [1.0, 0.0], [0.0, 1.0]
    with gpu_lib.Solver("linear", 2, alpha, h, N, [1.0], precision=precision,
                        history=hist) as s:
        got = s.solve(y0, y1=y1)
    ref = oracle.solve("linear", alpha, h, N, y0, params=[1.0], y1=y1)
    parity(rel_err(got, ref), 1e-12 if precision == "fp64" else 1e-6, hist or "fp64")


@pytest.mark.parametrize("precision,rec", [("fp64", None), ("split", "columns"),
                                            ("split", "targets")])
def test_forced_oscillator_batch_above_one(gpu_lib, parity, precision, rec):
    """A sweep of 300 forced oscillators at alpha = 1.3 with their own y'(0)
    and uneven lengths (600 columns: tensor history in split precision, both
    recurrence layouts)."""
    w = duffing_sweep(B=300, N=1500)
    alpha = 1.3
    y0 = uniform(SEED_BASE + 71, 2 * w.B, -0.5, 0.5).reshape(w.B, 2)
    y1 = uniform(SEED_BASE + 72, 2 * w.B, -0.5, 0.5).reshape(w.B, 2)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[::5] = 999
    with gpu_lib.Solver(w.rhs, w.dim, alpha, w.h, w.N, w.params, precision=precision,
                        recurrence=rec) as s:
        got = s.solve_batch(y0, traj_params=w.traj_params, N_each=ne, y1=y1)
    idx = np.r_[0:6, 147:151, 294:300]
    ref = oracle.solve_batch(w.rhs, alpha, w.h, w.N, y0[idx], params=w.params,
                             traj_params=w.traj_params[idx], N_each=ne[idx], y1=y1[idx])
    tol = 1e-12 if precision == "fp64" else 1e-6
    for j, b in enumerate(idx):
        n = ne[b]
        parity(rel_err(got[b, : n + 1], ref[j, : n + 1]), tol, b)


def test_y1_rejected_below_one(gpu_lib):
    with gpu_lib.Solver("linear", 1, 0.8, 1e-3, 100, [1.0]) as s:
        with pytest.raises(gpu_lib.FabmError) as e:
            s.solve([1.0], y1=[0.5])
    assert e.value.status == gpu_lib.FABM_EINVAL
