"""GPU parity of the FP64X2 precision (double-double history) against the oracle.

FP64X2 keeps the history sums to about twice double precision (weights in
double-double, exact products, compensated sums and combination) and the steps
of a block in double.  The bar is the FP64 one, max_n |y - y_oracle| / S_i <=
1e-12; the constant right-hand side, whose history telescopes to t^alpha
exactly, pins the sums to a few units in the last place of y.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from fabm_workloads import duffing_sweep, lcr_sweep, lorenz_single, ml_scalar

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


def test_x2_constant_rhs_is_t_to_the_alpha_to_a_few_ulp(gpu_lib, parity):
    """f = c: y_m = y0 + c (m h)^a / Gamma(a+1) exactly, so y_m / y_1 = m^a.
    Checked against m^a to 30 digits for every m up to 40000 (about 1250
    blocks of history)."""
    alpha, h, N, c = 0.7, 0.01, 40_000, 1.5
    with gpu_lib.Solver("const", 1, alpha, h, N, [c], precision="fp64x2") as s:
        y = s.solve([0.0])[:, 0]
    with gpu_lib.Solver("const", 1, alpha, h, N, [c], precision="fp64") as s:
        y64 = s.solve([0.0])[:, 0]
    getcontext().prec = 30
    a = Decimal(alpha)
    m = np.arange(1, N + 1)
    ref = np.array([float(Decimal(int(k)) ** a) for k in m])
    err_x2 = float(np.max(np.abs(y[1:] / y[1] - ref) / ref))
    err_64 = float(np.max(np.abs(y64[1:] / y64[1] - ref) / ref))
    parity(err_x2, 2e-15, "fp64x2")
    parity(err_64, TOL, "fp64 (for comparison)")


@pytest.mark.parametrize("case", ["ml", "lorenz"])
def test_x2_single_trajectory_vs_oracle(gpu_lib, parity, case):
    w = ml_scalar() if case == "ml" else lorenz_single(N=20_000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64x2") as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL, case)


def test_x2_batch_with_uneven_lengths_vs_oracle(gpu_lib, parity):
    w = duffing_sweep(B=70, N=3000)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[::9] = 1234
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64x2") as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params, N_each=ne)
    idx = np.r_[0:4, 33:36, 66:70]
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx], N_each=ne[idx])
    for j, b in enumerate(idx):
        n = ne[b]
        parity(rel_err(got[b, : n + 1], ref[j, : n + 1]), TOL, b)


def test_x2_two_orders_and_above_one_vs_oracle(gpu_lib, parity):
    """One order per component, one of them above 1 with y'(0)."""
    w = lcr_sweep(B=8, N=2000)
    alphas = [0.9, 1.2]
    y1 = np.zeros_like(w.y0)
    y1[:, 1] = 0.05
    with gpu_lib.Solver(w.rhs, w.dim, alphas, w.h, w.N, w.params, precision="fp64x2") as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params, y1=y1)
    ref = oracle.solve_batch(w.rhs, alphas, w.h, w.N, w.y0, params=w.params,
                             traj_params=w.traj_params, y1=y1)
    parity(rel_err(got, ref), TOL, "")


def test_x2_history_kernel_and_autotune(gpu_lib, parity):
    w = ml_scalar(N=3000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64x2") as s:
        assert gpu_lib.fabm_get_history_kernel(s.handle) == gpu_lib.HIST["auto"]
        with pytest.raises(gpu_lib.FabmError):
            gpu_lib.fabm_set_history_kernel(s.handle, "fp64")
        gpu_lib.fabm_set_history_kernel(s.handle, "x2")
        rep = s.autotune(w.y0, n_probe=1000)
        assert len(rep) == 4 and all(k == gpu_lib.HIST["x2"] for _, k, _ in rep)
        got = s.solve(w.y0[0])
        B, A, D = gpu_lib.fabm_copy_weights(s.handle, 100)
    Bh, _, Ah, _, Dh, _ = gpu_lib.fabm_weights_x2(w.alpha, 99)
    assert np.array_equal(B, Bh) and np.array_equal(A, Ah) and np.array_equal(D, Dh)
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL, "")
    with pytest.raises(gpu_lib.FabmError):
        gpu_lib.Server(1 << 30, precision="fp64x2")


@pytest.mark.parametrize("case", ["ml", "lorenz"])
def test_x2_against_the_binary128_oracle(gpu_lib, parity, case):
    """The double-double mode against the oracle run entirely in binary128 (its
    weights, sums and steps), which pins the oracle's own rounding too."""
    w = ml_scalar(N=2000) if case == "ml" else lorenz_single(N=2000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64x2") as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve_q(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL, case)


@pytest.mark.parametrize("alpha", [0.3, 0.95, 1.5])
def test_device_double_double_weights_match_binary128(gpu_lib, alpha):
    """The FP64X2 solver computes its weights on the device in double-double
    (printed differences up to d = 64, non-cancelling series beyond); they agree
    with the host's binary128 evaluation of the same weights (pinned against
    50-digit values on the CPU) to 1e-27 relative, and their high parts are the
    doubles nearest to them."""
    N = 70_000
    with gpu_lib.Solver("linear", 1, alpha, 1e-3, N, [1.0], precision="fp64x2") as s:
        Bh, Ah, Dh = s.weights(N + 1)
        Bl, Al, Dl = gpu_lib.fabm_copy_weights_lo(s.handle, N + 1)
    hb, lb, ha, la, hd, ld = gpu_lib.fabm_weights_x2(alpha, N)
    for name, dh, dl, rh, rl in (("B", Bh, Bl, hb, lb), ("A", Ah, Al, ha, la),
                                 ("D", Dh, Dl, hd, ld)):
        diff = (dh[1:] - rh[1:]) + (dl[1:] - rl[1:])
        rel = np.abs(diff) / np.abs(rh[1:])
        assert float(rel.max()) < 1e-27, (name, int(rel.argmax()) + 1, float(rel.max()))
        assert np.all(np.abs(dl[1:]) <= 0.5 * np.spacing(np.abs(dh[1:]))), name
        assert dh[0] == 0.0 and dl[0] == 0.0
