"""GPU parity of the plain FP64 path against the CPU oracle (needs a GPU).

Every solve goes through the C ABI (libfabm.so).  The bar is the FP64 one:
max over steps of |y_gpu - y_oracle| / S_i <= 1e-12, where S_i is the largest
|y_oracle| of component i of the trajectory (the solution scale; pointwise
relative error is meaningless at zero crossings).  The GPU sums the history
in blocked order and the oracle sequentially, so the two differ by rounding
order only.
"""
import math

import numpy as np
import pytest

import oracle
from fabm_workloads import (LORENZ_PARAMS, duffing_sweep, lcr_sweep, lorenz_long, lorenz_single,
                            ml_scalar, uniform, SEED_BASE)

pytestmark = pytest.mark.gpu
TOL_FP64 = 1e-12


def rel_err(got, ref):
    """max_n |got - ref| / max_n |ref| per component, maximised over components
    (and trajectories for batched arrays)."""
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


def test_weights_match_oracle(gpu_lib):
    for alpha in (0.3, 0.7, 0.95, 0.99):
        N = 70000
        with gpu_lib.Solver("linear", 1, alpha, 1e-3, N, [1.0]) as s:
            B, A, D = s.weights()
        b, a, c = oracle.weights(alpha, N)
        np.testing.assert_allclose(B[1:], b, rtol=2e-15, atol=0)
        np.testing.assert_allclose(A[1:], a, rtol=2e-15, atol=0)
        np.testing.assert_allclose(D[1:], c - a, rtol=4e-15, atol=0)
        assert B[0] == 0 and A[0] == 0 and D[0] == 0


def test_weights_large_distance(gpu_lib):
    N = 2 ** 20
    with gpu_lib.Solver("linear", 1, 0.95, 1e-4, N, [1.0]) as s:
        B, A, D = s.weights()
    b, a, c = oracle.weights(0.95, N)
    idx = np.r_[1:200, N - 200:N]
    np.testing.assert_allclose(B[idx], b[idx - 1], rtol=2e-15)
    np.testing.assert_allclose(A[idx], a[idx - 1], rtol=2e-15)
    np.testing.assert_allclose(D[idx], (c - a)[idx - 1], rtol=4e-15)


@pytest.mark.parametrize("N", [1, 2, 31, 32, 33, 63, 64, 65, 97, 1000, 1027])
def test_constant_rhs_closed_form(gpu_lib, N):
    """f = const: y = y0 + const t^a/Gamma(a+1) exactly (Sec. 2 weights integrate
    constants exactly); block edges and a ragged tail."""
    alpha, h = 0.6, 0.01
    with gpu_lib.Solver("const", 2, alpha, h, N, [1.5]) as s:
        y = s.solve([0.25, -1.0])
    t = np.arange(N + 1) * h
    ex = 1.5 * t ** alpha / math.gamma(alpha + 1)
    np.testing.assert_allclose(y[:, 0], 0.25 + ex, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(y[:, 1], -1.0 + ex, rtol=1e-14, atol=1e-15)


def test_time_rhs_closed_form(gpu_lib):
    alpha, h, N = 0.45, 0.02, 777
    with gpu_lib.Solver("time", 1, alpha, h, N) as s:
        y = s.solve([0.5])
    t = np.arange(N + 1) * h
    np.testing.assert_allclose(y[:, 0], 0.5 + t ** (alpha + 1) / math.gamma(alpha + 2),
                               rtol=1e-14, atol=1e-15)


def test_mittag_leffler_config_vs_oracle(gpu_lib, parity):
    w = ml_scalar()
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL_FP64, "")


def test_lorenz_config_vs_oracle(gpu_lib, parity):
    """Lorenz-type, a = 0.98, h = 5e-4, compared for t <= 10 (20,000 steps)."""
    w = lorenz_single(N=20_000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL_FP64, "")


def test_lorenz_full_size_prefix_vs_oracle(gpu_lib, parity):
    """The full N = 2^18 solve, as the bench launches it; its first 20,000 steps
    (t <= 10) against the oracle, the rest checked for finiteness and for the
    bound every trajectory of this system obeys (it stays in a ball of radius
    ~ rho + sigma around (0, 0, rho + sigma))."""
    w = lorenz_single()
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve(w.y0[0])
    n = w.compare_steps
    ref = oracle.solve(w.rhs, w.alpha, w.h, n, w.y0[0], params=w.params)
    parity(rel_err(got[: n + 1], ref), TOL_FP64, "")
    assert np.all(np.isfinite(got))
    c = np.array([0.0, 0.0, LORENZ_PARAMS[0] + LORENZ_PARAMS[1]])
    assert np.max(np.linalg.norm(got - c, axis=1)) < 2 * (LORENZ_PARAMS[0] + LORENZ_PARAMS[1])


def test_batch_uneven_lengths_and_params(gpu_lib, parity):
    """Duffing sweep shape: per-trajectory forcing, uneven N, ragged tails;
    rows past N_each stay untouched."""
    w = duffing_sweep(B=37, N=1500)
    ne = np.array([1500, 1, 32, 33, 1000, 1499] * 6 + [7], dtype=np.int64)
    y0 = uniform(SEED_BASE + 99, 2 * w.B, -0.5, 0.5).reshape(w.B, 2)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve_batch(y0, traj_params=w.traj_params, N_each=ne)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, y0, params=w.params,
                             traj_params=w.traj_params, N_each=ne)
    for b in range(w.B):
        parity(rel_err(got[b, : ne[b] + 1], ref[b, : ne[b] + 1]), TOL_FP64, b)
        assert np.all(np.isnan(got[b, ne[b] + 1:]))


def test_lcr_paper_system(gpu_lib, parity):
    w = lcr_sweep(B=8, N=3000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params,
                             traj_params=w.traj_params)
    parity(rel_err(got, ref), TOL_FP64, "")


def test_manufactured_solution(gpu_lib, parity):
    alpha = 0.8
    kappa = 2.0 / math.gamma(3.0 - alpha)
    N = 640
    with gpu_lib.Solver("manufactured", 1, alpha, 1.0 / N, N, [kappa, 2.0 - alpha, 2.0]) as s:
        got = s.solve([0.0])
    ref = oracle.solve("manufactured", alpha, 1.0 / N, N, [0.0], params=[kappa, 2.0 - alpha, 2.0])
    parity(rel_err(got, ref), TOL_FP64, "")
    t = np.arange(N + 1) / N
    assert np.max(np.abs(got[:, 0] - t * t)) < 1e-4


def test_lorenz_long_subset_vs_oracle(gpu_lib, parity):
    """4 trajectories of the long-horizon batch, t <= 5 at h = 1e-4 (50,000 steps)."""
    w = lorenz_long().subset(np.arange(4), N=50_000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        got = s.solve_batch(w.y0)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params)
    parity(rel_err(got, ref), TOL_FP64, "")


def test_batch_equals_singles_bitwise(gpu_lib):
    w = lorenz_single(N=700)
    y0 = np.concatenate([w.y0, w.y0 + 0.3, w.y0 - 0.2])
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        batch = s.solve_batch(y0)
        singles = [s.solve(y0[i]) for i in range(3)]
        again = s.solve_batch(y0)
    for i in range(3):
        assert np.array_equal(batch[i], singles[i])
    assert np.array_equal(batch, again)


def test_output_on_device(gpu_lib):
    torch = pytest.importorskip("torch")
    w = lorenz_single(N=300)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        dev = torch.empty((1, w.N + 1, 3), dtype=torch.float64, device="cuda")
        s.solve_batch(w.y0, out=dev)
        host = s.solve_batch(w.y0)
    assert np.array_equal(dev.cpu().numpy(), host)


def test_empty_batch_and_nonfinite_detection(gpu_lib):
    with gpu_lib.Solver("linear", 1, 0.9, 0.1, 5000, [-50.0]) as s:
        s.solve_batch(np.zeros((0, 1)))
        with pytest.raises(gpu_lib.FabmError) as ei:
            s.solve([1.0])
    assert ei.value.status == gpu_lib.FABM_ENONFINITE
    ref = oracle.solve("linear", 0.9, 0.1, 5000, [1.0], params=[-50.0])
    first_bad = int(np.argmax(~np.isfinite(ref[:, 0])))
    step = int(str(ei.value).split("step ")[-1])
    assert abs(step - first_bad) <= 1


def test_graph_replay_matches_direct_launches(gpu_lib):
    """The cached CUDA graph of a solve gives bit-identical results to direct
    launches, across new inputs of the same shape."""
    w = lorenz_single(N=1500)
    y0b = np.concatenate([w.y0, w.y0 + 0.1])
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params) as s:
        s.set_graphs(False)
        direct = s.solve_batch(y0b, N_each=[1500, 999])
        s.set_graphs(True)
        g1 = s.solve_batch(y0b, N_each=[1500, 999])
        g2 = s.solve_batch(y0b[::-1].copy(), N_each=[999, 1500])
    assert np.array_equal(direct[0], g1[0]) and np.array_equal(direct[1, :1000], g1[1, :1000])
    assert np.array_equal(g2[0, :1000], direct[1, :1000]) and np.array_equal(g2[1], direct[0])


@pytest.mark.parametrize("B", [1, 3, 16])
def test_persistent_solve_matches_the_oracle_and_the_graph_schedule(gpu_lib, parity, B):
    """The FP64 solve as one persistent cooperative launch (recurrence CTAs and
    history CTAs handing blocks over through device flags) against the oracle
    at 1e-12, and against the schedule of one launch per kernel and block;
    uneven lengths, including one inside the first far block and one on a
    block edge."""
    w = lorenz_single(N=6000)
    y0 = w.y0 + np.linspace(-0.05, 0.05, B)[:, None]
    ne = np.full(B, w.N, dtype=np.int64)
    if B > 1:
        ne[1] = 77
    if B > 2:
        ne[-1] = 4096
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, y0, params=w.params, N_each=ne,
                             threads=min(B, 16))
    out = {}
    for hist in ("fp64-persist", "fp64"):
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, history=hist) as s:
            out[hist] = s.solve_batch(y0, N_each=ne)
            if hist == "fp64-persist":
                assert s.last_launch_count <= 3  # initial values + the persistent launch
    for b in range(B):
        n = ne[b]
        for hist, got in out.items():
            parity(rel_err(got[b, : n + 1], ref[b, : n + 1]), TOL_FP64, f"{hist}-{b}")


def test_persistent_solve_scalar_and_manufactured(gpu_lib, parity):
    """One component (no exchange between warps): the Mittag-Leffler workload
    through the persistent launch."""
    w = ml_scalar()
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, history="fp64-persist") as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL_FP64, "ml")
