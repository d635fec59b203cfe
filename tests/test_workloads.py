"""The synthetic input recipe (no GPU): the seeded generators produce the
shapes, ranges and parameters the documented workloads state, and SplitMix64
matches its published definition."""
import numpy as np

from fabm_workloads import (LCR_PARAMS, LORENZ_PARAMS, SEED_BASE, duffing_sweep, lcr_sweep,
                            lorenz_long, lorenz_single, ml_scalar, served_stream, splitmix64,
                            uniform)


def _splitmix64_scalar(seed, n):
    """SplitMix64 written with Python integers, one output at a time."""
    m = (1 << 64) - 1
    x, out = seed & m, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & m
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_the_scalar_definition():
    for seed in (0, 1, SEED_BASE, 2 ** 64 - 1):
        assert [int(v) for v in splitmix64(seed, 64)] == _splitmix64_scalar(seed, 64)
    u = uniform(SEED_BASE, 10_000, -2.0, 3.0)
    assert u.min() >= -2.0 and u.max() < 3.0
    assert abs(u.mean() - 0.5) < 0.05  # 5 / sqrt(12 * 10^4) ~ 0.014


def test_single_trajectory_workloads():
    w = ml_scalar()
    assert (w.rhs, w.dim, w.alpha, w.h, w.N) == ("linear", 1, 0.8, 1e-3, 10_000)
    assert np.array_equal(w.y0, [[1.0]]) and w.params == (1.0,)
    w = lorenz_single()
    assert (w.rhs, w.dim, w.alpha, w.h, w.N) == ("lorenz", 3, 0.98, 5e-4, 2 ** 18)
    assert w.params == LORENZ_PARAMS
    assert np.all(np.abs(w.y0 - 1.0) <= 0.01) and w.compare_steps * w.h <= 10.0 + 1e-12


def test_duffing_sweep_grid():
    w = duffing_sweep()
    assert (w.B, w.dim, w.alpha, w.h, w.N) == (4096, 2, 0.95, 1e-3, 2 ** 16)
    F = w.traj_params[:, 2]
    assert F[0] == 0.1 and abs(F[-1] - 2.0) < 1e-12
    assert np.allclose(np.diff(F), 1.9 / 4095)
    assert np.all(w.traj_params[:, 0] == 0.1) and np.all(w.traj_params[:, 1] == 1.2)
    assert np.all(w.y0 == 0.0)


def test_lorenz_long_and_lcr_sweep():
    w = lorenz_long()
    assert (w.B, w.alpha, w.h, w.N) == (256, 0.95, 1e-4, 2 ** 20)
    assert np.all(np.abs(w.y0 - 1.0) <= 0.05) and w.compare_steps == 50_000
    w = lcr_sweep(B=1024)
    f = w.traj_params[:, 4]
    assert f[0] == 0.0 and abs(f[-1] - 0.2) < 1e-15 and np.all(np.diff(f) > 0)
    assert np.all(w.traj_params[:, :4] == np.array(LCR_PARAMS))
    assert np.all(np.abs(w.y0) <= 0.1) and w.compare_steps * w.h <= 40.0 + 1e-9


def test_served_stream_distribution():
    reqs = served_stream(n=6000, rate=100.0, k_lo=12, k_hi=18)
    arr = np.array([r.arrival for r in reqs])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    assert abs(np.mean(np.diff(arr)) - 1 / 100.0) < 0.1 / 100.0  # Poisson gaps, mean 1/rate
    kinds = [r.rhs for r in reqs]
    for rhs, dim in (("linear", 1), ("duffing", 2), ("lorenz", 3)):
        share = kinds.count(rhs) / len(reqs)
        assert abs(share - 1 / 3) < 0.03
        assert all(r.dim == dim for r in reqs if r.rhs == rhs)
    alphas = np.array([r.alpha for r in reqs])
    assert alphas.min() >= 0.7 and alphas.max() < 0.99
    ks = np.log2([r.N for r in reqs])
    assert set(np.round(ks).astype(int)) == set(range(12, 19))
    assert all(r.h == 1e-3 for r in reqs)
    # deterministic: the same seed gives the same stream
    again = served_stream(n=6000, rate=100.0, k_lo=12, k_hi=18)
    assert all(a.N == b.N and np.array_equal(a.y0, b.y0) for a, b in zip(reqs, again))
