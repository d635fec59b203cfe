"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (one batch solve with the output on the device; the served stream of
the served-mix line), on trajectories sampled across the batch that the
oracle computes one by one (needs a GPU).  Bars: 1e-6 of the solution scale
for the split path."""
import numpy as np
import pytest

import oracle
from fabm_workloads import duffing_sweep, lcr_sweep, lorenz_long, served_stream

pytestmark = pytest.mark.gpu


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


def _device_solve(gpu_lib, w):
    import torch
    Yd = torch.empty((w.B, w.N + 1, w.dim), dtype=torch.float64, device="cuda")
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision=w.precision) as s:
        s.solve_batch(w.y0, traj_params=w.traj_params, N_each=w.N_each, out=Yd)
        block = s.block
    return Yd, block


def _check_sampled(parity, w, Yd, idx, n_cmp, label):
    import torch
    assert bool(torch.isfinite(Yd).all())
    got = Yd[idx, : n_cmp + 1].cpu().numpy()
    sub = w.subset(idx, N=n_cmp)
    ref = oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n_cmp, sub.y0, params=sub.params,
                             traj_params=sub.traj_params)
    for j, b in enumerate(idx):
        parity(rel_err(got[j], ref[j]), 1e-6, f"{label}-traj{b}")


def test_duffing_sweep_full_size(gpu_lib, parity):
    """4096 oscillators x 2^16 steps (tensor history, blocks of 64); four
    amplitudes across the sweep against the oracle over the first 16384 steps."""
    w = duffing_sweep()
    Yd, block = _device_solve(gpu_lib, w)
    assert block == 64
    _check_sampled(parity, w, Yd, np.array([0, 1, 2047, 4095]), 16384, "duffing")
    assert float(Yd.abs().max()) < 10.0  # bounded forced oscillators


def test_lorenz_long_full_size_split(gpu_lib, parity):
    """256 Lorenz trajectories x 2^20 steps in split precision (the FP64 solve
    of this size takes ~45 min); three of them against the oracle over t <= 5
    (50,000 steps), the horizon the workload states."""
    w = lorenz_long()
    w.precision = "split"
    Yd, block = _device_solve(gpu_lib, w)
    assert block == 64
    _check_sampled(parity, w, Yd, np.array([0, 128, 255]), w.compare_steps, "lorenz-long-split")


def test_lcr_sweep_bench_size(gpu_lib, parity):
    """The bench's LCR sweep (1024 amplitudes x 2^14 steps, split); three
    trajectories against the oracle over t <= 40 (the sweep turns chaotic
    above f ~ 0.13, where a 1e-8 perturbation reaches 1e-6 from t ~ 54), the
    whole horizon bounded."""
    w = lcr_sweep(B=1024, N=2 ** 14)
    w.precision = "split"
    Yd, _ = _device_solve(gpu_lib, w)
    _check_sampled(parity, w, Yd, np.array([0, 511, 1023]), w.compare_steps, "lcr")
    assert float(Yd.abs().max()) < 10.0


def test_served_mix_bench_size(gpu_lib, parity):
    """The served-mix bench line's stream (2000 requests, N = 2^12..2^14, split),
    all queued at once; six requests against the oracle."""
    reqs = served_stream(n=2000, rate=1e9, k_lo=12, k_hi=14)
    with gpu_lib.Server(120 << 30, precision="split") as srv:
        tickets = [srv.submit(r.rhs, r.dim, r.alpha, r.h, r.N, r.y0, r.params) for r in reqs]
        while any(srv.poll(t) < gpu_lib.FABM_REQ_DONE for t in tickets):
            srv.step()
        pick = [0, 1, 2, 999, 1998, 1999]
        results = {i: srv.result(tickets[i]) for i in pick}
    for i in pick:
        r = reqs[i]
        ref = oracle.solve(r.rhs, r.alpha, r.h, r.N, r.y0, params=r.params)
        parity(rel_err(results[i], ref), 1e-6, f"req{i}-{r.rhs}-N{r.N}")
