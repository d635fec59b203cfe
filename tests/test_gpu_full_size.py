"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (one batch solve with the output on the device; the served stream of
the served-mix line), on trajectories sampled across the batch that the
oracle computes one by one (needs a GPU).  Bars: 1e-6 of the solution scale
for the split path."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from fabm_workloads import duffing_sweep, lcr_sweep, lorenz_long, served_stream

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _cores():
    return max(1, os.cpu_count() or 1)


def duffing_horizons():
    """(index, F, horizon) of the sampled oscillators (tests/golden/make_oracle_refs.py)."""
    out = []
    for ln in open(os.path.join(GOLDEN, "duffing_sweep_horizons.txt")):
        if ln.strip() and not ln.startswith("#"):
            i, F, H = ln.split()
            out.append((int(i), float(F), int(H)))
    return out


def served_live():
    """request id -> (rhs, k, horizon) of the k = 15, 16 requests."""
    out = {}
    for ln in open(os.path.join(GOLDEN, "served_horizons.txt")):
        if ln.strip() and not ln.startswith("#"):
            rid, rhs, k, H = ln.split()
            out[int(rid)] = (rhs, int(k), int(H))
    return out


def served_stored():
    """request id -> (rhs, k, horizon, stride, rows) of the k = 17, 18 requests."""
    out, cur = {}, None
    for ln in open(os.path.join(GOLDEN, "served_k17_k18.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        t = ln.split()
        if t[0] == "request":
            cur = int(t[1])
            out[cur] = [t[2], int(t[4]), int(t[6]), int(t[8]), []]
        else:
            out[cur][4].append([float(v) for v in t[1:]])
    return {k: (v[0], v[1], v[2], v[3], np.array(v[4])) for k, v in out.items()}


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
    """4096 oscillators x 2^16 steps (tensor history); 18 amplitudes across the
    sweep against the oracle, each over its whole pre-divergence horizon
    (tests/golden/duffing_sweep_horizons.txt: the full 65,536 steps where a
    1e-7 change of x0 never moves the oracle's solution by 1e-6 of its scale,
    0.8 x the step where it does on a chaotic attractor)."""
    w = duffing_sweep()
    Yd, block = _device_solve(gpu_lib, w)
    assert block == 64
    import torch
    assert bool(torch.isfinite(Yd).all())
    assert float(Yd.abs().max()) < 10.0  # bounded forced oscillators
    hz = duffing_horizons()
    idx = np.array([i for i, _, _ in hz])
    assert np.allclose([F for _, F, _ in hz], w.traj_params[idx, 2], rtol=0, atol=1e-15)
    sub = w.subset(idx)
    ref = oracle.solve_batch(sub.rhs, sub.alpha, sub.h, sub.N, sub.y0, params=sub.params,
                             traj_params=sub.traj_params, threads=_cores())
    got = Yd[idx].cpu().numpy()
    full = 0
    for j, (i, F, H) in enumerate(hz):
        full += H == w.N
        parity(rel_err(got[j, : H + 1], ref[j, : H + 1]), 1e-6, f"duffing-F{F:.3f}-to{H}")
    assert full >= len(hz) // 2, "most sampled amplitudes are compared over the whole run"


def test_lorenz_long_full_size_split(gpu_lib, parity):
    """256 Lorenz trajectories x 2^20 steps in split precision (the FP64 solve
    of this size takes ~45 min); three of them against the oracle over t <= 5
    (50,000 steps), the horizon the workload states."""
    w = lorenz_long()
    w.precision = "split"
    Yd, block = _device_solve(gpu_lib, w)
    assert block == 64
    _check_sampled(parity, w, Yd, np.array([0, 128, 255]), w.compare_steps, "lorenz-long-split")


def test_lorenz_long_fp64_launch_shape(gpu_lib, parity):
    """The FP64 path at the width of the long-horizon batch (256 Lorenz
    trajectories, 768 columns, lag-2 schedule on two history streams), cut to
    N = 2^17 (the full 2^20 takes ~45 min in FP64): four trajectories against
    the oracle over t <= 5 (50,000 steps) at the FP64 bar."""
    w = lorenz_long()
    w = w.subset(np.arange(w.B), N=2 ** 17)
    w.precision = "fp64"
    Yd, block = _device_solve(gpu_lib, w)
    assert block == 32
    import torch
    assert bool(torch.isfinite(Yd).all())
    idx = np.array([0, 85, 170, 255])
    n_cmp = 50_000
    got = Yd[idx, : n_cmp + 1].cpu().numpy()
    sub = w.subset(idx, N=n_cmp)
    ref = oracle.solve_batch(sub.rhs, sub.alpha, sub.h, n_cmp, sub.y0, params=sub.params,
                             threads=4)
    for j, b in enumerate(idx):
        parity(rel_err(got[j], ref[j]), 1e-12, f"lorenz-long-fp64-traj{b}")


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


def test_served_long_requests_against_the_oracle(gpu_lib, parity):
    """Requests of the full served stream (20,000 requests, k = 12..18) with
    N = 2^15 .. 2^18, one per right-hand side and k, served together with the
    stream's first 64 requests: k = 15, 16 against the oracle run here, k = 17,
    18 against stored oracle rows (tests/golden/served_k17_k18.txt, every
    N/512-th step), each over its pre-divergence horizon."""
    reqs = served_stream(n=20_000, rate=1e12, k_lo=12, k_hi=18)
    live, stored = served_live(), served_stored()
    picked = sorted(set(live) | set(stored))
    assert {live[i][1] for i in live} == {15, 16} and {v[1] for v in stored.values()} == {17, 18}
    with cf.ThreadPoolExecutor(len(live)) as ex:
        fut = {i: ex.submit(oracle.solve, reqs[i].rhs, reqs[i].alpha, reqs[i].h, reqs[i].N,
                            reqs[i].y0, params=reqs[i].params) for i in live}
        with gpu_lib.Server(120 << 30, precision="split") as srv:
            extra = [r for r in reqs[:64] if r.rid not in picked]
            tickets = {r.rid: srv.submit(r.rhs, r.dim, r.alpha, r.h, r.N, r.y0, r.params)
                       for r in [reqs[i] for i in picked] + extra}
            results = {i: srv.wait(tickets[i]) for i in picked}
        refs = {i: f.result() for i, f in fut.items()}
    for i in picked:
        r = reqs[i]
        got = results[i]
        assert got.shape == (r.N + 1, r.dim) and np.all(np.isfinite(got))
        if i in live:
            rhs, k, H = live[i]
            ref = refs[i][: H + 1]
            g = got[: H + 1]
        else:
            rhs, k, H, stride, rows = stored[i]
            steps = np.arange(rows.shape[0]) * stride
            keep = steps <= H
            ref, g = rows[keep], got[steps[keep]]
        assert rhs == r.rhs
        parity(rel_err(g, ref), 1e-6, f"req{i}-{rhs}-k{k}-to{H}")
