"""The paper's own LCR workload (Sec. 5) on the GPU: the forced series LCR
circuit swept over the forcing amplitude, its equilibria at f = 0, and the
stroboscopic sampling behind the bifurcation diagram (needs a GPU)."""
import math
import os

import numpy as np
import pytest

import oracle
from fabm_workloads import LCR_PARAMS, lcr_sweep

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lcr_section5.txt")


def golden():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def rel_err(got, ref):
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(got - ref) / scale))


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_equilibria_stay_fixed(gpu_lib, precision):
    """E0 and E+- of Sec. 5 (closed form printed there) are fixed points at f = 0."""
    g = golden()
    s, a, b = g["sigma"], g["a"], g["b"]
    xe = s * (a - b) / (1 + s * b)
    ye = (b - a) / (1 + s * b)
    y0 = np.array([[0.0, 0.0], [xe, ye], [-xe, -ye]])
    tp = np.array([[s, g["omega"], a, b, 0.0]] * 3)
    with gpu_lib.Solver("lcr", 2, g["alpha1"], 0.01, 2000, tp[0], precision=precision) as sv:
        Y = sv.solve_batch(y0, traj_params=tp)
    tol = 1e-12 if precision == "fp64" else 1e-6
    for k in range(3):
        dev = np.max(np.abs(Y[k] - y0[k]))
        assert dev <= tol * max(1.0, np.max(np.abs(y0[k]))), (k, dev)


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_stroboscope_of_sweep_vs_oracle(gpu_lib, parity, precision):
    """Bifurcation-diagram samples (once per forcing period) of a 16-amplitude
    sweep: GPU solve + GPU sampler against the oracle's trajectories sampled
    on the CPU."""
    import torch
    w = lcr_sweep(B=16, N=4000)
    period = 2 * math.pi / LCR_PARAMS[1]
    t0, ns = 0.5 * period, 4  # t = 5.7 .. 40.0, inside the horizon T = 40
    Yd = torch.empty((w.B, w.N + 1, 2), dtype=torch.float64, device="cuda")
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision=precision) as s:
        s.solve_batch(w.y0, traj_params=w.traj_params, out=Yd)
    ref_traj = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params,
                                  traj_params=w.traj_params)
    scale = np.max(np.abs(ref_traj), axis=1)  # (B, dim)
    for comp in (0, 1):
        got = gpu_lib.fabm_stroboscope(Yd, w.N, w.h, t0, period, ns, comp=comp).cpu().numpy()
        ref = oracle.stroboscope(ref_traj, w.h, t0, period, ns, comp=comp)
        assert not np.isnan(ref).any() and not np.isnan(got).any()
        err = float(np.max(np.abs(got - ref) / scale[:, comp:comp + 1]))
        parity(err, 1e-12 if precision == "fp64" else 1e-6, f"comp{comp}")
        # the sampler alone: same trajectories in, interpolation only (the two
        # ways of forming the weight t/h - n differ by rounding, ~1e-16 of t/h)
        mine = oracle.stroboscope(Yd.cpu().numpy(), w.h, t0, period, ns, comp=comp)
        assert np.max(np.abs(got - mine) / scale[:, comp:comp + 1]) <= 1e-13


def test_stroboscope_edges(gpu_lib):
    import torch
    B, N, dim, h = 3, 100, 2, 0.5
    t = np.arange(N + 1) * h
    Y = np.zeros((B, N + 1, dim))
    for b in range(B):
        Y[b, :, 0] = 1.0 + b + 0.25 * t       # linear: interpolation is exact
        Y[b, :, 1] = -t * (b + 1)
    Yd = torch.tensor(Y, device="cuda")
    # samples from before 0 to past the end, including grid points and t = N h
    t0, period, ns = -0.75, 2.5, 23
    got = gpu_lib.fabm_stroboscope(Yd, N, h, t0, period, ns, comp=1).cpu().numpy()
    tj = t0 + np.arange(ns) * period
    inside = (tj >= 0) & (tj <= N * h)
    assert np.all(np.isnan(got[:, ~inside]))
    ex = -np.outer(np.arange(1, B + 1), tj[inside])
    np.testing.assert_allclose(got[:, inside], ex, rtol=1e-15, atol=1e-13)
    # ragged lengths: samples past N_each[b] h are NaN
    ne = torch.tensor([100, 40, 1], dtype=torch.int64, device="cuda")
    got = gpu_lib.fabm_stroboscope(Yd, N, h, 0.0, 0.5, N + 1, comp=0, N_each=ne).cpu().numpy()
    for b, nb in enumerate([100, 40, 1]):
        np.testing.assert_allclose(got[b, : nb + 1], Y[b, : nb + 1, 0], rtol=1e-15)
        assert np.all(np.isnan(got[b, nb + 1:]))
    with pytest.raises(gpu_lib.FabmError) as e:
        gpu_lib.fabm_stroboscope(Yd, N, h, 0.0, 1.0, 4, comp=2)
    assert e.value.status == gpu_lib.FABM_EINVAL
