"""GPU parity of the split (tensor-core) path against the CPU oracle.

The history sums run as bf16 tcgen05 products of fixed-point slices; the bar
is the mixed-precision one: max_n |y_gpu - y_oracle| / S_i <= 1e-6, S_i the
largest |y_oracle| of component i of the trajectory.  Sizes span several
64-point segments, several 128-column tiles and ragged tails.  Both tensor
tilings run: "tensor-wide" (far history of pairs of blocks, 128 targets per
MMA, 128-point groups) and "tensor" (64 targets per MMA, 64-point segments).
"""
import math

import numpy as np
import pytest

import oracle
from fabm_workloads import (duffing_sweep, lcr_sweep, lorenz_long, lorenz_single, ml_scalar,
                            uniform, SEED_BASE)

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-6
HISTS = ["tensor-wide", "tensor", "fp32c"]
# history kernel and, on the tensor path, the recurrence layout
PATHS = [("tensor-wide", "columns"), ("tensor-wide", "targets"), ("tensor", "columns"),
         ("tensor", "targets"), ("fp32c", None)]


def rel_err(got, ref):
    ref = np.asarray(ref)
    scale = np.max(np.abs(ref), axis=-2, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(np.asarray(got) - ref) / scale))


@pytest.mark.parametrize("hist,rec", PATHS)
@pytest.mark.parametrize("N", [1, 31, 32, 33, 63, 64, 65, 128, 129, 193, 1000])
def test_split_constant_rhs_closed_form(gpu_lib, N, hist, rec):
    alpha, h = 0.7, 0.01
    with gpu_lib.Solver("const", 1, alpha, h, N, [1.5], precision="split", history=hist,
                        recurrence=rec) as s:
        y = s.solve([0.25])
    t = np.arange(N + 1) * h
    ex = 0.25 + 1.5 * t ** alpha / math.gamma(alpha + 1)
    assert np.max(np.abs(y[:, 0] - ex)) / np.max(np.abs(ex)) < TOL_SPLIT


@pytest.mark.parametrize("hist", HISTS)
def test_split_mittag_leffler(gpu_lib, parity, hist):
    w = ml_scalar()
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist) as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL_SPLIT, "")


@pytest.mark.parametrize("hist", HISTS)
def test_split_lorenz_prefix(gpu_lib, parity, hist):
    w = lorenz_single(N=20_000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist) as s:
        got = s.solve(w.y0[0])
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    parity(rel_err(got, ref), TOL_SPLIT, "")


@pytest.mark.parametrize("hist,rec", PATHS)
def test_split_duffing_batch_several_column_tiles(gpu_lib, parity, hist, rec):
    """300 trajectories x 2 = 600 columns: five 128-column tiles, the last one
    ragged; uneven lengths."""
    w = duffing_sweep(B=300, N=3000)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[::7] = 1777
    ne[3] = 1
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist,
                        recurrence=rec) as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params, N_each=ne)
    idx = np.r_[0:8, 150:154, 292:300]
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx], N_each=ne[idx])
    for j, b in enumerate(idx):
        n = ne[b]
        parity(rel_err(got[b, : n + 1], ref[j, : n + 1]), TOL_SPLIT, b)


@pytest.mark.parametrize("hist", ["tensor-wide", "tensor"])
@pytest.mark.parametrize("rec", ["columns", "targets"])
def test_split_lorenz_batch_partial_warps(gpu_lib, parity, rec, hist):
    """23 Lorenz trajectories on the tensor path: the column recurrence puts 10
    trajectories (30 columns) in a warp, so the warps hold 10, 10 and 3 of them
    and two lanes of each warp idle; lengths differ inside a warp, including
    one that ends inside the first block and one that ends on a block edge."""
    w = lorenz_long().subset(np.arange(23), N=2000)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[::6] = 777
    ne[[1, 13, 21]] = [5, 1280, 1999]
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                        history=hist, recurrence=rec) as s:
        got = s.solve_batch(w.y0, N_each=ne)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params, N_each=ne)
    for b in range(w.B):
        n = ne[b]
        parity(rel_err(got[b, : n + 1], ref[b, : n + 1]), TOL_SPLIT, b)


@pytest.mark.parametrize("hist", HISTS)
def test_split_matches_fp64_gpu_on_lcr(gpu_lib, parity, hist):
    w = lcr_sweep(B=16, N=4000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist) as s:
        sp = s.solve_batch(w.y0, traj_params=w.traj_params)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64") as s:
        dp = s.solve_batch(w.y0, traj_params=w.traj_params)
    parity(rel_err(sp, dp), TOL_SPLIT, "")


@pytest.mark.parametrize("hist", HISTS)
def test_split_lorenz_long_subset(gpu_lib, parity, hist):
    w = lorenz_long().subset(np.arange(4), N=50_000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist) as s:
        got = s.solve_batch(w.y0)
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0, params=w.params)
    parity(rel_err(got, ref), TOL_SPLIT, "")


@pytest.mark.parametrize("hist", HISTS)
def test_split_deterministic(gpu_lib, hist):
    w = lorenz_single(N=3000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split", history=hist) as s:
        a = s.solve(w.y0[0])
        b = s.solve(w.y0[0])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("rec", ["columns", "targets"])
def test_recurrence_layouts_agree_on_a_sweep(gpu_lib, parity, rec):
    """LCR sweep on the tensor path with either recurrence layout, against the
    oracle over the non-chaotic horizon, and both layouts against each other."""
    w = lcr_sweep(B=96, N=3000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                        history="tensor", recurrence=rec) as s:
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
        assert gpu_lib.fabm_get_recurrence_layout(s.handle) == gpu_lib.RECURRENCE[rec]
    idx = np.r_[0:3, 60:63, 93:96]
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx])
    for j, b in enumerate(idx):
        parity(rel_err(got[b, : w.compare_steps + 1], ref[j, : w.compare_steps + 1]), TOL_SPLIT, b)
    other = "targets" if rec == "columns" else "columns"
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                        history="tensor", recurrence=other) as s:
        alt = s.solve_batch(w.y0, traj_params=w.traj_params)
    n = w.compare_steps + 1
    assert rel_err(got[:, :n], alt[:, :n]) < TOL_SPLIT


def test_recurrence_layout_rejects_unknown(gpu_lib):
    with gpu_lib.Solver("linear", 1, 0.8, 1e-3, 100, [1.0], precision="split") as s:
        with pytest.raises(gpu_lib.FabmError):
            gpu_lib.fabm_set_recurrence_layout(s.handle, 7)


def test_auto_history_kernel_choice(gpu_lib):
    """Split precision picks tensor cores for wide batches (64+ columns) and the
    compensated fp32 kernel for narrow ones; the block length follows; the
    128-target far tiling where N^2 x columns reaches 2^40."""
    w = duffing_sweep(B=40, N=256)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split") as s:
        assert s.last_history_kernel is None
        s.solve_batch(w.y0[:2], traj_params=w.traj_params[:2])
        assert s.block == 32 and s.last_history_kernel == "fp32c"
        s.solve_batch(w.y0, traj_params=w.traj_params)
        assert s.block == 64 and s.last_history_kernel == "tensor"  # N <= 256: no far group
    # the 128-target far tiling from N^2 x columns >= 2^40 on
    w = duffing_sweep(B=40, N=257)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split") as s:
        s.solve_batch(w.y0, traj_params=w.traj_params)
        assert s.last_history_kernel == "tensor"
        gpu_lib.fabm_set_history_kernel(s.handle, "tensor-wide")
        s.solve_batch(w.y0, traj_params=w.traj_params)
        assert s.last_history_kernel == "tensor-wide"
    for B, N, kernel in ((512, 32767, "tensor"), (512, 32768, "tensor-wide")):
        w = duffing_sweep(B=B, N=N)  # 1024 columns: N^2 x 1024 just below / at 2^40
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split") as s:
            s.solve_batch(w.y0[:B], traj_params=w.traj_params[:B])
            assert s.last_history_kernel == kernel, (B, N)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="fp64") as s:
        with pytest.raises(gpu_lib.FabmError):
            gpu_lib.fabm_set_history_kernel(s.handle, "tensor")
        s.solve_batch(w.y0[:1], traj_params=w.traj_params[:1])
        assert s.last_history_kernel == "fp64"


def test_autotune_picks_a_candidate_and_stays_correct(gpu_lib, parity):
    w = duffing_sweep(B=96, N=2000)
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split") as s:
        rep = s.autotune(w.y0, traj_params=w.traj_params, n_probe=1024)
        assert len(rep) == 8 and all(ms > 0 for ms, _, _ in rep)
        assert {k for _, k, _ in rep} == {gpu_lib.FABM_HIST_TENSOR_WIDE, gpu_lib.FABM_HIST_TENSOR,
                                          gpu_lib.FABM_HIST_FP32C}
        best = min(rep)[1]
        assert gpu_lib.fabm_get_history_kernel(s.handle) == best
        assert gpu_lib.fabm_get_recurrence_warps(s.handle) in (0, 1, 2, 4, 8)
        got = s.solve_batch(w.y0[:4], traj_params=w.traj_params[:4])
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[:4], params=w.params,
                             traj_params=w.traj_params[:4])
    parity(rel_err(got, ref), TOL_SPLIT, "")


def test_recurrence_width_leaves_the_results_bit_for_bit(gpu_lib, parity):
    """Warps per CTA of the column recurrence, automatic or set (a partial last
    CTA included), change the launch only; after the autotuner (which may also
    move the SM reserve, hence the far chunking) the solve still meets the
    oracle."""
    w = duffing_sweep(B=200, N=700)  # 400 columns: 13 warps, the last one partial
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                        history="tensor-wide", recurrence="columns") as s:
        assert gpu_lib.fabm_get_recurrence_warps(s.handle) == 0
        ref = s.solve_batch(w.y0, traj_params=w.traj_params)
        for wp in (1, 3, 12):
            gpu_lib.fabm_set_recurrence_warps(s.handle, wp)
            assert gpu_lib.fabm_get_recurrence_warps(s.handle) == wp
            assert np.array_equal(s.solve_batch(w.y0, traj_params=w.traj_params), ref)
        for bad in (-1, 13):
            with pytest.raises(gpu_lib.FabmError) as e:
                gpu_lib.fabm_set_recurrence_warps(s.handle, bad)
            assert e.value.status == gpu_lib.FABM_EINVAL
        gpu_lib.fabm_set_recurrence_warps(s.handle, 0)
        s.autotune(w.y0, traj_params=w.traj_params, n_probe=700)
        assert gpu_lib.fabm_get_recurrence_warps(s.handle) in (0, 1, 2, 4, 8)
        got = s.solve_batch(w.y0, traj_params=w.traj_params)
    idx = np.array([0, 101, 199])
    orc = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx])
    parity(rel_err(got[idx], orc), TOL_SPLIT, "after-autotune")


@pytest.mark.parametrize("N", [255, 256, 257, 383, 384, 385, 511, 512, 513, 767, 769, 1025])
def test_wide_far_history_group_edges_closed_form(gpu_lib, N):
    """The 128-target far history starts at block 4 (target group 2, point group
    0) and steps by pairs of blocks; lengths around group and pair edges, on the
    constant right-hand side whose scheme is exact."""
    alpha, h = 0.7, 0.01
    B = 40  # 40 trajectories x 2 components = 80 columns: one column tile, ragged
    with gpu_lib.Solver("const", 2, alpha, h, N, [1.5], precision="split",
                        history="tensor-wide") as s:
        y = s.solve_batch(np.full((B, 2), 0.25))
        assert gpu_lib.fabm_get_history_kernel(s.handle) == gpu_lib.FABM_HIST_TENSOR_WIDE
    t = np.arange(N + 1) * h
    ex = 0.25 + 1.5 * t ** alpha / math.gamma(alpha + 1)
    assert np.max(np.abs(y - ex[None, :, None])) / np.max(np.abs(ex)) < TOL_SPLIT


def test_wide_and_narrow_tilings_agree_with_the_oracle(gpu_lib, parity):
    """Duffing batch (160 trajectories, 320 columns: three column tiles, the
    last ragged) with uneven lengths, order above one (weights growing with the
    distance) on the linear right-hand side, both tilings against the oracle."""
    w = duffing_sweep(B=160, N=2500)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[::5] = 1300
    ne[7] = 300
    idx = np.array([0, 7, 64, 100, 159])
    ref = oracle.solve_batch(w.rhs, w.alpha, w.h, w.N, w.y0[idx], params=w.params,
                             traj_params=w.traj_params[idx], N_each=ne[idx])
    for hist in ("tensor-wide", "tensor"):
        with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision="split",
                            history=hist) as s:
            got = s.solve_batch(w.y0, traj_params=w.traj_params, N_each=ne)
        for j, b in enumerate(idx):
            n = ne[b]
            parity(rel_err(got[b, : n + 1], ref[j, : n + 1]), TOL_SPLIT, f"{hist}-{b}")
    alpha, N = 1.4, 1500
    y0 = np.linspace(0.5, 1.5, 70).reshape(70, 1)
    y1 = np.linspace(-1.0, 1.0, 70).reshape(70, 1)
    refh = oracle.solve_batch("linear", alpha, 1e-3, N, y0[[0, 35, 69]], params=[1.0],
                              y1=y1[[0, 35, 69]])
    with gpu_lib.Solver("linear", 1, alpha, 1e-3, N, [1.0], precision="split",
                        history="tensor-wide") as s:
        goth = s.solve_batch(y0, y1=y1)
    for j, b in enumerate([0, 35, 69]):
        parity(rel_err(goth[b], refh[j]), TOL_SPLIT, f"alpha1.4-{b}")
