"""Output paths of fabm_solve_batch (needs a GPU).

A large output into pinned host memory is copied block group by block group
while the solve goes on; the result must equal the one written to device
memory bit for bit, and rows past a trajectory's N_each (which turn streaming
off) must stay untouched in the caller's buffer.
"""
import numpy as np
import pytest
import torch

from fabm_workloads import duffing_sweep, lorenz_long

pytestmark = pytest.mark.gpu


def _device_and_pinned(gpu_lib, w, precision, N_each=None):
    with gpu_lib.Solver(w.rhs, w.dim, w.alpha, w.h, w.N, w.params, precision=precision) as s:
        dev = torch.empty((w.B, w.N + 1, w.dim), dtype=torch.float64, device="cuda")
        s.solve_batch(w.y0, traj_params=w.traj_params, N_each=N_each, out=dev)
        host = torch.full((w.B, w.N + 1, w.dim), -7.0, dtype=torch.float64, pin_memory=True)
        s.solve_batch(w.y0, traj_params=w.traj_params, N_each=N_each, out=host)
        again = torch.full_like(host, -7.0).pin_memory()
        s.solve_batch(w.y0, traj_params=w.traj_params, N_each=N_each, out=again)  # cached graph
    return dev.cpu().numpy(), host.numpy(), again.numpy()


@pytest.mark.parametrize("precision,w", [
    ("split", duffing_sweep(B=530, N=8100)),            # 67 MB, tensor history, ragged last group
    ("fp64", lorenz_long().subset(np.arange(64), N=50_001)),  # 77 MB, CUDA-core history
])
def test_streamed_pinned_output_is_bitwise_the_device_result(gpu_lib, precision, w):
    dev, host, again = _device_and_pinned(gpu_lib, w, precision)
    assert w.B * (w.N + 1) * w.dim * 8 >= 64 << 20
    assert np.array_equal(dev, host)
    assert np.array_equal(dev, again)


def test_rows_past_n_each_stay_untouched_in_pinned_output(gpu_lib):
    w = duffing_sweep(B=530, N=8100)
    ne = np.full(w.B, w.N, dtype=np.int64)
    ne[5] = 3000
    dev, host, _ = _device_and_pinned(gpu_lib, w, "split", N_each=ne)
    assert np.all(host[5, 3001:] == -7.0)
    assert np.array_equal(dev[5, :3001], host[5, :3001])
    keep = np.arange(w.B) != 5
    assert np.array_equal(dev[keep], host[keep])
