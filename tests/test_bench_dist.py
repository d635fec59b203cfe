"""The multi-rank path of bench.py on CPU: two gloo ranks, each a replica.

There is no exchange of solver data between ranks (trajectories are
independent); ranks only agree on the slowest step time and the job's
throughput is every rank's units over that time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.dist_max(100.0 + 50.0 * rank, "cpu")
    ws, r, lr = bench._dist()
    value = bench.replica_throughput(262144.0, ws, ms)
    results[rank] = (ms, ws, r, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    assert res[0][0] == res[1][0] == 150.0
    assert [res[i][2] for i in range(world)] == [0, 1]
    assert all(res[i][1] == world for i in range(world))
    assert res[0][3] == pytest.approx(2 * 262144.0 / 0.150)


def test_single_process_is_unchanged():
    import bench
    assert bench.dist_max(3.5, "cpu") == 3.5
    assert bench.replica_throughput(10.0, 1, 1000.0) == pytest.approx(10.0)
