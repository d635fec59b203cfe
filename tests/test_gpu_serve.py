"""The continuous-batching server (needs a GPU).

Requests with different right-hand sides, dims, alphas and lengths are
admitted by an HBM budget, advanced together block by block, and must give the
same result alone and in the mix (bit for bit: a request's chunking depends
only on its own block index) and match the oracle on the solution scale (FP64:
1e-12, split: 1e-6); FP64 requests also match the standalone solver.
"""
import numpy as np
import pytest

import oracle
from fabm_workloads import LORENZ_PARAMS, served_stream

pytestmark = pytest.mark.gpu

MIX = [
    ("lorenz", 3, 0.95, 1e-3, 3000, [1.0, 1.02, 0.98], LORENZ_PARAMS),
    ("linear", 1, 0.8, 1e-3, 1000, [1.0], (1.0,)),
    ("duffing", 2, 0.9, 1e-3, 2047, [0.2, -0.1], (0.1, 1.2, 0.7)),
    ("lcr", 2, 0.9, 1e-2, 777, [0.05, 0.0], (1.015, 0.55, -1.02, -0.58, 0.1)),
    ("linear", 3, 0.7, 2e-3, 33, [1.0, -2.0, 0.5], (0.5,)),
    ("lorenz", 3, 0.75, 5e-4, 1, [1.0, 1.0, 1.0], LORENZ_PARAMS),
]


def rel_err(got, ref):
    scale = np.max(np.abs(ref), axis=0, keepdims=True)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(got - ref) / scale))


def run_to_completion(srv, tickets, max_steps=100000):
    for _ in range(max_steps):
        if all(srv.poll(t) >= 2 for t in tickets):
            return
        srv.step()
    raise AssertionError("server did not finish")


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_server_matches_standalone(gpu_lib, parity, precision):
    with gpu_lib.Server(8 << 30, precision=precision) as srv:
        tickets = [srv.submit(r, d, a, h, N, y0, p) for r, d, a, h, N, y0, p in MIX]
        run_to_completion(srv, tickets)
        results = [srv.result(t) for t in tickets]
    for (rhs, dim, a, h, N, y0, p), got in zip(MIX, results):
        assert got.shape == (N + 1, dim)
        ref = oracle.solve(rhs, a, h, N, y0, params=p)
        if precision == "fp64":
            parity(rel_err(got, ref), 1e-12, rhs)
            with gpu_lib.Solver(rhs, dim, a, h, N, p) as s:
                parity(rel_err(got, s.solve(y0)), 1e-12, f"{rhs}-vs-solver")
        else:
            parity(rel_err(got, ref), 1e-6, rhs)


def test_same_alone_and_in_mix_bitwise(gpu_lib):
    target = MIX[0]
    with gpu_lib.Server(8 << 30) as srv:
        t = srv.submit(*target[:5], target[5], target[6])
        run_to_completion(srv, [t])
        alone = srv.result(t)
    with gpu_lib.Server(8 << 30) as srv:
        others = [srv.submit(r, d, a, h, N, y0, p) for r, d, a, h, N, y0, p in MIX[1:4]]
        for _ in range(7):  # arrive while the others are in flight
            srv.step()
        t = srv.submit(*target[:5], target[5], target[6])
        late = [srv.submit(r, d, a, h, N, y0, p) for r, d, a, h, N, y0, p in MIX[3:]]
        run_to_completion(srv, [t] + others + late)
        mixed = srv.result(t)
    assert np.array_equal(alone, mixed)


def test_budget_admission_and_release(gpu_lib, parity):
    """A budget that holds two of these requests: the others wait until memory
    is released, then run; every result stays correct."""
    req = ("lorenz", 3, 0.9, 1e-3, 4000, [1.0, 1.0, 1.0], LORENZ_PARAMS)
    with gpu_lib.Server(1 << 30) as probe:  # one request's device footprint
        probe.submit(*req[:5], req[5], req[6])
        probe.step()
        per_req = probe.stats()["bytes_in_use"]
    assert per_req > 0
    with gpu_lib.Server(2 * per_req + per_req // 2) as srv:
        tickets = [srv.submit(*req[:5], np.asarray(req[5]) + 0.01 * i, req[6]) for i in range(4)]
        active, waiting = srv.step()
        assert (active, waiting) == (2, 2)
        assert srv.poll(tickets[2]) == gpu_lib.FABM_REQ_WAITING
        assert srv.stats()["bytes_in_use"] == 2 * per_req
        run_to_completion(srv, tickets)
        res = [srv.result(t) for t in tickets]
    y0s = np.stack([np.asarray(req[5]) + 0.01 * i for i in range(4)])
    refs = oracle.solve_batch(req[0], req[2], req[3], req[4], y0s, params=req[6])
    for i, got in enumerate(res):
        parity(rel_err(got, refs[i]), 1e-12, f"req{i}")


def test_failures_are_isolated(gpu_lib, parity):
    with gpu_lib.Server(64 << 20) as srv:
        bad = srv.submit("linear", 1, 0.9, 0.1, 5000, [1.0], (-50.0,))     # overflows
        huge = srv.submit("linear", 1, 0.9, 1e-3, 2 ** 24, [1.0], (1.0,))  # never fits
        good = srv.submit("linear", 1, 0.8, 1e-3, 500, [1.0], (1.0,))
        run_to_completion(srv, [bad, huge, good])
        assert srv.poll(bad) == gpu_lib.FABM_REQ_FAILED
        assert srv.poll(huge) == gpu_lib.FABM_REQ_FAILED
        with pytest.raises(gpu_lib.FabmError) as e1:
            srv.result(bad)
        assert e1.value.status == gpu_lib.FABM_ENONFINITE
        with pytest.raises(gpu_lib.FabmError) as e2:
            srv.result(huge)
        assert e2.value.status == gpu_lib.FABM_ENOMEM
        got = srv.result(good)
    ref = oracle.solve("linear", 0.8, 1e-3, 500, [1.0], params=[1.0])
    parity(rel_err(got, ref), 1e-12, "")


def test_served_stream_sample_continuous(gpu_lib, parity):
    """Requests of the mixed stream submitted while others are in flight; each
    matches the oracle at the split bar."""
    reqs = served_stream(n=24, rate=1e9, k_lo=9, k_hi=11)
    with gpu_lib.Server(8 << 30, precision="split") as srv:
        tickets = []
        for i, r in enumerate(reqs):
            tickets.append(srv.submit(r.rhs, r.dim, r.alpha, r.h, r.N, r.y0, r.params))
            if i % 3 == 2:
                srv.step()
        run_to_completion(srv, tickets)
        results = [srv.result(t) for t in tickets]
    for r, got in zip(reqs, results):
        ref = oracle.solve(r.rhs, r.alpha, r.h, r.N, r.y0, params=r.params)
        parity(rel_err(got, ref), 1e-6, "")


def _uninterrupted(gpu_lib, req, precision):
    with gpu_lib.Server(8 << 30, precision=precision) as srv:
        t = srv.submit(*req[:5], req[5], req[6])
        run_to_completion(srv, [t])
        return srv.result(t)


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("blocks", [0, 1, 2, 40])
def test_checkpoint_resume_on_another_server_bitwise(gpu_lib, precision, blocks):
    """A request checkpointed after `blocks` steps and resumed on a fresh
    server (in a mix) gives the uninterrupted result bit for bit."""
    req = MIX[0]
    ref = _uninterrupted(gpu_lib, req, precision)
    with gpu_lib.Server(8 << 30, precision=precision) as a:
        t = a.submit(*req[:5], req[5], req[6])
        other = a.submit(*MIX[2][:5], MIX[2][5], MIX[2][6])
        for _ in range(blocks):
            a.step()
        state = a.checkpoint(t)
        run_to_completion(a, [t, other])
        assert np.array_equal(a.result(t), ref)  # checkpointing does not disturb it
    with gpu_lib.Server(8 << 30, precision=precision) as b:
        mix = [b.submit(r, d, al, h, N, y0, p) for r, d, al, h, N, y0, p in MIX[1:4]]
        t2 = b.resume(state)
        assert b.shape(t2) == (req[4], req[1])
        run_to_completion(b, [t2] + mix)
        got = b.result(t2)
    assert np.array_equal(got, ref)


def test_evict_and_resume_releases_memory(gpu_lib):
    req = MIX[0]
    ref = _uninterrupted(gpu_lib, req, "fp64")
    with gpu_lib.Server(8 << 30) as srv:
        t = srv.submit(*req[:5], req[5], req[6])
        for _ in range(17):
            srv.step()
        assert srv.stats()["bytes_in_use"] > 0
        state = srv.checkpoint(t)
        srv.cancel(t)
        assert srv.stats()["bytes_in_use"] == 0
        with pytest.raises(gpu_lib.FabmError):
            srv.poll(t)
        t2 = srv.resume(state)
        run_to_completion(srv, [t2])
        assert np.array_equal(srv.result(t2), ref)


def test_checkpoint_errors(gpu_lib):
    req = MIX[1]
    with gpu_lib.Server(8 << 30) as srv:
        t = srv.submit(*req[:5], req[5], req[6])
        srv.step()
        state = bytearray(srv.checkpoint(t))
        with pytest.raises(gpu_lib.FabmError) as e:
            srv.resume(bytes(state[:-8]))               # truncated
        assert e.value.status == gpu_lib.FABM_EINVAL
        bad = bytearray(state)
        bad[0] ^= 0xFF                                  # not a checkpoint
        with pytest.raises(gpu_lib.FabmError):
            srv.resume(bytes(bad))
        with pytest.raises(gpu_lib.FabmError):
            srv.checkpoint(12345)                       # unknown ticket
        with pytest.raises(gpu_lib.FabmError):
            srv.cancel(12345)
        run_to_completion(srv, [t])
        with pytest.raises(gpu_lib.FabmError):
            srv.checkpoint(t)                           # finished
        srv.result(t)
    with gpu_lib.Server(8 << 30, precision="split") as other:
        with pytest.raises(gpu_lib.FabmError) as e:
            other.resume(bytes(state))                  # precision mismatch
        assert e.value.status == gpu_lib.FABM_EINVAL


def test_wait_steps_until_the_request_finishes(gpu_lib, parity):
    """fabm_server_wait on one request of a mix: the others advance with it and
    stay correct; a failed request reports its error; unknown tickets fail."""
    with gpu_lib.Server(8 << 30) as srv:
        tickets = [srv.submit(r, d, a, h, N, y0, p) for r, d, a, h, N, y0, p in MIX]
        got = srv.wait(tickets[1])                     # linear, 1000 steps
        assert srv.poll(tickets[0]) == gpu_lib.FABM_REQ_RUNNING   # lorenz, 3000 steps
        rest = [srv.wait(t) for t in tickets[2:]] + [srv.wait(tickets[0])]
        with pytest.raises(gpu_lib.FabmError):
            srv.wait(tickets[1])                       # already collected
        bad = srv.submit("linear", 1, 0.9, 0.1, 5000, [1.0], (-50.0,))
        with pytest.raises(gpu_lib.FabmError) as e:
            srv.wait(bad)
        assert e.value.status == gpu_lib.FABM_ENONFINITE
    r, d, a, h, N, y0, p = MIX[1]
    parity(rel_err(got, oracle.solve(r, a, h, N, y0, params=p)), 1e-12, "wait")
    assert rest[-1].shape == (MIX[0][4] + 1, 3)


def test_finished_lists_each_request_once(gpu_lib):
    with gpu_lib.Server(8 << 30) as srv:
        tickets = [srv.submit(r, d, a, h, N, y0, p) for r, d, a, h, N, y0, p in MIX]
        seen = []
        for _ in range(1000):
            srv.step()
            seen += srv.finished()
            if len(seen) == len(tickets):
                break
        assert sorted(seen) == sorted(tickets)
        assert all(srv.poll(t) == gpu_lib.FABM_REQ_DONE for t in tickets)
        assert srv.finished() == []


# 1 < alpha < 2 (Sec. 2: the Taylor part y0 + t y'(0)); y1 None means y'(0) = 0
HIGH = [
    ("linear", 2, 1.5, 1e-3, 2000, [1.0, -0.5], (1.0,), [0.3, 0.2]),
    ("duffing", 2, 1.8, 1e-3, 1500, [0.2, 0.0], (0.1, 1.2, 0.7), [0.0, 0.1]),
    ("lorenz", 3, 1.2, 5e-4, 1200, [1.0, 1.0, 1.0], LORENZ_PARAMS, None),
]


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_orders_between_one_and_two_against_the_oracle(gpu_lib, parity, precision):
    with gpu_lib.Server(8 << 30, precision=precision) as srv:
        tickets = [srv.submit(r, d, a, h, N, y0, p, y1=y1) for r, d, a, h, N, y0, p, y1 in HIGH]
        other = srv.submit(*MIX[1][:5], MIX[1][5], MIX[1][6])
        run_to_completion(srv, tickets + [other])
        results = [srv.result(t) for t in tickets]
    bar = 1e-12 if precision == "fp64" else 1e-6
    for (rhs, dim, a, h, N, y0, p, y1), got in zip(HIGH, results):
        assert got.shape == (N + 1, dim)
        ref = oracle.solve(rhs, a, h, N, y0, params=p, y1=y1)
        parity(rel_err(got, ref), bar, f"{rhs}-alpha{a}")


def test_orders_between_one_and_two_checkpoint_keeps_y1(gpu_lib):
    r, d, a, h, N, y0, p, y1 = HIGH[0]
    with gpu_lib.Server(8 << 30) as first:
        t = first.submit(r, d, a, h, N, y0, p, y1=y1)
        for _ in range(5):
            first.step()
        state = first.checkpoint(t)
        run_to_completion(first, [t])
        ref = first.result(t)
    with gpu_lib.Server(8 << 30) as second:
        t2 = second.resume(state)
        run_to_completion(second, [t2])
        assert np.array_equal(second.result(t2), ref)


def test_order_and_y1_checks_at_submission(gpu_lib):
    with gpu_lib.Server(1 << 30) as srv:
        for alpha, y1 in ((0.8, [0.1]), (2.0, None), (1.5, [float("nan")])):
            with pytest.raises(gpu_lib.FabmError) as e:
                srv.submit("linear", 1, alpha, 1e-3, 100, [1.0], (1.0,), y1=y1)
            assert e.value.status == gpu_lib.FABM_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_orders_between_one_and_two_long_request(gpu_lib, parity, precision):
    """A served request with 1 < alpha < 2 over 2^15 steps (1024 blocks, the far
    history in many chunks) beside shorter ones, against the oracle over the
    whole run: D^1.6 y = -y with y'(0) given, a decaying oscillation."""
    N = 1 << 15
    y0, y1, p = [1.0, -0.5], [0.3, 0.2], (1.0,)
    with gpu_lib.Server(8 << 30, precision=precision) as srv:
        t = srv.submit("linear", 2, 1.6, 1e-4, N, y0, p, y1=y1)
        others = [srv.submit(*MIX[1][:5], MIX[1][5], MIX[1][6]),
                  srv.submit(*HIGH[1][:5], HIGH[1][5], HIGH[1][6], y1=HIGH[1][7])]
        run_to_completion(srv, [t] + others)
        got = srv.result(t)
    ref = oracle.solve("linear", 1.6, 1e-4, N, y0, params=p, y1=y1)
    parity(rel_err(got, ref), 1e-12 if precision == "fp64" else 1e-6, f"linear-a1.6-N{N}")
