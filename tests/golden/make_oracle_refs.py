"""Writes the stored oracle references of the full-size parity tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``fabm_workloads.py``); nothing here touches the CUDA library.

1. ``duffing_sweep_horizons.txt``: for amplitudes sampled across the Duffing
   sweep (4096 oscillators, N = 2^16), the comparison horizon.  A forced
   oscillator on a chaotic attractor amplifies any error, so the split path
   (errors ~1e-7 of the solution scale per step) can only be held to its 1e-6
   bar while a perturbation of that size has not grown past the bar: each
   amplitude is solved twice by the oracle, from y0 and from y0 with x0 moved
   by 1e-7, and the horizon is 0.8 x the first step at which the two differ
   by more than 1e-6 of the solution scale (rounded down to a multiple of 64),
   or the whole run when they never do (periodic attractors contract
   perturbations).
2. ``served_k17_k18.txt``: requests of the full served stream (20,000 requests,
   N = 2^k, k = 12..18) too long for the oracle to run inside a GPU test
   (~5-10 min each): for each right-hand side the first request with k = 17
   and with k = 18, the same horizon rule, and every (N/512)-th row of the
   oracle's solution.  ``served_horizons.txt`` gives the horizons of the
   k = 15 and 16 requests, which the tests solve with the oracle themselves.

Usage: python tests/golden/make_oracle_refs.py [--jobs 8]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from fabm_workloads import duffing_sweep, served_stream  # noqa: E402

PERTURB = 1e-7
BAR = 1e-6
DUFFING_SAMPLE = [0, 1, 273, 546, 819, 1092, 1365, 1638, 1911, 2047, 2184, 2457, 2730, 3003,
                  3276, 3549, 3822, 4095]
SERVED_K_LIVE = (15, 16)
SERVED_K_STORED = (17, 18)
SERVED_N_REQ = 20_000


def horizon(rhs, alpha, h, N, y0, params):
    """Steps over which the oracle's solution is insensitive, at the 1e-6 bar,
    to a 1e-7 change of the initial state (0.8 x the first departure)."""
    y0 = np.asarray(y0, dtype=np.float64)
    yp = y0.copy()
    yp[0] += PERTURB * max(1.0, abs(y0[0]))
    both = oracle.solve_batch(rhs, alpha, h, N, np.stack([y0, yp]), params=params, threads=2)
    Y, Yp = both[0], both[1]
    scale = np.max(np.abs(Y), axis=0)
    scale = np.where(scale == 0, 1.0, scale)
    d = np.max(np.abs(Yp - Y) / scale, axis=1)
    over = np.nonzero(d > BAR)[0]
    if over.size == 0:
        return N, Y
    return int(0.8 * over[0]) // 64 * 64, Y


def _duffing_job(i):
    w = duffing_sweep()
    sub = w.subset(np.array([i]))
    H, _ = horizon(sub.rhs, sub.alpha, sub.h, sub.N, sub.y0[0], tuple(sub.traj_params[0]))
    return i, float(sub.traj_params[0][2]), H


def served_selection():
    """Indices of the first request of each right-hand side for each k in
    SERVED_K_LIVE + SERVED_K_STORED, in the full served stream."""
    reqs = served_stream(n=SERVED_N_REQ, rate=1e12, k_lo=12, k_hi=18)
    pick = {}
    for r in reqs:
        k = int(round(np.log2(r.N)))
        key = (r.rhs, k)
        if k in SERVED_K_LIVE + SERVED_K_STORED and key not in pick:
            pick[key] = r.rid
    return reqs, pick


def _served_job(req):
    H, Y = horizon(req.rhs, req.alpha, req.h, req.N, req.y0, req.params)
    stride = max(req.N // 512, 1)
    return req.rid, H, stride, Y[::stride].copy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--only", choices=["duffing", "served"], default=None)
    args = ap.parse_args()
    oracle.build()
    with cf.ThreadPoolExecutor(max_workers=args.jobs) as ex:
        if args.only in (None, "served"):
            reqs, pick = served_selection()
            order = sorted(pick.items(), key=lambda kv: -reqs[kv[1]].N)  # longest first
            futs = {ex.submit(_served_job, reqs[i]): (key, i) for key, i in order}
        if args.only in (None, "duffing"):
            duff = list(ex.map(_duffing_job, DUFFING_SAMPLE))
            with open(os.path.join(HERE, "duffing_sweep_horizons.txt"), "w") as fh:
                fh.write("# Duffing sweep (4096 x 2^16, alpha 0.95, h 1e-3): comparison horizon per\n"
                         "# sampled oscillator, written by tests/golden/make_oracle_refs.py (oracle\n"
                         f"# only): 0.8 x the first step at which a {PERTURB:g} change of x0 moves the\n"
                         f"# oracle's solution by more than {BAR:g} of its scale; N = never.\n"
                         "# index  F  horizon_steps\n")
                for i, F, H in duff:
                    fh.write(f"{i} {F:.17g} {H}\n")
        if args.only in (None, "served"):
            live, stored = [], []
            for fut in cf.as_completed(futs):
                (rhs, k), i = futs[fut]
                rid, H, stride, rows = fut.result()
                (stored if k in SERVED_K_STORED else live).append((rid, rhs, k, H, stride, rows))
            with open(os.path.join(HERE, "served_horizons.txt"), "w") as fh:
                fh.write("# Served stream (20,000 requests, k = 12..18): comparison horizons of the\n"
                         "# requests the GPU tests solve with the oracle themselves, written by\n"
                         "# tests/golden/make_oracle_refs.py (rule as in duffing_sweep_horizons.txt).\n"
                         "# request  rhs  k  horizon_steps\n")
                for rid, rhs, k, H, _, _ in sorted(live):
                    fh.write(f"{rid} {rhs} {k} {H}\n")
            with open(os.path.join(HERE, "served_k17_k18.txt"), "w") as fh:
                fh.write("# Served stream (20,000 requests, k = 12..18): oracle rows of the first\n"
                         "# request of each right-hand side with k = 17 and k = 18, written by\n"
                         "# tests/golden/make_oracle_refs.py (oracle only).  Per request a header\n"
                         "# 'request <id> <rhs> k <k> horizon <steps> stride <s> rows <n>' and n rows\n"
                         "# 'step y_1 .. y_dim' for steps 0, s, 2s, ..\n")
                for rid, rhs, k, H, stride, rows in sorted(stored):
                    fh.write(f"request {rid} {rhs} k {k} horizon {H} stride {stride} rows {len(rows)}\n")
                    for j, row in enumerate(rows):
                        fh.write(" ".join([str(j * stride)] + [f"{v:.17g}" for v in row]) + "\n")


if __name__ == "__main__":
    main()
