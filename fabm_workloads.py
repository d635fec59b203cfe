"""Seeded synthetic workloads for the fractional ABM solver.

This module only draws random numbers and lays out problem descriptions
(right-hand side, fractional order, step size, horizon, initial states,
parameters).  It contains none of the method's arithmetic, so both the CPU
oracle's tests and the CUDA path's tests and bench take their inputs from it.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so that every
platform draws the same values; a uniform double is the top 53 bits of an
output times 2^-53.  Seeds are 1710011330 + the workload's index.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1710011330
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started from ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z & _M64


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles in [lo, hi) from SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


LORENZ_PARAMS = (10.0, 28.0, 8.0 / 3.0)
DUFFING_GAMMA, DUFFING_OMEGA = 0.1, 1.2
# Sec. 5 parameter values of the forced series LCR circuit: sigma, omega, a, b.
LCR_PARAMS = (1.015, 0.55, -1.02, -0.58)


@dataclass
class Workload:
    """One batch of trajectories that share (rhs, dim, alpha, h, N)."""
    name: str
    rhs: str
    dim: int
    alpha: float
    h: float
    N: int
    y0: np.ndarray                       # (B, dim)
    params: tuple                        # shared right-hand-side parameters
    traj_params: np.ndarray | None = None  # (B, n_params) or None
    N_each: np.ndarray | None = None     # (B,) or None
    compare_steps: int | None = None     # oracle comparison horizon (steps)
    precision: str = "fp64"
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return self.y0.shape[0]

    @property
    def cols(self) -> int:
        return self.B * self.dim

    def history_macs(self) -> float:
        """Algorithmic history multiply-adds: N^2 per column (predictor and
        corrector sums together)."""
        ns = self.N_each if self.N_each is not None else np.full(self.B, self.N)
        return float(np.sum(ns.astype(np.float64) ** 2) * self.dim)

    def steps_traj(self) -> float:
        ns = self.N_each if self.N_each is not None else np.full(self.B, self.N)
        return float(np.sum(ns))

    def subset(self, idx, N: int | None = None) -> "Workload":
        idx = np.asarray(idx)
        N = self.N if N is None else N
        ne = None
        if self.N_each is not None:
            ne = np.minimum(self.N_each[idx], N)
        return Workload(self.name + "-subset", self.rhs, self.dim, self.alpha, self.h, N,
                        self.y0[idx].copy(), self.params,
                        None if self.traj_params is None else self.traj_params[idx].copy(),
                        ne, None, self.precision, self.note)


def ml_scalar(N: int = 10_000) -> Workload:
    """D^a y = -y, y(0) = 1, a = 0.8, h = 1e-3, T = 10 (N = 10,000 steps)."""
    return Workload("ml-scalar-a0.8-N10000", "linear", 1, 0.8, 1e-3, N,
                    np.ones((1, 1)), (1.0,), compare_steps=N,
                    note="exact solution E_a(-t^a)")


def lorenz_single(N: int = 2 ** 18) -> Workload:
    """3-dim fractional Lorenz-type system, a = 0.98, y0 = (1,1,1) + U(-0.01, 0.01),
    h = 5e-4, N = 2^18, one trajectory; oracle comparison for t <= 10."""
    y0 = 1.0 + uniform(SEED_BASE + 2, 3, -0.01, 0.01).reshape(1, 3)
    return Workload("lorenz-a0.98-h5e-4-N262144", "lorenz", 3, 0.98, 5e-4, N, y0,
                    LORENZ_PARAMS, compare_steps=min(N, 20_000))


def duffing_sweep(B: int = 4096, N: int = 2 ** 16) -> Workload:
    """Bifurcation sweep: B forced cubic oscillators D^a x = y,
    D^a y = -0.1 y - x - x^3 + F cos(1.2 t), F_i = 0.1 + 1.9 i/(B-1), a = 0.95,
    y0 = 0, h = 1e-3, N = 2^16."""
    F = 0.1 + np.arange(B) * (1.9 / max(B - 1, 1))
    tp = np.stack([np.full(B, DUFFING_GAMMA), np.full(B, DUFFING_OMEGA), F], axis=1)
    return Workload(f"duffing-sweep-B{B}-a0.95-N{N}", "duffing", 2, 0.95, 1e-3, N,
                    np.zeros((B, 2)), (DUFFING_GAMMA, DUFFING_OMEGA, 1.0), tp,
                    compare_steps=N, precision="split")


def lorenz_long(B: int = 256, N: int = 2 ** 20) -> Workload:
    """B Lorenz-type trajectories, a = 0.95, y0 in (1,1,1) + U(-0.05, 0.05)^3,
    h = 1e-4, N = 2^20; oracle comparison on 4 trajectories for t <= 5."""
    y0 = 1.0 + uniform(SEED_BASE + 5, 3 * B, -0.05, 0.05).reshape(B, 3)
    return Workload(f"lorenz-long-B{B}-a0.95-h1e-4-N{N}", "lorenz", 3, 0.95, 1e-4, N, y0,
                    LORENZ_PARAMS, compare_steps=min(N, 50_000))


def lcr_sweep(B: int = 64, N: int = 2 ** 14, alpha: float = 0.9, h: float = 1e-2,
              f_max: float = 0.2) -> Workload:
    """The paper's forced series LCR system (Sec. 5), alpha1 = alpha2 = alpha, forcing
    amplitude f swept over [0, f_max]; y0 seeded near the origin."""
    f = np.linspace(0.0, f_max, B)
    tp = np.stack([np.full(B, LCR_PARAMS[0]), np.full(B, LCR_PARAMS[1]),
                   np.full(B, LCR_PARAMS[2]), np.full(B, LCR_PARAMS[3]), f], axis=1)
    y0 = uniform(SEED_BASE + 6, 2 * B, -0.1, 0.1).reshape(B, 2)
    # amplitudes above ~0.13 are chaotic: an oracle run with y0 perturbed by 1e-8
    # departs by 1e-6 of the solution scale from t ~ 54 (f = 0.176) and t ~ 75
    # (f = 0.2), so trajectories are compared with the oracle for t <= 40
    return Workload(f"lcr-sweep-B{B}-a{alpha}-N{N}", "lcr", 2, alpha, h, N, y0,
                    LCR_PARAMS + (0.0,), tp, compare_steps=min(N, int(round(40.0 / h))))


# ------------------------------------------------------------ served stream --

SERVE_RHS = ("linear", "duffing", "lorenz")
SERVE_DIM = {"linear": 1, "duffing": 2, "lorenz": 3}


@dataclass
class Request:
    rid: int
    arrival: float       # seconds after the stream starts
    rhs: str
    dim: int
    alpha: float
    h: float
    N: int
    y0: np.ndarray
    params: tuple


def served_stream(n: int = 20_000, rate: float = 1000.0, k_lo: int = 12, k_hi: int = 18,
                  seed: int = SEED_BASE + 4) -> list[Request]:
    """Mixed request stream: rhs uniform over {linear, duffing, lorenz},
    alpha ~ U(0.7, 0.99), N = 2^k with k uniform on {k_lo..k_hi}, h = 1e-3, seeded
    initial states, Poisson arrivals at ``rate`` requests per second."""
    u = uniform(seed, 9 * n).reshape(n, 9)
    gaps = -np.log1p(-u[:, 0]) / rate
    arrival = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        rhs = SERVE_RHS[min(int(u[i, 1] * 3), 2)]
        alpha = 0.7 + 0.29 * u[i, 2]
        k = k_lo + min(int(u[i, 3] * (k_hi - k_lo + 1)), k_hi - k_lo)
        if rhs == "linear":
            y0 = np.array([0.5 + u[i, 4]])
            params = (0.5 + u[i, 5],)
        elif rhs == "duffing":
            y0 = np.array([u[i, 4] - 0.5, u[i, 5] - 0.5])
            params = (DUFFING_GAMMA, DUFFING_OMEGA, 0.1 + 1.9 * u[i, 6])
        else:
            y0 = 1.0 + 0.1 * (u[i, 4:7] - 0.5)
            params = LORENZ_PARAMS
        out.append(Request(i, float(arrival[i]), rhs, SERVE_DIM[rhs], float(alpha), 1e-3,
                           2 ** k, y0, params))
    return out
