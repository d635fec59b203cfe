"""CPU oracle for the fractional Adams-Bashforth-Moulton method -- TEST INFRASTRUCTURE.

A plain, slow FP64 restatement of the predictor-corrector of Section 2 of
arXiv:1710.01133 (Eq. abm and the corrector/weight formulas that follow it),
compiled from ``fabm_oracle.c`` with gcc and loaded with ctypes.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the CUDA library never does, and the two share no code.

Right-hand sides are named by string; the oracle keeps its own numbering.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fabm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# name -> (oracle id, dim or None for "any", number of params, default params)
RHS = {
    "const": (0, None, 1, (1.0,)),
    "time": (1, None, 0, ()),
    "linear": (2, None, 1, (1.0,)),
    "lorenz": (3, 3, 3, (10.0, 28.0, 8.0 / 3.0)),
    "duffing": (4, 2, 3, (0.1, 1.2, 1.0)),
    "manufactured": (5, 1, 3, None),
    "lcr": (6, 2, 5, (1.015, 0.55, -1.02, -0.58, 0.0)),
}


def build(force: bool = False) -> str:
    """Compile liboracle.so (idempotent).  Returns its path."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        P = ctypes.POINTER
        lib.fabm_oracle_weights.argtypes = [d, i64, P(d), P(d), P(d)]
        lib.fabm_oracle_constants.argtypes = [d, d, P(d), P(d)]
        lib.fabm_oracle_rhs.argtypes = [i, i, d, P(d), P(d), i, P(d)]
        lib.fabm_oracle_solve.argtypes = [i, d, d, i64, i, P(d), i, P(d), P(d), P(d), i]
        lib.fabm_oracle_solve_threaded.argtypes = [i, d, d, i64, i, P(d), i, P(d), P(d), i]
        lib.fabm_oracle_solve_q.argtypes = [i, d, d, i64, i, P(d), i, P(d), P(d), P(d)]
        lib.fabm_oracle_solve_w.argtypes = [i, d, i64, i, P(d), i, P(d), P(d), P(d), d, d,
                                            P(d), P(d), P(d), i]
        lib.fabm_oracle_solve_batch.argtypes = [i, d, d, i64, i, P(d), i, i64, P(d), P(d), P(d),
                                                P(ctypes.c_int64), P(d), i, i]
        lib.fabm_oracle_solve_batch_multi.argtypes = [i, P(d), d, i64, i, P(d), i, i64, P(d),
                                                      P(d), P(d), P(ctypes.c_int64), P(d), i]
        for f in ("fabm_oracle_weights", "fabm_oracle_constants", "fabm_oracle_rhs",
                  "fabm_oracle_solve", "fabm_oracle_solve_w", "fabm_oracle_solve_batch",
                  "fabm_oracle_solve_batch_multi", "fabm_oracle_solve_threaded",
                  "fabm_oracle_solve_q"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def _rhs(name, dim, params):
    rid, rdim, npar, dflt = RHS[name]
    if rdim is not None and dim != rdim:
        raise ValueError(f"rhs {name!r} needs dim {rdim}, got {dim}")
    if params is None:
        if dflt is None:
            raise ValueError(f"rhs {name!r} needs explicit params")
        params = dflt
    params = _f64(params).reshape(-1)
    if params.size < npar:
        raise ValueError(f"rhs {name!r} needs {npar} params")
    if params.size == 0:
        params = np.zeros(1)
    return rid, params


def weights(alpha: float, n: int):
    """(b, a, c), each of length n: the weights b_j, a_j, c_j, j = 0..n-1."""
    b, a, c = np.empty(n), np.empty(n), np.empty(n)
    _check(_load().fabm_oracle_weights(alpha, n, _dp(b), _dp(a), _dp(c)), "weights")
    return b, a, c


def constants(alpha: float, h: float):
    """(h^alpha, 1/Gamma(alpha+2))."""
    ha, ig = ctypes.c_double(), ctypes.c_double()
    _check(_load().fabm_oracle_constants(alpha, h, ctypes.byref(ha), ctypes.byref(ig)),
           "constants")
    return ha.value, ig.value


def rhs_eval(name: str, t: float, y, params=None):
    y = _f64(y).reshape(-1)
    rid, p = _rhs(name, y.size, params)
    out = np.empty_like(y)
    _check(_load().fabm_oracle_rhs(rid, y.size, t, _dp(y), _dp(p), p.size, _dp(out)), "rhs")
    return out


def _y1(y1, shape):
    return None if y1 is None else _f64(y1).reshape(shape)


def solve(name: str, alpha, h: float, N: int, y0, params=None,
          compensated: bool = True, y1=None):
    """One trajectory: returns y_0..y_N as an (N+1, dim) array.  y1 = y'(0)
    (the second Taylor term, 1 < alpha < 2 only; None: zero).  alpha may be a
    sequence of one order per component."""
    if np.ndim(alpha) > 0:
        return solve_batch(name, alpha, h, N, _f64(y0).reshape(1, -1), params=params,
                           compensated=compensated,
                           y1=None if y1 is None else _f64(y1).reshape(1, -1))[0]
    y0 = _f64(y0).reshape(-1)
    rid, p = _rhs(name, y0.size, params)
    y1 = _y1(y1, y0.shape)
    out = np.empty((N + 1, y0.size))
    _check(_load().fabm_oracle_solve(y0.size, alpha, h, N, rid, _dp(p), p.size, _dp(y0),
                                     _dp(y1), _dp(out), int(compensated)), "solve")
    return out


def solve_q(name: str, alpha: float, h: float, N: int, y0, params=None, y1=None):
    """One trajectory with every quantity in binary128 (weights, sums, t, f),
    y rounded to double once: the self-check of the double-precision oracle and
    the reference of the double-double mode.  O(N^2) binary128 operations."""
    y0 = _f64(y0).reshape(-1)
    rid, p = _rhs(name, y0.size, params)
    y1a = None if y1 is None else _f64(y1).reshape(-1)
    out = np.empty((N + 1, y0.size))
    _check(_load().fabm_oracle_solve_q(y0.size, alpha, h, N, rid, _dp(p), p.size, _dp(y0),
                                       _dp(y1a), _dp(out)), "solve_q")
    return out


def solve_threaded(name: str, alpha: float, h: float, N: int, y0, params=None,
                   threads: int = 4):
    """One trajectory (0 < alpha <= 1) with every step's k-sums split over
    `threads` threads (the paper's Alg. 2 layout); a timing reference, equal to
    solve() up to the order of the additions."""
    y0 = _f64(y0).reshape(-1)
    rid, p = _rhs(name, y0.size, params)
    out = np.empty((N + 1, y0.size))
    _check(_load().fabm_oracle_solve_threaded(y0.size, alpha, h, N, rid, _dp(p), p.size, _dp(y0),
                                              _dp(out), int(threads)), "solve_threaded")
    return out


def solve_with_weights(name: str, h: float, N: int, y0, b, a, c, h_alpha: float,
                       inv_gamma2: float, params=None, compensated: bool = True, y1=None):
    """One trajectory with caller-supplied weight vectors (length >= N)."""
    y0 = _f64(y0).reshape(-1)
    rid, p = _rhs(name, y0.size, params)
    b, a, c = _f64(b), _f64(a), _f64(c)
    if min(b.size, a.size, c.size) < N:
        raise ValueError("weight vectors shorter than N")
    y1 = _y1(y1, y0.shape)
    out = np.empty((N + 1, y0.size))
    _check(_load().fabm_oracle_solve_w(y0.size, h, N, rid, _dp(p), p.size, _dp(b), _dp(a),
                                       _dp(c), h_alpha, inv_gamma2, _dp(y0), _dp(y1), _dp(out),
                                       int(compensated)), "solve_w")
    return out


def solve_batch(name: str, alpha: float, h: float, N: int, y0, params=None,
                traj_params=None, N_each=None, threads: int | None = None,
                compensated: bool = True, out=None, y1=None):
    """B trajectories: y0 (and y1 = y'(0) for 1 < alpha < 2) are (B, dim);
    returns (B, N+1, dim).  Rows of trajectory t past N_each[t] are left as
    they were in ``out`` (NaN when out is None).  alpha may be a sequence of
    dim orders, one per component (y1 then serves the components above 1)."""
    y0 = _f64(y0)
    B, dim = y0.shape
    y1 = _y1(y1, y0.shape)
    rid, p = _rhs(name, dim, params)
    tp = None
    if traj_params is not None:
        tp = _f64(traj_params).reshape(B, -1)
        if tp.shape[1] != p.size:
            raise ValueError("traj_params rows must have as many entries as params")
    ne = None
    if N_each is not None:
        ne = np.ascontiguousarray(np.asarray(N_each, dtype=np.int64))
    if out is None:
        out = np.full((B, N + 1, dim), np.nan)
    if np.ndim(alpha) > 0:  # one order per component
        al = _f64(alpha).reshape(-1)
        if al.size != dim:
            raise ValueError("alpha must have dim entries")
        _check(_load().fabm_oracle_solve_batch_multi(
            dim, _dp(al), h, N, rid, _dp(p), p.size, B, _dp(y0), _dp(y1), _dp(tp),
            None if ne is None else ne.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            _dp(out), int(compensated)), "solve_batch_multi")
        return out
    threads = threads or os.cpu_count() or 1
    _check(_load().fabm_oracle_solve_batch(
        dim, alpha, h, N, rid, _dp(p), p.size, B, _dp(y0), _dp(y1), _dp(tp),
        None if ne is None else ne.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        _dp(out), int(threads), int(compensated)), "solve_batch")
    return out


def stroboscope(Y, h, t0, period, n_samples, comp=0):
    """Samples of trajectories Y (B x (N+1) x dim on t_n = n h) at
    t_j = t0 + j period, by linear interpolation between the two grid points
    around t_j (np.interp); NaN outside [0, N h].  This is the sampling of the
    bifurcation diagram of Sec. 5 (once per forcing period 2 pi / omega)."""
    Y = np.asarray(Y, dtype=np.float64)
    B, rows = Y.shape[0], Y.shape[1]
    t = t0 + np.arange(n_samples) * period
    grid = np.arange(rows) * h
    out = np.empty((B, n_samples))
    for b in range(B):
        out[b] = np.interp(t, grid, Y[b, :, comp])
    out[:, (t < 0) | (t > (rows - 1) * h)] = np.nan
    return out
