"""Pins of the oracle's right-hand sides from the mathematics of each system.

Every system the workloads use (Lorenz-type, forced cubic oscillator, the
paper's LCR circuit of Sec. 5) is checked through a whole oracle solve against
a result that does not come from the oracle's own formulas:

* exact equilibria that must stay fixed bit for bit;
* invariant subspaces on which the system reduces to D^a z = -beta z, whose
  solution is z0 E_a(-beta t^a) (Mittag-Leffler series at 40 digits);
* regions where the system is linear (small amplitudes, or the inner branch
  |x| < 1 of the LCR characteristic), where the solution of
  D^a Y = M Y + e g(t) is the matrix Mittag-Leffler series
      Y(t) = sum_k t^{ak}/Gamma(ak+1) M^k Y0
           + sum_k sum_j (-1)^j w^p t^{p+a(k+1)}/Gamma(p+a(k+1)+1) M^k e A
  with p = 2j for A cos(wt) forcing and p = 2j+1 for A sin(wt), obtained by
  applying the Riemann-Liouville integral I^{a(k+1)} to the power series of
  the forcing term by term;
* at order a = 1 the scheme is the trapezoidal rule with an explicit
  predictor, so the unforced, undamped oscillator conserves its energy
  v^2/2 + x^2/2 + x^4/4 up to O(h^2).

Each pin also checks that it discriminates: the same closed form for a
plausible slip (a flipped sign, sin for cos, a dropped term) lies far outside
the tolerance.  Tolerances: the scheme's own discretisation error at the step
used, bounded from above by the measured error at twice the step (the scheme
converges with order ~1+a, so halving h reduces the error), and at most 1e-4
of the solution scale, the bar the Mittag-Leffler pin of the scalar
configuration uses.
"""
import math

import numpy as np
import pytest

import oracle
from fabm_workloads import LCR_PARAMS

mp = pytest.importorskip("mpmath")


def _series(M, y0, alpha, t, forcing=None, dps=40):
    """Matrix Mittag-Leffler solution of D^alpha Y = M Y + e A f(w t), Y(0) = y0,
    at time t; forcing = (e, A, w, 'cos'|'sin') or None."""
    with mp.workdps(dps):
        a = mp.mpf(alpha)
        t = mp.mpf(t)
        Mm = mp.matrix([[mp.mpf(x) for x in row] for row in M])
        n = Mm.rows
        out = mp.matrix(n, 1)
        v = mp.matrix([mp.mpf(x) for x in y0])
        for k in range(400):
            c = t ** (a * k) / mp.gamma(a * k + 1) if k else mp.mpf(1)
            term = c * v
            out += term
            if k > 8 and mp.norm(term) < mp.mpf(10) ** (-dps + 5) * (1 + mp.norm(out)):
                break
            v = Mm * v
        if forcing is not None:
            e, A, w, kind = forcing
            w = mp.mpf(w)
            v = mp.matrix([mp.mpf(x) for x in e]) * mp.mpf(A)
            for k in range(400):
                beta = a * (k + 1)
                s = mp.mpf(0)
                for j in range(400):
                    p = 2 * j if kind == "cos" else 2 * j + 1
                    tj = (-1) ** j * w ** p * t ** (p + beta) / mp.gamma(p + beta + 1)
                    s += tj
                    if j > 4 and abs(tj) < mp.mpf(10) ** (-dps + 5) * (1 + abs(s)):
                        break
                term = s * v
                out += term
                if k > 8 and mp.norm(term) < mp.mpf(10) ** (-dps + 5) * (1 + mp.norm(out)):
                    break
                v = Mm * v
        return np.array([float(out[i]) for i in range(n)])


def _closed_form(M, y0, alpha, h, steps, forcing=None):
    return np.array([_series(M, y0, alpha, n * h, forcing) for n in steps])


def _rel(got, ref):
    scale = np.max(np.abs(ref), axis=0)
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(got - ref) / scale))


def _check_linear_pin(rhs, params, y0, alpha, h, N, M, forcing, wrong, comps=None):
    """The oracle against the closed form at h (and its error at 2h as the
    bound), and every mistaken closed form in `wrong` far outside it."""
    every = max(N // 16, 1)
    steps = np.arange(0, N + 1, every)
    ref = _closed_form(M, y0, alpha, h, steps, forcing)
    sl = slice(None) if comps is None else comps
    got = oracle.solve(rhs, alpha, h, N, y0, params=params)[steps][:, sl]
    coarse = oracle.solve(rhs, alpha, 2 * h, N // 2, y0, params=params)[steps // 2][:, sl]
    err, err2 = _rel(got, ref), _rel(coarse, ref)
    tol = min(err2, 1e-4)
    assert err <= tol, (err, err2)
    assert err < 0.7 * err2, (err, err2)  # halving h reduces the error: the limit is ref
    for name, (Mw, fw) in wrong.items():
        alt = _closed_form(Mw, y0, alpha, h, steps, fw)
        assert _rel(alt, ref) > 100 * tol, name
    return err


# ---------------------------------------------------------------- Lorenz --

def test_lorenz_nontrivial_equilibria_stay_fixed_bitwise():
    """With rho = 3, beta = 2 the equilibria C+- = (+-sqrt(beta(rho-1)),
    +-sqrt(beta(rho-1)), rho-1) = (+-2, +-2, 2) are exact in binary: f
    vanishes there exactly, so every step reproduces y0.  A flipped sign in
    the y or z equation (x(rho-z)+y, xy+beta z, ...) makes f nonzero."""
    for y0 in ((2.0, 2.0, 2.0), (-2.0, -2.0, 2.0)):
        Y = oracle.solve("lorenz", 0.9, 1e-2, 500, y0, params=(10.0, 3.0, 2.0))
        assert np.array_equal(Y, np.tile(np.array(y0), (501, 1)))
        f = oracle.rhs_eval("lorenz", 0.0, y0, params=(10.0, 3.0, 2.0))
        assert np.array_equal(f, np.zeros(3))


def test_lorenz_z_axis_is_invariant_with_mittag_leffler_decay():
    """x = y = 0 is invariant; on it D^a z = -beta z, so z(t) = z0 E_a(-beta t^a)."""
    alpha, h, N, beta = 0.95, 1e-3, 2000, 8.0 / 3.0
    Y = oracle.solve("lorenz", alpha, h, N, (0.0, 0.0, 1.5), params=(10.0, 28.0, beta))
    assert np.array_equal(Y[:, :2], np.zeros((N + 1, 2)))
    err = _check_linear_pin("lorenz", (10.0, 28.0, beta), (0.0, 0.0, 1.5), alpha, h, N,
                            [[0, 0, 0], [0, 0, 0], [0, 0, -beta]], None,
                            {"+beta z": ([[0, 0, 0], [0, 0, 0], [0, 0, beta]], None),
                             "-2 beta z": ([[0, 0, 0], [0, 0, 0], [0, 0, -2 * beta]], None)})
    assert err < 1e-4


def test_lorenz_linearisation_at_the_origin():
    """Amplitude 1e-8: z stays O(1e-16) and (x, y) follow the linear system
    D^a (x, y) = [[-sigma, sigma], [rho, -1]] (x, y) to relative O(1e-15); this
    pins the x equation sigma (y - x) (the equilibria above cannot, x = y there)."""
    s, r, b = 10.0, 28.0, 8.0 / 3.0
    alpha, h, N = 0.98, 1e-4, 4000
    y0 = (1e-8, -2e-8, 0.0)
    M = [[-s, s, 0], [r, -1, 0], [0, 0, -b]]
    wrong = {
        "sigma (x - y)": ([[s, -s, 0], [r, -1, 0], [0, 0, -b]], None),
        "x rho + y": ([[-s, s, 0], [r, 1, 0], [0, 0, -b]], None),
        "rho on y": ([[-s, s, 0], [-1, r, 0], [0, 0, -b]], None),
    }
    _check_linear_pin("lorenz", (s, r, b), y0, alpha, h, N, M, None, wrong)


# ------------------------------------------------------- forced oscillator --

def test_duffing_small_amplitude_damping_and_cosine_forcing():
    """F = 1e-4 keeps |x| ~ 1e-4, so x^3 is 1e-8 of x and the oscillator is the
    linear D^a (x, y) = [[0, 1], [-1, -gamma]] (x, y) + (0, F cos(w t))."""
    g, w, F = 0.1, 1.2, 1e-4
    alpha, h, N = 0.95, 1e-3, 3000
    M = [[0, 1], [-1, -g]]
    e = (0.0, 1.0)
    wrong = {
        "+gamma y": ([[0, 1], [-1, g]], (e, F, w, "cos")),
        "sin forcing": (M, (e, F, w, "sin")),
        "-F cos": (M, (e, -F, w, "cos")),
        "no -x": ([[0, 1], [0, -g]], (e, F, w, "cos")),
    }
    _check_linear_pin("duffing", (g, w, F), (0.0, 0.0), alpha, h, N, M, (e, F, w, "cos"), wrong)


def test_duffing_energy_is_conserved_at_order_one():
    """alpha = 1, gamma = F = 0: x'' + x + x^3 = 0 keeps E = v^2/2 + x^2/2 + x^4/4.
    The scheme is then the trapezoidal rule (b_j = a_j = 1, c_n = 1/2), second
    order: the drift of E shrinks ~4x when h halves.  With the cubic term's sign
    or factor wrong the drift of the true E would be O(1)."""
    def energy(Y, q=0.25):
        x, v = Y[:, 0], Y[:, 1]
        return 0.5 * v * v + 0.5 * x * x + q * x ** 4

    y0 = (1.0, 0.0)
    drift = {}
    for h in (2e-3, 1e-3):
        Y = oracle.solve("duffing", 1.0, h, int(round(10.0 / h)), y0, params=(0.0, 1.2, 0.0))
        E = energy(Y)
        drift[h] = float(np.max(np.abs(E - E[0])))
    assert drift[1e-3] < 1e-5, drift
    assert 3.0 < drift[2e-3] / drift[1e-3] < 5.0, drift
    for q in (-0.25, 0.5):  # the energy of a wrong cubic term is not conserved
        Y = oracle.solve("duffing", 1.0, 1e-3, 10_000, y0, params=(0.0, 1.2, 0.0))
        Ew = energy(Y, q)
        assert float(np.max(np.abs(Ew - Ew[0]))) > 1e3 * drift[1e-3]


# ------------------------------------------------------------ LCR (Sec. 5) --

def test_lcr_inner_branch_is_the_linear_circuit():
    """For |x| < 1, g(x) = a x (Eq. sys.LRC and the definition of g), so the
    circuit is D^a (x, y) = [[-a, 1], [-1, -sigma]] (x, y) + (0, f sin(w t)):
    checked with the Sec. 5 values sigma, w, a and f = 0.1 from (0.05, 0.02)
    while |x| stays below 1 (t <= 2)."""
    sg, w, a, b = LCR_PARAMS
    f = 0.1
    alpha, h, N = 0.9, 1e-3, 2000
    y0 = (0.05, 0.02)
    Y = oracle.solve("lcr", alpha, h, N, y0, params=(sg, w, a, b, f))
    assert float(np.max(np.abs(Y[:, 0]))) < 1.0
    M = [[-a, 1], [-1, -sg]]
    e = (0.0, 1.0)
    wrong = {
        "g = -a x": ([[a, 1], [-1, -sg]], (e, f, w, "sin")),
        "cos forcing": (M, (e, f, w, "cos")),
        "+sigma y": ([[-a, 1], [-1, sg]], (e, f, w, "sin")),
        "slope b inside": ([[-b, 1], [-1, -sg]], (e, f, w, "sin")),
    }
    _check_linear_pin("lcr", (sg, w, a, b, f), y0, alpha, h, N, M, (e, f, w, "sin"), wrong)


def test_series_reduces_to_the_scalar_mittag_leffler_function():
    """The matrix series helper itself, on a 1 x 1 matrix, against mpmath's
    own evaluation of E_a(-t^a) through its defining series at 50 digits and
    against the closed form of I^a cos at a = 1 (sin t)."""
    alpha = 0.8
    for t in (0.5, 2.0, 5.0):
        with mp.workdps(50):
            ml = mp.nsum(lambda k: (-mp.mpf(t) ** mp.mpf(alpha)) ** k / mp.gamma(mp.mpf(alpha) * k + 1),
                         [0, mp.inf])
        assert abs(_series([[-1.0]], [1.0], alpha, t)[0] - float(ml)) < 1e-14
    # D^1 y = cos(t), y(0) = 0 -> y = sin(t)
    for t in (0.3, 1.7):
        assert abs(_series([[0.0]], [0.0], 1.0, t, ((1.0,), 1.0, 1.0, "cos"))[0]
                   - math.sin(t)) < 1e-14
