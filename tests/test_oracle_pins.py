"""Pins of the CPU oracle to facts other than its own code (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: closed-form solutions, weight identities, the Mittag-Leffler solution of
the linear test equation, the convergence order, equilibria printed in the
paper, exact invariances, and a 50-digit evaluation at tiny N.  The last group
plants plausible mistakes in the oracle's weights and checks that a pin fails.
"""
import math
import os

import numpy as np
import pytest

import oracle
from fabm_workloads import LCR_PARAMS, lorenz_single, ml_scalar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(h, N):
    return np.arange(N + 1, dtype=np.float64) * h


# ------------------------------------------------------------- weights ---

@pytest.mark.parametrize("alpha", [0.3, 0.7, 0.95, 0.99, 1.3, 1.7])
def test_weight_telescoping_identities(alpha):
    """sum_{j<=n} b_j = (n+1)^a/G(a+1) and c_n + sum_{j<n} a_j + 1/G(a+2) =
    (n+1)^a/G(a+1): the product-rectangle and product-trapezoid rules integrate
    constants exactly (Sec. 2 weights)."""
    n = 4000
    b, a, c = oracle.weights(alpha, n)
    g1, g2 = math.gamma(alpha + 1), math.gamma(alpha + 2)
    for m in (1, 2, 3, 10, 257, 1999, n - 1):
        exact = (m + 1) ** alpha / g1
        assert math.fsum(b[: m + 1]) == pytest.approx(exact, rel=4e-15 * math.log2(m + 2))
        tot = math.fsum(list(a[:m]) + [c[m], 1.0 / g2])
        assert tot == pytest.approx(exact, rel=4e-15 * math.log2(m + 2))


def test_weight_special_values():
    """0^p = 0 convention: b_0 = 1/G(a+1), c_0 = a/G(a+2), a_0 = (2^{a+1}-2)/G(a+2);
    and all weights positive and decreasing for 0 < a < 1."""
    for alpha in (0.25, 0.8, 0.98):
        b, a, c = oracle.weights(alpha, 2000)
        g1, g2 = math.gamma(alpha + 1), math.gamma(alpha + 2)
        assert b[0] == pytest.approx(1 / g1, rel=2e-16)
        assert c[0] == pytest.approx(alpha / g2, rel=2e-16)
        assert a[0] == pytest.approx((2 ** (alpha + 1) - 2) / g2, rel=1e-15)
        assert np.all(b > 0) and np.all(a > 0) and np.all(c > 0)
        assert np.all(np.diff(b) < 0) and np.all(np.diff(a) < 0)


def test_weight_asymptotics_large_n():
    """For large j the weights follow their Taylor expansions in 1/j:
    b_j ~ a j^{a-1}/G(a+1) (1 + (a-1)/(2j)), a_j ~ a j^{a-1}/G(a+1) (1 + (a-1)/j),
    c_j ~ a j^{a-1}/(2 G(a+1)).  The direct FP64 formulas lose up to 1e-4 of a_j
    at j ~ 2^20 through cancellation; the oracle's binary128 route does not."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    alpha = 0.95
    n = 2 ** 20
    b, a, c = oracle.weights(alpha, n)
    A = mp.mpf(alpha)
    g1, g2 = mp.gamma(A + 1), mp.gamma(A + 2)
    for j in (2 ** 10, 2 ** 16, n - 2):
        J = mp.mpf(j)
        # exact values from the series of (1+u)^p in u = 1/j (no cancellation)
        def second_diff(p, X):  # (X+1)^p - 2 X^p + (X-1)^p
            s = mp.mpf(0)
            for k in range(1, 40):
                s += 2 * mp.binomial(p, 2 * k) / X ** (2 * k)
            return X ** p * s
        a_ex = second_diff(A + 1, J + 1) / g2
        b_ex = J ** A * (mp.power(1 + 1 / J, A) - 1) / g1
        c_ex = (J ** (A + 1) - (J - A) * (J + 1) ** A) / g2
        assert abs(a[j] / float(a_ex) - 1) < 2.3e-16
        assert abs(b[j] / float(b_ex) - 1) < 2.3e-16
        assert abs(c[j] / float(c_ex) - 1) < 2.3e-16
        lead = float(A * J ** (A - 1) / g1)
        assert a[j] == pytest.approx(lead * (1 + (alpha - 1) / j), rel=2.0 / j ** 2)
        assert b[j] == pytest.approx(lead * (1 + (alpha - 1) / (2 * j)), rel=2.0 / j ** 2)
        assert c[j] == pytest.approx(lead / 2, rel=3.0 / j)


# ------------------------------------------------------ closed forms -------

@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.8, 0.99])
def test_constant_rhs_is_exact(alpha):
    """f = const reproduces y = y0 + const t^a/G(a+1) at every grid point: both the
    predictor (product rectangle) and the corrector (product trapezoid) integrate
    constants exactly."""
    h, N = 0.013, 700
    y = oracle.solve("const", alpha, h, N, [0.25], params=[1.5])
    t = _grid(h, N)
    ex = 0.25 + 1.5 * t ** alpha / math.gamma(alpha + 1)
    np.testing.assert_allclose(y[:, 0], ex, rtol=4e-15, atol=0)


@pytest.mark.parametrize("alpha", [0.3, 0.6, 0.9])
def test_linear_in_time_rhs_corrector_is_exact(alpha):
    """f = t: the corrector integrates linear functions exactly, so
    y = y0 + t^{a+1}/G(a+2) at every grid point."""
    h, N = 0.02, 500
    y = oracle.solve("time", alpha, h, N, [-0.5, 2.0])
    t = _grid(h, N)
    ex = t ** (alpha + 1) / math.gamma(alpha + 2)
    np.testing.assert_allclose(y[:, 0], -0.5 + ex, rtol=5e-15, atol=1e-15)
    np.testing.assert_allclose(y[:, 1], 2.0 + ex, rtol=5e-15, atol=1e-15)


def _mittag_leffler(mp, alpha, z):
    s, k = mp.mpf(0), 0
    while True:
        term = z ** k / mp.gamma(alpha * k + 1)
        s += term
        k += 1
        if k > 10 and abs(term) < mp.mpf(10) ** -40:
            return s


def test_mittag_leffler_config():
    """D^a y = -y, y0 = 1 has the solution E_a(-t^a) (Mittag-Leffler).  On the
    a = 0.8, h = 1e-3, T = 10 workload the oracle must be within 1e-4 (it is
    within ~2e-7), and halving h must shrink the error."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    w = ml_scalar()
    y = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    A = mp.mpf(w.alpha)
    errs = []
    for T in (0.5, 1, 2, 5, 10):
        n = int(round(T / w.h))
        ex = float(_mittag_leffler(mp, A, -mp.mpf(n * w.h) ** A))
        errs.append(abs(y[n, 0] - ex))
    assert max(errs) < 1e-4
    assert max(errs) < 1e-6
    # refinement at T = 1
    y2 = oracle.solve(w.rhs, w.alpha, w.h / 2, 2000, w.y0[0], params=w.params)
    ex1 = float(_mittag_leffler(mp, A, -mp.mpf(1) ** A))
    assert abs(y2[2000, 0] - ex1) < 0.6 * abs(y[1000, 0] - ex1)


@pytest.mark.parametrize("alpha", [0.5, 0.8, 0.95])
def test_convergence_order_manufactured(alpha):
    """y = t^2 solves D^a y = 2 t^{2-a}/G(3-a) + t^2 - y, y(0) = 0.  For this smooth
    solution the fractional Adams method converges with order 1 + a (Diethelm,
    Ford, Freed, Numer. Algorithms 36 (2004)); the paper's scheme must show it."""
    kappa = 2.0 / math.gamma(3.0 - alpha)
    params = [kappa, 2.0 - alpha, 2.0]
    errs = []
    Ns = [40, 80, 160, 320, 640, 1280]
    for N in Ns:
        h = 1.0 / N
        y = oracle.solve("manufactured", alpha, h, N, [0.0], params=params)
        t = _grid(h, N)
        errs.append(np.max(np.abs(y[:, 0] - t * t)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(orders[-1] - (1 + alpha)) < 0.1, orders


# --------------------------------------------------- invariants / paper ---

def _lcr_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "lcr_section5.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_lcr_equilibria_from_paper():
    """Sec. 5: at f = 0 the LCR system has the equilibria E0 = (0,0) and
    E+- = (+-s(a-b)/(1+s b), +-(b-a)/(1+s b)).  The oracle's right-hand side must
    vanish there, and a solve started there must stay there."""
    g = _lcr_golden()
    s, om, a, b = g["sigma"], g["omega"], g["a"], g["b"]
    assert (s, om, a, b) == LCR_PARAMS
    params = [s, om, a, b, 0.0]
    x = s * (a - b) / (1 + s * b)
    yv = (b - a) / (1 + s * b)
    for E in ([0.0, 0.0], [x, yv], [-x, -yv]):
        f = oracle.rhs_eval("lcr", 0.3, E, params)
        assert np.max(np.abs(f)) < 1e-15
        traj = oracle.solve("lcr", g["alpha1"], 0.01, 400, E, params=params)
        assert np.max(np.abs(traj - np.asarray(E))) < 1e-14
    # forcing switched on: leaves the equilibrium
    traj = oracle.solve("lcr", 0.9, 0.01, 400, [x, yv], params=[s, om, a, b, 0.1])
    assert np.max(np.abs(traj[-1] - [x, yv])) > 1e-3


def test_lorenz_origin_is_fixed_bitwise():
    y = oracle.solve("lorenz", 0.9, 1e-3, 300, [0.0, 0.0, 0.0])
    assert np.all(y == 0.0)


def test_linear_rhs_scaling_is_exact():
    """f = -lambda y is linear, and scaling by a power of two is exact in binary
    floating point, so y(4 y0) == 4 y(y0) bit for bit."""
    y1 = oracle.solve("linear", 0.7, 0.01, 600, [0.3, -1.1], params=[0.9])
    y4 = oracle.solve("linear", 0.7, 0.01, 600, [1.2, -4.4], params=[0.9])
    assert np.array_equal(y4, 4.0 * y1)


def test_batch_equals_singles_and_prefixes():
    w = lorenz_single(N=600)
    y0 = np.concatenate([w.y0, w.y0 + 0.01, w.y0 - 0.02])
    ne = np.array([600, 250, 1], dtype=np.int64)
    out = oracle.solve_batch("lorenz", 0.98, 5e-4, 600, y0, N_each=ne, threads=3)
    for t in range(3):
        single = oracle.solve("lorenz", 0.98, 5e-4, int(ne[t]), y0[t])
        assert np.array_equal(out[t, : ne[t] + 1], single)
        assert np.all(np.isnan(out[t, ne[t] + 1:]))


@pytest.mark.parametrize("alpha,y1", [(0.63, None), (1.45, (0.5, -1.0, 2.0))])
def test_tiny_N_against_50_digit_evaluation(alpha, y1):
    """Brute force at N <= 8: the scheme evaluated step by step in 50-digit
    arithmetic; the FP64 oracle must agree to ~1e-15.  For 1 < a < 2 the
    Taylor part is y0 + t y'(0)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    h, N = 0.002, 8
    A, H = mp.mpf(alpha), mp.mpf(h)
    p = [mp.mpf(v) for v in (10.0, 28.0, 8.0 / 3.0)]

    def f(t, y):
        return [p[0] * (y[1] - y[0]), y[0] * (p[1] - y[2]) - y[1], y[0] * y[1] - p[2] * y[2]]

    def pw(x, e):
        return mp.mpf(0) if x == 0 else mp.power(x, e)

    g1, g2 = mp.gamma(A + 1), mp.gamma(A + 2)
    bw = lambda j: (pw(j + 1, A) - pw(j, A)) / g1
    aw = lambda j: (pw(j + 2, A + 1) - 2 * pw(j + 1, A + 1) + pw(j, A + 1)) / g2
    cw = lambda j: (pw(j, A + 1) - (j - A) * pw(j + 1, A)) / g2
    y0 = [mp.mpf(v) for v in (0.1, -0.2, 0.3)]
    d1 = [mp.mpf(v) for v in (y1 or (0, 0, 0))]
    ys, fs = [y0], [f(0, y0)]
    for n in range(N):
        t1 = (n + 1) * mp.mpf(h)
        T = [y0[i] + t1 * d1[i] for i in range(3)]
        yp = [T[i] + H ** A * sum(bw(n - k) * fs[k][i] for k in range(n + 1)) for i in range(3)]
        fp = f(t1, yp)
        yc = [T[i] + H ** A * (cw(n) * fs[0][i] + sum(aw(n - k) * fs[k][i]
                                                       for k in range(1, n + 1))
                               + fp[i] / g2) for i in range(3)]
        ys.append(yc)
        fs.append(f(t1, yc))
    ref = np.array([[float(v) for v in row] for row in ys])
    got = oracle.solve("lorenz", alpha, h, N, [0.1, -0.2, 0.3], y1=y1)
    scale = np.max(np.abs(ref), axis=0)
    assert np.max(np.abs(got - ref) / scale) < 2e-15


# ------------------------------------------------- orders 1 < a < 2 -------
# Sec. 2 writes the Taylor part as sum_{k < ceil(a)} t^k/k! y^(k)(0); for
# 1 < a < 2 that is y0 + t y'(0), and the weights are the same formulas.

def test_weight_special_values_above_one():
    """b_0, c_0, a_0 as for a < 1; the weights now grow with j (like j^{a-1})."""
    for alpha in (1.2, 1.5, 1.9):
        b, a, c = oracle.weights(alpha, 3000)
        g1, g2 = math.gamma(alpha + 1), math.gamma(alpha + 2)
        assert b[0] == pytest.approx(1 / g1, rel=2e-16)
        assert c[0] == pytest.approx(alpha / g2, rel=2e-16)
        assert a[0] == pytest.approx((2 ** (alpha + 1) - 2) / g2, rel=1e-15)
        assert np.all(np.diff(b) > 0) and np.all(np.diff(a[1:]) > 0)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.9])
def test_constant_rhs_is_exact_above_one(alpha):
    """f = c: y = y0 + y'(0) t + c t^a/G(a+1) at every grid point; without the
    y'(0) t term the pin fails."""
    h, N = 0.011, 600
    t = _grid(h, N)
    y = oracle.solve("const", alpha, h, N, [0.25, -1.0], params=[1.5], y1=[-0.7, 2.0])
    ex = 1.5 * t ** alpha / math.gamma(alpha + 1)
    np.testing.assert_allclose(y[:, 0], 0.25 - 0.7 * t + ex, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(y[:, 1], -1.0 + 2.0 * t + ex, rtol=1e-14, atol=1e-14)
    y_no = oracle.solve("const", alpha, h, N, [0.25, -1.0], params=[1.5])
    assert np.max(np.abs(y_no[:, 0] - (0.25 - 0.7 * t + ex))) > 1.0


def test_linear_in_time_rhs_is_exact_above_one():
    alpha, h, N = 1.5, 0.02, 400
    t = _grid(h, N)
    y = oracle.solve("time", alpha, h, N, [0.3], y1=[0.9])
    ex = 0.3 + 0.9 * t + t ** (alpha + 1) / math.gamma(alpha + 2)
    np.testing.assert_allclose(y[:, 0], ex, rtol=1e-14, atol=1e-14)


def _mittag_leffler2(mp, alpha, beta, z):
    s, k = mp.mpf(0), 0
    while True:
        term = z ** k / mp.gamma(alpha * k + beta)
        s += term
        k += 1
        if k > 10 and abs(term) < mp.mpf(10) ** -40:
            return s


def test_mittag_leffler_above_one():
    """D^a y = -y for a = 1.5: y(0) = 1, y'(0) = 0 gives E_a(-t^a); y(0) = 0,
    y'(0) = 1 gives t E_{a,2}(-t^a) (damped oscillations).  h = 1e-3, T = 5:
    both within 1e-5."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    alpha, h, N = 1.5, 1e-3, 5000
    y = oracle.solve("linear", alpha, h, N, [1.0, 0.0], params=[1.0], y1=[0.0, 1.0])
    A = mp.mpf(alpha)
    for T in (0.5, 1, 2, 3.5, 5):
        n = int(round(T / h))
        z = -mp.mpf(n * h) ** A
        assert abs(y[n, 0] - float(_mittag_leffler2(mp, A, 1, z))) < 1e-5
        assert abs(y[n, 1] - float(mp.mpf(n * h) * _mittag_leffler2(mp, A, 2, z))) < 1e-5


@pytest.mark.parametrize("alpha", [1.25, 1.5, 1.8])
def test_convergence_order_above_one(alpha):
    """y = t^3 solves D^a y = 6 t^{3-a}/G(4-a) + t^3 - y, y(0) = y'(0) = 0; its
    D^a y is C^1 for a < 2, and for a >= 1 the method then converges with order
    2 (Diethelm, Ford, Freed, Numer. Algorithms 36 (2004))."""
    kappa = 6.0 / math.gamma(4.0 - alpha)
    errs = []
    for N in (40, 80, 160, 320, 640):
        h = 1.0 / N
        y = oracle.solve("manufactured", alpha, h, N, [0.0], params=[kappa, 3.0 - alpha, 3.0])
        errs.append(np.max(np.abs(y[:, 0] - _grid(h, N) ** 3)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(orders[-1] - 2.0) < 0.15, orders


# ----------------------------------------- planted mistakes must be caught --

def _pins_hold(wfun, ha_fun, ig, alpha):
    """Run the closed-form pins (f = const, f = t) and the convergence-order pin
    on weights produced by ``wfun(n) -> (b, a, c)``; True iff all hold."""
    h, N = 0.01, 300
    b, a, c = wfun(N + 1)
    t = _grid(h, N)
    y = oracle.solve_with_weights("const", h, N, [0.0], b, a, c, ha_fun(h), ig, params=[1.0])
    if np.max(np.abs(y[:, 0] - t ** alpha / math.gamma(alpha + 1))) > 1e-12:
        return False
    y = oracle.solve_with_weights("time", h, N, [0.0], b, a, c, ha_fun(h), ig)
    if np.max(np.abs(y[:, 0] - t ** (alpha + 1) / math.gamma(alpha + 2))) > 1e-12:
        return False
    kappa = 2.0 / math.gamma(3.0 - alpha)
    errs = []
    for N in (320, 640):
        h = 1.0 / N
        b, a, c = wfun(N + 1)
        y = oracle.solve_with_weights("manufactured", h, N, [0.0], b, a, c, ha_fun(h), ig,
                                      params=[kappa, 2.0 - alpha, 2.0])
        errs.append(np.max(np.abs(y[:, 0] - _grid(h, N) ** 2)))
    if not np.all(np.isfinite(errs)) or errs[1] == 0:
        return False
    return abs(math.log2(errs[0] / errs[1]) - (1 + alpha)) < 0.1


def test_planted_mistakes_are_caught():
    """Each plausible mistake in the weights or constants (the printed '+' sign of
    b_n, the garbled c_{n-k} of the printed algorithm, index shifts, a missing
    self-term, h in place of h^a) must break one of the pins; the correct
    weights pass them all."""
    alpha = 0.7
    g1 = math.gamma(alpha + 1)
    ig = 1.0 / math.gamma(alpha + 2)
    ha = lambda h: oracle.constants(alpha, h)[0]
    good = lambda n: oracle.weights(alpha, n)

    def b_plus(n):
        b, a, c = good(n)
        j = np.arange(n, dtype=np.float64)
        return ((j + 1) ** alpha + j ** alpha) / g1, a, c

    def shift(which):
        def w(n):
            v = list(good(n + 1))
            v[which] = v[which][1:]
            return tuple(x[:n] for x in v)
        return w

    def swap(dst, src):
        def w(n):
            v = list(good(n))
            v[dst] = v[src]
            return tuple(v)
        return w

    assert _pins_hold(good, ha, ig, alpha)
    mistakes = {
        "b with + sign": (b_plus, ha, ig),
        "b index shifted": (shift(0), ha, ig),
        "a index shifted": (shift(1), ha, ig),
        "corrector uses c_{n-k}": (swap(1, 2), ha, ig),
        "c_n replaced by a_n": (swap(2, 1), ha, ig),
        "self term dropped": (good, ha, 0.0),
        "h^a replaced by h": (good, lambda h: h, ig),
    }
    for name, (w, hf, g) in mistakes.items():
        assert not _pins_hold(w, hf, g, alpha), name


def test_stroboscope_exact_on_linear_trajectories():
    """Linear interpolation reproduces a trajectory linear in t at any sample
    time; samples outside [0, N h] are NaN (the sampling of Sec. 5's
    bifurcation diagram)."""
    h, N = 0.25, 40
    t = np.arange(N + 1) * h
    Y = np.stack([np.stack([2.0 - 3.0 * t, 0.5 * t], axis=1),
                  np.stack([1.0 + t, -t], axis=1)])
    tj = -0.3 + np.arange(12) * 0.97
    s = oracle.stroboscope(Y, h, -0.3, 0.97, 12, comp=0)
    inside = (tj >= 0) & (tj <= N * h)
    np.testing.assert_allclose(s[0, inside], 2.0 - 3.0 * tj[inside], rtol=1e-14)
    np.testing.assert_allclose(s[1, inside], 1.0 + tj[inside], rtol=1e-14)
    assert np.all(np.isnan(s[:, ~inside]))


# ------------------------------------------- one order per component -------
# Sec. 5's systems carry one order per equation (alpha1, alpha2); each
# component then uses the weights and constants of its own order.

def test_multi_order_independent_components_split_exactly():
    """Uncoupled components (linear RHS) solved as one system with orders
    (0.5, 0.9, 1.4) equal, bit for bit, the three scalar solves."""
    al = [0.5, 0.9, 1.4]
    y0, y1 = [1.0, -0.5, 2.0], [0.0, 0.0, 0.3]
    h, N = 0.01, 500
    y = oracle.solve("linear", al, h, N, y0, params=[0.7], y1=y1)
    for i, a in enumerate(al):
        yi = oracle.solve("linear", a, h, N, [y0[i]], params=[0.7],
                          y1=[y1[i]] if a > 1 else None)
        assert np.array_equal(y[:, i], yi[:, 0]), i


def test_multi_order_equal_orders_is_the_single_order_scheme():
    al = 0.83
    a = oracle.solve("lorenz", al, 1e-3, 700, [1.0, 1.0, 1.0])
    b = oracle.solve("lorenz", [al, al, al], 1e-3, 700, [1.0, 1.0, 1.0])
    assert np.array_equal(a, b)


def test_multi_order_constant_rhs_is_exact():
    al = [0.3, 0.75, 1.6]
    h, N = 0.02, 300
    t = _grid(h, N)
    y = oracle.solve("const", al, h, N, [0.1, 0.2, 0.3], params=[1.5], y1=[9.0, 9.0, -0.4])
    for i, a in enumerate(al):
        ex = [0.1, 0.2, 0.3][i] + (-0.4 * t if a > 1 else 0.0) + 1.5 * t ** a / math.gamma(a + 1)
        np.testing.assert_allclose(y[:, i], ex, rtol=1e-14, atol=1e-14)


def test_multi_order_lcr_equilibria():
    """E+- of Sec. 5 stay fixed at f = 0 for different orders alpha1, alpha2."""
    g = _lcr_golden()
    s, a, b = g["sigma"], g["a"], g["b"]
    x = s * (a - b) / (1 + s * b)
    yv = (b - a) / (1 + s * b)
    for E in ([x, yv], [-x, -yv]):
        traj = oracle.solve("lcr", [0.9, 0.7], 0.01, 300, E, params=[s, g["omega"], a, b, 0.0])
        assert np.max(np.abs(traj - np.array(E))) < 1e-12


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_k_reduction_equals_the_sequential_oracle(threads):
    """The Alg. 2-style timing variant splits every step's k-sums over threads:
    one thread reproduces the sequential oracle bit for bit, more threads
    change only the order of the additions."""
    w = lorenz_single(N=1500)
    ref = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params)
    got = oracle.solve_threaded(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=w.params,
                                threads=threads)
    if threads == 1:
        assert np.array_equal(got, ref)
    scale = np.max(np.abs(ref), axis=0)
    assert np.max(np.abs(got - ref) / scale) < 1e-13


# ---- binary128 self-check of the oracle ----

def _exact_power_law(y0, y1, c, alpha, h, N):
    """y0 + y1 t + c t^alpha / Gamma(alpha+1) at t_n = n h, 40 digits."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    a = mpmath.mpf(alpha)
    g = mpmath.gamma(a + 1)
    out = []
    for n in range(N + 1):
        t = mpmath.mpf(n) * mpmath.mpf(h)
        out.append(float(mpmath.mpf(y0) + mpmath.mpf(y1) * t + mpmath.mpf(c) * t ** a / g))
    return np.array(out)


@pytest.mark.parametrize("alpha,y1", [(0.7, None), (0.3, None), (1.5, 0.4)])
def test_binary128_oracle_is_correctly_rounded_on_the_power_law(alpha, y1):
    """f = c: the scheme reproduces y0 (+ y1 t) + c t^a / Gamma(a+1) exactly, so
    the binary128 run, rounded once, must give the nearest doubles."""
    h, N, c = 0.01, 600, 1.5
    got = oracle.solve_q("const", alpha, h, N, [0.25], params=[c],
                         y1=None if y1 is None else [y1])[:, 0]
    ex = _exact_power_law(0.25, y1 or 0.0, c, alpha, h, N)
    ulps = np.abs(got - ex) / np.spacing(np.abs(ex))
    assert np.max(ulps) <= 1.0


def test_binary128_oracle_time_rhs_corrector_is_exact():
    """f = t: the corrector integrates the linear interpolant of f exactly, so
    y_n = y0 + t_n^(a+1) / Gamma(a+2) to binary128 precision."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    alpha, h, N = 0.6, 0.02, 400
    got = oracle.solve_q("time", alpha, h, N, [0.5])[:, 0]
    a = mpmath.mpf(alpha)
    ex = np.array([float(mpmath.mpf(0.5) + (mpmath.mpf(n) * mpmath.mpf(h)) ** (a + 1)
                         / mpmath.gamma(a + 2)) for n in range(N + 1)])
    assert np.max(np.abs(got - ex) / np.spacing(np.abs(ex))) <= 1.0


@pytest.mark.parametrize("case", ["ml", "lorenz", "duffing", "lcr"])
def test_double_oracle_rounding_against_binary128(case):
    """The double-precision oracle (compensated sums, weights rounded once)
    stays within a few units in the last place of the binary128 run: its own
    rounding is far below the GPU bars it is used for."""
    from fabm_workloads import duffing_sweep, lcr_sweep
    if case == "ml":
        w = ml_scalar(N=1500)
    elif case == "lorenz":
        w = lorenz_single(N=1500)
    elif case == "duffing":
        w = duffing_sweep(B=8, N=1500).subset([5])
    else:
        w = lcr_sweep(B=8, N=1500).subset([6])
    p = w.params if w.traj_params is None else w.traj_params[0]
    q = oracle.solve_q(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=p)
    d = oracle.solve(w.rhs, w.alpha, w.h, w.N, w.y0[0], params=p)
    scale = np.max(np.abs(q), axis=0)
    assert np.max(np.abs(d - q) / scale) < 1e-14
