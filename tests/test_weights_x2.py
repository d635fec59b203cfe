"""Double-double weights of the FP64X2 precision (host code, no GPU).

fabm_weights_x2 evaluates B(d) = b_{d-1}, A(d) = a_{d-1} and D(m) = c_{m-1} -
a_{m-1} (Sec. 2's predictor and corrector weights in distance form) in
binary128 from rewrites of the printed differences.  Pinned here against the
printed formulas evaluated with 50-digit arithmetic, and against the oracle's
weights (the printed formulas in binary128, rounded to double): the high parts
must be those doubles, up to one unit in the last place.
"""
import numpy as np
import pytest

import oracle
import paper_1710_01133_gb300 as fabm

DISTANCES = [1, 2, 3, 4, 7, 15, 16, 17, 31, 63, 64, 65, 127, 500, 1023, 4096, 40000, 65535, 65536]


@pytest.mark.parametrize("alpha", [0.1, 0.5, 0.8, 0.98, 1.0, 1.3, 1.95])
def test_weights_x2_match_50_digit_printed_formulas(alpha):
    mpmath = pytest.importorskip("mpmath")
    Bh, Bl, Ah, Al, Dh, Dl = fabm.fabm_weights_x2(alpha, 1 << 16)
    assert Bh[0] == Bl[0] == Ah[0] == Al[0] == Dh[0] == Dl[0] == 0.0
    mp = mpmath.mp
    mp.dps = 50
    a = mp.mpf(alpha)
    g1, g2 = mp.gamma(a + 1), mp.gamma(a + 2)

    def pw(x, p):  # 0^p = 0
        return mp.mpf(0) if x == 0 else mp.mpf(x) ** p

    worst = 0.0
    for d in DISTANCES:
        n = d - 1  # paper index of the weight at distance d
        b = (pw(n + 1, a) - pw(n, a)) / g1
        an = (pw(n + 2, a + 1) - 2 * pw(n + 1, a + 1) + pw(n, a + 1)) / g2
        cn = (pw(n, a + 1) - (n - a) * pw(n + 1, a)) / g2
        for ex, hi, lo in ((b, Bh[d], Bl[d]), (an, Ah[d], Al[d]), (cn - an, Dh[d], Dl[d])):
            err = abs(mp.mpf(hi) + mp.mpf(lo) - ex) / abs(ex)
            worst = max(worst, float(err))
            # hi is the double nearest the value, lo at most half an ulp of hi
            assert abs(lo) <= np.spacing(abs(hi)) / 2
    assert worst < 1e-26, worst


@pytest.mark.parametrize("alpha", [0.3, 0.9, 1.5])
def test_weights_x2_high_parts_are_the_oracle_doubles(alpha):
    n = 20_000
    Bh, _, Ah, _, Dh, _ = fabm.fabm_weights_x2(alpha, n)
    b, a, c = oracle.weights(alpha, n)  # index j = d - 1
    ulp = lambda v: np.spacing(np.abs(v))  # noqa: E731
    assert np.all(np.abs(Bh[1:] - b) <= ulp(b))
    assert np.all(np.abs(Ah[1:] - a) <= ulp(a))
    assert np.all(np.abs(Dh[1:] - (c - a)) <= 4 * ulp(c - a))  # c - a rounds once more


def test_weights_x2_rejects_bad_arguments():
    for alpha in (0.0, 2.0, float("nan")):
        with pytest.raises(fabm.FabmError):
            fabm.fabm_weights_x2(alpha, 10)
    with pytest.raises(fabm.FabmError):
        fabm.fabm_weights_x2(0.5, -1)
