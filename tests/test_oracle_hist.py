"""Pins of the oracle's weighted histograms (Sec. 5, Fig. 2 observables):
observables and bins of a hand-made event, the sum rules that tie the
histograms to the event weights, and the analytic transverse-momentum
spectrum of u ubar -> 2 gamma at fixed sqrt(s-hat)."""
import math

import numpy as np
import pytest

ALPHA = 1 / 137.035999
Q = 2 / 3

PT_MAX, PT, ETA, DR, DR_MIN, SQRT_S = range(6)


def _event(rs, photons):
    """Momenta (n+2, 4) of one event: p1, p2 along +-z with energy rs/2 and
    photons given as (pT, eta, px-direction, py-direction) with exact unit
    directions."""
    rows = [[rs / 2, 0.0, 0.0, rs / 2], [rs / 2, 0.0, 0.0, -rs / 2]]
    for pt, eta, cx, cy in photons:
        rows.append([pt * math.cosh(eta), pt * cx, pt * cy, pt * math.sinh(eta)])
    return np.array(rows)


def test_hand_made_event(oracle):
    """Photons of pT 30, 55, 75 GeV at eta 0, 1, -1 and phi 0, 3pi/4, -3pi/4,
    lab shift y = 0.25, sqrt(s-hat) = 400 GeV, weight 2.5.  Then max pT = 75;
    the eta_lab are 0.25, 1.25, -0.75; Delta phi is 3pi/4 for the pairs with
    photon 1 and pi/2 (folded from 3pi/2) for photons 2 and 3, so the Delta R
    are sqrt(1 + 9pi^2/16) = 2.5597 (twice) and sqrt(4 + pi^2/4) = 2.5431, the
    smallest 2.5431."""
    r = math.sqrt(0.5)
    mom = _event(400.0, [(30.0, 0.0, 1.0, 0.0), (55.0, 1.0, -r, r), (75.0, -1.0, -r, -r)])[None]
    w = np.array([2.5])
    specs = [(PT_MAX, 5, 0.0, 50.0),     # 75 -> overflow
             (PT, 10, 0.0, 100.0),       # 30 (a left edge) -> bin 4, 55 -> 6, 75 -> 8
             (ETA, 10, -2.5, 2.5),       # 0.25 -> 6, 1.25 -> 8, -0.75 -> 4
             (ETA, 4, 0.0, 2.0),         # -0.75 -> underflow, 0.25 -> 1, 1.25 -> 3
             (DR, 10, 2.5, 2.6),         # 2.5597 -> 6 (twice), 2.5431 -> 5
             (DR_MIN, 4, 1.0, 3.0),      # 2.5431 -> 4
             (SQRT_S, 10, 0.0, 1000.0)]  # 400 (a left edge) -> 5
    want = [{6: 1}, {4: 1, 6: 1, 8: 1}, {6: 1, 8: 1, 4: 1}, {0: 1, 1: 1, 3: 1}, {6: 2, 5: 1}, {4: 1}, {5: 1}]
    got = oracle.hist(3, mom, np.array([0.25]), w, specs)
    for h, sp, wb in zip(got, specs, want):
        expect = np.zeros((sp[1] + 2, 2))
        for b, c in wb.items():
            expect[b] = [2.5 * c, 6.25 * c]
        np.testing.assert_array_equal(h, expect)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_sum_rules(oracle, n):
    """Over all bins, including under- and overflow, each histogram holds
    every entry: sum w = (entries per event) * sum of the weights, and the
    same for w^2; the smallest Delta R never exceeds an event's Delta R."""
    ps = oracle.phase_space(n, 0x4403 + n, 5, 3000, oracle.toy_pdf(), oracle.cuts())
    w = np.random.default_rng(n).exponential(size=3000) * ps["mask"]
    specs = [(PT_MAX, 20, 20.0, 400.0), (PT, 20, 20.0, 400.0), (ETA, 10, -2.5, 2.5), (DR, 16, 0.0, 8.0),
             (DR_MIN, 16, 0.0, 8.0), (SQRT_S, 20, 0.0, 2000.0)]
    got = oracle.hist(n, ps["momenta"], ps["y"], w, specs)
    mult = [1, n, n, n * (n - 1) // 2, 1, 1]
    S1, S2 = math.fsum(w), math.fsum(w * w)
    for h, m in zip(got, mult):
        assert math.fsum(h[:, 0]) == pytest.approx(m * S1, rel=1e-13)
        assert math.fsum(h[:, 1]) == pytest.approx(m * S2, rel=1e-13)
    # cumulative: the smallest Delta R lies below any threshold whenever one pair does
    dr, drmin = np.cumsum(got[3][:, 0]), np.cumsum(got[4][:, 0])
    assert np.all(drmin >= dr / (n * (n - 1) // 2) - 1e-12 * S1)
    # every passing photon satisfies the cuts: pT > 20 and |eta| < 2.5 leave no under/overflow
    assert got[1][0, 0] == 0 and got[2][0, 0] == 0 and got[2][-1, 0] == 0


def test_n2_transverse_momentum_spectrum(oracle):
    """u ubar -> 2 gamma at sqrt(s) = 500 GeV with pT > 20, |eta| < 2.5: the
    photons are back to back with pT = 250 sin(theta), and
    dsigma/dcos(theta) = (pi alpha^2 Q^4 / 3s) (1 + c^2)/(1 - c^2) for
    |c| < tanh 2.5, so the sigma of a pT bin [a, b) is
    2 K [F(c)] between sqrt(1 - (b/250)^2) and min(tanh 2.5, sqrt(1 - (a/250)^2)),
    F(c) = 2 atanh(c) - c.  Every bin of the MC histogram agrees within 5
    standard errors."""
    N = 100_000
    S, Cc = oracle.fixed(500.0), oracle.cuts(20.0, 2.5, -1.0)
    seed = 0x0908440300000001
    w, mask, _ = oracle.event_weights(2, seed, 0, N, S, Cc)
    ps = oracle.phase_space(2, seed, 0, N, S, Cc)
    assert np.array_equal(ps["mask"], mask)
    nb = 10
    (h,) = oracle.hist(2, ps["momenta"], ps["y"], w, [(PT_MAX, nb, 0.0, 250.0)])
    K = math.pi * ALPHA**2 * Q**4 / (3 * 500.0**2) * 0.3893793721e12
    c0 = math.tanh(2.5)
    F = lambda c: 2 * math.atanh(c) - c
    for k in range(nb):
        a, b = 250.0 * k / nb, 250.0 * (k + 1) / nb
        clo, chi = math.sqrt(1 - (b / 250.0) ** 2), min(c0, math.sqrt(1 - (a / 250.0) ** 2))
        exact = 2 * K * (F(chi) - F(clo)) if chi > clo else 0.0
        sw, sw2 = h[k + 1]
        est = sw / N
        err = math.sqrt(max(sw2 / N - est * est, 0.0) / (N - 1))
        if exact == 0.0:
            assert sw == 0.0
        else:
            assert abs(est - exact) < 5 * err + 1e-12, (k, est, exact, err)
    assert h[0, 0] == 0 and h[-1, 0] == 0
    # the bins add up to the total cross section of the n = 2 pin
    assert math.fsum(h[:, 0]) / N == pytest.approx(K * (10 - 2 * c0), rel=5 * 0.01)
