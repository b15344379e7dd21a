"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, textbook closed forms, limits, symmetries and
independent routes (no polarisation vectors; phase-space recursion).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from helpers import (boost_matrix, helicity_index, mask_words, mdot,
                     rotation_matrix, transform)

E2_DEFAULT = 4 * math.pi / 137.035999
Q = 2.0 / 3.0
GEV2_TO_FB = 0.3893793721e12   # (hbar c)^2 in GeV^2 fb
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cm_points(O, n, N, seed=2024, rs=500.0):
    return O.phase_space(n, seed, 0, N, O.fixed(rs))["momenta"]


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------

def test_philox_known_answers(oracle):
    """Philox4x32-10 reproduces the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_layout_and_range(oracle):
    """Draw d of (seed, point, stream) is (m + 1/2) 2^-52 of Philox words 2(d&1), 2(d&1)+1."""
    seed, point, stream = 0x0908440300000002, (1 << 33) + 5, 1
    for d in range(6):
        w = oracle.philox4x32_10([point & 0xFFFFFFFF, point >> 32, d >> 1, stream],
                                 [seed & 0xFFFFFFFF, seed >> 32])
        lo, hi = int(w[2 * (d & 1)]), int(w[2 * (d & 1) + 1])
        m = ((hi << 32) | lo) >> 12
        assert oracle.uniform_draw(seed, point, stream, d) == (m + 0.5) / 2.0**52
    u = np.array([oracle.uniform_draw(7, i, 0, d) for i in range(500) for d in range(8)])
    assert np.all((u > 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-4


# --------------------------------------------------------------------------
# amplitude: closed forms
# --------------------------------------------------------------------------

def test_n2_closed_form(oracle):
    """sum_h |M|^2 = 8 e^4 Q^4 (u/t + t/u) for q qbar -> 2 gamma (massless)."""
    p = cm_points(oracle, 2, 40)
    a = oracle.amp2(2, p)
    p1, k1, k2 = p[:, 0], p[:, 2], p[:, 3]
    t = mdot(p1 - k1, p1 - k1)
    u = mdot(p1 - k2, p1 - k2)
    ref = 8 * E2_DEFAULT**2 * Q**4 * (u / t + t / u)
    np.testing.assert_allclose(a, ref, rtol=1e-12)


def _classic_nphoton(n, m):
    """16 e^6 Q^6 s sum_j t_j u_j (t_j^2 + u_j^2) / prod_i t_i u_i at n = 3
    (massless e+e- -> 3 gamma); the n = 2 member of the same family is the
    formula above.  t_i = 2 p1.k_i, u_i = 2 p2.k_i."""
    p1, p2, ks = m[0], m[1], m[2:]
    s = mdot(p1 + p2, p1 + p2)
    t = np.array([2 * mdot(p1, k) for k in ks])
    u = np.array([2 * mdot(p2, k) for k in ks])
    c = 4.0 ** (n - 1) * (E2_DEFAULT * Q * Q) ** n
    return c * s ** (n - 2) * np.sum(t * u * (t**2 + u**2)) / np.prod(t * u)


def test_n3_closed_form(oracle):
    p = cm_points(oracle, 3, 20, seed=5)
    a = oracle.amp2(3, p)
    ref = np.array([_classic_nphoton(3, m) for m in p])
    np.testing.assert_allclose(a, ref, rtol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_mhv_closed_form(oracle, n):
    """Single-minority photon helicity (MHV) amplitudes, any n:
    |M_h|^2 = (2 e^2 Q^2)^n s^(n-2) s_aj^3 s_bj / prod_i s_1i s_2i,
    with s_ci = 2 p_c.k_i, from the Parke-Taylor form of a fermion line with n
    photons.  For s1 = +, s2 = - the cubed invariant belongs to p1 when the
    minority photon has helicity -, to p2 when it has helicity +; flipping all
    helicities (s1 = -) swaps the roles."""
    m = cm_points(oracle, n, 1, seed=100 + n)[0]
    p1, p2, ks = m[0], m[1], m[2:]
    s = mdot(p1 + p2, p1 + p2)
    s1 = np.array([2 * mdot(p1, k) for k in ks])
    s2 = np.array([2 * mdot(p2, k) for k in ks])
    pref = (2 * E2_DEFAULT * Q * Q) ** n * s ** (n - 2) / np.prod(s1 * s2)
    js = range(n) if n <= 6 else [0, n - 1]
    for sig in (+1, -1):
        for minority in (+1, -1):
            for j in js:
                lam = [-minority] * n
                lam[j] = minority
                h = helicity_index(sig, -sig, lam)
                val = abs(oracle.amp_hel(n, m, h)[0]) ** 2
                cube_p1 = (minority < 0) == (sig > 0)
                ref = pref * (s1[j] ** 3 * s2[j] if cube_p1 else s2[j] ** 3 * s1[j])
                assert val == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_metric_polarisation_sum(oracle, n):
    """Independent route: sum_lambda eps eps* -> -g (no polarisation vectors)."""
    p = cm_points(oracle, n, 3, seed=31 + n)
    a = oracle.amp2(n, p)
    for i in range(3):
        assert oracle.amp2_metric(n, p[i]) == pytest.approx(a[i], rel=1e-12)


def _soft_config(O, n, eps, seed):
    """n hard photons recoiling against one soft photon of energy eps*sqrt(s)/2."""
    rng = np.random.default_rng(seed)
    rs = 500.0
    r = rng.uniform(0.05, 0.95, size=4 * n)
    c, ph = rng.uniform(-0.8, 0.8), rng.uniform(0, 2 * math.pi)
    ksoft = eps * rs / 2 * np.array([1, math.sqrt(1 - c * c) * math.cos(ph),
                                     math.sqrt(1 - c * c) * math.sin(ph), c])
    P = np.array([rs, 0, 0, 0]) - ksoft
    M = math.sqrt(mdot(P, P))
    hard, _ = O.rambo(n, M, r)
    hard = transform(hard, boost_matrix(P[1:] / P[0]))
    p1 = np.array([rs / 2, 0, 0, rs / 2])
    p2 = np.array([rs / 2, 0, 0, -rs / 2])
    hard0, _ = O.rambo(n, rs, r)
    full = np.vstack([p1, p2, hard, ksoft])
    base = np.vstack([p1, p2, hard0])
    return full, base, p1, p2, ksoft


@pytest.mark.parametrize("n", [2, 3, 4])
def test_soft_photon_limit(oracle, n):
    """sum|M_{n+1}|^2 -> 2 e^2 Q^2 (p1.p2)/((p1.k)(p2.k)) sum|M_n|^2 as k -> 0."""
    for seed in range(3):
        full, base, p1, p2, k = _soft_config(oracle, n, 1e-6, seed)
        a_full = oracle.amp2(n + 1, full[None])[0]
        a_base = oracle.amp2(n, base[None])[0]
        eik = 2 * E2_DEFAULT * Q * Q * mdot(p1, p2) / (mdot(p1, k) * mdot(p2, k))
        assert a_full == pytest.approx(eik * a_base, rel=1e-4)


# --------------------------------------------------------------------------
# amplitude: symmetries and identities
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_ward_identity(oracle, n):
    """Replacing any photon polarisation by its momentum kills the ordering sum."""
    m = cm_points(oracle, n, 1, seed=41 + n)[0]
    hs = range(1 << (n + 2))
    scale = max(abs(oracle.amp_hel(n, m, h)[0]) for h in hs)
    for i in range(n):
        for h in hs:
            amp, sum_abs = oracle.amp_hel(n, m, h, ward=i)
            assert abs(amp) <= 1e-12 * scale
    # individual orderings do not vanish: the cancellation is between diagrams
    amp, sum_abs = oracle.amp_hel(n, m, helicity_index(1, -1, [1] * n), ward=0)
    assert sum_abs > 1e-3 * scale


@pytest.mark.parametrize("n", [2, 3, 4])
def test_lorentz_invariance(oracle, n):
    """|M_h|^2 is invariant under boosts and rotations (generic-frame spinors)."""
    rng = np.random.default_rng(7 + n)
    p = cm_points(oracle, n, 2, seed=51 + n)
    for m in p:
        L = boost_matrix(rng.uniform(-0.5, 0.5, 3)) @ rotation_matrix(rng.normal(size=3), 1.1)
        mb = transform(m, L)
        np.testing.assert_allclose(oracle.amp2(n, mb[None]), oracle.amp2(n, m[None]), rtol=1e-10)
        for h in [helicity_index(1, -1, [1] + [-1] * (n - 1)), helicity_index(-1, 1, [1, -1] * (n // 2) + [1] * (n % 2))]:
            a = abs(oracle.amp_hel(n, m, h)[0]) ** 2
            b = abs(oracle.amp_hel(n, mb, h)[0]) ** 2
            assert b == pytest.approx(a, rel=1e-10)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_photon_permutation_symmetry(oracle, n):
    rng = np.random.default_rng(n)
    m = cm_points(oracle, n, 1, seed=61 + n)[0]
    perm = rng.permutation(n)
    mp = np.vstack([m[:2], m[2:][perm]])
    assert oracle.amp2(n, mp[None])[0] == pytest.approx(oracle.amp2(n, m[None])[0], rel=1e-12)
    lam = [1, -1, -1, 1, 1][:n]
    h = helicity_index(1, -1, lam)
    hp = helicity_index(1, -1, [lam[i] for i in perm])
    assert abs(oracle.amp_hel(n, mp, hp)[0]) ** 2 == pytest.approx(
        abs(oracle.amp_hel(n, m, h)[0]) ** 2, rel=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_parity_and_helicity_selection(oracle, n):
    """|M_{-h}|^2 = |M_h|^2; s1 = s2 vanishes exactly (chirality); all photons of
    one helicity vanish by cancellation; 2(2^n - 2) helicities survive."""
    m = cm_points(oracle, n, 1, seed=71 + n)[0]
    full = (1 << (n + 2)) - 1
    vals = np.array([abs(oracle.amp_hel(n, m, h)[0]) ** 2 for h in range(full + 1)])
    top = vals.max()
    for h in range(full + 1):
        assert vals[h ^ full] == pytest.approx(vals[h], rel=1e-12, abs=1e-13 * top)
        s1, s2 = h & 1, (h >> 1) & 1
        lam = h >> 2
        if s1 == s2:
            assert vals[h] == 0.0
        elif lam == 0 or lam == (1 << n) - 1:
            assert vals[h] < 1e-24 * top
    assert int(np.sum(vals > 1e-20 * top)) == 2 * (2**n - 2)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_scaling(oracle, n):
    m = cm_points(oracle, n, 1, seed=81 + n)[0]
    lam = 3.7
    assert oracle.amp2(n, (lam * m)[None])[0] == pytest.approx(
        lam ** (4 - 2 * n) * oracle.amp2(n, m[None])[0], rel=1e-12)


def test_helicity_mask(oracle):
    n = 3
    m = cm_points(oracle, n, 1, seed=90)[0]
    hs = [5, 6, 9, 30, 17]
    direct = sum(abs(oracle.amp_hel(n, m, h)[0]) ** 2 for h in hs)
    assert oracle.amp2(n, m[None], hel_mask=mask_words(n, hs))[0] == pytest.approx(direct, rel=1e-14)


# --------------------------------------------------------------------------
# phase space
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_rambo_conservation_and_masslessness(oracle, n):
    ps = oracle.phase_space(n, 3, 0, 200, oracle.toy_pdf(), None)
    mom, rs = ps["momenta"], ps["sqrt_s"]
    tot = mom[:, 2:].sum(axis=1)
    inc = mom[:, 0] + mom[:, 1]
    scale = rs[:, None]
    np.testing.assert_allclose(tot / scale, inc / scale, atol=1e-13)
    m2 = mdot(mom[:, 2:], mom[:, 2:]) / (rs[:, None] ** 2)
    assert np.max(np.abs(m2)) < 1e-13
    assert np.all(mom[:, 2:, 0] > 0)


def test_phase_space_volume(oracle):
    """Phi_2 = 1/(8 pi), Phi_3 = s/(256 pi^3), and the recursion
    Phi_n(s) = int_0^s dm2/(2 pi) (1 - m2/s)/(8 pi) Phi_{n-1}(m2)."""
    s = 500.0**2
    assert oracle.phase_space_volume(2, s) == pytest.approx(1 / (8 * math.pi), rel=1e-14)
    assert oracle.phase_space_volume(3, s) == pytest.approx(s / (256 * math.pi**3), rel=1e-14)
    for n in range(3, 9):
        val, _ = integrate.quad(lambda m2: (1 - m2 / s) / (8 * math.pi) / (2 * math.pi)
                                * oracle.phase_space_volume(n - 1, m2), 0, s, epsrel=1e-12)
        assert oracle.phase_space_volume(n, s) == pytest.approx(val, rel=1e-10)
    # RAMBO returns the same constant weight
    assert oracle.rambo(4, 500.0, np.full(16, 0.3))[1] == oracle.phase_space_volume(4, s)


def test_rambo_two_body_isotropy(oracle):
    ps = oracle.phase_space(2, 11, 0, 4000, oracle.fixed(500.0), None)
    k = ps["momenta"][:, 2]
    cth = k[:, 3] / k[:, 0]
    phi = np.arctan2(k[:, 2], k[:, 1])
    assert stats.kstest(cth, stats.uniform(-1, 2).cdf).pvalue > 1e-4
    assert stats.kstest(phi, stats.uniform(-math.pi, 2 * math.pi).cdf).pvalue > 1e-4
    np.testing.assert_allclose(k[:, 0], 250.0, rtol=1e-10)


def test_rambo_three_body_dalitz_flat(oracle):
    """Massless 3-body: (x1, x2) = 2(E1, E2)/sqrt(s) uniform on x1, x2 <= 1, x1 + x2 >= 1."""
    ps = oracle.phase_space(3, 12, 0, 4000, oracle.fixed(500.0), None)
    x = 2 * ps["momenta"][:, 2:, 0] / 500.0
    x1, x2 = x[:, 0], x[:, 1]
    assert np.all(x1 <= 1 + 1e-12) and np.all(x1 + x2 >= 1 - 1e-12)
    assert stats.kstest(x1**2, "uniform").pvalue > 1e-4
    assert stats.kstest((x2 - (1 - x1)) / x1, "uniform").pvalue > 1e-4


def test_toy_pdf_marginal_is_beta(oracle):
    """Without the floor, x1 and x2 follow the normalised x^(-1/2)(1-x)^3 = Beta(1/2, 4)."""
    S = oracle.toy_pdf(floor=0.0)
    ps = oracle.phase_space(2, 13, 0, 4000, S, None)
    tau = ps["sqrt_s"] / 14000.0
    x1, x2 = tau * np.exp(ps["y"]), tau * np.exp(-ps["y"])
    beta = stats.beta(0.5, 4)
    assert stats.kstest(x1, beta.cdf).pvalue > 1e-4
    assert stats.kstest(x2, beta.cdf).pvalue > 1e-4
    assert np.all(ps["tries"] == 1)


def test_toy_pdf_floor_acceptance(oracle):
    """Acceptance of sqrt(x1 x2) 14 TeV > 100 GeV against its integral."""
    S = oracle.toy_pdf()
    ps = oracle.phase_space(2, 14, 0, 20000, S, None)
    assert np.all(ps["sqrt_s"] > 100.0)
    tau0 = (100.0 / 14000.0) ** 2
    beta = stats.beta(0.5, 4)
    rej, _ = integrate.quad(lambda x1: beta.pdf(x1) * beta.cdf(min(1.0, tau0 / x1)),
                            0, 1, points=[tau0], limit=400)
    p_acc = 1 - rej
    N, T = ps["tries"].size, ps["tries"].sum()
    est = N / T
    sigma = math.sqrt(p_acc * (1 - p_acc) / T)
    assert abs(est - p_acc) < 5 * sigma


def test_fixed_and_uniform_samplers(oracle):
    """The fixed sampler gives sqrt(s-hat) itself; the uniform one is uniform
    on [lo, hi] (KS test against the library's uniform law); both have y = 0
    and one attempt per point."""
    ps = oracle.phase_space(3, 15, 0, 50, oracle.fixed(500.0), None)
    assert np.all(ps["sqrt_s"] == 500.0) and np.all(ps["y"] == 0) and np.all(ps["tries"] == 1)
    ps = oracle.phase_space(3, 16, 0, 4000, oracle.uniform(200.0, 2000.0), None)
    rs = ps["sqrt_s"]
    assert np.all((rs > 200.0) & (rs < 2000.0))
    assert stats.kstest(rs, stats.uniform(loc=200.0, scale=1800.0).cdf).pvalue > 1e-4
    assert np.all(ps["y"] == 0) and np.all(ps["tries"] == 1)


# --------------------------------------------------------------------------
# cuts and cross section
# --------------------------------------------------------------------------

def _photon(pt, eta, phi):
    return np.array([pt * math.cosh(eta), pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(eta)])


def test_cut_decisions(oracle):
    C = oracle.cuts(20.0, 2.5, 0.4)
    good = [_photon(30, 0.1, 0.0), _photon(40, -1.0, 2.0)]
    assert oracle.pass_cuts(2, np.array(good), 0.0, C)
    assert not oracle.pass_cuts(2, np.array([_photon(19.9, 0.1, 0.0), good[1]]), 0.0, C)
    assert not oracle.pass_cuts(2, np.array([_photon(30, 2.51, 0.0), good[1]]), 0.0, C)
    assert oracle.pass_cuts(2, np.array([_photon(30, 2.4, 0.0), good[1]]), 0.0, C)
    # boost rapidity shifts eta: 2.4 + 0.2 fails
    assert not oracle.pass_cuts(2, np.array([_photon(30, 2.4, 0.0), good[1]]), 0.2, C)
    # Delta R: 0.3 in eta at equal phi fails; wrapped phi (pi - 0.1 vs -pi + 0.1) -> 0.2 fails
    assert not oracle.pass_cuts(2, np.array([_photon(30, 0.0, 1.0), _photon(30, 0.3, 1.0)]), 0.0, C)
    assert not oracle.pass_cuts(2, np.array([_photon(30, 0.0, math.pi - 0.1),
                                            _photon(30, 0.0, -math.pi + 0.1)]), 0.0, C)
    assert oracle.pass_cuts(2, np.array([_photon(30, 0.0, math.pi - 0.3),
                                        _photon(30, 0.0, -math.pi + 0.3)]), 0.0, C)
    # no Delta R cut when dr_min <= 0
    assert oracle.pass_cuts(2, np.array([_photon(30, 0.0, 1.0), _photon(30, 0.3, 1.0)]), 0.0,
                            oracle.cuts(20.0, 2.5, -1.0))


def test_n2_cut_acceptance_and_cross_section(oracle):
    """sqrt(s) = 500 GeV, pT > 20, |eta| < 2.5: pass fraction tanh 2.5 and
    sigma-hat = pi alpha^2 Q^4 (10 - 2 tanh 2.5) / (3 s) = 137.71 fb."""
    N = 40000
    S, Cc = oracle.fixed(500.0), oracle.cuts(20.0, 2.5, -1.0)
    w, mask, tries = oracle.event_weights(2, 0x0908440300000001, 0, N, S, Cc)
    frac = mask.mean()
    c0 = math.tanh(2.5)
    assert abs(frac - c0) < 5 * math.sqrt(c0 * (1 - c0) / N)
    sig, err = oracle.xsec_from_weights(w)
    alpha = 1 / 137.035999
    exact = math.pi * alpha**2 * Q**4 * (10 - 2 * c0) / (3 * 500.0**2) * 0.3893793721e12
    assert exact == pytest.approx(137.71, abs=0.01)
    assert abs(sig - exact) < 5 * err
    assert err / sig < 0.01


def _toy_pdf_sigma_n2(pt_min=20.0, eta_max=2.5, e_beam=7000.0, floor=100.0, alpha=1 / 137.035999):
    """u ubar -> 2 gamma cross section under the toy PDF by quadrature.

    x1, x2 each follow Beta(1/2, 4), sqrt(s-hat) = 2 e_beam sqrt(x1 x2) must
    exceed `floor`, either beam may carry the quark (a factor 2, Sec. 2.1
    eq. (1)), and the photons must pass the cuts of Sec. 2.2 in the lab
    frame, boosted by y = ln(x1/x2)/2 from the partonic one.  At n = 2 the
    partonic cross section is known in closed form: the photons are back to
    back at cos(theta*) = +-c, so pT = (sqrt(s-hat)/2) sqrt(1 - c^2), the lab
    pseudorapidities are +-atanh(c) + y, Delta R >= pi passes any cut below
    pi, and
        d sigma-hat / d c = pi alpha^2 Q^4 (1 + c^2) / (3 s-hat (1 - c^2)),
    whose integral over |c| < c_max is pi alpha^2 Q^4 (4 atanh c_max - 2 c_max)
    / (3 s-hat), with c_max = min(tanh(eta_max - |y|), sqrt(1 - 4 pT_min^2 /
    s-hat)).  With u_i = sqrt(x_i) the Beta density becomes 2 (1 - u^2)^3 / B
    (B = B(1/2, 4) = 32/35), and with tau = u1 u2, rho = ln(u1/u2) = y
    (du1 du2 = dtau drho / 2) the integral runs over floor / (2 e_beam) <
    tau < 1, |rho| < -ln tau."""
    B = 32.0 / 35.0
    E = 2 * e_beam

    def partonic_over_shat(shat, rho):   # sigma-hat s-hat / (pi alpha^2 Q^4 / 3)
        if abs(rho) >= eta_max:
            return 0.0
        c = min(math.tanh(eta_max - abs(rho)), math.sqrt(1 - 4 * pt_min**2 / shat))
        return 4 * math.atanh(c) - 2 * c

    def inner(s):   # tau = e^s
        tau = math.exp(s)
        shat = (tau * E) ** 2
        rmax = min(-s, eta_max)
        kink = eta_max - math.atanh(math.sqrt(1 - 4 * pt_min**2 / shat))

        def g(rho):
            u1s, u2s = tau * math.exp(rho), tau * math.exp(-rho)
            return (1 - u1s) ** 3 * (1 - u2s) ** 3 * partonic_over_shat(shat, rho)

        v, _ = integrate.quad(g, 0.0, rmax, points=[kink] if 0 < kink < rmax else None, limit=200,
                              epsabs=0, epsrel=1e-11)
        return 2 * v * tau / shat   # both signs of rho; dtau = tau ds

    I, _ = integrate.quad(inner, math.log(floor / E), 0.0, limit=400, epsabs=0, epsrel=1e-10)
    return 2 * (2 / B) ** 2 * 0.5 * I * math.pi * alpha**2 * Q**4 / 3 * GEV2_TO_FB


def test_toy_pdf_cross_section_scale(oracle):
    """The toy-PDF cross section sigma = 2 P_acc <w> (Sec. 2.1 eq. (1)-(2):
    the q <-> qbar factor 2, the acceptance of the sqrt(s-hat) floor from the
    draw counts, and the weights of eq. (2) with the cuts of Sec. 2.2) against
    the same integral done by quadrature at n = 2, where the partonic cross
    section is known in closed form."""
    exact = _toy_pdf_sigma_n2()
    assert exact == pytest.approx(193.766, rel=1e-5)
    w, mask, tries = oracle.event_weights(2, 0x0908440300000321, 0, 400_000, oracle.toy_pdf(), oracle.cuts())
    sig, err = oracle.xsec_from_weights(w, tries, 2)
    assert err / sig < 0.01
    assert abs(sig - exact) < 5 * err


def test_identical_photon_factor_by_soft_emission(oracle):
    """The 1/n! of eq. (2) beyond n = 2, from soft-photon factorisation.
    Events of u ubar -> 3 gamma at sqrt(s) = 500 GeV with exactly one photon
    of energy in [a, b] << sqrt(s) and every photon at |cos theta| < c0 carry,
    to O(b / sqrt(s)),
        sigma_3 = 3 (f(3) / f(2)) sigma_2(c0) I,
    with f(n) the identical-photon factor, 3 the choices of the soft photon,
    sigma_2(c0) = pi alpha^2 Q^4 (4 atanh c0 - 2 c0) / (3 s) the analytic n = 2
    cross section at |cos theta| < c0, and I the eikonal integral over the
    soft photon: d^3k / ((2 pi)^3 2E) e^2 Q^2 2 p1.p2 / (p1.k p2.k) gives
    I = 4 alpha Q^2 ln(b / a) atanh(c0) / pi.  With f(n) = 1/n! the prefactor
    is 1 (1/n would give 2)."""
    rs, a, b, c0, N = 500.0, 2.0, 10.0, 0.8, 4_000_000
    ps = oracle.phase_space(3, 0x0908440300000303, 0, N, oracle.fixed(rs), None)
    k = ps["momenta"][:, 2:, :]
    E, cos = k[:, :, 0], k[:, :, 3] / k[:, :, 0]
    sel = (((E > a) & (E < b)).sum(axis=1) == 1) & np.all(np.abs(cos) < c0, axis=1)
    idx = np.nonzero(sel)[0]
    a2 = oracle.amp2(3, ps["momenta"][idx])
    w = np.array([oracle.event_weight(3, rs**2, a2[j], ps["weight"][i]) for j, i in enumerate(idx)])
    sigma3 = w.sum() / N
    err = math.sqrt(((w**2).sum() / N - sigma3**2) / N)
    alpha = 1 / 137.035999
    sigma2 = math.pi * alpha**2 * Q**4 * (4 * math.atanh(c0) - 2 * c0) / (3 * rs**2) * 0.3893793721e12
    eikonal = 4 * alpha * Q**2 * math.log(b / a) * math.atanh(c0) / math.pi
    assert err / sigma3 < 0.02
    assert abs(sigma3 / (sigma2 * eikonal) - 1) < 0.08


def test_propagators_spacelike(oracle):
    """Every ordering prefix gives t = (p1 - K)^2 <= 0 at physical points."""
    n = 5
    p = oracle.phase_space(n, 15, 0, 200, oracle.toy_pdf(), None)["momenta"]
    for m in p:
        p1, ks = m[0], m[2:]
        for mask in range(1, (1 << n) - 1):
            K = sum(ks[i] for i in range(n) if mask >> i & 1)
            q = p1 - K
            assert mdot(q, q) <= 1e-9 * m[0, 0] ** 2
