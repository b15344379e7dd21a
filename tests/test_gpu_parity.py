"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 chain within helpers.fp64_tolerance per point (a 1e-12
floor for rounding-order differences over up to n! 2^(n+2) terms, plus input
rounding amplified by the smallest propagator denominator); FP32 chain median
<= 1e-4 and max <= 1e-3 relative; phase-space momenta within 1e-12 sqrt(s)
(FP64 rounding amplified by the RAMBO boost); integer outputs (cut mask,
sampler attempts) bit-exact.
"""
import math

import numpy as np
import pytest

from helpers import fp64_tolerance, helicity_index, mask_words, mdot

pytestmark = pytest.mark.gpu

SEED = 0x0908440300000000


def torch_mod():
    import torch
    return torch


def dev(a, dtype=None):
    torch = torch_mod()
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=dtype) if dtype else t.cuda()


def gpu_amp2(H, ctx, n, mom, precision, mask=None):
    torch = torch_mod()
    N = mom.shape[0]
    m = dev(mom.astype(np.float64))
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    mk = dev(mask.astype(np.uint32).view(np.int32)) if mask is not None else None
    H.heget_amp2(ctx, n, N, m, out, hel_mask=mk, precision=precision)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rel(a, b):
    return np.abs(a - b) / np.abs(b)


# --------------------------------------------------------------------------
# phase space
# --------------------------------------------------------------------------

SAMPLERS = {
    "fixed": lambda O, H: (O.fixed(500.0), H.sampler_fixed(500.0)),
    "uniform": lambda O, H: (O.uniform(200.0, 2000.0), H.sampler_uniform(200.0, 2000.0)),
    "toy": lambda O, H: (O.toy_pdf(), H.sampler_toy_pdf()),
}


@pytest.mark.parametrize("n", [2, 4, 6, 8])
@pytest.mark.parametrize("kind", ["fixed", "uniform", "toy"])
def test_phase_space_matches_oracle(oracle, heget_lib, gpu, n, kind):
    torch = torch_mod()
    H = heget_lib
    so, sh = SAMPLERS[kind](oracle, H)
    N, i0 = 3001, 12345
    ref = oracle.phase_space(n, SEED + 1, i0, N, so, oracle.cuts())
    mom = torch.empty((N, n + 2, 4), dtype=torch.float64, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    rs = torch.empty(N, dtype=torch.float64, device="cuda")
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    mask = torch.empty(N, dtype=torch.uint8, device="cuda")
    tries = torch.empty(N, dtype=torch.int32, device="cuda")
    H.heget_phase_space_ex(gpu, SEED + 1, i0, N, n, sh, mom, w, rs, y, mask, tries)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(tries.cpu().numpy(), ref["tries"])
    np.testing.assert_allclose(rs.cpu().numpy(), ref["sqrt_s"], rtol=1e-15)
    np.testing.assert_allclose(y.cpu().numpy(), ref["y"], rtol=0, atol=1e-14)
    scale = ref["sqrt_s"][:, None, None]
    np.testing.assert_allclose(mom.cpu().numpy() / scale, ref["momenta"] / scale, rtol=0, atol=1e-12)
    np.testing.assert_allclose(w.cpu().numpy(), ref["weight"], rtol=1e-13)
    np.testing.assert_array_equal(mask.cpu().numpy(), ref["mask"])


def test_phase_space_fixed_entry_point(oracle, heget_lib, gpu):
    torch = torch_mod()
    n, N = 3, 257
    mom = torch.empty((N, n + 2, 4), dtype=torch.float64, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    heget_lib.heget_phase_space(gpu, SEED, N, n, 500.0, mom, w)
    torch.cuda.synchronize()
    ref = oracle.phase_space(n, SEED, 0, N, oracle.fixed(500.0))
    np.testing.assert_allclose(mom.cpu().numpy() / 500.0, ref["momenta"] / 500.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(w.cpu().numpy(), ref["weight"], rtol=1e-13)


# --------------------------------------------------------------------------
# |M|^2
# --------------------------------------------------------------------------

N_BY_N = {2: 5003, 3: 1001, 4: 301, 5: 77, 6: 21, 7: 6}


def oracle_points(O, n, N, seed):
    return O.phase_space(n, seed, 0, N, O.toy_pdf())["momenta"]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_amp2_fp64_matches_oracle(oracle, heget_lib, gpu, n):
    mom = oracle_points(oracle, n, N_BY_N[n], SEED + 10 + n)
    ref = oracle.amp2(n, mom)
    got = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP64)
    assert np.all(rel(got, ref) < fp64_tolerance(mom))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_amp2_fp32_accuracy(oracle, heget_lib, gpu, n):
    mom = oracle_points(oracle, n, N_BY_N[n], SEED + 10 + n)
    ref = oracle.amp2(n, mom)
    got = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP32)
    r = rel(got, ref)
    assert np.median(r) <= 1e-4
    assert np.max(r) <= 1e-3


def test_amp2_n8_full_sum(oracle, heget_lib, gpu):
    n = 8
    mom = oracle_points(oracle, n, 2, SEED + 18)
    ref = oracle.amp2(n, mom)
    got64 = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP64)
    got32 = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP32)
    assert np.all(rel(got64, ref) < fp64_tolerance(mom))
    assert np.max(rel(got32, ref)) < 1e-3


@pytest.mark.parametrize("n", [6, 8])
def test_amp2_mhv_closed_form(oracle, heget_lib, gpu, n):
    """Single-minority-helicity amplitudes against their closed form (no brute force)."""
    e2 = 4 * math.pi / 137.035999
    Q = 2 / 3
    mom = oracle_points(oracle, n, 24, SEED + 30 + n)
    for minority in (+1, -1):
        hs = []
        for j in range(n):
            lam = [-minority] * n
            lam[j] = minority
            hs.append(helicity_index(1, -1, lam))
        mask = mask_words(n, hs)
        got64 = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP64, mask)
        got32 = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP32, mask)
        p1, p2, ks = mom[:, 0], mom[:, 1], mom[:, 2:]
        s = mdot(p1 + p2, p1 + p2)
        s1 = 2 * mdot(p1[:, None], ks)
        s2 = 2 * mdot(p2[:, None], ks)
        pref = (2 * e2 * Q * Q) ** n * s ** (n - 2) / np.prod(s1 * s2, axis=1)
        a, b = (s1, s2) if minority < 0 else (s2, s1)
        ref = pref * np.sum(a ** 3 * b, axis=1)
        assert np.all(rel(got64, ref) < fp64_tolerance(mom))
        assert np.max(rel(got32, ref)) < 1e-3


@pytest.mark.parametrize("n", [3, 4, 5])
def test_amp2_helicity_masks(oracle, heget_lib, gpu, n):
    rng = np.random.default_rng(n)
    mom = oracle_points(oracle, n, 33, SEED + 40 + n)
    for trial in range(3):
        hs = rng.choice(1 << (n + 2), size=1 + trial * 5, replace=False)
        mask = mask_words(n, hs)
        ref = oracle.amp2(n, mom, hel_mask=mask)
        got = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP64, mask)
        scale = oracle.amp2(n, mom)
        assert np.all(np.abs(got - ref) / scale < fp64_tolerance(mom))


def test_amp2_rejects_bad_points(oracle, heget_lib, gpu):
    n = 3
    mom = oracle_points(oracle, n, 40, SEED + 50)
    mom[5, 3, 1] = np.nan          # non-finite photon component
    mom[17, 0, 1] = 1.0            # p1 not along +z
    got = gpu_amp2(heget_lib, gpu, n, mom, heget_lib.HEGET_FP64)
    assert np.isnan(got[5]) and np.isnan(got[17])
    good = np.ones(40, dtype=bool)
    good[[5, 17]] = False
    assert np.all(rel(got[good], oracle.amp2(n, mom[good])) < fp64_tolerance(mom[good]))
    with pytest.raises(heget_lib.HegetError) as ei:
        heget_lib.heget_check(gpu)
    assert ei.value.status == heget_lib.HEGET_EINVAL
    heget_lib.heget_check(gpu)     # flag cleared


def test_amp2_host_argument_checks(heget_lib, gpu):
    torch = torch_mod()
    x = torch.zeros((4, 6, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for bad in [dict(n=1), dict(n=9), dict(precision=16)]:
        kw = dict(n=4, precision=heget_lib.HEGET_FP64)
        kw.update(bad)
        with pytest.raises(heget_lib.HegetError):
            heget_lib.heget_amp2(gpu, kw["n"], 4, x, out, precision=kw["precision"])
    heget_lib.heget_amp2(gpu, 4, 0, x, out)      # N = 0 is a no-op


# --------------------------------------------------------------------------
# cross section and accumulation
# --------------------------------------------------------------------------

def gpu_xsec(H, ctx, n, N, seed, sampler, precision, i0=0, want_w=False):
    torch = torch_mod()
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda") if want_w else None
    H.heget_xsec_async(ctx, n, seed, i0, N, sampler, precision, res, w)
    torch.cuda.synchronize()
    r = H.result_from_tensor(res)
    return r, (w.cpu().numpy() if want_w else None)


def test_xsec_n2_analytic(heget_lib, gpu):
    """sqrt(s) = 500 GeV, pT > 20, |eta| < 2.5: sigma = pi a^2 Q^4 (10 - 2 tanh 2.5)/(3 s)."""
    H = heget_lib
    H.heget_set_params(gpu, dr_min=-1.0)
    try:
        r = H.heget_xsec(gpu, 2, 65536, SEED + 1, H.sampler_fixed(500.0), H.HEGET_FP64)
    finally:
        H.heget_set_params(gpu)
    alpha, Q, c0 = 1 / 137.035999, 2 / 3, math.tanh(2.5)
    exact = math.pi * alpha**2 * Q**4 * (10 - 2 * c0) / (3 * 500.0**2) * 0.3893793721e12
    assert r.n_total == 65536 and r.n_tries == 65536
    assert abs(r.sigma_fb - exact) < 5 * r.err_fb
    assert abs(r.n_pass / 65536 - c0) < 5 * math.sqrt(c0 * (1 - c0) / 65536)


def _edge_event(theta, e1=100.0, rs=500.0):
    """u ubar -> 3 gamma at sqrt(s) = rs with photon 1 (energy e1) at angle
    theta to the incoming u and photons 2, 3 sharing the rest back to back
    in their own rest frame."""
    e = rs / 2
    k1 = e1 * np.array([1.0, math.sin(theta), 0.0, math.cos(theta)])
    P = np.array([rs, 0.0, 0.0, 0.0]) - k1
    m = math.sqrt(P[0] ** 2 - P[1:] @ P[1:])
    beta = P[1:] / P[0]
    g = 1 / math.sqrt(1 - beta @ beta)

    def boost(p):
        bp = beta @ p[1:]
        return np.concatenate([[g * (p[0] + bp)], p[1:] + ((g - 1) * bp / (beta @ beta) + g * p[0]) * beta])

    q = m / 2
    return np.array([[e, 0, 0, e], [e, 0, 0, -e], k1,
                     boost(np.array([q, 0, q, 0])), boost(np.array([q, 0, -q, 0]))])


@pytest.mark.parametrize("kind", ["collinear", "soft"])
def test_nearly_collinear_and_soft_photons(oracle, heget_lib, gpu, kind):
    """The method's singular limits: a photon at 1e-2 .. 1e-4 rad from the
    beam (|M|^2 grows as 1/theta^2), or of 1 .. 1e-3 GeV at 1 rad (as 1/E^2),
    where the propagator condition grows as well.  FP64 within the rounding
    tolerance of the input; FP32 finite."""
    torch = torch_mod()
    H = heget_lib
    if kind == "collinear":
        mom = np.stack([_edge_event(t) for t in (1e-2, 3e-3, 1e-3, 3e-4, 1e-4)])
    else:
        mom = np.stack([_edge_event(1.0, e1) for e1 in (1.0, 1e-1, 1e-2, 1e-3)])
    ref = oracle.amp2(3, mom)
    assert np.all(np.diff(ref) > 0)   # closer to the limit, larger |M|^2
    m = dev(mom)
    for prec in (H.HEGET_FP64, H.HEGET_FP32):
        out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
        H.heget_amp2(gpu, 3, mom.shape[0], m, out, precision=prec)
        H.heget_check(gpu)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        if prec == H.HEGET_FP64:
            assert np.all(rel(got, ref) <= fp64_tolerance(mom))


@pytest.mark.parametrize("n", [3, 5])
def test_other_quark_charges_couplings_and_cuts(oracle, heget_lib, gpu, n):
    """Context parameters reach every step: d dbar -> n gamma (Q = -1/3, the
    other subprocesses of Sec. 2.1 differ from u ubar only in the charge), a
    different alpha and different cuts, against the oracle with the same
    parameters: |M|^2 in FP64, and the fused path's cut masks (bit for bit)
    and weights."""
    torch = torch_mod()
    H = heget_lib
    alpha, Q, cut = 1 / 128.0, -1 / 3, (30.0, 2.0, 0.6)
    seed, N = SEED + 80 + n, {3: 1500, 5: 200}[n]
    H.heget_set_params(gpu, alpha=alpha, q_charge=Q, pt_min=cut[0], eta_max=cut[1], dr_min=cut[2])
    try:
        mom = oracle_points(oracle, n, N, seed)
        ref = oracle.amp2(n, mom, alpha=alpha, Q=Q)
        m = dev(mom)
        out = torch.empty(N, dtype=torch.float64, device="cuda")
        H.heget_amp2(gpu, n, N, m, out, precision=H.HEGET_FP64)
        torch.cuda.synchronize()
        assert np.all(rel(out.cpu().numpy(), ref) <= fp64_tolerance(mom))
        wo, mask, tries = oracle.event_weights(n, seed, 0, N, oracle.toy_pdf(), oracle.cuts(*cut), alpha=alpha, Q=Q)
        r64, w64 = gpu_xsec(H, gpu, n, N, seed, H.sampler_toy_pdf(), H.HEGET_FP64, want_w=True)
        r32, w32 = gpu_xsec(H, gpu, n, N, seed, H.sampler_toy_pdf(), H.HEGET_FP32, want_w=True)
    finally:
        H.heget_set_params(gpu)
    np.testing.assert_array_equal(w64 != 0, mask != 0)
    np.testing.assert_array_equal(w32 != 0, mask != 0)
    assert 0 < mask.sum() < N and r64.n_pass == r32.n_pass == int(mask.sum())
    nz = wo != 0
    assert np.max(rel(w64[nz], wo[nz])) < 1e-11
    assert np.max(rel(w32[nz], wo[nz])) < 1e-3


@pytest.mark.parametrize("n,N", [(2, 4099), (3, 2051), (4, 1030), (5, 130)])
def test_xsec_event_weights_match_oracle(oracle, heget_lib, gpu, n, N):
    H = heget_lib
    seed, i0 = SEED + 60 + n, 777
    wo, mask, tries = oracle.event_weights(n, seed, i0, N, oracle.toy_pdf(), oracle.cuts())
    r64, w64 = gpu_xsec(H, gpu, n, N, seed, H.sampler_toy_pdf(), H.HEGET_FP64, i0=i0, want_w=True)
    r32, w32 = gpu_xsec(H, gpu, n, N, seed, H.sampler_toy_pdf(), H.HEGET_FP32, i0=i0, want_w=True)
    np.testing.assert_array_equal(w64 != 0, mask != 0)
    nz = wo != 0
    assert np.max(rel(w64[nz], wo[nz])) < 1e-11
    assert np.max(rel(w32[nz], wo[nz])) < 1e-3
    assert r64.n_pass == int(mask.sum()) and r64.n_tries == int(tries.sum()) and r64.n_total == N
    assert r64.sum_w == pytest.approx(math.fsum(w64), rel=1e-15)
    sig, err = oracle.xsec_from_weights(wo, tries, 2)
    assert r64.sigma_fb == pytest.approx(sig, rel=1e-11)
    assert r64.err_fb == pytest.approx(err, rel=1e-9)


def test_xsec_deterministic(heget_lib, gpu):
    H = heget_lib
    a, wa = gpu_xsec(H, gpu, 4, 50000, SEED + 70, H.sampler_toy_pdf(), H.HEGET_FP32, want_w=True)
    b, wb = gpu_xsec(H, gpu, 4, 50000, SEED + 70, H.sampler_toy_pdf(), H.HEGET_FP32, want_w=True)
    assert a.sum_w == b.sum_w and a.sum_w2 == b.sum_w2 and a.err_fb == b.err_fb
    np.testing.assert_array_equal(wa, wb)


def test_compensated_sum_vs_fsum(heget_lib, gpu):
    """Double-double accumulation: within 1 ulp of the exactly rounded sum."""
    torch = torch_mod()
    rng = np.random.default_rng(5)
    N = 1 << 20
    x = rng.standard_normal(N) * 10.0 ** rng.uniform(-10, 10, N)
    x[::7] *= -1
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    heget_lib.heget_sum(gpu, dev(x), N, out)
    torch.cuda.synchronize()
    s, s2 = out.cpu().numpy()
    exact = math.fsum(x)
    assert abs(s - exact) <= np.spacing(abs(exact))
    exact2 = math.fsum(x * x)
    assert abs(s2 - exact2) <= np.spacing(abs(exact2))
