"""Kinematic distributions on the device (heget_hist; Sec. 5, Fig. 2)
against the oracle's histograms of the same events: bin sums of the FP64
and FP32 event weights within their parity tolerances, entry counts (unit
weights) bit for bit, and at the full size of the n = 4 toy-PDF workload the
properties that hold at any size: every histogram holds the cross section's
sum of weights times its entries per event, the cuts leave nothing outside
pT > 20, |eta| < 2.5 and Delta R > 0.4, and the sums are reproducible."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x090844030000B000
PT_MAX, PT, ETA, DR, DR_MIN, SQRT_S = range(6)
SPECS = [(PT_MAX, 40, 0.0, 400.0), (PT, 40, 0.0, 400.0), (ETA, 25, -2.5, 2.5), (DR, 30, 0.0, 6.0),
         (DR_MIN, 30, 0.0, 6.0), (SQRT_S, 50, 0.0, 2500.0)]


def _split(flat, specs):
    out, off = [], 0
    for sp in specs:
        out.append(flat[2 * off:2 * (off + sp[1] + 2)].reshape(sp[1] + 2, 2))
        off += sp[1] + 2
    return out


def _dev_hist(H, ctx, n, seed, i0, w, specs, sampler):
    import torch
    out = torch.empty(H.hist_bins(specs), dtype=torch.float64, device="cuda")
    H.heget_hist(ctx, n, seed, i0, w.numel(), sampler, w, specs, out)
    torch.cuda.synchronize()
    return _split(out.cpu().numpy(), specs)


def _dev_weights(H, ctx, n, seed, i0, N, sampler, prec):
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_xsec_async(ctx, n, seed, i0, N, sampler, prec, res, w)
    torch.cuda.synchronize()
    return w, H.result_from_tensor(res)


CASES = [(2, "fixed", 2309), (4, "toy", 3001), (5, "toy", 1000), (6, "uniform", 300)]


def _samplers(H, O, kind):
    if kind == "fixed":
        return H.sampler_fixed(500.0), O.fixed(500.0)
    if kind == "uniform":
        return H.sampler_uniform(200.0, 2000.0), O.uniform(200.0, 2000.0)
    return H.sampler_toy_pdf(), O.toy_pdf()


@pytest.mark.parametrize("n,kind,N", CASES + [(8, "uniform", 700)])
def test_counts_bit_exact(oracle, heget_lib, gpu, n, kind, N):
    """Unit weights: every event's entries counted, each in the oracle's bin."""
    import torch
    H = heget_lib
    sd, so = _samplers(H, oracle, kind)
    seed, i0 = SEED + n, 77
    ones = torch.ones(N, dtype=torch.float64, device="cuda")
    got = _dev_hist(H, gpu, n, seed, i0, ones, SPECS, sd)
    ps = oracle.phase_space(n, seed, i0, N, so, oracle.cuts())
    ref = oracle.hist(n, ps["momenta"], ps["y"], np.ones(N), SPECS)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("n,kind,N", CASES)
def test_weighted_sums_match_oracle(oracle, heget_lib, gpu, n, kind, N):
    H = heget_lib
    sd, so = _samplers(H, oracle, kind)
    seed, i0 = SEED + 10 + n, 5
    wo, mask, _ = oracle.event_weights(n, seed, i0, N, so, oracle.cuts())
    ps = oracle.phase_space(n, seed, i0, N, so, oracle.cuts())
    ref = oracle.hist(n, ps["momenta"], ps["y"], wo, SPECS)
    for prec, tol in ((H.HEGET_FP64, 1e-10), (H.HEGET_FP32, 1e-4)):
        w, _ = _dev_weights(H, gpu, n, seed, i0, N, sd, prec)
        got = _dev_hist(H, gpu, n, seed, i0, w, SPECS, sd)
        scale = math.fsum(wo)
        for g, r in zip(got, ref):
            assert np.max(np.abs(g[:, 0] - r[:, 0])) <= tol * scale
            assert np.max(np.abs(g[:, 1] - r[:, 1])) <= tol * math.fsum(wo * wo)


def test_full_size_properties(heget_lib, gpu):
    """n = 4 toy PDF, 1,048,576 points (the bench's step), FP32 weights."""
    import torch
    H = heget_lib
    n, N, seed = 4, 1 << 20, SEED + 99
    S = H.sampler_toy_pdf()
    w, r = _dev_weights(H, gpu, n, seed, 0, N, S, H.HEGET_FP32)
    specs = [(PT_MAX, 50, 20.0, 520.0), (PT, 50, 20.0, 520.0), (ETA, 50, -2.5, 2.5), (DR, 40, 0.4, 8.4),
             (DR_MIN, 40, 0.4, 8.4), (SQRT_S, 50, 0.0, 5000.0)]
    got = _dev_hist(H, gpu, n, seed, 0, w, specs, S)
    mult = [1, n, n, n * (n - 1) // 2, 1, 1]
    for h, m in zip(got, mult):
        assert math.fsum(h[:, 0]) == pytest.approx(m * r.sum_w, rel=1e-12)
        assert math.fsum(h[:, 1]) == pytest.approx(m * r.sum_w2, rel=1e-12)
    for k in (0, 1, 3, 4):   # pT > 20 and Delta R > 0.4: nothing below lo
        assert got[k][0, 0] == 0.0
    assert got[2][0, 0] == 0.0 and got[2][-1, 0] == 0.0   # |eta| < 2.5
    again = _dev_hist(H, gpu, n, seed, 0, w, specs, S)
    for a, b in zip(got, again):
        np.testing.assert_array_equal(a, b)
    # two halves add up to the whole (to rounding)
    half = N // 2 + 13
    lo = _dev_hist(H, gpu, n, seed, 0, w[:half].contiguous(), specs, S)
    hi = _dev_hist(H, gpu, n, seed, half, w[half:].contiguous(), specs, S)
    for a, b, c in zip(lo, hi, got):
        np.testing.assert_allclose(a + b, c, rtol=1e-13, atol=1e-15 * abs(r.sum_w))


def test_hist_argument_checks(heget_lib, gpu):
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    w = torch.ones(10, dtype=torch.float64, device="cuda")
    out = torch.full((64,), 7.0, dtype=torch.float64, device="cuda")
    for bad in ([(9, 4, 0.0, 1.0)], [(PT, 0, 0.0, 1.0)], [(PT, 4, 1.0, 1.0)], [(PT, 4, 0.0, float("inf"))],
                [(PT, 1023, 0.0, 1.0)], [(PT, 4, 0.0, 1.0)] * 9, [], [(PT, 4, 0.0, 1e-310)]):
        with pytest.raises(H.HegetError):
            H.heget_hist(gpu, 4, 1, 0, 10, S, w, bad, out)
    with pytest.raises(H.HegetError):
        H.heget_hist(gpu, 9, 1, 0, 10, S, w, [(PT, 4, 0.0, 1.0)], out)
    with pytest.raises(H.HegetError):
        H.heget_hist(gpu, 4, 1, 0, 10, S, None, [(PT, 4, 0.0, 1.0)], out)
    H.heget_hist(gpu, 4, 1, 0, 0, S, None, [(PT, 4, 0.0, 1.0)], out)   # N = 0: zeros
    torch.cuda.synchronize()
    assert torch.all(out[:12] == 0) and torch.all(out[12:] == 7.0)
