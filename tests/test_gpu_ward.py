"""GPU gauge check (heget_ward): with a photon's polarisation replaced by
k/k^0 the sum over orderings vanishes for momentum-conserving points, so the
returned ratio is rounding noise -- at the FP64 level in FP64, several orders
larger in FP32 -- and the same inputs give O(1) ratios when the replacement
is wrong (checked on the oracle side by the Ward pin)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0908440300006000


def _points(O, n, N, seed):
    ps = O.phase_space(n, seed, 0, N, O.toy_pdf(), O.cuts())
    keep = ps["mask"] == 1
    return ps["momenta"][keep]


def _ward(H, ctx, n, mom, photon, prec):
    import torch
    m = torch.from_numpy(np.ascontiguousarray(mom)).cuda()
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    H.heget_ward(ctx, n, mom.shape[0], m, photon, out, precision=prec)
    H.heget_check(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("n,N", [(2, 400), (3, 300), (4, 200), (5, 60), (6, 24), (8, 2)])
def test_ward_ratio_is_rounding_noise(oracle, heget_lib, gpu, n, N):
    H = heget_lib
    mom = _points(oracle, n, N, SEED + n)
    assert mom.shape[0] > 0
    for photon in sorted({0, n // 2, n - 1}):
        r64 = _ward(H, gpu, n, mom, photon, H.HEGET_FP64)
        r32 = _ward(H, gpu, n, mom, photon, H.HEGET_FP32)
        assert np.all(np.isfinite(r64)) and np.all(np.isfinite(r32))
        assert np.max(r64) <= 1e-12, (photon, np.max(r64))
        assert np.median(r32) <= 1e-5 and np.max(r32) <= 1e-3, (photon, np.median(r32), np.max(r32))
        # the numerator is computed, not dropped: rounding noise that scales with the precision
        assert np.mean(r64 > 0) > 0.9
        assert np.median(r32) > 1e3 * np.median(r64)


def test_ward_matches_oracle_scale_of_noise(oracle, heget_lib, gpu):
    """Oracle and device both put the gauge-replaced sum at the FP64 rounding
    level relative to the largest helicity amplitude."""
    H = heget_lib
    n = 3
    mom = _points(oracle, n, 20, SEED + 33)
    r64 = _ward(H, gpu, n, mom, 1, H.HEGET_FP64)
    for p in range(mom.shape[0]):
        big = max(abs(oracle.amp_hel(n, mom[p], h)[0]) for h in range(1 << (n + 2)))
        wmax = max(abs(oracle.amp_hel(n, mom[p], h, ward=1)[0]) for h in range(1 << (n + 2)))
        assert wmax / big <= 1e-12
        assert r64[p] <= 1e-12


def test_ward_argument_checks_and_bad_points(heget_lib, gpu):
    import torch
    H = heget_lib
    m = torch.zeros((4, 6, 4), dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for bad in (-1, 4, 7):
        with pytest.raises(H.HegetError):
            H.heget_ward(gpu, 4, 4, m, bad, out)
    with pytest.raises(H.HegetError):
        H.heget_ward(gpu, 4, 4, None, 0, out)
    # an all-zero row fails the device input check: NaN and EINVAL from heget_check
    H.heget_ward(gpu, 4, 4, m, 0, out)
    with pytest.raises(H.HegetError):
        H.heget_check(gpu)
    assert np.all(np.isnan(out.cpu().numpy()))
