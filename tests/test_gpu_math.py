"""Device elementary functions of RAMBO, checked against the host.

The logarithm of the RAMBO energies (Tang's table-driven method) against the
host libm logarithm: within 3 ulp of the result everywhere on the inputs
RAMBO produces (products of two uniforms in (0, 1)), at every table
breakpoint and midpoint, next to 1 (where the ln 2 terms cancel) and at the
extreme exponents.  The cosine and sine of the azimuth 2 pi r against
extended-precision host values: within 2.5 ulp.  The records' integer
double -> float conversion against the hardware one: bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev_log(H, x):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.empty_like(xd)
    H.heget_log_table(xd, yd, x.size)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_log_table_within_three_ulp(heget_lib, gpu):
    H = heget_lib
    rng = np.random.default_rng(4403)
    m = rng.integers(0, 2**52, size=(2, 400_000), dtype=np.uint64)
    u = (m.astype(np.float64) + 0.5) * 2.0**-52          # the uniforms of the RNG layout
    xs = [u[0] * u[1], u[0]]
    j = np.arange(257)
    xs.append(1.0 + j / 256.0)
    xs.append((1.0 + (j + 0.5) / 256.0)[:-1])
    xs.append(np.nextafter(1.0 + (j + 0.5) / 256.0, 0.0)[:-1])
    xs.append(np.nextafter(1.0, 0.0) - np.arange(64) * 2.0**-53)
    xs.append(0.5 + np.arange(1, 64) * 2.0**-60)
    xs.append(np.ldexp(1.0 + rng.random(2000), rng.integers(-1021, 1023, 2000)))
    xs.append(np.array([2.0**-106, 2.0**-1022, 0.75, 1.5, 3.0, 1e300]))
    x = np.concatenate(xs)
    got = _dev_log(H, x)
    ref = np.log(x)
    nz = ref != 0
    assert np.all(got[~nz] == 0.0)
    err = _ulps(got[nz], ref[nz])
    assert err.max() <= 3.0, (err.max(), x[nz][np.argmax(err)])
    assert np.mean(err <= 1.0) > 0.99


def test_log_table_argument_checks(heget_lib, gpu):
    H = heget_lib
    with pytest.raises(H.HegetError):
        H.heget_log_table(None, None, 4)
    H.heget_log_table(None, None, 0)


def _two_pi_long():
    return np.longdouble("6.283185307179586476925286766559005768394")


def test_sincos_2pi_within_two_and_a_half_ulp(heget_lib, gpu):
    """The RAMBO azimuth (table of 2 pi j/512 plus Taylor series of the
    remainder) against cos and sin of 2 pi r in extended precision: random
    uniforms, every breakpoint and the midpoints between them (where the
    table index switches), the quarter turns (exact zeros of one factor) and
    the ends of (0, 1)."""
    import torch
    H = heget_lib
    rng = np.random.default_rng(2 * 4403)
    m = list(rng.integers(0, 2**52, size=200_000, dtype=np.uint64))
    for j in range(513):
        for off in (-(1 << 42) - 1, -(1 << 42), -1, 0, 1, (1 << 42) - 1, 1 << 42):
            c = j * (1 << 43) + off
            if 0 <= c < (1 << 52):
                m.append(np.uint64(c))
    m += [np.uint64(v) for v in (0, 1, (1 << 52) - 1, (1 << 52) - 2)]
    m = np.array(m, dtype=np.uint64)
    low = rng.integers(0, 1 << 12, size=m.size, dtype=np.uint64)
    bits = (m << np.uint64(12)) | low
    words = np.stack([(bits & np.uint64(0xFFFFFFFF)).astype(np.uint32), (bits >> np.uint64(32)).astype(np.uint32)], 1)
    wd = torch.from_numpy(words.view(np.int32).copy()).cuda()
    cs = torch.empty((m.size, 2), dtype=torch.float64, device="cuda")
    H.heget_sincos_2pi(wd, cs, m.size)
    torch.cuda.synchronize()
    got = cs.cpu().numpy()
    r = (2 * m.astype(np.longdouble) + 1) / np.longdouble(2.0**53)
    phi = _two_pi_long() * r
    for k, ref in enumerate((np.cos(phi), np.sin(phi))):
        refd = ref.astype(np.float64)
        err = np.abs(got[:, k].astype(np.longdouble) - ref) / np.spacing(np.abs(refd)).astype(np.longdouble)
        err = err.astype(np.float64)
        assert err.max() <= 2.5, (k, err.max(), m[np.argmax(err)])
        assert np.mean(err <= 1.0) > 0.99


def test_sincos_2pi_argument_checks(heget_lib, gpu):
    H = heget_lib
    with pytest.raises(H.HegetError):
        H.heget_sincos_2pi(None, None, 4)
    H.heget_sincos_2pi(None, None, 0)


def test_f32_round_matches_the_hardware_conversion(heget_lib, gpu):
    """The records' double -> float conversion (integer operations) against
    the hardware conversion, bit for bit, over the normal float range: random
    values, ties and near-ties of the dropped 29 bits, carries into the
    exponent, the largest finite float and the overflow boundary, infinities
    and NaN; below 2^-126 it gives a signed zero."""
    import torch
    H = heget_lib
    rng = np.random.default_rng(3 * 4403)
    xs = [rng.standard_normal(100_000) * np.exp2(rng.integers(-120, 120, 100_000)),
          rng.random(50_000), -rng.random(50_000)]
    base = np.float32(rng.random(2000) + 1.0).astype(np.float64)
    ulp = np.spacing(np.float32(base)).astype(np.float64)
    for f in (0.5, 0.5 - 2.0**-30, 0.5 + 2.0**-30, 1.0 - 2.0**-30, 2.0**-29):
        xs += [base + f * ulp, -(base + f * ulp)]
    fmax = float(np.finfo(np.float32).max)
    xs.append(np.array([0.0, -0.0, 2.0**-126, -(2.0**-126), fmax, -fmax, np.nextafter(2.0**128 - 2.0**103, 0.0),
                        2.0**128 - 2.0**103, 2.0**129, np.inf, -np.inf, 1.9999999403953552, 0.99999997, 1e30]))
    x = np.concatenate(xs)
    x = x[(np.abs(x) >= 2.0**-126) | (x == 0)]   # the hardware keeps subnormals; the records never hold them
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty(x.size, dtype=torch.float32, device="cuda")
    H.heget_f32_round(xd, yd, x.size)
    torch.cuda.synchronize()
    got = yd.cpu().numpy()
    ref = xd.float().cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    tiny = np.array([1e-39, -1e-40, 2.0**-127], dtype=np.float64)
    H.heget_f32_round(torch.from_numpy(tiny).cuda(), yd, tiny.size)
    torch.cuda.synchronize()
    assert np.all(yd[:3].cpu().numpy() == 0.0) and np.signbit(yd[1].item())
    nan = torch.tensor([np.nan], dtype=torch.float64, device="cuda")
    H.heget_f32_round(nan, yd, 1)
    torch.cuda.synchronize()
    assert np.isnan(yd[0].item())


def test_f32_round_argument_checks(heget_lib, gpu):
    H = heget_lib
    with pytest.raises(H.HegetError):
        H.heget_f32_round(None, None, 4)
    H.heget_f32_round(None, None, 0)
