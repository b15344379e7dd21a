"""The device logarithm of the RAMBO energies (Tang's table-driven method)
against the host libm logarithm: within 3 ulp of the result everywhere on the
inputs RAMBO produces (products of two uniforms in (0, 1)), at every table
breakpoint and midpoint, next to 1 (where the ln 2 terms cancel) and at the
extreme exponents."""
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
    j = np.arange(65)
    xs.append(1.0 + j / 64.0)
    xs.append((1.0 + (j + 0.5) / 64.0)[:-1])
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
