"""Device |M|^2 under the symmetries of the amplitude.

These properties hold at any size, so they reach sizes and inputs the oracle
cannot: rotations about the beam axis, boosts along it (p1 and p2 then have
unequal energies, a frame heget_amp2 accepts), the exchange of the incoming
u and ubar (followed by the rotation by pi about x that puts them back on
+z / -z), photon permutations, and the scaling |M|^2(lambda p) =
lambda^(4-2n) |M|^2(p).  The boosted frame is also compared with the oracle
directly.  Tolerances: FP64 within the rounding tolerance of both inputs;
FP32 against the FP64 result with the FP32 parity bar."""
import math

import numpy as np
import pytest

from helpers import boost_matrix, fp64_tolerance, rotation_matrix, transform

pytestmark = pytest.mark.gpu

SEED = 0x090844030000D000


def _points(H, ctx, n, N, seed):
    """Cut-passing toy-PDF points generated on the device."""
    import torch
    mom = torch.empty((N, n + 2, 4), dtype=torch.float64, device="cuda")
    mask = torch.empty(N, dtype=torch.uint8, device="cuda")
    H.heget_phase_space_ex(ctx, seed, 0, N, n, H.sampler_toy_pdf(), momenta=mom, mask=mask)
    torch.cuda.synchronize()
    m = mom.cpu().numpy()
    return m[mask.cpu().numpy() == 1]


def _amp2(H, ctx, n, mom, prec):
    import torch
    m = torch.from_numpy(np.ascontiguousarray(mom, dtype=np.float64)).cuda()
    out = torch.empty(m.shape[0], dtype=torch.float64, device="cuda")
    H.heget_amp2(ctx, n, m.shape[0], m, out, precision=prec)
    H.heget_check(ctx)   # every transformed input still has p1, p2 massless along +z / -z
    return out.cpu().numpy()


def _variants(n, mom):
    swap = mom.copy()
    swap[:, [0, 1]] = swap[:, [1, 0]]
    swap = transform(swap, np.diag([1.0, 1.0, -1.0, -1.0]))   # rotation by pi about x, exact
    perm = np.random.default_rng(n).permutation(n)
    permuted = mom.copy()
    permuted[:, 2:] = mom[:, 2:][:, perm]
    return {
        "rotation about z": transform(mom, rotation_matrix([0, 0, 1], 0.7)),
        "boost along z": transform(mom, boost_matrix([0, 0, 0.6])),
        "boost along -z": transform(mom, boost_matrix([0, 0, -0.35])),
        "u <-> ubar": swap,
        "photon permutation": permuted,
    }


@pytest.mark.parametrize("n,N", [(3, 20000), (4, 20000), (6, 2000), (8, 64)])
def test_invariances(heget_lib, gpu, n, N):
    H = heget_lib
    mom = _points(H, gpu, n, N, SEED + n)
    assert mom.shape[0] > 0
    base = _amp2(H, gpu, n, mom, H.HEGET_FP64)
    tol0 = fp64_tolerance(mom)
    for name, v in _variants(n, mom).items():
        a64 = _amp2(H, gpu, n, v, H.HEGET_FP64)
        rel = np.abs(a64 - base) / base
        assert np.all(rel <= tol0 + fp64_tolerance(v)), (name, float(rel.max()))
        a32 = _amp2(H, gpu, n, v, H.HEGET_FP32)
        r32 = np.abs(a32 - base) / base
        assert np.median(r32) <= 1e-4 and r32.max() <= 1e-3, (name, float(np.median(r32)), float(r32.max()))


@pytest.mark.parametrize("n", [3, 6])
def test_scaling(heget_lib, gpu, n):
    """Doubling every momentum is exact in FP64, so |M|^2 scales by exactly
    2^(4-2n) up to the last rounding of the result."""
    H = heget_lib
    mom = _points(H, gpu, n, 3000 if n == 3 else 400, SEED + 20 + n)
    for prec in (H.HEGET_FP64, H.HEGET_FP32):
        base = _amp2(H, gpu, n, mom, prec)
        scaled = _amp2(H, gpu, n, 2.0 * mom, prec)
        np.testing.assert_allclose(scaled, base * 2.0 ** (4 - 2 * n), rtol=1e-14, atol=0)


def test_boosted_frame_against_the_oracle(oracle, heget_lib, gpu):
    """p1 and p2 of unequal energies: the device against the oracle on the
    same boosted momenta."""
    H = heget_lib
    n = 4
    mom = oracle.phase_space(n, SEED + 30, 0, 400, oracle.toy_pdf(), oracle.cuts())
    m = mom["momenta"][mom["mask"] == 1]
    b = transform(m, boost_matrix([0, 0, 0.8]))
    assert np.all(b[:, 0, 0] > 8.9 * b[:, 1, 0])   # E1 = 9 E2 after the boost
    ref = oracle.amp2(n, b)
    a64 = _amp2(H, gpu, n, b, H.HEGET_FP64)
    assert np.all(np.abs(a64 - ref) / ref <= fp64_tolerance(b))
    a32 = _amp2(H, gpu, n, b, H.HEGET_FP32)
    r32 = np.abs(a32 - ref) / ref
    assert np.median(r32) <= 1e-4 and r32.max() <= 1e-3
    assert math.isfinite(float(a64.sum()))
