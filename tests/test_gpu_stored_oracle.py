"""GPU parity at n = 7 and n = 8 against stored oracle samples.

The FP64 oracle takes about a minute of one core per point at n = 8, so the
expected values of these tests were written once by
tests/golden/gen_oracle_samples.py, which calls only oracle/ (phase-space
points regenerated from the seed, |M|^2 summed over all 2^(n+2) helicities,
event weights of Sec. 2.1 eq. (2)).  Here the device evaluates the same
points through the C ABI:
  * |M|^2 of 32 cut-passing points per n, with the prefix tree and the subset
    recursion, in FP64 (per-point tolerance of helpers.fp64_tolerance) and
    FP32 (median <= 1e-4, max <= 1e-3 relative);
  * the fused cross-section path's event weights of points 0..255 (about 70
    pass the cuts), both algorithms, FP32 (max <= 1e-3) and FP64 (<= 1e-11),
    with the cut masks bit for bit.
"""
import os

import numpy as np
import pytest

from helpers import fp64_tolerance

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SEED = 0x0908440300000002
SAMPLERS = {8: ("uniform", 200.0, 2000.0), 7: ("toy",)}


def _read(path):
    head, rows = [], []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                head.append(line)
            elif line.strip():
                rows.append([float(x) for x in line.split()])
    return head, np.array(rows)


def _samplers(H, O, n):
    s = SAMPLERS[n]
    if s[0] == "uniform":
        return H.sampler_uniform(s[1], s[2]), O.uniform(s[1], s[2])
    return H.sampler_toy_pdf(), O.toy_pdf()


def _amp2(H, ctx, n, mom, precision):
    import torch
    N = mom.shape[0]
    m = torch.from_numpy(np.ascontiguousarray(mom)).cuda()
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_amp2(ctx, n, N, m, out, precision=precision)
    H.heget_check(ctx)
    return out.cpu().numpy()


@pytest.fixture(params=[0, 1], ids=["tree", "subset"])
def alg(request, heget_lib, gpu):
    heget_lib.heget_set_algorithm(gpu, request.param)
    yield request.param
    heget_lib.heget_set_algorithm(gpu, heget_lib.HEGET_ALG_TREE)


@pytest.mark.parametrize("n", [7, 8])
def test_amp2_against_stored_oracle(oracle, heget_lib, gpu, alg, n):
    H = heget_lib
    head, rows = _read(os.path.join(GOLDEN, f"oracle_amp2_n{n}.txt"))
    assert f"seed {SEED:#x}" in head[1]
    idx = rows[:, 0].astype(int)
    ref = rows[:, 1]
    assert len(idx) >= 32
    _, so = _samplers(H, oracle, n)
    mom = oracle.phase_space(n, SEED, 0, int(idx.max()) + 1, so, oracle.cuts())["momenta"][idx]
    got64 = _amp2(H, gpu, n, mom, H.HEGET_FP64)
    got32 = _amp2(H, gpu, n, mom, H.HEGET_FP32)
    assert np.all(np.abs(got64 - ref) / ref < fp64_tolerance(mom))
    r = np.abs(got32 - ref) / ref
    assert np.median(r) <= 1e-4 and np.max(r) <= 1e-3


@pytest.mark.parametrize("n", [7, 8])
def test_event_weights_against_stored_oracle(oracle, heget_lib, gpu, alg, n):
    import torch
    H = heget_lib
    head, rows = _read(os.path.join(GOLDEN, f"oracle_weights_n{n}.txt"))
    assert f"seed {SEED:#x}" in head[1]
    N = rows.shape[0]
    mask, w_or = rows[:, 1].astype(bool), rows[:, 3]
    assert np.count_nonzero(mask) >= 64
    sd, _ = _samplers(H, oracle, n)
    for prec, tol in ((H.HEGET_FP32, 1e-3), (H.HEGET_FP64, 1e-11)):
        res = torch.zeros(80, dtype=torch.uint8, device="cuda")
        w = torch.empty(N, dtype=torch.float64, device="cuda")
        H.heget_xsec_async(gpu, n, SEED, 0, N, sd, prec, res, w)
        torch.cuda.synchronize()
        got = w.cpu().numpy()
        np.testing.assert_array_equal(got != 0, mask)
        assert H.result_from_tensor(res).n_pass == int(mask.sum())
        r = np.abs(got[mask] - w_or[mask]) / w_or[mask]
        assert np.max(r) < tol, (prec, float(np.max(r)))
        if prec == H.HEGET_FP32:
            assert np.median(r) <= 1e-4
