"""Parity at the benchmark's full sizes, in the launch configuration the
bench times (the default fused path of heget_xsec_async: with the tree the
warp-specialised kernel at n <= 5 and the tile kernel above, with the subset
recursion the warp-specialised kernel in FP32 and the tile kernel in FP64):
per-event weights of sampled points (blocks at the start, the middle and the
ragged end of the range) against the oracle, computed one by one; cut
decisions bit for bit; and the result's counts and sums against the full
weight array, for both ordering-sum algorithms."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x090844030000D000
# (n, sampler, points, sampled block length, FP64 checked too)
FULL = [(2, "fixed", 65536, 64, True), (4, "toy", 1 << 20, 64, True), (6, "toy", 1 << 20, 24, True),
        (8, "uniform", 65536, 8, True)]


def _samplers(H, O, kind):
    if kind == "fixed":
        return H.sampler_fixed(500.0), O.fixed(500.0), O.cuts(20.0, 2.5, -1.0)
    if kind == "uniform":
        return H.sampler_uniform(200.0, 2000.0), O.uniform(200.0, 2000.0), O.cuts()
    return H.sampler_toy_pdf(), O.toy_pdf(), O.cuts()


@pytest.mark.parametrize("n,kind,N,B,fp64", FULL)
def test_full_size_sampled_parity(oracle, heget_lib, gpu, n, kind, N, B, fp64):
    import torch
    H = heget_lib
    sd, so, cut = _samplers(H, oracle, kind)
    if kind == "fixed":
        H.heget_set_params(gpu, dr_min=-1.0)
    try:
        seed = SEED + n
        starts = [N - B] if n == 8 else [0, N // 2 + 7, N - B]
        ref = {s: oracle.event_weights(n, seed, s, B, so, cut) for s in starts}
        for alg, prec, tol in ((H.HEGET_ALG_TREE, H.HEGET_FP32, 1e-3), (H.HEGET_ALG_TREE, H.HEGET_FP64, 1e-11),
                               (H.HEGET_ALG_SUBSET, H.HEGET_FP32, 1e-3), (H.HEGET_ALG_SUBSET, H.HEGET_FP64, 1e-11)):
            if prec == H.HEGET_FP64 and not fp64:
                continue
            H.heget_set_algorithm(gpu, alg)
            res = torch.zeros(80, dtype=torch.uint8, device="cuda")
            w = torch.empty(N, dtype=torch.float64, device="cuda")
            H.heget_xsec_async(gpu, n, seed, 0, N, sd, prec, res, w)
            torch.cuda.synchronize()
            r = H.result_from_tensor(res)
            wh = w.cpu().numpy()
            assert r.n_total == N and r.n_pass == int(np.count_nonzero(wh))
            assert r.sum_w == pytest.approx(math.fsum(wh), rel=1e-13)
            for s, (wo, mask, _) in ref.items():
                got = wh[s:s + B]
                np.testing.assert_array_equal(got != 0, mask.astype(bool))
                nz = wo != 0
                if nz.any():
                    assert np.max(np.abs(got[nz] - wo[nz]) / wo[nz]) < tol
    finally:
        H.heget_set_algorithm(gpu, H.HEGET_ALG_TREE)
        H.heget_set_params(gpu)
