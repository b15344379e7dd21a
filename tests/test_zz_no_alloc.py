"""heget_xsec_noalloc: the cross section for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc: applications whose device
memory belongs to a framework arena or a custom allocator, and
latency-critical paths that cannot take cudaMalloc's implicit
synchronisation.  heget_xsec_noalloc keeps its scratch (per-block partial
sums) in a static device array instead.  This file checks, through the C ABI,
that two calls in a row give the same result as heget_xsec_async (which uses
the context workspace): bit for bit, since both launch the same kernel with
the same shape and combine the block partials in the same fixed order.  It
also checks the largest accepted size of a tile-kernel case and the
refusals.  It is collected last so that a run stopping at the first failure
has run every other test first.
"""
import ctypes
import math

import pytest

pytestmark = pytest.mark.gpu

XSEC_TILE_N7 = 32          # default xsec tile at n = 7 (points per block of the tile kernel)
NOALLOC_MAX_BLOCKS = 4096  # the static scratch holds this many block partials


def _run_async(H, ctx, n, seed, N, sampler, precision):
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    H.heget_xsec_async(ctx, n, seed, 0, N, sampler, precision, res)
    torch.cuda.synchronize()
    return H.result_from_tensor(res)


def _run_noalloc(H, n, seed, N, sampler, precision):
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    H.heget_xsec_noalloc(0, n, seed, 0, N, sampler, precision, res)
    torch.cuda.synchronize()
    return H.result_from_tensor(res)


def _same(a, b):
    assert a.n_total == b.n_total and a.n_pass == b.n_pass and a.n_tries == b.n_tries
    for f in ("sigma_fb", "err_fb", "sum_w", "sum_w2"):
        assert getattr(a, f) == getattr(b, f), f
    assert math.isfinite(a.sigma_fb) and a.sigma_fb > 0


@pytest.mark.parametrize("n,N,precision", [(4, 100_003, 32), (3, 20_000, 64), (6, 60_001, 32),
                                           (7, NOALLOC_MAX_BLOCKS * XSEC_TILE_N7, 32)])
def test_noalloc_matches_xsec_async_twice(heget_lib, gpu, n, N, precision):
    H = heget_lib
    sampler = H.sampler_toy_pdf()
    # two calls in a row: the shared static scratch must not carry anything over
    for seed in (0x0908440300000101, 0x0908440300000202):
        ref = _run_async(H, gpu, n, seed, N, sampler, precision)
        got = _run_noalloc(H, n, seed, N, sampler, precision)
        _same(got, ref)


def test_noalloc_refuses_oversized_calls(heget_lib, gpu):
    import torch
    H = heget_lib
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    lib = H.load()
    s = H.sampler_toy_pdf()
    st = lib.heget_xsec_noalloc(0, 8, 1, 0, 1 << 20, ctypes.byref(s), None, 32, res.data_ptr(), None)
    assert st == H.HEGET_EINVAL
    assert b"no-allocation path" in lib.heget_last_error()
    # one point past the largest accepted size at n = 7
    st = lib.heget_xsec_noalloc(0, 7, 1, 0, NOALLOC_MAX_BLOCKS * XSEC_TILE_N7 + 1, ctypes.byref(s), None, 32,
                                res.data_ptr(), None)
    assert st == H.HEGET_EINVAL


def test_noalloc_refuses_what_set_params_refuses(heget_lib, gpu):
    import torch
    H = heget_lib
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    lib = H.load()
    s = H.sampler_toy_pdf()
    good = H.heget_params(1.0 / 137.035999, 2.0 / 3.0, 20.0, 2.5, 0.4)
    assert lib.heget_xsec_noalloc(0, 4, 1, 0, 1000, ctypes.byref(s), ctypes.byref(good), 32, res.data_ptr(),
                                  None) == H.HEGET_OK
    torch.cuda.synchronize()
    for bad in (H.heget_params(1.0 / 137.035999, float("nan"), 20.0, 2.5, 0.4),
                H.heget_params(1.0 / 137.035999, 0.0, 20.0, 2.5, 0.4),
                H.heget_params(float("inf"), 2.0 / 3.0, 20.0, 2.5, 0.4),
                H.heget_params(1.0 / 137.035999, 2.0 / 3.0, 20.0, float("inf"), 0.4),
                H.heget_params(1.0 / 137.035999, 2.0 / 3.0, 20.0, 2.5, float("nan"))):
        st = lib.heget_xsec_noalloc(0, 4, 1, 0, 1000, ctypes.byref(s), ctypes.byref(bad), 32, res.data_ptr(), None)
        assert st == H.HEGET_EINVAL
    # point indices past int64
    st = lib.heget_xsec_noalloc(0, 4, 1, (1 << 63) - 10, 1000, ctypes.byref(s), None, 32, res.data_ptr(), None)
    assert st == H.HEGET_EINVAL
