"""heget_xsec_noalloc: the cross section for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc: code running while a
stream is captured into a CUDA graph, applications whose device memory
belongs to a framework arena, latency-critical paths.  heget_xsec_noalloc
keeps its scratch (per-block partial sums) in a static device array instead.
This file checks, through the C ABI, that two calls in a row give the same
result as heget_xsec_async (which uses the context workspace), and that
sizes beyond the static array are refused.  It is collected last so that a
run stopping at the first failure has run every other test first.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


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


def _close(a, b):
    # the tolerance of the xsec parity tests: 1e-11 relative on sigma and sums
    assert a.n_total == b.n_total and a.n_pass == b.n_pass and a.n_tries == b.n_tries
    for f in ("sigma_fb", "sum_w", "sum_w2"):
        x, y = getattr(a, f), getattr(b, f)
        assert x == pytest.approx(y, rel=1e-11, abs=0.0), f
    assert a.err_fb == pytest.approx(b.err_fb, rel=1e-9)


@pytest.mark.parametrize("n,N,precision", [(4, 100_003, 32), (3, 20_000, 64)])
def test_noalloc_matches_xsec_async_twice(heget_lib, gpu, n, N, precision):
    H = heget_lib
    sampler = H.sampler_toy_pdf()
    # two calls in a row: the shared static scratch must not carry anything over
    for seed in (0x0908440300000101, 0x0908440300000202):
        ref = _run_async(H, gpu, n, seed, N, sampler, precision)
        got = _run_noalloc(H, n, seed, N, sampler, precision)
        _close(got, ref)


def test_noalloc_refuses_oversized_calls(heget_lib, gpu):
    import torch
    H = heget_lib
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    lib = H.load()
    s = H.sampler_toy_pdf()
    st = lib.heget_xsec_noalloc(0, 8, 1, 0, 1 << 20, ctypes.byref(s), None, 32, res.data_ptr(), None)
    assert st == H.HEGET_EINVAL
    assert b"no-allocation path" in lib.heget_last_error()
