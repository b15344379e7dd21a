"""GPU tests of the launch machinery: mixed-n batches, CUDA-graph replay,
autotuned launch shapes.  Results must not depend on how work is launched."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0908440300005000


def _res(H, t):
    import torch
    torch.cuda.synchronize()
    return H.result_from_tensor(t)


def _buf():
    import torch
    return torch.zeros(80, dtype=torch.uint8, device="cuda")


def _async(H, ctx, n, seed, N, S, prec, i0=0):
    r = _buf()
    H.heget_xsec_async(ctx, n, seed, i0, N, S, prec, r)
    return _res(H, r)


def _same(a, b):
    return (a.sum_w == b.sum_w and a.sum_w2 == b.sum_w2 and a.n_pass == b.n_pass and a.n_total == b.n_total
            and a.n_tries == b.n_tries and a.sigma_fb == b.sigma_fb and a.err_fb == b.err_fb)


MIX = [(2, 7001, 32), (5, 513, 32), (3, 3000, 64), (4, 4097, 32), (6, 77, 32), (2, 1, 64), (4, 0, 32),
       (7, 9, 32), (3, 1500, 32), (8, 3, 32)]


def test_batch_alone_equals_in_mix_and_matches_single_runs(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    reqs = []
    for k, (n, N, prec) in enumerate(MIX):
        reqs.append(dict(n=n, precision=prec, seed=SEED + k, i0=11 * k, N=N, sampler=S, result_dev=_buf()))
    H.heget_xsec_batch(gpu, reqs)
    mixed = [_res(H, r["result_dev"]) for r in reqs]
    for k, r in enumerate(reqs):
        alone = dict(r, result_dev=_buf())
        H.heget_xsec_batch(gpu, [alone])
        assert _same(_res(H, alone["result_dev"]), mixed[k]), f"request {k} differs alone vs in the mix"
        ref = _async(H, gpu, r["n"], r["seed"], r["N"], S, r["precision"], i0=r["i0"])
        got = mixed[k]
        assert got.n_total == ref.n_total == r["N"]
        assert got.n_pass == ref.n_pass and got.n_tries == ref.n_tries
        if r["N"]:
            # FP64: the same arithmetic in another tile order; FP32: heget_xsec_async runs the
            # warp-specialised kernel (n <= 5) or a tile kernel of another block size (n = 6, 7), whose
            # sums over orderings run in another order: per-point FP32 rounding differences (~1e-6)
            rel = 1e-12 if r["precision"] == 64 else 1e-5
            assert got.sum_w == pytest.approx(ref.sum_w, rel=rel, abs=0)
            assert got.sigma_fb == pytest.approx(ref.sigma_fb, rel=rel, abs=0)


def test_batch_weights_match_oracle(oracle, heget_lib, gpu):
    import torch
    H = heget_lib
    reqs = []
    for k, (n, N) in enumerate([(3, 300), (2, 1000), (4, 120)]):
        reqs.append(dict(n=n, precision=64, seed=SEED + 50 + k, i0=5, N=N, sampler=H.sampler_toy_pdf(),
                         result_dev=_buf(), w_out=torch.empty(N, dtype=torch.float64, device="cuda")))
    H.heget_xsec_batch(gpu, reqs)
    torch.cuda.synchronize()
    for r in reqs:
        wo, mask, tries = oracle.event_weights(r["n"], r["seed"], r["i0"], r["N"], oracle.toy_pdf(),
                                               oracle.cuts())
        w = r["w_out"].cpu().numpy()
        nz = wo != 0
        np.testing.assert_array_equal(w != 0, nz)
        assert np.max(np.abs(w[nz] - wo[nz]) / wo[nz]) < 1e-11


def test_batch_rejects_bad_requests(heget_lib, gpu):
    H = heget_lib
    bad = dict(n=9, precision=32, seed=1, N=10, sampler=H.sampler_toy_pdf(), result_dev=_buf())
    with pytest.raises(H.HegetError):
        H.heget_xsec_batch(gpu, [bad])
    with pytest.raises(H.HegetError):
        H.heget_xsec_batch(gpu, [dict(bad, n=3, result_dev=None)])


@pytest.mark.parametrize("n,prec", [(4, 32), (6, 32), (3, 64)])
def test_graph_replay_matches_direct_launch(heget_lib, gpu, n, prec):
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    N = {4: 50_000, 6: 3_000, 3: 20_000}[n]
    res = _buf()
    g = H.heget_graph_xsec(gpu, n, N, S, prec, res)
    try:
        stream = torch.cuda.Stream()
        for seed, i0 in [(SEED + 1, 0), (SEED + 2, 1000), (SEED + 1, 0)]:
            H.heget_graph_launch(g, seed, i0, stream=stream)
            stream.synchronize()
            got = H.result_from_tensor(res)
            ref = _async(H, gpu, n, seed, N, S, prec, i0=i0)
            assert _same(got, ref)
    finally:
        H.heget_graph_destroy(g)


def test_autotune_picks_a_shape_that_agrees(heget_lib, gpu, tmp_path):
    H = heget_lib
    S = H.sampler_toy_pdf()
    base = _async(H, gpu, 3, SEED + 9, 30_000, S, 32)
    tile, ms = H.heget_autotune(gpu, 3, 32, 1, 30_000)
    assert ms > 0 and (tile == 0 or tile % 32 == 0)
    assert H.heget_get_tile(gpu, 3, 32, 1) == (tile if tile else 128)
    tuned = _async(H, gpu, 3, SEED + 9, 30_000, S, 32)
    assert tuned.n_pass == base.n_pass
    assert tuned.sum_w == pytest.approx(base.sum_w, rel=1e-12)
    t2, _ = H.heget_autotune(gpu, 5, 32, 0, 4_000)
    path = tmp_path / "tune.txt"
    H.heget_autotune_save(gpu, path)
    H.heget_set_tile(gpu, 3, 32, 1, 0)
    H.heget_set_tile(gpu, 5, 32, 0, 0)
    H.heget_autotune_load(gpu, path)
    if tile:
        assert H.heget_get_tile(gpu, 3, 32, 1) == tile
    if t2:
        assert H.heget_get_tile(gpu, 5, 32, 0) == t2
    H.heget_set_tile(gpu, 3, 32, 1, 0)
    H.heget_set_tile(gpu, 5, 32, 0, 0)


def test_failed_call_leaves_no_stale_cuda_error(heget_lib, gpu):
    """A launch shape whose shared memory exceeds the device limit fails on the
    host with HEGET_ECUDA before any launch; the runtime error it reports does
    not linger for the caller's next CUDA call."""
    import torch
    H = heget_lib
    H.heget_set_tile(gpu, 8, 64, 1, 4096)
    try:
        with pytest.raises(H.HegetError) as e:
            H.heget_xsec_async(gpu, 8, SEED, 0, 5000, H.sampler_toy_pdf(), 64, _buf())
        assert e.value.status == H.HEGET_ECUDA
        x = torch.ones(1000, device="cuda").sum()   # would raise on a leftover error
        assert float(x) == 1000.0
    finally:
        H.heget_set_tile(gpu, 8, 64, 1, 0)


def test_point_ranges_and_params_are_checked_on_the_host(heget_lib, gpu):
    """Point indices i0 .. i0+N-1 must fit in int64, and the physics
    parameters must be finite: every entry point refuses the call before it
    launches anything, and the context keeps its parameters."""
    H = heget_lib
    S = H.sampler_toy_pdf()
    top = 2 ** 63 - 10

    def refused(call, what="overflow"):
        with pytest.raises(H.HegetError) as e:
            call()
        assert e.value.status == H.HEGET_EINVAL and what in str(e.value)

    refused(lambda: H.heget_phase_space_ex(gpu, 1, top, 100, 4, S))
    refused(lambda: H.heget_xsec_launch(gpu, 4, 1, top, 100, S, H.HEGET_FP32))
    refused(lambda: H.heget_hist(gpu, 4, 1, top, 100, S, None, [(0, 10, 0.0, 100.0)], None))
    refused(lambda: H.heget_xsec_batch(gpu, [dict(n=4, precision=32, seed=1, i0=top, N=100, sampler=S,
                                                  result_dev=_buf())]))
    refused(lambda: H.heget_phase_space_ex(gpu, 1, -1, 100, 4, S), "< 0")
    refused(lambda: H.heget_xsec_batch(gpu, [dict(n=8, precision=32, seed=1, N=2 ** 40, sampler=S,
                                                  result_dev=_buf())]), "split")
    res = _buf()
    g = H.heget_graph_xsec(gpu, 4, 1000, S, H.HEGET_FP32, res)
    try:
        refused(lambda: H.heget_graph_launch(g, 1, top))
        H.heget_graph_launch(g, 1, top - 10_000)        # indices near the top of the range still run
        assert _res(H, res).n_total == 1000
    finally:
        H.heget_graph_destroy(g)
    srv = H.heget_server_start(gpu)
    try:
        refused(lambda: H.heget_submit(srv, 4, 1, 100, S, i0=top))
        with pytest.raises(H.HegetError) as e:
            H.heget_submit(srv, 8, 1, 2 ** 40, S)           # more tile partials than the arena holds
        assert e.value.status == H.HEGET_ENOMEM
    finally:
        H.heget_server_stop(srv)

    before = H.heget_get_params(gpu)
    for bad in (dict(dr_min=float("nan")), dict(eta_max=float("inf")), dict(pt_min=float("inf")),
                dict(alpha=float("inf")), dict(q_charge=0.0)):
        with pytest.raises(H.HegetError) as e:
            H.heget_set_params(gpu, **bad)
        assert e.value.status == H.HEGET_EINVAL
    after = H.heget_get_params(gpu)
    assert [getattr(after, f) for f, _ in after._fields_] == [getattr(before, f) for f, _ in before._fields_]


@pytest.mark.parametrize("n,N,prec", [(4, 70_001, 32), (6, 3_001, 32), (3, 9_999, 64)])
def test_launch_and_finalize_pair_equals_the_async_call(heget_lib, gpu, n, N, prec):
    """heget_xsec_launch + heget_xsec_finalize (the bench's step) give the
    same result as heget_xsec_async; finalising again rereads the same
    partials; a NULL result buffer is refused."""
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    ref = _async(H, gpu, n, SEED + 700 + n, N, S, prec, i0=123)
    H.heget_xsec_launch(gpu, n, SEED + 700 + n, 123, N, S, prec)
    r1, r2 = _buf(), _buf()
    H.heget_xsec_finalize(gpu, r1)
    H.heget_xsec_finalize(gpu, r2)
    a, b = _res(H, r1), _res(H, r2)
    assert _same(a, ref) and _same(b, ref) and a.n_total == N
    with pytest.raises(H.HegetError) as e:
        H.heget_xsec_finalize(gpu, None)
    assert e.value.status == H.HEGET_EINVAL
    torch.cuda.synchronize()


def test_fma_peak_probe(heget_lib, gpu):
    """The FFMA/DFMA throughput probe reports rates of the right size for a
    GB300 (FP32 tens of TFLOP/s, FP64 about 1/64 of it) and refuses bad
    arguments."""
    H = heget_lib
    f32 = H.heget_measure_fma_peak(gpu, H.HEGET_FP32)
    f64 = H.heget_measure_fma_peak(gpu, H.HEGET_FP64)
    assert 20 < f32 < 200 and 0.2 < f64 < 5 and 20 < f32 / f64 < 200
    with pytest.raises(H.HegetError) as e:
        H.heget_measure_fma_peak(gpu, 16)
    assert e.value.status == H.HEGET_EINVAL
