"""GPU tests of the run-time launch shapes (the autotuner's search space) and
of the CUDA graphs of the mixed-n launches.

Every tile-kernel shape of the FP32 prefix tree computes the same cross
section as the default (sums over orderings and helicities in another order:
FP32 rounding only); a tuned context gives the bits of a direct launch with
the same shape and tile, and so does a graph of the tuned step; batch and
server launches replayed from graphs give the bits of direct launches."""
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x090844030000A000


def _buf():
    import torch
    return torch.zeros(80, dtype=torch.uint8, device="cuda")


def _res(H, t):
    import torch
    torch.cuda.synchronize()
    return H.result_from_tensor(t)


def _async(H, ctx, n, seed, N, S, prec):
    r = _buf()
    H.heget_xsec_async(ctx, n, seed, 0, N, S, prec, r)
    return _res(H, r)


def _same(a, b):
    return (a.sum_w == b.sum_w and a.sum_w2 == b.sum_w2 and a.n_pass == b.n_pass and a.n_total == b.n_total
            and a.n_tries == b.n_tries and a.sigma_fb == b.sigma_fb and a.err_fb == b.err_fb)


@pytest.fixture
def reset_shapes(heget_lib, gpu):
    yield
    for n in range(2, 9):
        for p in (32, 64):
            heget_lib.heget_set_shape(gpu, n, p, 0)
            heget_lib.heget_set_tile(gpu, n, p, 1, 0)


@pytest.mark.parametrize("n,N", [(6, 20_000), (7, 3_000), (8, 400)])
def test_every_shape_gives_the_default_cross_section(heget_lib, gpu, reset_shapes, n, N):
    H = heget_lib
    S = H.sampler_toy_pdf()
    base = _async(H, gpu, n, SEED + n, N, S, 32)
    for shape in (1, 2, 3):
        threads, rows, groups = H.heget_shape_info(n, 32, shape)
        assert threads > 0 and rows in (1, 4) and groups >= 1
        H.heget_set_shape(gpu, n, 32, shape)
        assert H.heget_get_shape(gpu, n, 32) == shape
        got = _async(H, gpu, n, SEED + n, N, S, 32)
        assert got.n_pass == base.n_pass and got.n_total == base.n_total and got.n_tries == base.n_tries
        assert got.sum_w == pytest.approx(base.sum_w, rel=1e-5), shape
        assert got.sigma_fb == pytest.approx(base.sigma_fb, rel=1e-5), shape
    H.heget_set_shape(gpu, n, 32, 0)


def test_shape_arguments_are_checked(heget_lib, gpu):
    H = heget_lib
    lib = H.load()
    assert lib.heget_set_shape(gpu, 6, 32, 4) == H.HEGET_EINVAL
    assert lib.heget_set_shape(gpu, 4, 32, 1) == H.HEGET_EINVAL   # one shape below n = 6
    assert lib.heget_set_shape(gpu, 6, 64, 1) == H.HEGET_EINVAL   # FP64 keeps its default
    assert lib.heget_set_shape(gpu, 9, 32, 0) == H.HEGET_EINVAL
    assert lib.heget_get_shape(gpu, 6, 16) == -1
    assert H.heget_shape_info(6, 32, 0) == (0, 0, 0)


def test_tuned_context_and_its_graph_equal_direct_launches(heget_lib, gpu, reset_shapes, tmp_path):
    H = heget_lib
    S = H.sampler_toy_pdf()
    n, N = 6, 30_000
    shape, tile, ms = H.heget_autotune_shape(gpu, n, 32, 16_384)
    assert ms > 0 and 0 <= shape < 4
    assert H.heget_get_shape(gpu, n, 32) == shape
    tuned = _async(H, gpu, n, SEED + 1, N, S, 32)
    # the same launch set by hand on another context
    ctx2 = H.heget_create(0)
    try:
        H.heget_set_shape(ctx2, n, 32, shape)
        H.heget_set_tile(ctx2, n, 32, 1, tile)
        direct = _async(H, ctx2, n, SEED + 1, N, S, 32)
    finally:
        H.heget_destroy(ctx2)
    assert _same(tuned, direct)
    # a graph of the tuned step, replayed for the same seed
    r = _buf()
    g = H.heget_graph_xsec(gpu, n, N, S, 32, r)
    try:
        H.heget_graph_launch(g, SEED + 1, 0)
        assert _same(_res(H, r), tuned)
    finally:
        H.heget_graph_destroy(g)
    # saved and restored with the tile
    path = tmp_path / "tune.txt"
    H.heget_autotune_save(gpu, path)
    H.heget_set_shape(gpu, n, 32, 0)
    H.heget_set_tile(gpu, n, 32, 1, 0)
    H.heget_autotune_load(gpu, path)
    assert H.heget_get_shape(gpu, n, 32) == shape


MIX = [(2, 7001, 32), (5, 513, 32), (3, 3000, 64), (4, 4097, 32), (6, 77, 32), (2, 1, 64), (7, 9, 32),
       (8, 3, 32)]


def _batch(H, ctx, k0):
    import torch
    S = H.sampler_toy_pdf()
    reqs = [dict(n=n, precision=p, seed=SEED + k0 + k, i0=11 * k, N=N, sampler=S, result_dev=_buf())
            for k, (n, N, p) in enumerate(MIX)]
    H.heget_xsec_batch(ctx, reqs)
    torch.cuda.synchronize()
    return [H.result_from_tensor(r["result_dev"]) for r in reqs]


def test_batch_graphs_replay_the_direct_bits(heget_lib, gpu):
    H = heget_lib
    direct = [_batch(H, gpu, 0), _batch(H, gpu, 100)]
    H.heget_set_graphs(gpu, 1)
    try:
        first = _batch(H, gpu, 0)     # captures one graph per precision
        second = _batch(H, gpu, 100)  # same buckets, new request contents: replays
        on, captures, replays = H.heget_get_graphs(gpu)
        assert on == 1 and captures >= 2 and replays >= 2
    finally:
        H.heget_set_graphs(gpu, 0)
    for a, b in zip(direct[0], first):
        assert _same(a, b)
    for a, b in zip(direct[1], second):
        assert _same(a, b)


def test_server_graphs_replay_the_direct_bits(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    reqs = [(4, 40_000, 32), (6, 500, 32), (3, 9_000, 64)] * 3

    def serve():
        srv = H.heget_server_start(gpu, max_launch_work=5e9)
        try:
            t = [H.heget_submit(srv, n, SEED + 7, N, S, p) for (n, N, p) in reqs]
            return [H.heget_wait(srv, x, 120.0) for x in t]
        finally:
            H.heget_server_stop(srv)

    direct = serve()
    H.heget_set_graphs(gpu, 1)
    try:
        graphed = serve()
    finally:
        H.heget_set_graphs(gpu, 0)
    for a, b in zip(direct, graphed):
        assert a.status == H.HEGET_OK and b.status == H.HEGET_OK
        assert _same(a.result, b.result)
