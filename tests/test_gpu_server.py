"""GPU tests of the request server: every result is bitwise the batch result
of the same request alone, whatever shared its launches; admission, bounded
waits and error statuses behave as declared."""
import threading
import time

import pytest

pytestmark = pytest.mark.gpu

SEED = 0x0908440300007000


def _buf():
    import torch
    return torch.zeros(80, dtype=torch.uint8, device="cuda")


def _alone(H, ctx, n, prec, seed, i0, N, S):
    import torch
    r = _buf()
    H.heget_xsec_batch(ctx, [dict(n=n, precision=prec, seed=seed, i0=i0, N=N, sampler=S, result_dev=r)])
    torch.cuda.synchronize()
    return H.result_from_tensor(r)


def _same(a, b):
    return (a.sum_w == b.sum_w and a.sum_w2 == b.sum_w2 and a.n_pass == b.n_pass and a.n_total == b.n_total
            and a.n_tries == b.n_tries and a.sigma_fb == b.sigma_fb and a.err_fb == b.err_fb)


MIX = [(2, 7001, 32), (5, 513, 32), (3, 3000, 64), (4, 40_097, 32), (6, 77, 32), (2, 1, 64), (4, 1, 32),
       (7, 9, 32), (3, 1500, 32), (8, 3, 32), (4, 300_000, 32), (5, 2000, 64)]


def test_server_results_equal_batch_alone(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    srv = H.heget_server_start(gpu, max_launch_work=5e9)   # small launches: requests share several
    try:
        tickets = [H.heget_submit(srv, n, SEED + k, N, S, prec, i0=7 * k) for k, (n, N, prec) in enumerate(MIX)]
        got = [H.heget_wait(srv, t, 120.0) for t in tickets]
    finally:
        H.heget_server_stop(srv)
    for k, ((n, N, prec), g) in enumerate(zip(MIX, got)):
        assert g.status == H.HEGET_OK
        assert g.t_submit <= g.t_admit <= g.t_done
        ref = _alone(H, gpu, n, prec, SEED + k, 7 * k, N, S)
        assert _same(g.result, ref), f"request {k} (n={n}, N={N}) differs from the batch alone"


def test_server_concurrent_submitters(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    srv = H.heget_server_start(gpu, max_launch_work=2e10)
    out, errors = {}, []

    def client(c):
        try:
            for j in range(6):
                n = 2 + (c + j) % 5
                N = 500 + 977 * ((c * 7 + j) % 11)
                t = H.heget_submit(srv, n, SEED + 100 * c + j, N, S, H.HEGET_FP32)
                out[(c, j)] = (n, N, H.heget_wait(srv, t, 120.0))
        except Exception as e:   # noqa: BLE001 -- reported below
            errors.append(e)

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    try:
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=300)
    finally:
        H.heget_server_stop(srv)
    assert not errors, errors
    assert len(out) == 24
    for (c, j), (n, N, g) in out.items():
        assert g.status == H.HEGET_OK
        assert _same(g.result, _alone(H, gpu, n, H.HEGET_FP32, SEED + 100 * c + j, 0, N, S))


def test_server_admits_in_order_under_an_inflight_limit(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    srv = H.heget_server_start(gpu, max_inflight=1)
    try:
        reqs = [(4, 20_000), (3, 5_000), (5, 1_000), (2, 30_000)]
        tickets = [H.heget_submit(srv, n, SEED + 300 + k, N, S) for k, (n, N) in enumerate(reqs)]
        got = [H.heget_wait(srv, t, 120.0) for t in tickets]
    finally:
        H.heget_server_stop(srv)
    for a, b in zip(got, got[1:]):
        assert b.t_admit >= a.t_done          # one request in flight at a time, FIFO
    for k, ((n, N), g) in enumerate(zip(reqs, got)):
        assert _same(g.result, _alone(H, gpu, n, H.HEGET_FP32, SEED + 300 + k, 0, N, S))


def test_server_small_arena_queues_until_space(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    # each request below needs a few KiB of partials; 16 KiB holds only some at once
    srv = H.heget_server_start(gpu, arena_bytes=16 << 10)
    try:
        tickets = [H.heget_submit(srv, 4, SEED + 400 + k, 20_000 + 1000 * k, S) for k in range(8)]
        got = [H.heget_wait(srv, t, 120.0) for t in tickets]
        with pytest.raises(H.HegetError) as e:
            H.heget_submit(srv, 4, 1, 10_000_000, S)   # could never fit
        assert e.value.status == H.HEGET_ENOMEM
    finally:
        H.heget_server_stop(srv)
    for k, g in enumerate(got):
        assert _same(g.result, _alone(H, gpu, 4, H.HEGET_FP32, SEED + 400 + k, 0, 20_000 + 1000 * k, S))


def test_server_wait_timeout_poll_and_errors(heget_lib, gpu):
    H = heget_lib
    S = H.sampler_toy_pdf()
    srv = H.heget_server_start(gpu)
    try:
        t = H.heget_submit(srv, 8, SEED + 500, 6_000, S, H.HEGET_FP32)   # ~0.1 s of work
        for bad in (-1.0, float("nan")):
            with pytest.raises(H.HegetError) as e:
                H.heget_wait(srv, t, bad)
            assert e.value.status == H.HEGET_EINVAL
        with pytest.raises(H.HegetError) as e:
            H.heget_wait(srv, t, 1e-4)
        assert e.value.status == H.HEGET_ETIMEOUT
        g = H.heget_wait(srv, t, 120.0)                    # the ticket stays valid after a timeout
        assert g.status == H.HEGET_OK and g.result.n_total == 6_000
        with pytest.raises(H.HegetError) as e:
            H.heget_poll(srv, t)                           # released once claimed
        assert e.value.status == H.HEGET_ENOTFOUND
        with pytest.raises(H.HegetError) as e:
            H.heget_wait(srv, 987_654_321, 0.01)
        assert e.value.status == H.HEGET_ENOTFOUND
        for bad in [dict(n=9, N=10), dict(n=1, N=10), dict(n=4, N=0), dict(n=4, N=-5)]:
            with pytest.raises(H.HegetError) as e:
                H.heget_submit(srv, bad["n"], 1, bad["N"], S)
            assert e.value.status == H.HEGET_EINVAL
        with pytest.raises(H.HegetError):
            H.heget_submit(srv, 4, 1, 10, S, precision=16)
        t2 = H.heget_submit(srv, 2, SEED + 501, 100, S)
        g2, t_end = None, time.monotonic() + 60
        while g2 is None and time.monotonic() < t_end:
            g2 = H.heget_poll(srv, t2)
        assert g2 is not None and g2.status == H.HEGET_OK
        t3 = H.heget_submit(srv, 2, SEED + 502, 100, S)
        assert H.heget_wait(srv, t3, 1e300).status == H.HEGET_OK   # an unbounded wait is capped, not overflowed
    finally:
        H.heget_server_stop(srv)
