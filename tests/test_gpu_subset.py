"""GPU parity of the subset recursion (HEGET_ALG_SUBSET): the same ordering
sum as the prefix tree, regrouped by photon set.  Checked against the FP64
oracle exactly like the tree (per-point FP64 tolerance, FP32 median/max),
against the MHV closed form and helicity masks, and through every path that
runs amplitudes (amp2, fused xsec incl. the warp-specialised n <= 4 kernel,
batch, graph replay)."""
import math

import numpy as np
import pytest

from helpers import fp64_tolerance, helicity_index, mask_words, mdot

pytestmark = pytest.mark.gpu

SEED = 0x0908440300009000
N_BY_N = {2: 5003, 3: 1001, 4: 301, 5: 77, 6: 21, 7: 6, 8: 2}


@pytest.fixture
def subset(heget_lib, gpu):
    heget_lib.heget_set_algorithm(gpu, heget_lib.HEGET_ALG_SUBSET)
    assert heget_lib.heget_get_algorithm(gpu) == heget_lib.HEGET_ALG_SUBSET
    yield gpu
    heget_lib.heget_set_algorithm(gpu, heget_lib.HEGET_ALG_TREE)


def _amp2(H, ctx, n, mom, precision, mask=None):
    import torch
    N = mom.shape[0]
    m = torch.from_numpy(np.ascontiguousarray(mom)).cuda()
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    mk = torch.from_numpy(mask.astype(np.uint32).view(np.int32)).cuda() if mask is not None else None
    H.heget_amp2(ctx, n, N, m, out, hel_mask=mk, precision=precision)
    H.heget_check(ctx)
    return out.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_subset_amp2_matches_oracle(oracle, heget_lib, subset, n):
    H = heget_lib
    mom = oracle.phase_space(n, SEED + n, 0, N_BY_N[n], oracle.toy_pdf())["momenta"]
    ref = oracle.amp2(n, mom)
    got64 = _amp2(H, subset, n, mom, H.HEGET_FP64)
    got32 = _amp2(H, subset, n, mom, H.HEGET_FP32)
    assert np.all(_rel(got64, ref) < fp64_tolerance(mom))
    r = _rel(got32, ref)
    assert np.median(r) <= 1e-4 and np.max(r) <= 1e-3


@pytest.mark.parametrize("n", [5, 6, 8])
def test_subset_agrees_with_tree(heget_lib, gpu, n):
    """Both algorithms on the same device momenta, FP64: equal to rounding."""
    import torch
    H = heget_lib
    N = {5: 2000, 6: 300, 8: 8}[n]
    mom = torch.empty((N, n + 2, 4), dtype=torch.float64, device="cuda")
    H.heget_phase_space_ex(gpu, SEED + 20 + n, 0, N, n, H.sampler_uniform(200.0, 2000.0), momenta=mom)
    out = {}
    for alg in (H.HEGET_ALG_TREE, H.HEGET_ALG_SUBSET):
        H.heget_set_algorithm(gpu, alg)
        a = torch.empty(N, dtype=torch.float64, device="cuda")
        H.heget_amp2(gpu, n, N, mom, a, precision=H.HEGET_FP64)
        out[alg] = a.cpu().numpy()
    H.heget_set_algorithm(gpu, H.HEGET_ALG_TREE)
    assert np.all(_rel(out[H.HEGET_ALG_SUBSET], out[H.HEGET_ALG_TREE]) < fp64_tolerance(mom.cpu().numpy()))


@pytest.mark.parametrize("n", [4, 6])
def test_subset_mhv_and_masks(oracle, heget_lib, subset, n):
    H = heget_lib
    e2, Q = 4 * math.pi / 137.035999, 2 / 3
    mom = oracle.phase_space(n, SEED + 40 + n, 0, 16, oracle.toy_pdf())["momenta"]
    hs = []
    for j in range(n):
        lam = [-1] * n
        lam[j] = 1
        hs.append(helicity_index(1, -1, lam))
    got = _amp2(H, subset, n, mom, H.HEGET_FP64, mask_words(n, hs))
    p1, p2, ks = mom[:, 0], mom[:, 1], mom[:, 2:]
    s = mdot(p1 + p2, p1 + p2)
    s1, s2 = 2 * mdot(p1[:, None], ks), 2 * mdot(p2[:, None], ks)
    ref = (2 * e2 * Q * Q) ** n * s ** (n - 2) / np.prod(s1 * s2, axis=1) * np.sum(s2 ** 3 * s1, axis=1)
    assert np.all(_rel(got, ref) < fp64_tolerance(mom))
    rng = np.random.default_rng(n)
    hs = rng.choice(1 << (n + 2), size=9, replace=False)
    mask = mask_words(n, hs)
    ref = oracle.amp2(n, mom, hel_mask=mask)
    got = _amp2(H, subset, n, mom, H.HEGET_FP64, mask)
    assert np.all(np.abs(got - ref) / oracle.amp2(n, mom) < fp64_tolerance(mom))


@pytest.mark.parametrize("n,N", [(2, 2003), (3, 1001), (4, 1030), (5, 130), (6, 40)])
def test_subset_xsec_weights_match_oracle(oracle, heget_lib, subset, n, N):
    import torch
    H = heget_lib
    seed, i0 = SEED + 60 + n, 321
    wo, mask, tries = oracle.event_weights(n, seed, i0, N, oracle.toy_pdf(), oracle.cuts())
    nz = wo != 0
    for prec, tol in ((H.HEGET_FP64, 1e-11), (H.HEGET_FP32, 1e-3)):
        res = torch.zeros(80, dtype=torch.uint8, device="cuda")
        w = torch.empty(N, dtype=torch.float64, device="cuda")
        H.heget_xsec_async(subset, n, seed, i0, N, H.sampler_toy_pdf(), prec, res, w)
        torch.cuda.synchronize()
        w = w.cpu().numpy()
        np.testing.assert_array_equal(w != 0, nz)
        assert np.max(_rel(w[nz], wo[nz])) < tol
        r = H.result_from_tensor(res)
        assert r.n_pass == int(mask.sum()) and r.n_tries == int(tries.sum())


def test_subset_batch_and_graph(heget_lib, subset):
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    reqs = [dict(n=n, precision=p, seed=SEED + 80 + n, i0=0, N=N, sampler=S,
                 result_dev=torch.zeros(80, dtype=torch.uint8, device="cuda"))
            for n, N, p in [(3, 3000, 32), (6, 100, 32), (7, 9, 64), (5, 400, 64)]]
    H.heget_xsec_batch(subset, reqs)
    torch.cuda.synchronize()
    mixed = [H.result_from_tensor(r["result_dev"]) for r in reqs]
    for r, m in zip(reqs, mixed):
        alone = dict(r, result_dev=torch.zeros(80, dtype=torch.uint8, device="cuda"))
        H.heget_xsec_batch(subset, [alone])
        torch.cuda.synchronize()
        a = H.result_from_tensor(alone["result_dev"])
        assert a.sum_w == m.sum_w and a.n_pass == m.n_pass
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    g = H.heget_graph_xsec(subset, 6, 500, S, 32, res)
    try:
        st = torch.cuda.Stream()
        H.heget_graph_launch(g, SEED + 90, 0, stream=st)
        st.synchronize()
        got = H.result_from_tensor(res)
    finally:
        H.heget_graph_destroy(g)
    ref = torch.zeros(80, dtype=torch.uint8, device="cuda")
    H.heget_xsec_async(subset, 6, SEED + 90, 0, 500, S, 32, ref)
    torch.cuda.synchronize()
    assert got.sum_w == H.result_from_tensor(ref).sum_w


def test_algorithm_argument_checks(heget_lib, gpu):
    H = heget_lib
    with pytest.raises(H.HegetError):
        H.heget_set_algorithm(gpu, 7)
    assert H.heget_get_algorithm(gpu) == H.HEGET_ALG_TREE
    assert H.load().heget_get_algorithm(None) == -1


def test_subset_server_equals_batch_and_async(heget_lib, subset):
    """With the subset recursion the server runs the subset batch kernel with
    its own tiles: every result is bitwise the batch result of the request
    alone, and within FP32/FP64 rounding of heget_xsec_async (another launch
    shape, so another summation order)."""
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    mix = [(8, 300, 32), (7, 700, 64), (2, 9000, 32), (6, 2500, 64), (5, 4000, 32), (8, 40, 64), (4, 20_000, 32)]
    srv = H.heget_server_start(subset, max_launch_work=2e9)   # several launches per request
    try:
        tickets = [H.heget_submit(srv, n, SEED + 200 + k, N, S, p, i0=5 * k) for k, (n, N, p) in enumerate(mix)]
        got = [H.heget_wait(srv, t, 120.0) for t in tickets]
    finally:
        H.heget_server_stop(srv)
    for k, ((n, N, p), g) in enumerate(zip(mix, got)):
        assert g.status == H.HEGET_OK
        r = torch.zeros(80, dtype=torch.uint8, device="cuda")
        H.heget_xsec_batch(subset, [dict(n=n, precision=p, seed=SEED + 200 + k, i0=5 * k, N=N, sampler=S,
                                         result_dev=r)])
        torch.cuda.synchronize()
        alone = H.result_from_tensor(r)
        assert alone.sum_w == g.result.sum_w and alone.sum_w2 == g.result.sum_w2, f"request {k} (n={n})"
        assert alone.n_pass == g.result.n_pass and alone.n_tries == g.result.n_tries
        res = torch.zeros(80, dtype=torch.uint8, device="cuda")
        H.heget_xsec_async(subset, n, SEED + 200 + k, 5 * k, N, S, p, res)
        torch.cuda.synchronize()
        ref = H.result_from_tensor(res)
        assert ref.n_pass == alone.n_pass and ref.n_total == alone.n_total == N
        rel = 1e-12 if p == 64 else 1e-5
        assert alone.sum_w == pytest.approx(ref.sum_w, rel=rel, abs=0)


def test_batch_graphs_follow_the_algorithm(heget_lib, gpu):
    """The batch kernel is compiled once per algorithm, and its CUDA graphs
    are kept per algorithm: with graphs on, alternating the context between
    the tree and the subset recursion gives each algorithm's direct bits."""
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    reqs = [(6, 200, 32), (3, 3000, 64), (8, 20, 32)]

    def run():
        bufs = [torch.zeros(80, dtype=torch.uint8, device="cuda") for _ in reqs]
        H.heget_xsec_batch(gpu, [dict(n=n, precision=p, seed=SEED + 300 + k, i0=0, N=N, sampler=S, result_dev=b)
                                 for k, ((n, N, p), b) in enumerate(zip(reqs, bufs))])
        torch.cuda.synchronize()
        return [H.result_from_tensor(b) for b in bufs]

    try:
        tree = run()
        H.heget_set_algorithm(gpu, H.HEGET_ALG_SUBSET)
        sub = run()
        H.heget_set_graphs(gpu, 1)
        sub_g = run()                        # captures the subset kernel's graphs
        H.heget_set_algorithm(gpu, H.HEGET_ALG_TREE)
        tree_g = run()                       # captures the tree's
        H.heget_set_algorithm(gpu, H.HEGET_ALG_SUBSET)
        sub_g2 = run()                       # replays the subset kernel's
        on, captures, replays = H.heget_get_graphs(gpu)
        assert on == 1 and captures >= 4 and replays >= 2
    finally:
        H.heget_set_graphs(gpu, 0)
        H.heget_set_algorithm(gpu, H.HEGET_ALG_TREE)
    for a, b in zip(tree, tree_g):
        assert a.sum_w == b.sum_w and a.n_pass == b.n_pass
    for a, b, c in zip(sub, sub_g, sub_g2):
        assert a.sum_w == b.sum_w == c.sum_w and a.n_pass == b.n_pass
    for a, b in zip(tree, sub):
        assert a.n_pass == b.n_pass and a.sum_w == pytest.approx(b.sum_w, rel=1e-5)
