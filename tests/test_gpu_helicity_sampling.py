"""Helicity sampling (heget_set_helicity_sampling): the paper's events carry
one random helicity combination each (Sec. 3).  Per-event weights against
the oracle's 2^(n+2) |M_h|^2 for the same drawn h (the zeros of
sigma1 = sigma2 included, bit for bit), through both ordering-sum
algorithms and the warp-specialised and tile kernels; the sampled estimate
agrees with the full helicity sum on the same events within its error; and
forced FP32 -> FP64 escalation reproduces the FP64 sampled weights."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x090844030000C000


@pytest.fixture
def sampling(heget_lib, gpu):
    heget_lib.heget_set_helicity_sampling(gpu, 1)
    assert heget_lib.heget_get_helicity_sampling(gpu) == 1
    yield gpu
    heget_lib.heget_set_helicity_sampling(gpu, 0)
    heget_lib.heget_set_algorithm(gpu, heget_lib.HEGET_ALG_TREE)
    heget_lib.heget_set_escalation(gpu, 0.0)


def _weights(H, ctx, n, seed, i0, N, prec, S=None):
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_xsec_async(ctx, n, seed, i0, N, S or H.sampler_toy_pdf(), prec, res, w)
    torch.cuda.synchronize()
    return w.cpu().numpy(), H.result_from_tensor(res)


def _oracle_sampled(oracle, n, seed, i0, N):
    """Oracle weights with the drawn helicities, and which points are exact
    zeros (cut failures, and h with sigma1 = sigma2)."""
    ps = oracle.phase_space(n, seed, i0, N, oracle.toy_pdf(), oracle.cuts())
    ref, zero = np.zeros(N), np.ones(N, dtype=bool)
    for j in range(N):
        if not ps["mask"][j]:
            continue
        h = int(oracle.uniform_draw(seed, i0 + j, 2, 0) * 2 ** (n + 2))
        zero[j] = (h & 1) == ((h >> 1) & 1)
        M, _ = oracle.amp_hel(n, ps["momenta"][j], h)
        ref[j] = oracle.event_weight(n, ps["sqrt_s"][j] ** 2, 2 ** (n + 2) * abs(M) ** 2, ps["weight"][j], 1)
    return ref, zero


@pytest.mark.parametrize("n,N,alg", [(2, 700, 0), (4, 600, 0), (4, 600, 1), (6, 60, 0), (6, 60, 1)])
def test_sampled_weights_match_oracle(oracle, heget_lib, sampling, n, N, alg):
    """Exact zeros bit for bit; elsewhere within the precision's tolerance,
    with a floor for the helicities that vanish only by cancellation (all
    photons of one helicity), where both sides give rounding noise."""
    H = heget_lib
    H.heget_set_algorithm(sampling, alg)
    seed, i0 = SEED + n, 11
    ref, zero = _oracle_sampled(oracle, n, seed, i0, N)
    assert 0 < zero.sum() < N and np.all(ref[zero] == 0)
    big = np.max(ref)
    for prec, tol in ((H.HEGET_FP64, 1e-11), (H.HEGET_FP32, 1e-3)):
        w, _ = _weights(H, sampling, n, seed, i0, N, prec)
        assert np.all(w[zero] == 0)
        nz = ~zero
        assert np.all(np.abs(w[nz] - ref[nz]) <= tol * ref[nz] + 1e-10 * big)


def test_sampled_mean_agrees_with_full_sum(heget_lib, sampling):
    """Same events: E[2^(n+2) |M_h|^2] = sum_h |M_h|^2 (5 standard errors)."""
    H = heget_lib
    n, N, seed = 4, 200_000, SEED + 40
    ws, rs = _weights(H, sampling, n, seed, 0, N, H.HEGET_FP32)
    H.heget_set_helicity_sampling(sampling, 0)
    wf, rf = _weights(H, sampling, n, seed, 0, N, H.HEGET_FP32)
    d = ws - wf
    err = d.std(ddof=1) / math.sqrt(N)
    assert abs(d.mean()) < 5 * err
    assert rs.n_pass == rf.n_pass and ws.std() > wf.std()


@pytest.mark.parametrize("n,N", [(4, 3000), (6, 150)])
def test_forced_escalation_with_sampling(heget_lib, sampling, n, N):
    """The condition bound uses the sampled lane's weight: with every point
    of nonzero weight escalated, the FP32 launch returns the FP64 sampled
    weights."""
    H = heget_lib
    w64, r64 = _weights(H, sampling, n, SEED + 60 + n, 3, N, H.HEGET_FP64)
    H.heget_set_escalation(sampling, 1e-30)
    w32, r32 = _weights(H, sampling, n, SEED + 60 + n, 3, N, H.HEGET_FP32)
    # every point with a nonzero sampled weight escalates; those that drew a
    # vanishing helicity (sigma1 = sigma2) have weight and bound exactly 0
    assert r32.n_pass == r64.n_pass > r32.n_escalated == np.count_nonzero(w64) > 0
    # escalated points are recomputed with the subset recursion: rounding
    # differs from the FP64 launch (the tree) by ~1e-15 relative
    assert np.all(np.abs(w32 - w64) <= 1e-13 * np.abs(w64) + 1e-13 * np.max(w64))


def test_helicity_sampling_argument_checks(heget_lib, gpu):
    H = heget_lib
    with pytest.raises(H.HegetError):
        H.heget_set_helicity_sampling(gpu, 2)
    assert H.heget_get_helicity_sampling(gpu) == 0
    assert H.load().heget_get_helicity_sampling(None) == -1
    assert H.load().heget_set_helicity_sampling(None, 1) == H.HEGET_EINVAL


def test_sampling_through_the_batch(heget_lib, sampling):
    """The mixed-n batch samples the same helicities: each request's sums
    equal those of a direct launch over the same points (FP64, to rounding;
    the two paths tile the points differently)."""
    import torch
    H = heget_lib
    S = H.sampler_toy_pdf()
    reqs = [dict(n=n, precision=64, seed=SEED + 90 + n, i0=5, N=N, sampler=S,
                 result_dev=torch.zeros(80, dtype=torch.uint8, device="cuda"))
            for n, N in [(2, 3000), (4, 1500), (6, 80)]]
    H.heget_xsec_batch(sampling, reqs)
    torch.cuda.synchronize()
    for r in reqs:
        got = H.result_from_tensor(r["result_dev"])
        _, ref = _weights(H, sampling, r["n"], r["seed"], r["i0"], r["N"], H.HEGET_FP64)
        assert got.n_pass == ref.n_pass
        assert got.sum_w == pytest.approx(ref.sum_w, rel=1e-12)
        assert got.sum_w2 == pytest.approx(ref.sum_w2, rel=1e-12)
