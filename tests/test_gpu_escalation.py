"""FP32 -> FP64 escalation: the per-point error bound flags points, an FP64
kernel recomputes them, and the flagged points count with their FP64 values.

Forcing every point to escalate (tau ~ 0) must reproduce the FP64 results
through both fused kernels (warp-specialised and tile) and both ordering-sum
algorithms; tau = 0 must escalate nothing; and with tau = 2e-7 every point must end within
2 n tau of the FP64 oracle, which checks that the bound really bounds the
FP32 error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x090844030000A000


@pytest.fixture
def esc(heget_lib, gpu):
    yield gpu
    heget_lib.heget_set_escalation(gpu, 0.0)
    heget_lib.heget_set_algorithm(gpu, heget_lib.HEGET_ALG_TREE)


def _xsec(H, ctx, n, N, seed, prec):
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_xsec_async(ctx, n, seed, 3, N, H.sampler_toy_pdf(), prec, res, w)
    torch.cuda.synchronize()
    return H.result_from_tensor(res), w.cpu().numpy()


@pytest.mark.parametrize("n,N,alg", [(3, 3001, 0), (6, 150, 0), (6, 150, 1), (4, 2000, 1)])
def test_forced_escalation_gives_fp64_results(heget_lib, esc, n, N, alg):
    H = heget_lib
    H.heget_set_algorithm(esc, alg)
    H.heget_set_escalation(esc, 1e-30)
    r32, w32 = _xsec(H, esc, n, N, SEED + n, H.HEGET_FP32)
    r64, w64 = _xsec(H, esc, n, N, SEED + n, H.HEGET_FP64)
    assert r32.n_escalated == r32.n_pass == r64.n_pass > 0
    assert r64.n_escalated == 0
    nz = w64 != 0
    np.testing.assert_array_equal(w32 != 0, nz)
    assert np.max(np.abs(w32[nz] - w64[nz]) / w64[nz]) < 1e-13
    assert r32.sum_w == pytest.approx(r64.sum_w, rel=1e-12, abs=0)
    assert r32.sum_w2 == pytest.approx(r64.sum_w2, rel=1e-12, abs=0)


def test_escalation_off_and_default(heget_lib, esc):
    H = heget_lib
    H.heget_set_escalation(esc, 0.0)
    assert H.heget_get_escalation(esc) == 0.0
    r0, w0 = _xsec(H, esc, 5, 2000, SEED + 50, H.HEGET_FP32)
    assert r0.n_escalated == 0
    H.heget_set_escalation(esc, 1e-4)
    r1, w1 = _xsec(H, esc, 5, 2000, SEED + 50, H.HEGET_FP32)
    assert r1.n_pass == r0.n_pass and r1.n_escalated <= r1.n_pass // 100
    nz = w0 != 0
    assert np.max(np.abs(w1[nz] - w0[nz]) / w0[nz]) < 1e-3


@pytest.mark.parametrize("n", [5, 6])
def test_bound_holds_against_the_oracle(oracle, heget_lib, esc, n):
    """tau = 2e-7 (a few u32): unescalated points have a bound below tau, so
    their FP32 error must stay within the bound's constant (2 n rounding
    steps per chain); escalated ones are FP64."""
    import torch
    H = heget_lib
    mom = oracle.phase_space(n, SEED + 60 + n, 0, 60 if n == 5 else 16, oracle.toy_pdf())["momenta"]
    ref = oracle.amp2(n, mom)
    tau = 2e-7
    H.heget_set_escalation(esc, tau)
    m = torch.from_numpy(mom).cuda()
    out = torch.empty(mom.shape[0], dtype=torch.float64, device="cuda")
    H.heget_amp2(esc, n, mom.shape[0], m, out, precision=H.HEGET_FP32)
    got = out.cpu().numpy()
    k = H.heget_amp2_escalated(esc)
    assert 0 <= k <= mom.shape[0]
    assert np.max(np.abs(got - ref) / ref) < 2 * n * tau


def test_forced_amp2_escalation(heget_lib, esc):
    import torch
    H = heget_lib
    n, N = 5, 3000
    mom = torch.empty((N, n + 2, 4), dtype=torch.float64, device="cuda")
    H.heget_phase_space_ex(esc, SEED + 70, 0, N, n, H.sampler_uniform(200.0, 2000.0), momenta=mom)
    a64 = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_amp2(esc, n, N, mom, a64, precision=H.HEGET_FP64)
    H.heget_set_escalation(esc, 1e-30)
    a32 = torch.empty(N, dtype=torch.float64, device="cuda")
    H.heget_amp2(esc, n, N, mom, a32, precision=H.HEGET_FP32)
    assert H.heget_amp2_escalated(esc) == N
    a32, a64 = a32.cpu().numpy(), a64.cpu().numpy()
    assert np.max(np.abs(a32 - a64) / a64) < 1e-13


def test_graph_replay_with_escalation(heget_lib, esc):
    import torch
    H = heget_lib
    H.heget_set_escalation(esc, 1e-30)
    S = H.sampler_toy_pdf()
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    g = H.heget_graph_xsec(esc, 4, 5000, S, H.HEGET_FP32, res)
    try:
        st = torch.cuda.Stream()
        for seed, i0 in [(SEED + 1, 0), (SEED + 2, 777)]:
            H.heget_graph_launch(g, seed, i0, stream=st)
            st.synchronize()
            got = H.result_from_tensor(res)
            ref = torch.zeros(80, dtype=torch.uint8, device="cuda")
            H.heget_xsec_async(esc, 4, seed, i0, 5000, S, H.HEGET_FP32, ref)
            torch.cuda.synchronize()
            ref = H.result_from_tensor(ref)
            assert got.sum_w == ref.sum_w and got.n_escalated == ref.n_escalated == ref.n_pass > 0
    finally:
        H.heget_graph_destroy(g)


def test_escalation_argument_checks(heget_lib, gpu):
    H = heget_lib
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(H.HegetError):
            H.heget_set_escalation(gpu, bad)
    assert H.heget_get_escalation(gpu) == 0.0   # off unless enabled
