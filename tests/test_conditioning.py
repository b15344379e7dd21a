"""Condition of the ordering sum on the benchmark workloads (oracle only).

For one helicity, kappa_h = sum_pi |A_pi| / |sum_pi A_pi| says how many
digits the sum over the n! orderings can lose; for the helicity sum the
relevant figure is kappa = sqrt(sum_h (sum_pi |A_pi,h|)^2 / sum_h |M_h|^2).
On the cut-passing points of the toy-PDF workloads the helicity sum stays
within a few units and no helicity that carries weight (|M_h| above 1e-3 of
the point's largest) comes near 1e4, the level at which a point would need
its own tolerance.  So the ordering sum costs at most a few bits, and the
FP32 and FP64 differences against the oracle come from the chain's rounding
and the denominators, not from cancellation between orderings."""
import numpy as np
import pytest

SEED = 0x0908440300000002


@pytest.mark.parametrize("n,N", [(2, 200), (3, 200), (4, 200), (5, 60), (6, 24), (7, 6)])
def test_ordering_sum_is_well_conditioned(oracle, n, N):
    ps = oracle.phase_space(n, SEED, 0, N, oracle.toy_pdf(), oracle.cuts())
    k_sum, k_hel = [], []
    for j in np.nonzero(ps["mask"])[0]:
        m = ps["momenta"][j]
        amp, sabs = [], []
        for h in range(1 << (n + 2)):
            if (h & 1) == ((h >> 1) & 1):
                continue   # sigma1 = sigma2: exactly zero
            a, s = oracle.amp_hel(n, m, h)
            amp.append(abs(a))
            sabs.append(s)
        amp, sabs = np.array(amp), np.array(sabs)
        k_sum.append(np.sqrt((sabs**2).sum() / (amp**2).sum()))
        big = amp > 1e-3 * amp.max()
        k_hel.append((sabs[big] / amp[big]).max())
    assert len(k_sum) > 0
    print(f"n={n}: {len(k_sum)} points, kappa of the helicity sum <= {max(k_sum):.3g}, "
          f"of a weighted helicity <= {max(k_hel):.3g}")
    assert max(k_sum) < 5
    assert max(k_hel) < 1e4
