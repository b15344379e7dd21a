"""The algorithmic flop counts behind bench.py's roofline, pinned by brute
force: the tree's chain steps are the distinct ordered prefixes of 2..n-1
photons (n-2 with the two-ended finish, from n = 4), its closures the n!
orderings; the subset recursion's currents are the (set, helicities) pairs
of the two sides met in the middle, and its contraction one product per set
of half the photons and helicity configuration."""
import importlib.util
import itertools
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("n", range(2, 8))
def test_tree_flops_by_enumeration(bench, n):
    two_ended = n >= 4
    deepest = n - 2 if two_ended else n - 1
    prefixes = set()
    for perm in itertools.permutations(range(n)):
        for l in range(2, deepest + 1):
            prefixes.add(perm[:l])
    steps = len(prefixes)   # the first photon is a table row, not a step
    closures = math.factorial(n)
    pairs = n * (n - 1) * 4 * 32 if two_ended else 0
    assert bench.tree_flops_per_point(n) == (1 << n) * (28 * steps + 16 * closures) + pairs
    # FP64 counts the same tree
    assert bench.tree_flops_per_point(n, fp64=True) == bench.tree_flops_per_point(n)


@pytest.mark.parametrize("n", range(2, 9))
def test_subset_flops_by_enumeration(bench, n):
    """Met in the middle at m = n // 2: every (set, helicities) current of
    the vbar side up to m photons and of the u side up to n - m - 1 photons
    costs 12 FMA per photon attached last (sets of 2 or more) plus 12 for its
    Q, the size-(n-m) R currents 12 per photon, and each of the 2^n
    configurations 8 per set T of m photons in the contraction."""
    m, mk = n // 2, n - n // 2
    fma = 0
    for side_max in (m, mk - 1):
        for k in range(1, side_max + 1):
            for S in itertools.combinations(range(n), k):
                for _lam in range(1 << k):
                    fma += (12 * len(S) if k >= 2 else 0) + 12
    if mk >= 2:
        for V in itertools.combinations(range(n), mk):
            fma += (1 << mk) * 12 * len(V)
    for T in itertools.combinations(range(n), m):
        fma += (1 << n) * 8
    assert bench.subset_flops_per_point(n) == 2 * fma
    if n == 8:
        assert fma == 315_776


@pytest.mark.parametrize("n", range(2, 9))
def test_helas4_flops_by_enumeration(bench, n):
    """The 4-component comparison count: every ordered prefix of 1..n-1
    photons is a step, every ordering a closure, for 2^(n+1) helicities."""
    prefixes = set()
    for perm in itertools.permutations(range(n)):
        for l in range(1, n):
            prefixes.add(perm[:l])
    assert bench.helas4_flops_per_point(n) == (1 << (n + 1)) * (128 * len(prefixes) + 88 * math.factorial(n))


def test_roofline_fields(bench):
    """The headline roofline: FP64 flops and FP64 instructions per point (one
    instruction per issue slot, 2 slots per SM and clock) over the kernel
    time; the subset recursion's step on the FP32 pipe by its own count."""
    N, kern_s, n_eval = 1 << 20, 1.2e-3, 600_000
    r = bench.roofline(4, N, kern_s, 70.0, 1.0, n_eval=n_eval)
    assert r["pipe"] == "fp64" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.FP64_FLOPS_PER_POINT[4] * N / kern_s / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK)
    slots = bench.SMS * 2 * bench.SM_GHZ * 1e9
    assert r["fp64_issue_frac"] == pytest.approx(bench.FP64_INSTR_PER_POINT[4] * N / kern_s / slots)
    # flops per instruction lie between 1 (DADD, DMUL) and 2 (DFMA)
    assert bench.FP64_INSTR_PER_POINT[4] <= bench.FP64_FLOPS_PER_POINT[4] <= 2 * bench.FP64_INSTR_PER_POINT[4]
    assert r["fp32_tree"]["achieved"] == pytest.approx(bench.tree_flops_per_point(4) * n_eval / kern_s / 1e12)
    s = bench.roofline(8, N, kern_s, 70.0, 1.0, n_eval=n_eval, subset=True)
    assert s["pipe"] == "fp32 fma" and s["flops_per_point"] == bench.subset_flops_per_point(8)
    assert s["frac"] == pytest.approx(bench.subset_flops_per_point(8) * n_eval / kern_s / 1e12 / bench.FP32_PEAK)
    t = bench.roofline(6, N, kern_s, 70.0, 1.0, n_eval=n_eval)
    assert t["kernel"] == "xsec_kernel<float,6,160>" and t["flops_per_point"] == bench.tree_flops_per_point(6)
