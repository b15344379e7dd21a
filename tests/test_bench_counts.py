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
