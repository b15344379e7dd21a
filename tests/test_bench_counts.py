"""The algorithmic flop counts behind bench.py's roofline, pinned by brute
force: the tree's chain steps are the distinct ordered prefixes of 2..n-1
photons (n-2 with the two-ended finish, from n = 4), its closures the n!
orderings; the subset recursion's steps are the (set, photon, helicities)
triples of sets of 2..n-1 photons."""
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
    steps = 0
    for k in range(2, n):
        for S in itertools.combinations(range(n), k):
            steps += len(S) * (1 << k)   # each photon of S attached last, every helicity of S
    assert bench.subset_flops_per_point(n) == 32 * steps + 16 * n * (1 << n)


@pytest.mark.parametrize("n", range(2, 9))
def test_helas4_flops_by_enumeration(bench, n):
    """The 4-component comparison count: every ordered prefix of 1..n-1
    photons is a step, every ordering a closure, for 2^(n+1) helicities."""
    prefixes = set()
    for perm in itertools.permutations(range(n)):
        for l in range(1, n):
            prefixes.add(perm[:l])
    assert bench.helas4_flops_per_point(n) == (1 << (n + 1)) * (128 * len(prefixes) + 88 * math.factorial(n))
