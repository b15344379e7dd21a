"""Write the stored oracle samples of the largest photon counts.

The FP64 oracle evaluates all n! orderings of all 2^(n+2) helicities with
explicit 4x4 Dirac matrices: about 50 s of one core per point at n = 8.  The
parity tests and the benchmark's error columns at n = 7 and n = 8 therefore
read their expected values from the files this script writes; every value in
them comes from ``oracle/`` alone (phase-space points regenerated from the
seed, |M|^2 of Sec. 2.1 eqs. (6)-(8) summed over helicities, event weights of
eq. (2)).

    python tests/golden/gen_oracle_samples.py [--threads T] [n ...]

Files (text, one record per line, '#' comments):
  oracle_weights_n<n>.txt : the workload's points 0 .. N-1 in order:
                            index, mask, tries, weight (fb)
  oracle_amp2_n<n>.txt    : the first cut-passing points of that sample:
                            index, sum_h |M_h|^2 (GeV^(4-2n))
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

SEED = 0x0908440300000002

# n -> (sampler description, sampler factory, points of the weight sample,
#       cut-passing points whose |M|^2 is stored)
SAMPLES = {
    8: ("uniform 200..2000 GeV", lambda: O.uniform(200.0, 2000.0), 256, 32),
    7: ("toy PDF", lambda: O.toy_pdf(), 256, 32),
}


def write(n: int, threads: int) -> None:
    desc, smp, N, n_amp = SAMPLES[n]
    cut = O.cuts()
    t0 = time.time()
    w, mask, tries = O.event_weights(n, SEED, 0, N, smp(), cut, threads=threads)
    t_w = time.time() - t0
    path = os.path.join(HERE, f"oracle_weights_n{n}.txt")
    with open(path, "w") as fh:
        fh.write(f"# u ubar -> {n} gamma event weights (fb) from the FP64 oracle, written by gen_oracle_samples.py\n")
        fh.write(f"# n {n} seed {SEED:#x} i0 0 N {N} sampler {desc} cuts pT>20 |eta|<2.5 dR>0.4\n")
        fh.write(f"# alpha {O.ALPHA!r} Q {O.Q_U!r}; {int(mask.sum())} points pass the cuts; {t_w:.0f} s on "
                 f"{threads} threads\n")
        fh.write("# index mask tries weight\n")
        for i in range(N):
            fh.write(f"{i} {int(mask[i])} {int(tries[i])} {float(w[i])!r}\n")
    ps = O.phase_space(n, SEED, 0, N, smp(), cut)
    idx = [i for i in range(N) if ps["mask"][i]][:n_amp]
    t0 = time.time()
    a = O.amp2(n, ps["momenta"][idx], threads=threads)
    t_a = time.time() - t0
    path = os.path.join(HERE, f"oracle_amp2_n{n}.txt")
    with open(path, "w") as fh:
        fh.write(f"# u ubar -> {n} gamma: sum over all 2^(n+2) helicities of |M_h|^2 (couplings included, no colour,"
                 f" spin average or 1/n!) from the FP64 oracle, written by gen_oracle_samples.py\n")
        fh.write(f"# momenta: points of n {n} seed {SEED:#x} sampler {desc} (oracle.phase_space), the first "
                 f"{len(idx)} that pass the cuts; {t_a:.0f} s on {threads} threads\n")
        fh.write("# index amp2\n")
        for i, v in zip(idx, a):
            fh.write(f"{i} {float(v)!r}\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("n", type=int, nargs="*", default=sorted(SAMPLES))
    args = ap.parse_args()
    O.build()
    for n in args.n:
        write(n, args.threads)


if __name__ == "__main__":
    main()
