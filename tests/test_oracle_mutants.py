"""The pins must catch plausible mistakes in the oracle.

Each mutant below is a copy of ``oracle/heget_oracle.c`` (or of the Python
wrappers in ``oracle/__init__.py``) with one small edit
of the kind a careful reader could still make while restating the paper --
a dropped term, a wrong sign, a transposed index, a missing conjugation, a
wrong normalisation.  Every copy is built in a scratch directory and the
oracle's pin suite (``test_oracle_pins.py``, ``test_oracle_hist.py``) runs
against it in a child process; at least one pin has to fail.  The unmodified
source runs through the same harness first and has to pass, so a broken
harness cannot pass for a strong suite.

Mistakes that cannot show in any quantity the method computes (a common phase
of every amplitude, the order in which equal momenta are visited, the side a
measure-zero tie falls on) are not mutants.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["test_oracle_pins.py", "test_oracle_hist.py"]

# (name, exact text in heget_oracle.c, replacement)
MUTANTS = [
    # Philox4x32-10 and the draw layout
    ("philox multiplier", "M0 = 0xD2511F53u", "M0 = 0xD2511F55u"),
    ("philox key schedule", "k1 += W1;", "k1 += W0;"),
    ("philox output words swapped", "uint32_t y0 = (uint32_t)(b >> 32) ^ x1 ^ k0;",
     "uint32_t y0 = (uint32_t)(a >> 32) ^ x1 ^ k0;"),
    ("uniform without the half-ulp offset", "((double)m + 0.5) * 0x1p-52", "((double)m) * 0x1p-52"),
    ("counter uses draw instead of draw/2", "draw >> 1,\n", "draw,\n"),
    # Dirac algebra and external states
    ("gamma^i lower block sign", "G[i].m[2 + a][b] = -s[i][a][b];", "G[i].m[2 + a][b] = s[i][a][b];"),
    ("sigma_y transposed", "s[2][0][1] = -I; s[2][1][0] = I;", "s[2][0][1] = I; s[2][1][0] = -I;"),
    ("slash with the wrong metric sign", "- G[1].m[x][y] * a[1]", "+ G[1].m[x][y] * a[1]"),
    ("Minkowski product drops a sign", "- a[3] * b[3];", "+ a[3] * b[3];"),
    ("spinor phase sign", "u.v[3] = nrm * cexp(I * ph) * sh;", "u.v[3] = nrm * cexp(-I * ph) * sh;"),
    ("spinor normalisation", "double nrm = sqrt(2 * p[0]);", "double nrm = sqrt(p[0]);"),
    ("polarisation: e_phi sign", "(-lam * eth[i] - I * ephi[i])", "(-lam * eth[i] + I * ephi[i])"),
    ("polarisation: no conjugate for outgoing photons", "e[mu] = conj(e[mu]);", "e[mu] = e[mu];"),
    ("polarisation: e_theta z component sign", "double eth[3] = {c * cp, c * sp, -s};",
     "double eth[3] = {c * cp, c * sp, s};"),
    # the chain and the ordering sum
    ("momentum flow: q = p1 + K", "q[mu] -= k[mu];", "q[mu] += k[mu];"),
    ("vertex ignores the ordering", "psi = matvec(&V[perm[l]], &psi);", "psi = matvec(&V[l], &psi);"),
    ("propagator without 1/q^2", "S = mat_scale(&S, 1.0 / mdot(q, q));", "S = mat_scale(&S, 1.0);"),
    ("permutations not fully enumerated", "t = a[l]; a[l] = a[r]; a[r] = t;", "t = a[l];"),
    ("compensated sum: wrong correction sign", "*c[k] += (*s[k] - t) + v[k];", "*c[k] += (*s[k] - t) - v[k];"),
    ("coupling e^2 = alpha instead of 4 pi alpha", "double e = sqrt(4 * M_PI * cpl->alpha);",
     "double e = sqrt(cpl->alpha);"),
    ("half of the helicities summed", "for (int h = 0; h < (1 << (n + 2)); ++h) {\n        if (!mask_bit",
     "for (int h = 0; h < (1 << (n + 1)); ++h) {\n        if (!mask_bit"),
    ("helicity bit of the quark spins swapped", "int s1 = (h & 1) ? 1 : -1, s2 = (h & 2) ? 1 : -1;\n    spin4 u1 = u_spinor(mom, s1);\n    spin4 vb2 = vbar_spinor(mom + 4, s2);\n    mat4 V[ORACLE_MAXN];\n    for (int i = 0; i < n; ++i) {",
     "int s1 = (h & 2) ? 1 : -1, s2 = (h & 1) ? 1 : -1;\n    spin4 u1 = u_spinor(mom, s1);\n    spin4 vb2 = vbar_spinor(mom + 4, s2);\n    mat4 V[ORACLE_MAXN];\n    for (int i = 0; i < n; ++i) {"),
    ("photon helicity bit off by one", "int lam = (h >> (2 + i)) & 1 ? 1 : -1;", "int lam = (h >> (1 + i)) & 1 ? 1 : -1;"),
    # RAMBO and the phase-space volume
    ("RAMBO: cos(theta) not centred", "double c = 2 * r[4 * i] - 1;", "double c = r[4 * i];"),
    ("RAMBO: q0 from one uniform", "double q0 = -log(r[4 * i + 2] * r[4 * i + 3]);", "double q0 = -log(r[4 * i + 2]);"),
    ("RAMBO: boost direction", "double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};",
     "double b[3] = {Q[1] / M, Q[2] / M, Q[3] / M};"),
    ("RAMBO: a = 1/gamma", "double a = 1 / (1 + gam);", "double a = 1 / gam;"),
    ("RAMBO: energy without the boost term", "out[4 * i] = x * (gam * q[i][0] + bq);", "out[4 * i] = x * (gam * q[i][0]);"),
    ("phase-space volume: (pi/2)^n", "pow(M_PI / 2, n - 1)", "pow(M_PI / 2, n)"),
    ("phase-space volume: (n-1)! twice", "for (int i = 2; i <= n - 2; ++i) fact2 *= i;",
     "for (int i = 2; i <= n - 1; ++i) fact2 *= i;"),
    # samplers and cuts
    ("toy PDF: proposal x = u", "double x = u * u;", "double x = u;"),
    ("toy PDF: acceptance (1-x)^2", "if (v < pow(1 - x, b)) return x;", "if (v < pow(1 - x, b - 1)) return x;"),
    ("toy PDF: floor test reversed", "if (rs > S->floor) {", "if (rs < S->floor) {"),
    ("toy PDF: y = ln(x1/x2)", "*y = 0.5 * log(x1 / x2);", "*y = log(x1 / x2);"),
    ("toy PDF: attempts not counted", "            return t;\n", "            return 1;\n"),
    ("incoming ubar along +z", "p[7] = -rs / 2;", "p[7] = rs / 2;"),
    ("metric route: sign of the time component", "sign *= (mu == 0) ? -1.0 : 1.0;", "sign *= (mu == 0) ? 1.0 : -1.0;"),
    ("uniform sampler: range from lo to hi - lo", "*sqrt_s = S->lo + (S->hi - S->lo) * u;", "*sqrt_s = (S->hi - S->lo) * u;"),
    ("cuts: boost subtracted", "eta[i] = asinh(p[3] / pt) + y;", "eta[i] = asinh(p[3] / pt) - y;"),
    ("cuts: Delta phi not folded", "if (dphi > M_PI) dphi = 2 * M_PI - dphi;\n                double deta",
     "double deta"),
    ("cuts: |eta| test on eta", "if (!(fabs(eta[i]) < C->eta_max)) return 0;", "if (!(eta[i] < C->eta_max)) return 0;"),
    # the event weight
    ("weight: colour average 1/3 instead of 1/9", "(1.0 / 4) * (1.0 / 9) * 3", "(1.0 / 4) * (1.0 / 3) * 3"),
    ("weight: flux 1/s", "(1.0 / (2 * s))", "(1.0 / s)"),
    ("weight: (hbar c)^2 in pb", "#define GEV2_TO_FB 0.3893793721e12", "#define GEV2_TO_FB 0.3893793721e9"),
    ("weight: 1/n instead of 1/n!", "amp2 / nfact * phi_n", "amp2 / n * phi_n"),
    # histograms
    ("hist: bins counted from 0", "return 1 + (int)t;", "return (int)t;"),
    ("hist: largest pT taken as the smallest", "if (pt[i] > x[0]) x[0] = pt[i];", "if (pt[i] < x[0]) x[0] = pt[i];"),
    ("hist: smallest Delta R taken as the largest", "if (dr[p] < x[0]) x[0] = dr[p];", "if (dr[p] > x[0]) x[0] = dr[p];"),
    ("hist: eta without the boost", "eta[i] = asinh(k[4 * i + 3] / pt[i]) + y[j];", "eta[i] = asinh(k[4 * i + 3] / pt[i]);"),
    ("hist: Delta phi not folded", "if (dphi > M_PI) dphi = 2 * M_PI - dphi;\n                const double deta",
     "const double deta"),
    ("hist: w instead of w^2", "nsum_add(&sw2[b], w[j] * w[j]);", "nsum_add(&sw2[b], w[j]);"),
    ("hist: sqrt(s-hat) as E1", "x[0] = ev[0] + ev[4];", "x[0] = ev[0];"),
]


# The same for the Python wrappers (``oracle/__init__.py``): the arithmetic
# they hold (the toy-PDF cross-section scale of the summation step) and the
# order of the arguments they marshal.
PY_MUTANTS = [
    ("toy-PDF sigma without the q <-> qbar factor 2", "scale = 2.0 * N / float(np.sum(tries))",
     "scale = N / float(np.sum(tries))"),
    ("toy-PDF acceptance inverted", "scale = 2.0 * N / float(np.sum(tries))",
     "scale = 2.0 * float(np.sum(tries)) / N"),
    ("toy-PDF scale applied to the wrong sampler", "if sampler_kind == 2:", "if sampler_kind == 1:"),
    ("event weights: alpha and Q swapped", "alpha, Q, th, _ptr(w), _ptr(mask), _ptr(tries))",
     "Q, alpha, th, _ptr(w), _ptr(mask), _ptr(tries))"),
    ("amp2: alpha and Q swapped", "_ptr(mw), alpha, Q, th, _ptr(out))", "_ptr(mw), Q, alpha, th, _ptr(out))"),
    ("phase space: sqrt(s-hat) and y outputs swapped", "_ptr(mom), _ptr(w), _ptr(rs), _ptr(y), _ptr(mask)",
     "_ptr(mom), _ptr(w), _ptr(y), _ptr(rs), _ptr(mask)"),
]


def _sandbox(base, name, src, py_src=None):
    """A scratch tree with the pin tests and an oracle package built from `src`
    (and `py_src` as its wrappers, else the repository's)."""
    d = os.path.join(base, name.replace(" ", "_").replace("/", "_").replace(":", "").replace("^", "")
                     .replace("<->", "to").replace("(", "").replace(")", ""))
    os.makedirs(os.path.join(d, "oracle"))
    if py_src is None:
        shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), os.path.join(d, "oracle"))
    else:
        with open(os.path.join(d, "oracle", "__init__.py"), "w") as f:
            f.write(py_src)
    with open(os.path.join(d, "oracle", "heget_oracle.c"), "w") as f:
        f.write(src)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    for f in ["conftest.py", "helpers.py"] + PINS:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(d, "tests"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    return d


def _run(d):
    """Exit status of the pin suite in sandbox d (0 pass, 1 a pin failed)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", PYTHONDONTWRITEBYTECODE="1")
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + [os.path.join("tests", f) for f in PINS],
                       cwd=d, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout[-2000:] + p.stderr[-2000:]


def test_pins_catch_every_mutant(tmp_path):
    src = open(os.path.join(ROOT, "oracle", "heget_oracle.c")).read()
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    for name, find, repl in MUTANTS:
        assert src.count(find) == 1, f"mutant {name!r}: its text must occur exactly once"
    for name, find, repl in PY_MUTANTS:
        assert py.count(find) == 1, f"mutant {name!r}: its text must occur exactly once"
    cases = ([("unmodified", src, None)] + [(name, src.replace(find, repl), None) for name, find, repl in MUTANTS]
             + [(name, src, py.replace(find, repl)) for name, find, repl in PY_MUTANTS])
    dirs = [_sandbox(str(tmp_path), name, s, p) for name, s, p in cases]
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run, dirs))
    rc0, out0 = results[0]
    assert rc0 == 0, f"the unmodified oracle fails its pins in the harness:\n{out0}"
    survived, broken = [], []
    for (name, _, _), (rc, out) in zip(cases[1:], results[1:]):
        if rc == 0:
            survived.append(name)
        elif rc != 1:   # 1 = tests failed; anything else is a harness or build problem
            broken.append(f"{name}: exit {rc}\n{out}")
    assert not broken, "\n".join(broken)
    assert not survived, f"mutants no pin catches: {survived}"
