"""The constant tables of the device elementary functions, pinned against an
independent high-precision evaluation (mpmath at 200 bits): every entry of
the RAMBO azimuth table (cos, sin of 2 pi j/512) and of the logarithm's
breakpoint table (ln(1 + j/256) as a double-double, 1/(1 + j/256)) must be the
correctly rounded value."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0908_4403_gb300", "csrc")
HEX = r"(-?0x[0-9a-fA-Fp.+-]+)"


def _rows(name, width):
    text = open(os.path.join(CSRC, name)).read()
    pat = r"\{" + r",\s*".join([HEX] * width) + r"\}"
    return [tuple(float.fromhex(v) for v in m) for m in re.findall(pat, text)]


def test_sincos_table_is_correctly_rounded():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rows = _rows("heget_sincostab.h", 2)
    assert len(rows) == 512
    for j, (c, s) in enumerate(rows):
        a = 2 * mpmath.pi * j / 512
        for got, ref in ((c, mpmath.cos(a)), (s, mpmath.sin(a))):
            want = 0.0 if abs(ref) < mpmath.mpf(10) ** -40 else float(ref)
            assert got == want, (j, got, want)


def test_log_table_is_correctly_rounded():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rows = _rows("heget_logtab.h", 3)
    assert len(rows) == 257
    for j, (hi, lo, inv) in enumerate(rows):
        F = mpmath.mpf(256 + j) / 256
        ln = mpmath.log(F)
        assert hi == float(ln) and lo == float(ln - mpmath.mpf(hi)), j
        assert inv == float(1 / F), j
    text = open(os.path.join(CSRC, "heget_logtab.h")).read()
    hi = float.fromhex(re.search(r"kLn2Hi = " + HEX, text).group(1))
    lo = float.fromhex(re.search(r"kLn2Lo = " + HEX, text).group(1))
    ln2 = mpmath.log(2)
    assert hi == float(ln2) and lo == float(ln2 - mpmath.mpf(hi))


@pytest.mark.parametrize("gen,header", [("gen_logtab.py", "heget_logtab.h"), ("gen_sincostab.py", "heget_sincostab.h")])
def test_committed_tables_match_their_generators(tmp_path, gen, header):
    import subprocess
    import sys
    out = tmp_path / header
    subprocess.run([sys.executable, os.path.join(CSRC, gen), str(out)], check=True)
    assert out.read_bytes() == open(os.path.join(CSRC, header), "rb").read()
