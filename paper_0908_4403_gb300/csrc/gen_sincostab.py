#!/usr/bin/env python3
"""Writes heget_sincostab.h: the breakpoint table of the RAMBO azimuth in
heget_ps.cuh.  For j = 0..511 it stores (cos a_j, sin a_j), a_j = 2 pi j/512,
each correctly rounded to double: pi from Machin's formula and the two
Taylor series, all in 60-digit decimal arithmetic.  Run from anywhere:
python gen_sincostab.py"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
TABLE = 512


def atan_inv(k: int) -> Decimal:
    """atan(1/k) by its alternating series."""
    x = Decimal(1) / k
    x2 = x * x
    term, total, n = x, Decimal(0), 0
    eps = Decimal(10) ** -(getcontext().prec + 2)
    while abs(term) > eps:
        total += term / (2 * n + 1) * (1 if n % 2 == 0 else -1)
        term *= x2
        n += 1
    return total


PI = 16 * atan_inv(5) - 4 * atan_inv(239)


def cos_sin(a: Decimal):
    c, s = Decimal(0), Decimal(0)
    term, k = Decimal(1), 0          # a^k / k!
    eps = Decimal(10) ** -(getcontext().prec + 2)
    while k < 8 or abs(term) > eps:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
    return c, s


def rounded(v: Decimal) -> float:
    return 0.0 if abs(v) < Decimal(10) ** -40 else float(v)   # exact zeros at the quarter turns


def main(out=None):
    lines = [
        "// heget_sincostab.h -- generated by gen_sincostab.py; do not edit.",
        f"// (cos, sin) of 2 pi j/{TABLE}, j = 0..{TABLE - 1}, each correctly rounded.",
        "#pragma once",
        "",
        "namespace heget {",
        "",
        f"constexpr int kSinCosTable = {TABLE};",
        f"__device__ const double2 kSinCosTab[{TABLE}] = {{",
    ]
    for j in range(TABLE):
        c, s = cos_sin(2 * PI * j / TABLE)
        lines.append(f"    {{{rounded(c).hex()}, {rounded(s).hex()}}},")
    lines += ["};", "", "}  // namespace heget", ""]
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "heget_sincostab.h")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    import sys
    main(sys.argv[1] if len(sys.argv) > 1 else None)
