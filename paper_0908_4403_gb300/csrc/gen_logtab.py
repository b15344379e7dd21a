#!/usr/bin/env python3
"""Writes heget_logtab.h: the breakpoint table of the table-driven natural
logarithm in heget_ps.cuh (Tang, ACM TOMS 16 (1990) 378).  For j = 0..256 and
F_j = 1 + j/256 it stores ln F_j as a double-double (hi + lo, computed with
40-digit decimal arithmetic) and 1/F_j rounded to double.  ln 2 itself is
stored the same way.  Run from anywhere: python gen_logtab.py [output path]"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 40
TABLE = 256


def dd(v: Decimal):
    hi = float(v)
    lo = float(v - Decimal(hi))
    return hi, lo


def main(out=None):
    lines = [
        "// heget_logtab.h -- generated by gen_logtab.py; do not edit.",
        f"// ln(1 + j/{TABLE}) = hi + lo (double-double) and 1/(1 + j/{TABLE}), j = 0..{TABLE}.",
        "#pragma once",
        "",
        "namespace heget {",
        "",
        f"constexpr int kLogTable = {TABLE};",
        f"__device__ const double kLogTab[{TABLE + 1}][3] = {{",
    ]
    for j in range(TABLE + 1):
        F = Decimal(TABLE + j) / Decimal(TABLE)
        hi, lo = dd(F.ln())
        inv = float(Decimal(1) / F)
        lines.append(f"    {{{hi.hex()}, {lo.hex()}, {inv.hex()}}},")
    lines.append("};")
    hi, lo = dd(Decimal(2).ln())
    lines += ["", f"constexpr double kLn2Hi = {hi.hex()};", f"constexpr double kLn2Lo = {lo.hex()};", "",
              "}  // namespace heget", ""]
    out = out or os.path.join(os.path.dirname(os.path.abspath(__file__)), "heget_logtab.h")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    import sys
    main(sys.argv[1] if len(sys.argv) > 1 else None)
