#!/usr/bin/env python3
"""Writes heget_logtab.h: the breakpoint table of the table-driven natural
logarithm in heget_ps.cuh (Tang, ACM TOMS 16 (1990) 378).  For j = 0..64 and
F_j = 1 + j/64 it stores ln F_j as a double-double (hi + lo, computed with
40-digit decimal arithmetic) and 1/F_j rounded to double.  ln 2 itself is
stored the same way.  Run from anywhere: python gen_logtab.py"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 40


def dd(v: Decimal):
    hi = float(v)
    lo = float(v - Decimal(hi))
    return hi, lo


def main():
    lines = [
        "// heget_logtab.h -- generated by gen_logtab.py; do not edit.",
        "// ln(1 + j/64) = hi + lo (double-double) and 1/(1 + j/64), j = 0..64.",
        "#pragma once",
        "",
        "namespace heget {",
        "",
        "__device__ const double kLogTab[65][3] = {",
    ]
    for j in range(65):
        F = Decimal(64 + j) / Decimal(64)
        hi, lo = dd(F.ln())
        inv = float(Decimal(1) / F)
        lines.append(f"    {{{hi.hex()}, {lo.hex()}, {inv.hex()}}},")
    lines.append("};")
    hi, lo = dd(Decimal(2).ln())
    lines += ["", f"constexpr double kLn2Hi = {hi.hex()};", f"constexpr double kLn2Lo = {lo.hex()};", "",
              "}  // namespace heget", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heget_logtab.h")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
