"""Writes dd_tables.cuh: the double-double constant tables of dd.cuh.

Values: log(1 + j/128) for j = 0..128 and atan(j/64) for j = 0..64 from
mpmath at 50 digits, and the rationals 1/(2k+1) for k = 0..8; each split into
hi = the nearest double and lo = the nearest double to the remainder.
Run: python paper_2208_02382_b300/csrc/gen_dd_tables.py
"""
import os
from fractions import Fraction

import mpmath as mp

mp.mp.dps = 50
HERE = os.path.dirname(os.path.abspath(__file__))


def split_mp(v):
    hi = float(v)
    return hi, float(v - mp.mpf(hi))


def split_fr(f):
    hi = float(f)
    return hi, float(f - Fraction(hi))


def array(qual, name, vals):
    out, line = [f"{qual} double {name}[{len(vals)}] = {{"], "    "
    for x in vals:
        item = repr(x) + ", "
        if len(line) + len(item) > 96:
            out.append(line.rstrip())
            line = "    "
        line += item
    out.append(line.rstrip().rstrip(",") + "};")
    return "\n".join(out)


def main():
    logt = [split_mp(mp.log(1 + mp.mpf(j) / 128)) for j in range(129)]
    atant = [split_mp(mp.atan(mp.mpf(j) / 64)) for j in range(65)]
    odd = [split_fr(Fraction(1, 2 * k + 1)) for k in range(9)]
    parts = [
        "// Generated by gen_dd_tables.py: log(1 + j/128), j = 0..128, and atan(j/64),",
        "// j = 0..64 (50-digit mpmath values), and 1/(2k+1), k = 0..8, each as",
        "// double-double (hi = nearest double, lo = nearest double to the rest).",
        "#pragma once",
        "namespace bt {",
        array("__device__ const", "DD_LOGTAB_HI", [v[0] for v in logt]),
        array("__device__ const", "DD_LOGTAB_LO", [v[1] for v in logt]),
        array("__device__ const", "DD_ATANTAB_HI", [v[0] for v in atant]),
        array("__device__ const", "DD_ATANTAB_LO", [v[1] for v in atant]),
        array("__constant__", "DD_INVODD_HI", [v[0] for v in odd]),
        array("__constant__", "DD_INVODD_LO", [v[1] for v in odd]),
        "}  // namespace bt",
        "",
    ]
    with open(os.path.join(HERE, "dd_tables.cuh"), "w") as f:
        f.write("\n".join(parts))


if __name__ == "__main__":
    main()
