"""Writes esdc_exp_table.h: 2^(j/2048) for j = 0..2047, each the double nearest
to the exact value (computed with 60 significant decimal digits, then rounded
by Python's correctly rounded decimal-to-binary conversion).  Run from this
directory: python gen_exp_table.py"""
import decimal
import os

N = 2048


def table():
    decimal.getcontext().prec = 60
    ln2 = decimal.Decimal(2).ln()
    return [float((ln2 * j / N).exp()) for j in range(N)]


def main():
    vals = table()
    lines = ["// 2^(j/2048), j = 0..2047, each the double nearest to the exact value.",
             "// Written by gen_exp_table.py (60-digit decimal arithmetic); do not edit.",
             "#pragma once", "", "namespace esdc {", "",
             "static __device__ const double g_exp2_table[2048] = {"]
    for i in range(0, N, 4):
        lines.append("    " + ", ".join(v.hex() for v in vals[i:i + 4]) + ",")
    lines += ["};", "", "}  // namespace esdc", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "esdc_exp_table.h")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
