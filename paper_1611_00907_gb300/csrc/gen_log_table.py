"""Write log_table.h: the constants of the FP64 logarithm of the step kernels
(log_tab in device_common.cuh, after Tang's table-driven method, ACM TOMS
16(4), 1990).

Entry j (0..128) holds, for F_j = 1 + j/128, the double nearest 1/F_j and
ln F_j split as hi + lo: hi is ln F_j rounded to a multiple of 2^-32, lo the
double nearest the rest.  LN2_HI is ln 2 rounded to a multiple of 2^-32 too,
so that m * LN2_HI + hi is exact for any binary exponent m of a double (the
two terms cancel almost entirely for arguments just below 1, and only the
small terms carry rounding errors), and LN2_LO the double nearest
ln 2 - LN2_HI.  The logarithms are evaluated in 50-digit decimal arithmetic
and rounded once, so every constant is the nearest double.
Run from this directory:

    python gen_log_table.py > log_table.h
"""
import decimal
import sys
from fractions import Fraction

N = 128
D = decimal.Context(prec=50)


def nearest(x):
    """The double nearest the decimal x (one correct rounding)."""
    return float(x)


def ln(fr):
    """ln of a positive fraction, to 50 digits."""
    return D.ln(D.divide(decimal.Decimal(fr.numerator), decimal.Decimal(fr.denominator)))


def split(value):
    """value (a decimal) as hi, a multiple of 2^-32, and lo, the double
    nearest value - hi."""
    scale = 1 << 32
    hi = Fraction(round(Fraction(value) * scale), scale)
    lo = Fraction(value) - hi
    return float(hi), nearest(D.divide(decimal.Decimal(lo.numerator),
                                       decimal.Decimal(lo.denominator)))


def ln2_split():
    return split(ln(Fraction(2)))


def entries():
    for j in range(N + 1):
        F = Fraction(N + j, N)
        hi, lo = split(ln(F))
        yield j, float(1 / F), hi, lo


def header():
    hi, lo = ln2_split()
    rows = list(entries())
    out = ["// Generated by gen_log_table.py; do not edit.",
           "// Constants of the FP64 logarithm (log_tab in device_common.cuh):",
           "// ln 2 and ln F_j split as hi (a multiple of 2^-32) + lo, and the",
           "// breakpoints F_j = 1 + j/128 as {1/F_j, hi of ln F_j} and lo of ln F_j.",
           "#pragma once",
           "",
           "namespace cplbm {",
           "",
           "constexpr double LN2_HI = %s;" % hi.hex(),
           "constexpr double LN2_LO = %s;" % lo.hex(),
           "constexpr int LOG_TABLE_N = %d;" % N,
           "__device__ const double2 kLogTable[LOG_TABLE_N + 1] = {"]
    for j, inv, lh, _ in rows:
        out.append("    {%s, %s},  // %d" % (inv.hex(), lh.hex(), j))
    out += ["};", "__device__ const double kLogTableLo[LOG_TABLE_N + 1] = {"]
    for j, _, _, ll in rows:
        out.append("    %s,  // %d" % (ll.hex(), j))
    out += ["};", "", "}  // namespace cplbm", ""]
    return "\n".join(out)


if __name__ == "__main__":
    sys.stdout.write(header())
