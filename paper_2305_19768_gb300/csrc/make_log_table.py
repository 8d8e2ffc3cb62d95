"""Write qmc_log_table.h: the table of the evaluator's table-driven FP64
logarithm (Tang, "Table-driven implementation of the logarithm function in
IEEE floating-point arithmetic", ACM TOMS 16 (1990)).

For j = 0..1024, F_j = 1 + j/1024 and
    INVF[j]          = RN(1/F_j)
    LOGF_HI[j]       = ln(F_j) rounded to a multiple of 2^-42
    LOGF_LO[j]       = RN(ln(F_j) - LOGF_HI[j])
and LN2_HI = ln 2 rounded to a multiple of 2^-42, LN2_LO = RN(ln 2 - LN2_HI).
Rounding the leading parts to the 2^-42 grid makes e * LN2_HI + LOGF_HI[j]
exact for every binary exponent |e| < 2^10. Values come from mpmath at 60
digits and are written as C99 hexadecimal floating constants.

The same header carries the table of the evaluator's two-argument arctangent:
for j = 0..64, ATAN_HI[j] = RN(atan(j/64)), ATAN_LO[j] = RN(atan(j/64) -
ATAN_HI[j]), and pi/2, pi as (RN, RN(remainder)) pairs.

Usage: python make_log_table.py   (rewrites qmc_log_table.h beside it)
"""
import os

import mpmath as mp

mp.mp.dps = 60
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qmc_log_table.h")


def rn(x) -> float:
    """Round an mpf to the nearest double (ties to even)."""
    return float(mp.mpf(x))


def grid42(x) -> float:
    return float(mp.nint(mp.mpf(x) * 2 ** 42) / 2 ** 42)


def main():
    rows = []
    for j in range(1025):
        F = mp.mpf(1) + mp.mpf(j) / 1024
        L = mp.log(F)
        hi = grid42(L)
        lo = rn(L - mp.mpf(hi))
        rows.append((rn(1 / F), hi, lo))
    ln2 = mp.log(2)
    ln2_hi = grid42(ln2)
    ln2_lo = rn(ln2 - mp.mpf(ln2_hi))
    atan_rows = []
    for j in range(65):
        a = mp.atan(mp.mpf(j) / 64)
        ah = rn(a)
        atan_rows.append((ah, rn(a - mp.mpf(ah))))
    pio2 = mp.pi / 2
    pio2_hi = rn(pio2)
    pio2_lo = rn(pio2 - mp.mpf(pio2_hi))
    pi_hi = rn(mp.pi)
    pi_lo = rn(mp.pi - mp.mpf(pi_hi))
    with open(OUT, "w") as fh:
        fh.write("// Table of the evaluator's FP64 logarithm (written by make_log_table.py).\n")
        fh.write("// Row j: RN(1/F_j), ln(F_j) on the 2^-42 grid, RN(remainder); F_j = 1 + j/1024.\n")
        fh.write("#pragma once\n")
        fh.write(f"#define QMC_LN2_HI {ln2_hi.hex()}\n#define QMC_LN2_LO {ln2_lo.hex()}\n")
        fh.write("#define QMC_LOG_TABLE_ROWS 1025\n")
        fh.write("#define QMC_LOG_TABLE_INIT { \\\n")
        for inv, hi, lo in rows:
            fh.write(f"    {inv.hex()}, {hi.hex()}, {lo.hex()}, \\\n")
        fh.write("}\n")
        fh.write("// Row j: RN(atan(j/64)), RN(remainder).\n")
        fh.write(f"#define QMC_PIO2_HI {pio2_hi.hex()}\n#define QMC_PIO2_LO {pio2_lo.hex()}\n")
        fh.write(f"#define QMC_PI_HI {pi_hi.hex()}\n#define QMC_PI_LO {pi_lo.hex()}\n")
        fh.write("#define QMC_ATAN_TABLE_ROWS 65\n")
        fh.write("#define QMC_ATAN_TABLE_INIT { \\\n")
        for hi, lo in atan_rows:
            fh.write(f"    {hi.hex()}, {lo.hex()}, \\\n")
        fh.write("}\n")


if __name__ == "__main__":
    main()
