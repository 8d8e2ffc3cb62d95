"""Write qmc_log_table.h: the table of the evaluator's fixed-point logarithm
(qmc_ilog.h; Tang, "Table-driven implementation of the logarithm function in
IEEE floating-point arithmetic", ACM TOMS 16 (1990)).

For j = 0..1024, F_j = 1 + j/1024, row j holds three 64-bit words:
    RN(2^63 / F_j),  RN(2^116 ln F_j) mod 2^64,  RN(2^116 ln F_j) div 2^64.
Values come from mpmath at 80 digits.

The same header carries the table of the evaluator's two-argument arctangent:
for j = 0..64, ATAN_HI[j] = RN(atan(j/64)), ATAN_LO[j] = RN(atan(j/64) -
ATAN_HI[j]), and pi/2, pi as (RN, RN(remainder)) pairs.

Usage: python make_log_table.py   (rewrites qmc_log_table.h beside it)
"""
import os

import mpmath as mp

mp.mp.dps = 80
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qmc_log_table.h")


def rn(x) -> float:
    """Round an mpf to the nearest double (ties to even)."""
    return float(mp.mpf(x))


def main():
    rows = []
    for j in range(1025):
        F = mp.mpf(1) + mp.mpf(j) / 1024
        inv = int(mp.nint(mp.mpf(2) ** 63 / F))
        L = int(mp.nint(mp.log(F) * mp.mpf(2) ** 116))
        rows.append((inv, L & (2 ** 64 - 1), L >> 64))
    ln2 = int(mp.nint(mp.log(2) * mp.mpf(2) ** 116))
    assert ln2 & (2 ** 64 - 1) == 0x9ABC9E3B39803F2F and ln2 >> 64 == 0xB17217F7D1CF7   # qmc_ilog.h
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
        fh.write("// Table of the evaluator's fixed-point logarithm (written by make_log_table.py).\n")
        fh.write("// Row j: RN(2^63/F_j), RN(2^116 ln F_j) low and high words; F_j = 1 + j/1024.\n")
        fh.write("#pragma once\n")
        fh.write("#define QMC_LOG_TABLE_ROWS 1025\n")
        fh.write("#define QMC_LOG_TABLE_INIT { \\\n")
        for inv, lo, hi in rows:
            fh.write(f"    {inv:#x}ULL, {lo:#x}ULL, {hi:#x}ULL, \\\n")
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
