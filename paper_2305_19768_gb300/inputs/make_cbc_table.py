"""Write ``cbc_table.txt``: fast-CBC generating vectors (d = 6) for a ladder of
prime lattice sizes from 10^3 to 10^8.

Sizes: the next prime at or above m * 10^k for m in {1, 1.25, 1.6, 2, 2.5,
3.2, 4, 5, 6.4, 8} and k = 3..7, plus 10^8. Because CBC builds the vector
component by component, the first d entries of a row are the d-dimensional
CBC vector for that n.

Usage: python -m paper_2305_19768_gb300.inputs.make_cbc_table [--max N]
"""
from __future__ import annotations

import argparse
import time

from .lattice import DMAX_TABLE, TABLE_PATH, cbc_fast, next_prime, worst_case_error_sq

MULTIPLIERS = (1.0, 1.25, 1.6, 2.0, 2.5, 3.2, 4.0, 5.0, 6.4, 8.0)


def ladder(nmax: int):
    sizes = []
    for k in range(3, 8):
        for m in MULTIPLIERS:
            sizes.append(next_prime(int(round(m * 10 ** k))))
    sizes.append(next_prime(10 ** 8))
    return sorted(set(s for s in sizes if s <= nmax))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max", type=int, default=10 ** 8 + 100)
    args = ap.parse_args()
    rows = []
    for n in ladder(args.max):
        t0 = time.time()
        z = cbc_fast(n, DMAX_TABLE)
        e2 = worst_case_error_sq(n, z) if n <= 2_000_000 else float("nan")
        rows.append((n, z))
        print(f"n={n} z={z} e2={e2:.3e} {time.time() - t0:.1f}s", flush=True)
    with open(TABLE_PATH, "w") as fh:
        fh.write("# n z_1 ... z_6 : fast-CBC rank-1 lattice generating vectors, Korobov space\n")
        fh.write("# smoothness 2, product weights gamma_j = 1 (written by make_cbc_table.py)\n")
        for n, z in rows:
            fh.write(" ".join(str(v) for v in (n, *z)) + "\n")


if __name__ == "__main__":
    main()
