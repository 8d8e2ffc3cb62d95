"""Algorithmic FP64 work per integrand evaluation (roofline numerator).

One evaluation = one lattice point of one sector for one shift, all eps
orders, all subtraction corners. The count follows the evaluator's
formulation of the method and charges:

* +, -, x as 1 flop, fused multiply-add as 2, a division as 1;
* each library transcendental at a fixed algorithmic cost: log, exp and
  atan2 20 flops, sincos 30 (a minimax polynomial of degree ~10 plus range
  reduction), so that the figure does not depend on how the GPU's math
  library happens to implement them.

The count is per sector (it depends on d, the singular variables, the
monomial tables and the number of eps orders) and averaged over the
sectors of a workload weighted by their lattice points.
"""
from __future__ import annotations

LOG = EXP = ATAN2 = 20
SINCOS = 30


def sector_flops(sector, lo: int, norders: int, deform: bool = False) -> int:
    d = sector.d
    ns = len(sector.singular)
    hi = lo + norders - 1
    L = hi + ns + 1
    f = 0
    f += 2 * d                     # r / n, + delta
    f += d * (2 + 6)               # korobov3 t (u^2, u^4, three fma, one mul)
    f += d * (5 + 1)               # weight 140 u^3 (1-u)^3 and the product W
    emax = max(max(sector.U.max_var_exponent(), sector.F.max_var_exponent()), 1)
    f += d * max(emax - 1, 0)      # power table
    for P in (sector.U, sector.F):
        for e, _ in P.terms.items():
            f += sum(1 for x in e if x) + 1   # products + accumulation
    f += 2 * ns * (1 << max(ns - 1, 0))     # subset sums of the corner polynomials
    corners = 1 << ns
    per_corner = 0
    need_log = L > 1
    if need_log:
        per_corner += (LOG + 2) * (1 if sector.u1 else 0) + (LOG + 2) * (1 if sector.f1 else 0)
    per_corner += abs(int(sector.u0)) + abs(int(sector.f0)) + 2   # integer powers, one division
    f += corners * per_corner
    f += ns * (1 + (LOG if need_log else 0))   # 1/t and ln t of singular variables
    # regular variables with eps exponents
    for j in range(d):
        if sector.a[j] != -1 and sector.b[j] != 0 and need_log:
            f += LOG + 2
    # assembly: for each pole set P, D_P over supersets (L terms each), exp series, convolution
    for P in range(corners):
        npop = bin(P).count("1")
        sup = 1 << (ns - npop)
        f += sup * (1 + 3 * (L - 1))
        f += 2 * ns + 3 * (L - 1)
        f += L * (L + 1)  # convolution (fma per term)
        f += 2 * norders
    f += 2 * norders               # weight x value into the accumulator
    if deform:
        f += 4 * d * d + 40            # J, z, rho
        f += 60                        # complex determinant (d <= 3)
        f += 4 * (len(sector.U) + len(sector.F)) * 2
        f += 10                        # complex reciprocal
    return f


def workload_flops(integral, lo: int, norders: int, deform: bool = False) -> float:
    """Mean FP64 flops per evaluation over the integral's sectors (equal lattices)."""
    fs = [sector_flops(s, lo, norders, deform) for s in integral.sectors]
    return sum(fs) / len(fs)
