"""Algorithmic FP64 work per integrand evaluation (roofline numerator).

One evaluation = one lattice point of one sector for one shift, all eps
orders, all subtraction corners. The count follows the evaluator's
formulation of the method (Section "Kernels" of the design notes):

* +, -, x, division and reciprocal count 1 flop, a fused multiply-add 2;
* each transcendental counts a fixed algorithmic cost: log and exp 20
  flops, atan2 20, sincos 30 (a minimax polynomial of degree ~10 plus range
  reduction), independent of how a math library implements them;
* only the terms the requested orders need are counted: corner V carries
  its eps exponent (one log of U^u1 F^f1) only if hi + |V| >= 1, the ln t of
  a singular variable only if hi + ns - 1 >= 1, and so on.

The figure is per sector; workloads average it over their sectors.
"""
from __future__ import annotations

LOG = EXP = ATAN2 = 20
SINCOS = 30


def _monomial_flops(P) -> int:
    f = 0
    for e, _ in P.terms.items():
        nv = sum(1 for x in e if x)
        f += (nv - 1) + 2 if nv else 1
    return f


def sector_flops(sector, lo: int, norders: int, deform: bool = False) -> int:
    d = sector.d
    ns = len(sector.singular)
    hi = lo + norders - 1
    f = 0
    f += 2 * d                          # r / n and + delta
    f += 9 * d                          # korobov3 t
    f += 3 * d + 3                      # weight: u(1-u), product, cube, 140^d
    emax = max(sector.U.max_var_exponent(), sector.F.max_var_exponent(), 1)
    f += d * (emax - 1)                 # power table
    f += _monomial_flops(sector.U) + _monomial_flops(sector.F)
    f += 2 * ns * (1 << max(ns - 1, 0))  # subset sums of both polynomials
    u0, f0, u1, f1 = int(sector.u0), int(sector.f0), int(sector.u1), int(sector.f1)
    for V in range(1 << ns):
        nV = hi + bin(V).count("1") + 1
        f += (1 if f0 < 0 else 0) + (1 if u0 < 0 else 0) + max(abs(u0) + abs(f0) - 1, 0) + 1
        if nV > 1:
            f += max(abs(u1) + abs(f1) - 1, 0) + LOG + 1
            f += 2 * (nV - 1)           # corner series B Lambda^i / i!
    f += ns                              # 1/t of singular variables
    if hi + ns - 1 >= 1:
        f += ns * LOG
    need_lam = hi + ns >= 1
    for j in range(d):
        if sector.a[j] != -1 and sector.b[j] != 0 and need_lam:
            f += LOG + 2
    for q in range(ns):                  # superset Moebius transform
        for P in range(1 << ns):
            if not P & (1 << q):
                f += max(hi + bin(P).count("1") + 1, 0)
    for P in range(1 << ns):
        np_ = bin(P).count("1")
        nP = hi + np_ + 1
        if nP < 1:
            continue
        f += ns                          # A_P
        if nP > 1:
            f += 2 * (ns - np_) + 2 * (nP - 1)   # E_P and its series
        for k in range(max(0, lo + np_), nP):
            f += 2 * k                   # convolution term k
        f += 2 * min(norders, nP)        # res += A PE
    f += 2 * norders                     # weight x value into the accumulator
    if deform:
        f += 4 * d * d + 40              # J, z, rho
        f += 60                          # complex determinant (d <= 3)
        f += 4 * (len(sector.U) + len(sector.F)) * 2
        f += 10                          # complex reciprocal
    return f


def workload_flops(integral, lo: int, norders: int, deform: bool = False) -> float:
    """Mean FP64 flops per evaluation over the integral's sectors (equal lattices)."""
    fs = [sector_flops(s, lo, norders, deform) for s in integral.sectors]
    return sum(fs) / len(fs)
