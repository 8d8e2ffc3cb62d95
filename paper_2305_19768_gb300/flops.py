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


def sector_flops(sector, lo: int, norders: int) -> int:
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
    return f


CMUL = 6        # complex product: 2 FMA + 2 MUL (or 4 MUL + 2 ADD)
CFMA_REAL = 4   # real coefficient times complex value added in: 2 FMA


def _derivative_flops(P, d: int):
    """Real flops of all first and second derivatives of P at a real point
    (each derivative monomial: its products and one FMA with the coefficient)."""
    f = 0
    for e in P.terms:
        vars_ = [j for j in range(d) if e[j]]
        nv = len(vars_)
        f += nv * (max(nv - 2, 0) + 2)                       # dP/dt_j
        f += (nv * (nv + 1) // 2) * (max(nv - 3, 0) + 2)     # d2P/dt_j dt_k
    return f


def _complex_poly_flops(P) -> int:
    f = 0
    for e in P.terms:
        nv = sum(1 for x in e if x)
        f += max(nv - 1, 0) * CMUL + CFMA_REAL
    return f


def deformed_sector_flops(sector, lo: int, norders: int) -> int:
    """The deformed evaluator's formulation: korobov3 of u and of 1 - u; at
    each corner V the derivatives of F, the real matrix V_jk and det J in
    closed form, z and rho, U and F at z in complex arithmetic, the prefactor
    num/den with one complex reciprocal and, where the corner needs its eps
    exponent, one complex log of the product of its factors (a real log of
    the squared modulus and an atan2); then the assembly in complex
    arithmetic."""
    d = sector.d
    ns = len(sector.singular)
    hi = lo + norders - 1
    u0, f0, u1, f1 = int(sector.u0), int(sector.f0), int(sector.u1), int(sector.f1)
    f = 2 * d + 18 * d + 3 * d + 3       # lattice, korobov3 of u and 1 - u, weight
    f += ns + (ns * LOG if hi + ns - 1 >= 1 else 0)   # 1/t, ln t of singular variables
    per_corner = _derivative_flops(sector.F, d)
    per_corner += 4 * d * d + 3 * d      # V_jk, z, rho
    per_corner += {1: 0, 2: 5, 3: 26}.get(d, 26)      # det J (closed form)
    per_corner += _complex_poly_flops(sector.U) + _complex_poly_flops(sector.F)
    per_corner += 1                      # sign check
    nreg_a = sum(1 for j in range(d) if sector.a[j] > 0)
    per_corner += CMUL * (ns + abs(u0) + abs(f0) + nreg_a) + 6 + CMUL   # num/den, 1/den, num x (1/den)
    nb = sum(1 for j in range(d) if sector.b[j] != 0)
    lam_corner = CMUL * (nb + abs(u1) + abs(f1)) + CMUL + 6 + 2 + LOG + ATAN2 + 3
    for V in range(1 << ns):
        f += per_corner
        if hi + bin(V).count("1") >= 1:
            f += lam_corner
            f += 2 * CMUL * (hi + bin(V).count("1"))     # corner series B Lambda^i / i!
    # Moebius transform and pole-set assembly on complex values
    for q in range(ns):
        for P in range(1 << ns):
            if not P & (1 << q):
                f += 2 * max(hi + bin(P).count("1") + 1, 0)
    for P in range(1 << ns):
        np_ = bin(P).count("1")
        nP = hi + np_ + 1
        if nP < 1:
            continue
        f += ns
        if nP > 1:
            f += 2 * (ns - np_) + 2 * (nP - 1)
        for k in range(max(0, lo + np_), nP):
            f += 2 * k * 2
        f += 4 * min(norders, nP)
    f += 4 * norders
    return f


def workload_flops(integral, lo: int, norders: int, deform: bool = False) -> float:
    """Mean FP64 flops per evaluation over the integral's sectors (equal lattices)."""
    fs = [deformed_sector_flops(s, lo, norders) if deform else sector_flops(s, lo, norders)
          for s in integral.sectors]
    return sum(fs) / len(fs)
