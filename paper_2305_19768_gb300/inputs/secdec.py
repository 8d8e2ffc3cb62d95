"""Primary and iterative sector decomposition (input preparation).

The paper takes sector decomposition as given (its section on the program's
structure names the `geometric` and `iterative` strategies and delegates the
details to earlier pySecDec work); the integrator consumes the resulting
per-sector monomial tables. This module produces such tables for the
workloads the integrator is run on:

* primary sectors: x_k = 1, x_j = t_j in [0,1] for j != k (valid because the
  projective integrand of the Feynman representation is homogeneous of
  degree -N);
* iterative decomposition: while U (first) or else F vanishes identically on
  some set S of variables set to zero (the smallest such set, first in
  lexicographic order), split the sector into |S| subsectors
  t_j -> t_l t_j (j in S, j != l), factor the powers of t_l out of U and F,
  and accumulate the monomial prefactor prod_j t_j^{a_j + b_j eps}.
  Treating U before F (rather than their product) is what makes the
  recursion terminate for the planar double box (282 sectors).

Every finished sector has U and F with a non-zero constant term and a
monomial prefactor with integer a_j >= -1; variables with a_j = -1 are the
logarithmically singular ones that the integrator subtracts.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from typing import List

from .polynomial import LinPoly, minimal_vanishing_subset


@dataclass
class Sector:
    d: int
    a: List[int]
    b: List[Fraction]
    U: LinPoly
    F: LinPoly
    u0: Fraction
    u1: Fraction
    f0: Fraction
    f1: Fraction
    deform: bool = False
    origin: str = ""
    weight: int = 1          # constant factor of the sector (|det N| of a geometric sector)

    @property
    def singular(self) -> List[int]:
        """Variables with a_j <= -1 (subtracted endpoint singularities)."""
        return [j for j in range(self.d) if self.a[j] <= -1]


def _normalize(U: LinPoly, F: LinPoly, a, b, u0, u1, f0, f1):
    for j in range(U.nvars):
        ku = U.min_exponent(j)
        kf = F.min_exponent(j)
        if ku:
            U = U.divide_power(j, ku)
        if kf:
            F = F.divide_power(j, kf)
        a[j] += ku * u0 + kf * f0
        b[j] += ku * u1 + kf * f1
    return U, F


class DecompositionError(RuntimeError):
    pass


def decompose(U: LinPoly, F: LinPoly, u0, u1, f0, f1, *, deform=False, max_depth=40,
              max_sectors=20000) -> List[Sector]:
    """All finished sectors of U^{u0+u1 eps} F^{f0+f1 eps} over the simplex."""
    N = U.nvars
    out: List[Sector] = []

    def rec(Us, Fs, a, b, depth, origin):
        if depth > max_depth:
            raise DecompositionError(f"iterative decomposition exceeded depth {max_depth}")
        S = minimal_vanishing_subset([Us], Us.nvars)
        if S is None:
            S = minimal_vanishing_subset([Fs], Fs.nvars)
        if S is None:
            aa = []
            for j, x in enumerate(a):
                if Fraction(x).denominator != 1:
                    raise DecompositionError("non-integer monomial exponent")
                aa.append(int(x))
                if aa[-1] < -4:
                    raise DecompositionError(f"sector {origin}: exponent a_{j}={aa[-1]} < -4 "
                                             "needs subtraction beyond degree 3")
                if aa[-1] <= -1 and b[j] == 0:
                    raise DecompositionError(f"sector {origin}: unregulated singularity in t_{j}")
            out.append(Sector(Us.nvars, aa, [Fraction(x) for x in b], Us, Fs,
                              Fraction(u0), Fraction(u1), Fraction(f0), Fraction(f1),
                              deform, origin))
            if len(out) > max_sectors:
                raise DecompositionError("too many sectors")
            return
        for l in S:
            rest = [j for j in S if j != l]
            U2 = Us.rescale(l, rest)
            F2 = Fs.rescale(l, rest)
            a2 = list(a)
            b2 = list(b)
            a2[l] += len(rest) + sum(a[j] for j in rest)
            b2[l] += sum(b[j] for j in rest)
            U2, F2 = _normalize(U2, F2, a2, b2, u0, u1, f0, f1)
            rec(U2, F2, a2, b2, depth + 1, f"{origin}.{l}")

    for k in range(N):
        Uk = U.set_one(k)
        Fk = F.set_one(k)
        a = [Fraction(0)] * (N - 1)
        b = [Fraction(0)] * (N - 1)
        Uk, Fk = _normalize(Uk, Fk, a, b, u0, u1, f0, f1)
        rec(Uk, Fk, a, b, 0, f"p{k}")
    return out
