"""Feynman-parameter representation of scalar loop integrals.

Convention (the paper delegates it to the earlier pySecDec papers; this is
the standard one): propagators 1/(q_e^2 - m_e^2 + i0) with unit powers,
integration measure d^D l / (i pi^{D/2}) per loop, D = D0 - 2 eps, and

    I = (-1)^N Gamma(N - L D/2) Int_{x>=0} delta(1 - sum x)
            U^{N-(L+1)D/2} (F - i0)^{-(N - L D/2)},

    U = sum over spanning trees T of prod_{e not in T} x_e,
    F = - sum over 2-forests (T1, T2) of (p_T1)^2 prod_{e not in T1+T2} x_e
        + U sum_e m_e^2 x_e,

with p_T1 the external momentum flowing into T1. With this sign the
Euclidean region has F > 0. No exp(gamma_E eps) factor is included.

Exponents in the D0 - 2 eps expansion:
    U^{u0 + u1 eps}:  u0 = N - (L+1) D0/2,  u1 = L + 1
    F^{f0 + f1 eps}:  f0 = -(N - L D0/2),   f1 = -L
and the prefactor (-1)^N Gamma(N - L D0/2 + L eps).

This module is an input generator: it produces polynomials and a numeric
prefactor series that both the CUDA path and the CPU oracle consume.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from itertools import combinations
from typing import Callable, FrozenSet, List, Sequence, Tuple

from .polynomial import Coef, LinPoly


@dataclass
class Kinematics:
    """External kinematics: invariant names and the map leg-subset -> (sum p)^2.

    ``square`` returns the linear form (c_0, c_1..c_k) of (sum_{i in A} p_i)^2
    in the invariants. Legs are numbered 0..E-1.
    """

    invariants: List[str]
    nlegs: int
    square: Callable[[FrozenSet[int]], Coef]

    @property
    def ncoef(self) -> int:
        return 1 + len(self.invariants)


def kin_numeric_3pt(p1sq, p2sq, p3sq) -> Kinematics:
    """Three-point kinematics with fixed numeric p_i^2 (no free invariants)."""
    psq = [Fraction(p1sq), Fraction(p2sq), Fraction(p3sq)]

    def square(legs: FrozenSet[int]) -> Coef:
        legs = frozenset(legs)
        if len(legs) in (0, 3):
            return (Fraction(0),)
        if len(legs) == 2:
            legs = frozenset({0, 1, 2}) - legs
        (i,) = tuple(legs)
        return (psq[i],)

    return Kinematics([], 3, square)


def kin_massless_4pt() -> Kinematics:
    """Four massless legs, invariants s=(p0+p1)^2, t=(p1+p2)^2, u=-s-t."""

    def square(legs: FrozenSet[int]) -> Coef:
        legs = frozenset(legs)
        if len(legs) > 2:
            legs = frozenset(range(4)) - legs
        if len(legs) <= 1:
            return (Fraction(0), Fraction(0), Fraction(0))
        if legs in (frozenset({0, 1}), frozenset({2, 3})):
            return (Fraction(0), Fraction(1), Fraction(0))
        if legs in (frozenset({1, 2}), frozenset({0, 3})):
            return (Fraction(0), Fraction(0), Fraction(1))
        return (Fraction(0), Fraction(-1), Fraction(-1))  # u = -s - t

    return Kinematics(["s", "t"], 4, square)


def _unit(names, which) -> Coef:
    return (Fraction(0),) + tuple(Fraction(1 if n == which else 0) for n in names)


def kin_2pt(name: str, names=None) -> Kinematics:
    """Two-point kinematics p^2 = <name>, over the invariant list ``names``
    (default: just <name>)."""
    names = list(names) if names else [name]
    one, zero = _unit(names, name), (Fraction(0),) * (len(names) + 1)

    def square(legs: FrozenSet[int]) -> Coef:
        return one if len(frozenset(legs)) == 1 else zero

    return Kinematics(names, 2, square)


def kin_3pt_one_offshell(name: str, names=None) -> Kinematics:
    """Three-point kinematics with p_0^2 = <name>, p_1^2 = p_2^2 = 0."""
    names = list(names) if names else [name]
    one, zero = _unit(names, name), (Fraction(0),) * (len(names) + 1)

    def square(legs: FrozenSet[int]) -> Coef:
        legs = frozenset(legs)
        if len(legs) == 2:
            legs = frozenset({0, 1, 2}) - legs
        return one if legs == frozenset({0}) else zero

    return Kinematics(names, 3, square)


@dataclass
class Graph:
    """Loop graph: internal edges (vertex pairs, numeric m^2) and external legs
    (the vertex each leg attaches to, in leg order)."""

    edges: List[Tuple[int, int]]
    masses_sq: List[Fraction]
    legs: List[int]
    kin: Kinematics
    name: str = "graph"

    @property
    def nvertices(self) -> int:
        vs = set()
        for a, b in self.edges:
            vs.add(a)
            vs.add(b)
        vs.update(self.legs)
        return len(vs)

    @property
    def nloops(self) -> int:
        return len(self.edges) - self.nvertices + 1


def _components(nv: int, edges: Sequence[Tuple[int, int]]) -> List[int]:
    parent = list(range(nv))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    return [find(v) for v in range(nv)]


def symanzik(graph: Graph) -> Tuple[LinPoly, LinPoly]:
    """First and second Symanzik polynomials U, F of ``graph`` (see module doc)."""
    E = len(graph.edges)
    nv = graph.nvertices
    ncoef = graph.kin.ncoef
    U = LinPoly(E, ncoef)
    F0 = LinPoly(E, ncoef)
    one = (Fraction(1),) + (Fraction(0),) * (ncoef - 1)
    for forest_size, ncomp in ((nv - 1, 1), (nv - 2, 2)):
        if forest_size < 0:
            continue
        for sub in combinations(range(E), forest_size):
            comp = _components(nv, [graph.edges[e] for e in sub])
            roots = sorted(set(comp))
            if len(roots) != ncomp:
                continue  # contains a cycle (fewer edges than needed to span)
            exps = tuple(0 if e in sub else 1 for e in range(E))
            if ncomp == 1:
                U._acc(exps, one)
            else:
                r1 = roots[0]
                legs_in_1 = frozenset(i for i, v in enumerate(graph.legs) if comp[v] == r1)
                sq = graph.kin.square(legs_in_1)
                F0._acc(exps, tuple(-x for x in sq))
    mass_poly = LinPoly(E, ncoef)
    for e, m2 in enumerate(graph.masses_sq):
        if m2 != 0:
            mass_poly._acc(tuple(1 if k == e else 0 for k in range(E)),
                           (Fraction(m2),) + (Fraction(0),) * (ncoef - 1))
    F = F0 + U.mul_numeric(mass_poly) if len(mass_poly) else F0
    return U, F


def exponents(N: int, L: int, D0: int):
    """(u0, u1, f0, f1) of U^{u0+u1 eps} F^{f0+f1 eps} for D = D0 - 2 eps."""
    u0 = Fraction(N) - Fraction((L + 1) * D0, 2)
    f0 = -(Fraction(N) - Fraction(L * D0, 2))
    return u0, Fraction(L + 1), f0, Fraction(-L)


def _exp_series(c: List[float], order: int) -> List[float]:
    """Coefficients of exp(sum_{k>=1} c[k] x^k) up to x^order (c[0] ignored)."""
    out = [0.0] * (order + 1)
    out[0] = 1.0
    # a_n = (1/n) sum_{k=1}^{n} k c_k a_{n-k}
    for nn in range(1, order + 1):
        out[nn] = sum(k * c[k] * out[nn - k] for k in range(1, nn + 1)) / nn
    return out


def gamma_series(a: int, scale: int, order: int):
    """Laurent series of Gamma(a + scale*eps) for integer ``a``.

    Returns (lowest_order, coefficients) with coefficients of eps^lo .. eps^order.
    Uses Gamma(1+x) = exp(-gamma x + sum_{k>=2} (-1)^k zeta(k) x^k / k) and the
    recurrence Gamma(a+x) = Gamma(1+x) * prod (shifts).
    """
    from scipy.special import zeta

    nmax = order + 4
    c = [0.0] * (nmax + 1)
    c[1] = -0.57721566490153286061
    for k in range(2, nmax + 1):
        c[k] = (-1) ** k * float(zeta(k)) / k
    g1 = _exp_series(c, nmax)  # Gamma(1+x) in x
    # Gamma(a+x) = Gamma(1+x) * R(x):
    #   a >= 1: R = prod_{j=1}^{a-1} (j + x)
    #   a <= 0: R = 1 / prod_{j=a}^{0} (j + x)   (contains 1/x)
    poly = [1.0]
    lo = 0
    if a >= 1:
        # multiply by (j + x) successively
        for j in range(1, a):
            new = [0.0] * (len(poly) + 1)
            for i, p in enumerate(poly):
                new[i] += j * p
                new[i + 1] += p
            poly = new
        ser = [0.0] * (nmax + 1)
        for i, p in enumerate(poly):
            for k in range(nmax + 1 - i):
                ser[i + k] += p * g1[k]
    else:
        # 1/x * prod_{j=a}^{-1} 1/(j + x);  1/(j+x) = (1/j) sum (-x/j)^k
        inv = [0.0] * (nmax + 1)
        inv[0] = 1.0
        for j in range(a, 0):
            term = [(1.0 / j) * (-1.0 / j) ** k for k in range(nmax + 1)]
            new = [0.0] * (nmax + 1)
            for i in range(nmax + 1):
                if inv[i] == 0.0:
                    continue
                for k in range(nmax + 1 - i):
                    new[i + k] += inv[i] * term[k]
            inv = new
        ser = [0.0] * (nmax + 1)
        for i in range(nmax + 1):
            for k in range(nmax + 1 - i):
                ser[i + k] += inv[i] * g1[k]
        lo = -1
    # substitute x = scale*eps: coefficient of x^i (times x^lo) -> scale^(i+lo) eps^(i+lo)
    coeffs = []
    for i in range(order - lo + 1):
        coeffs.append(ser[i] * float(scale) ** (i + lo))
    return lo, coeffs


def prefactor_series(N: int, L: int, D0: int, order: int):
    """(-1)^N Gamma(N - L D0/2 + L eps) as (lowest order, real coefficients)."""
    a2 = 2 * N - L * D0
    if a2 % 2:
        raise ValueError("odd D0 (half-integer Gamma arguments) not supported")
    lo, coeffs = gamma_series(a2 // 2, L, order)
    sign = -1.0 if N % 2 else 1.0
    return lo, [sign * x for x in coeffs]


def gamma_series_check(a: int, scale: int, order: int) -> float:
    """Largest deviation of ``gamma_series`` from math.gamma at a few small eps
    (a self-check used by the input tests)."""
    lo, cs = gamma_series(a, scale, order)
    worst = 0.0
    for eps in (1e-3, -2e-3, 3e-3):
        approx = sum(c * eps ** (lo + i) for i, c in enumerate(cs))
        exact = math.gamma(a + scale * eps)
        worst = max(worst, abs(approx - exact) / abs(exact))
    return worst
