"""Sparse polynomials in Feynman parameters whose coefficients are linear
forms in the kinematic invariants.

A polynomial P(x_0..x_{n-1}) is stored as ``{exponent tuple: coefficient}``
where each coefficient is a tuple ``(c_0, c_1, ..., c_k)`` of exact
``Fraction`` values meaning ``c_0 + c_1*inv_1 + ... + c_k*inv_k``.
Symanzik polynomials of one- and two-loop graphs with numeric masses are of
this form (U has numeric coefficients, F is linear in the Mandelstam
invariants), and so are all sector polynomials derived from them by the
substitutions of sector decomposition, which only relabel exponents.

This module is part of the input generators: it builds the monomial tables
that both the CUDA path and the CPU oracle read. It holds none of the
lattice-rule arithmetic.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations
from typing import Dict, Iterable, Tuple

Exp = Tuple[int, ...]
Coef = Tuple[Fraction, ...]


def _cadd(a: Coef, b: Coef) -> Coef:
    return tuple(x + y for x, y in zip(a, b))


def _cscale(a: Coef, s) -> Coef:
    return tuple(x * s for x in a)


def _czero(a: Coef) -> bool:
    return all(x == 0 for x in a)


class LinPoly:
    """Polynomial with linear-form coefficients (see module docstring)."""

    __slots__ = ("nvars", "ncoef", "terms")

    def __init__(self, nvars: int, ncoef: int, terms: Dict[Exp, Coef] | None = None):
        self.nvars = nvars
        self.ncoef = ncoef
        self.terms: Dict[Exp, Coef] = {}
        if terms:
            for e, c in terms.items():
                self._acc(tuple(e), tuple(Fraction(x) for x in c))

    # -- construction -----------------------------------------------------
    def _acc(self, e: Exp, c: Coef) -> None:
        assert len(e) == self.nvars and len(c) == self.ncoef
        if e in self.terms:
            s = _cadd(self.terms[e], c)
            if _czero(s):
                del self.terms[e]
            else:
                self.terms[e] = s
        elif not _czero(c):
            self.terms[e] = c

    @classmethod
    def monomial(cls, nvars: int, ncoef: int, exps: Iterable[int], coef: Iterable) -> "LinPoly":
        return cls(nvars, ncoef, {tuple(exps): tuple(coef)})

    def copy(self) -> "LinPoly":
        p = LinPoly(self.nvars, self.ncoef)
        p.terms = dict(self.terms)
        return p

    # -- arithmetic ---------------------------------------------------------
    def __add__(self, other: "LinPoly") -> "LinPoly":
        assert self.nvars == other.nvars and self.ncoef == other.ncoef
        p = self.copy()
        for e, c in other.terms.items():
            p._acc(e, c)
        return p

    def scale(self, s) -> "LinPoly":
        return LinPoly(self.nvars, self.ncoef, {e: _cscale(c, Fraction(s)) for e, c in self.terms.items()})

    def mul_numeric(self, other: "LinPoly") -> "LinPoly":
        """Product where ``other`` has purely numeric coefficients (c_1..c_k = 0).

        Keeping one factor numeric keeps the result linear in the invariants.
        """
        assert self.nvars == other.nvars
        p = LinPoly(self.nvars, self.ncoef)
        for e2, c2 in other.terms.items():
            if any(x != 0 for x in c2[1:]):
                raise ValueError("mul_numeric: second factor has invariant-dependent coefficients")
            for e1, c1 in self.terms.items():
                p._acc(tuple(a + b for a, b in zip(e1, e2)), _cscale(c1, c2[0]))
        return p

    # -- substitutions used by sector decomposition ------------------------
    def set_one(self, k: int) -> "LinPoly":
        """Substitute x_k = 1 and drop the variable (primary sectors)."""
        p = LinPoly(self.nvars - 1, self.ncoef)
        for e, c in self.terms.items():
            p._acc(e[:k] + e[k + 1:], c)
        return p

    def vanishes_at_zero(self, subset: Iterable[int]) -> bool:
        """True if P is identically zero when all variables in ``subset`` are 0."""
        s = tuple(subset)
        return not any(all(e[j] == 0 for j in s) for e in self.terms)

    def rescale(self, l: int, subset: Iterable[int]) -> "LinPoly":
        """Substitute t_j -> t_l * t_j for every j in ``subset`` (l not in subset)."""
        s = tuple(subset)
        p = LinPoly(self.nvars, self.ncoef)
        for e, c in self.terms.items():
            e2 = list(e)
            e2[l] += sum(e[j] for j in s)
            p._acc(tuple(e2), c)
        return p

    def min_exponent(self, j: int) -> int:
        return min(e[j] for e in self.terms)

    def divide_power(self, j: int, k: int) -> "LinPoly":
        """Divide by t_j^k (k must not exceed the minimal exponent of t_j)."""
        p = LinPoly(self.nvars, self.ncoef)
        for e, c in self.terms.items():
            e2 = list(e)
            e2[j] -= k
            assert e2[j] >= 0
            p._acc(tuple(e2), c)
        return p

    def has_constant_term(self) -> bool:
        return tuple([0] * self.nvars) in self.terms

    def degree(self) -> int:
        return max((sum(e) for e in self.terms), default=0)

    def max_var_exponent(self) -> int:
        return max((max(e) if e else 0 for e in self.terms), default=0)

    # -- evaluation (host side, used by tests of the generators only) -------
    def evaluate(self, x, inv=()):
        """Numeric value at real/complex point ``x`` with invariants ``inv``."""
        inv = tuple(inv)
        assert len(inv) == self.ncoef - 1
        total = 0
        for e, c in self.terms.items():
            cv = float(c[0]) + sum(float(ci) * v for ci, v in zip(c[1:], inv))
            m = cv
            for xj, ej in zip(x, e):
                if ej:
                    m = m * xj ** ej
            total = total + m
        return total

    def sorted_terms(self):
        return sorted(self.terms.items(), key=lambda kv: kv[0])

    def __len__(self) -> int:
        return len(self.terms)

    def __repr__(self) -> str:
        return f"LinPoly(nvars={self.nvars}, nterms={len(self.terms)})"


def minimal_vanishing_subset(polys, nvars: int):
    """Smallest variable subset (first in lexicographic order of each size)
    on which at least one polynomial in ``polys`` vanishes identically, or None.
    """
    for size in range(1, nvars + 1):
        for s in combinations(range(nvars), size):
            if any(p.vanishes_at_zero(s) for p in polys):
                return s
    return None
