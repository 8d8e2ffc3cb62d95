"""Amplitude coefficients given as arithmetic expressions (section "Weighted
sums of integrals": coefficient strings, evaluated at the user's values with
arbitrary-precision rationals and expanded into a series in the regulator).

A coefficient is a string over
- numbers (integers, decimals, exponent notation; all read exactly);
- the invariant names and the regulator (`eps` by default);
- + - * / ^ (or **, integer exponents), unary minus and parentheses.

`series(expr, values, order)` substitutes exact rational values for the
invariants and returns the Laurent series in the regulator with exact
rational coefficients:
    (lowest order, [c_lo, c_lo+1, ..., c_order]).
The value is kept exactly as a rational function of the regulator and
expanded at the end, so a denominator that vanishes at eps = 0 raises the pole
order, as it must. `leading_order(expr, values)` is the lowest order (the
leading pole), which fixes how deep the integrals must be expanded.

A coefficient matrix row is either a list over all integrals or a dict
{integral index: expression} (missing entries are zero). `coefficient_array`
turns rows at many kinematic points into the C-ABI's coef[npoints][namp][nint]
[ncoef] array of complex doubles (the exact rationals rounded once, at the
end).

This is input preparation on the host; no part of it runs in the integrand.
"""
from __future__ import annotations

import re
from fractions import Fraction
from typing import Dict, List, Sequence, Tuple, Union

import numpy as np

Series = Tuple[int, List[Fraction]]   # (lowest order, coefficients from there up)

_TOKEN = re.compile(r"\s*(?:(\d+\.?\d*(?:[eE][+-]?\d+)?|\.\d+(?:[eE][+-]?\d+)?)|([A-Za-z_]\w*)|(\*\*|[-+*/^()]))")


class ParseError(ValueError):
    pass


def _tokens(text: str):
    pos, out = 0, []
    text = text.strip()
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            raise ParseError(f"unexpected character at {pos}: {text[pos:pos + 10]!r}")
        num, name, op = m.groups()
        if num is not None:
            out.append(("num", Fraction(num)))
        elif name is not None:
            out.append(("name", name))
        else:
            out.append(("op", "^" if op == "**" else op))
        pos = m.end()
    out.append(("end", None))
    return out


class _Parser:
    """Recursive descent: sum := term (('+'|'-') term)*; term := unary (('*'|'/') unary)*;
    unary := ('-'|'+') unary | power; power := atom ('^' unary)?; atom := number | name | '(' sum ')'."""

    def __init__(self, text: str):
        self.t = _tokens(text)
        self.i = 0

    def peek(self):
        return self.t[self.i]

    def take(self):
        tok = self.t[self.i]
        self.i += 1
        return tok

    def expect(self, op):
        tok = self.take()
        if tok != ("op", op):
            raise ParseError(f"expected {op!r}, got {tok[1]!r}")

    def parse(self):
        node = self.sum()
        if self.peek()[0] != "end":
            raise ParseError(f"trailing input at token {self.peek()[1]!r}")
        return node

    def sum(self):
        node = self.term()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()[1]
            node = (op, node, self.term())
        return node

    def term(self):
        node = self.unary()
        while self.peek() in (("op", "*"), ("op", "/")):
            op = self.take()[1]
            node = (op, node, self.unary())
        return node

    def unary(self):
        if self.peek() == ("op", "-"):
            self.take()
            return ("neg", self.unary())
        if self.peek() == ("op", "+"):
            self.take()
            return self.unary()
        return self.power()

    def power(self):
        base = self.atom()
        if self.peek() == ("op", "^"):
            self.take()
            return ("^", base, self.unary())
        return base

    def atom(self):
        kind, val = self.take()
        if kind == "num":
            return ("num", val)
        if kind == "name":
            return ("name", val)
        if (kind, val) == ("op", "("):
            node = self.sum()
            self.expect(")")
            return node
        raise ParseError(f"unexpected token {val!r}")


def parse(text: str):
    return _Parser(text).parse()


# ---------------------------------------------------------------- exact rational functions of eps
# With the invariants substituted, every coefficient is a rational function of
# the regulator: kept exactly as numerator / denominator polynomials (lists of
# Fractions, index = power of eps), reduced by their gcd, and expanded into a
# Laurent series only at the end, so that nothing is truncated early.
Poly = List[Fraction]


def _strip(p: Poly) -> Poly:
    while p and p[-1] == 0:
        p = p[:-1]
    return p


def _padd(a: Poly, b: Poly) -> Poly:
    n = max(len(a), len(b))
    return _strip([(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)])


def _pmul(a: Poly, b: Poly) -> Poly:
    if not a or not b:
        return []
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return _strip(out)


def _pdivmod(a: Poly, b: Poly):
    a = list(a)
    q = [Fraction(0)] * max(len(a) - len(b) + 1, 1)
    while len(_strip(a)) >= len(b) and _strip(a):
        a = _strip(a)
        k = len(a) - len(b)
        c = a[-1] / b[-1]
        q[k] = c
        for i, y in enumerate(b):
            a[i + k] -= c * y
    return _strip(q), _strip(a)


def _pgcd(a: Poly, b: Poly) -> Poly:
    while b:
        _, r = _pdivmod(a, b)
        a, b = b, r
    return [c / a[-1] for c in a] if a else [Fraction(1)]


def _norm(n: Poly, d: Poly):
    n, d = _strip(n), _strip(d)
    if not d:
        raise ZeroDivisionError("division by zero")
    if not n:
        return [], [Fraction(1)]
    g = _pgcd(n, d)
    if len(g) > 1:
        n, _ = _pdivmod(n, g)
        d, _ = _pdivmod(d, g)
    c = d[-1]
    return [x / c for x in n], [x / c for x in d]


def _eval(node, values: Dict[str, Fraction], reg: str):
    kind = node[0]
    if kind == "num":
        return _strip([node[1]]), [Fraction(1)]
    if kind == "name":
        if node[1] == reg:
            return [Fraction(0), Fraction(1)], [Fraction(1)]
        if node[1] not in values:
            raise KeyError(f"no value for {node[1]!r}")
        return _strip([Fraction(values[node[1]])]), [Fraction(1)]
    if kind == "neg":
        n, d = _eval(node[1], values, reg)
        return [-x for x in n], d
    if kind == "^":
        e_n, e_d = _eval(node[2], values, reg)
        if len(e_d) != 1 or len(e_n) > 1 or (e_n and e_n[0].denominator != 1):
            raise ParseError("exponents must be integer constants")
        p = int(e_n[0] / e_d[0]) if e_n else 0
        bn, bd = _eval(node[1], values, reg)
        if p < 0:
            bn, bd, p = bd, bn, -p
        n, d = [Fraction(1)], [Fraction(1)]
        while p:
            if p & 1:
                n, d = _pmul(n, bn), _pmul(d, bd)
            bn, bd = _pmul(bn, bn), _pmul(bd, bd)
            p >>= 1
        return _norm(n, d)
    n1, d1 = _eval(node[1], values, reg)
    n2, d2 = _eval(node[2], values, reg)
    if kind == "+":
        return _norm(_padd(_pmul(n1, d2), _pmul(n2, d1)), _pmul(d1, d2))
    if kind == "-":
        return _norm(_padd(_pmul(n1, d2), [-x for x in _pmul(n2, d1)]), _pmul(d1, d2))
    if kind == "*":
        return _norm(_pmul(n1, n2), _pmul(d1, d2))
    if kind == "/":
        return _norm(_pmul(n1, d2), _pmul(d1, n2))
    raise ParseError(f"unknown node {kind}")


def rational_function(expr: Union[str, tuple], values, regulator: str = "eps"):
    """(numerator, denominator) polynomials in the regulator, exact, reduced."""
    node = parse(expr) if isinstance(expr, str) else expr
    return _eval(node, {k: Fraction(v) for k, v in values.items()}, regulator)


def series(expr: Union[str, tuple], values: Dict[str, Union[Fraction, float, int, str]], order: int,
           regulator: str = "eps") -> Series:
    """Exact Laurent series of `expr` in the regulator up to `order` (inclusive),
    with the invariants set to `values` (read exactly: floats by their binary
    value, strings as decimals or fractions)."""
    n, d = rational_function(expr, values, regulator)
    if not n:
        return (order + 1, [])
    vn = next(i for i, x in enumerate(n) if x)
    vd = next(i for i, x in enumerate(d) if x)
    nh, dh = n[vn:], d[vd:]
    lo = vn - vd
    cnt = order - lo + 1
    if cnt <= 0:
        return (lo, [])
    out = []
    for k in range(cnt):                 # nh / dh as a power series (dh[0] != 0)
        acc = nh[k] if k < len(nh) else Fraction(0)
        for j in range(1, min(k, len(dh) - 1) + 1):
            acc -= dh[j] * out[k - j]
        out.append(acc / dh[0])
    return lo, out


def leading_order(expr: str, values, regulator: str = "eps") -> int:
    """Lowest order of the coefficient's series in the regulator (its leading pole)."""
    n, d = rational_function(expr, values, regulator)
    if not n:
        raise ValueError("the coefficient vanishes identically")
    return next(i for i, x in enumerate(n) if x) - next(i for i, x in enumerate(d) if x)


def coefficient_array(rows: Sequence[Sequence[Union[Sequence[str], Dict[int, str]]]], nint: int,
                      points: Sequence[Dict[str, object]], lowest: int, ncoef: int,
                      regulator: str = "eps") -> np.ndarray:
    """coef[npoints][namp][nint][ncoef] (complex128) of orders lowest..lowest+ncoef-1
    for amplitude rows given per point as lists or {integral: expression} dicts
    (`rows` has one entry per amplitude; every row applies at every point)."""
    out = np.zeros((len(points), len(rows), nint, ncoef), dtype=np.complex128)
    parsed = []
    for row in rows:
        items = row.items() if isinstance(row, dict) else enumerate(row)
        parsed.append([(int(i), parse(e)) for i, e in items if not (isinstance(e, str) and e.strip() == "0")])
    hi = lowest + ncoef - 1
    for p, vals in enumerate(points):
        for k, row in enumerate(parsed):
            for i, node in row:
                if not 0 <= i < nint:
                    raise IndexError(f"integral index {i} out of range")
                lo, c = series(node, vals, hi, regulator)
                if c and lo < lowest:
                    raise ValueError(f"coefficient of integral {i} has a pole of order {-lo} below {lowest}")
                for o, v in enumerate(c):
                    if lowest <= lo + o <= hi:
                        out[p, k, i, lo + o - lowest] = float(v)
    return out


def coefficient_series(rows, nint: int, points: Sequence[Dict[str, object]], highest: int,
                       regulator: str = "eps"):
    """(coef array, lowest order) for the C-ABI's qmc_sum_spec: the lowest order
    is the deepest leading pole over all entries and points (it decides how
    far the integrals are expanded), the array runs from there to `highest`."""
    lo = highest
    for row in rows:
        items = row.values() if isinstance(row, dict) else row
        for e in items:
            if isinstance(e, str) and e.strip() == "0":
                continue
            for vals in points:
                try:
                    lo = min(lo, leading_order(e, vals, regulator))
                except ValueError:
                    pass            # vanishes at this point
    return coefficient_array(rows, nint, points, lo, highest - lo + 1, regulator), lo
