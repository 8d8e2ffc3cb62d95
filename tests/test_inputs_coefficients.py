"""Coefficient strings (section "Weighted sums of integrals"): parsed,
evaluated at exact rational values and expanded in the regulator with exact
rationals. Checked against sympy's series expansion (an independent
implementation), against cancellations that floating point cannot survive,
and against the amplitude's polynomial coefficients."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2305_19768_gb300.inputs import coefficients as C
from paper_2305_19768_gb300.inputs import workloads as w

EXPRS = [
    "(s^2 - 3*t)/(s*t + 1)",
    "1/eps + 2 + eps",
    "(1+eps)^2/(eps*(1-2*eps))",
    "(s - t*eps)^3 / (eps^2 * (s + eps)) - 7/(2*eps)",
    "((s+t)/(s-t))^-2 * (1 - 4*eps + eps^2)",
    "s*t/((1-eps)*(1-2*eps)*(1-3*eps)) + 1.25e-1*s",
    "(eps^2 + s*eps)/(eps^3 - t*eps^2)",
]


@pytest.mark.parametrize("expr", EXPRS)
def test_series_matches_sympy(expr):
    sympy = pytest.importorskip("sympy")
    s_, t_, e_ = sympy.symbols("s t eps")
    vals = {"s": Fraction(7, 3), "t": Fraction(-5, 2)}
    order = 3
    lo, c = C.series(expr, vals, order)
    sexpr = sympy.sympify(expr.replace("^", "**"), locals={"s": s_, "t": t_, "eps": e_}, rational=True)
    sexpr = sexpr.subs({s_: sympy.Rational(7, 3), t_: sympy.Rational(-5, 2)})
    ser = sympy.series(sexpr, e_, 0, order + 1).removeO()
    for k in range(lo, order + 1):
        ref = sympy.Rational(ser.coeff(e_, k)) if k else sympy.Rational(ser.subs(e_, 0) if lo >= 0 else
                                                                        ser.coeff(e_, 0))
        got = c[k - lo] if 0 <= k - lo < len(c) else Fraction(0)
        assert Fraction(int(ref.p), int(ref.q)) == got, (expr, k, got, ref)
    # nothing below the leading order
    lead = min((k for k in range(-6, order + 1) if ser.coeff(e_, k) != 0), default=None)
    assert lead == lo


def test_exact_where_floating_point_cancels():
    assert C.series("(s + 1e20) - 1e20", {"s": 1}, 0) == (0, [Fraction(1)])
    x = Fraction(1, 3)
    lo, c = C.series("((s + 1e-12)^5 - s^5) / 1e-12", {"s": x}, 0)
    exact = ((x + Fraction(1, 10**12)) ** 5 - x ** 5) * 10**12
    assert lo == 0 and c[0] == exact
    # a denominator vanishing at eps = 0 only after cancellation raises the pole order
    assert C.leading_order("1/((s + eps)^2 - s^2)", {"s": 3}) == -1
    assert C.leading_order("s/(eps^2*(s-2))", {"s": 3}) == -2


def test_parse_errors():
    for bad in ("2*(s+", "s^t", "s $ t", "(s))", "s^(1/2)", "u + 1"):
        with pytest.raises((C.ParseError, KeyError)):
            C.series(bad, {"s": 1, "t": Fraction(1, 2)}, 0)
    assert C.series("s^t", {"s": 3, "t": -2}, 0) == (0, [Fraction(1, 9)])   # a constant integer exponent


def test_coefficient_array_rows_lists_and_dicts_and_the_amplitude_polynomials():
    coefs = w.amplitude_coefficients(10)
    pts = w.amplitude_grid(4, 4)
    rows_list = [[" + ".join(f"({c})*{m}" for c, m in zip(row, ("1", "s", "t", "s^2", "s*t", "t^2")))
                  for row in coefs]]
    rows_dict = [{i: r for i, r in enumerate(rows_list[0]) if i % 3 == 0}]
    vals = [{"s": float(p[0]), "t": float(p[1])} for p in pts]
    A = C.coefficient_array(rows_list, 10, vals, 0, 1)
    ref = w.amplitude_coefficient_values(pts, coefs)
    assert np.allclose(A[:, 0, :, 0].real, ref, rtol=1e-14, atol=1e-12)
    B = C.coefficient_array(rows_dict, 10, vals, 0, 1)
    assert np.array_equal(B[:, 0, ::3, 0], A[:, 0, ::3, 0])
    assert np.all(B[:, 0, [i for i in range(10) if i % 3], 0] == 0)
    # a pole below the requested lowest order is reported
    with pytest.raises(ValueError):
        C.coefficient_array([["1/eps"]], 1, [{}], 0, 1)
