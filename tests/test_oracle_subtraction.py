"""Pins of the oracle's Taylor subtraction for endpoint singularities
t_j^{-p + b_j eps} with p >= 2 (a_j <= -2), in one to four singular variables.

Two independent checks:
- pointwise: the oracle's eps-expanded integrand at interior points against
  the same subtracted integrand built by exact symbolic differentiation
  (sympy) and expanded in eps by high-precision numerical Taylor expansion
  (mpmath). Per singular variable t_q the subtraction applies
      g -> t^{-p+b eps} g(t) + sum_{k<p} g_k [1/(k - p + 1 + b eps) - t^{k-p+b eps}],
  g_k the k-th Taylor coefficient at t_q = 0; in several variables the
  operators are applied one variable after the other. No jets, no binomial
  series, no enumeration of corner states: a slip in any of those in the
  oracle shows here.
- integrated: polynomial G, whose sector integral is the exact finite sum
  sum_k c_k prod_q 1/(k_q - p_q + 1 + b_q eps), through the randomized
  lattice rule with the baker transform.

Why baker: the subtracted integrand t^{-p}(g - sum_{k<p} g_k t^k) cancels
p orders of t near the border, so its FP64 value carries an error of about
2^-53 |g| t^{-p}. Under korobov3 (t ~ 35 u^4, weight ~ 140 u^3) that is
2^-53 u^{3-4p} per unit of u at the smallest lattice coordinates: for p = 2
at n ~ 10^4 the eps^0 estimate is off by O(10^2) and its shift spread is as
large, so a within-n-sigma check is empty. Under the tent map (t = 2u,
weight 1) it is 2^-53 (2u)^{-p}, small enough for p <= 3 at these sizes.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import combine
from paper_2305_19768_gb300.inputs.lattice import cbc_fast, next_prime
from subtraction_cases import CASES, DEFORMED_CASES
from test_oracle_pins import _series_of_inverse_linear, _toy_integral

sp = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")


# ---------------------------------------------------------------- exact integrand
def _exact_integrand(d, a, b, Uterms, u0, u1, Fterms, f0, f1, tpoint, lo, norders, lam=None):
    """Laurent coefficients eps^lo.. of the subtracted sector integrand at tpoint
    (rationals), by symbolic differentiation and a numerical eps expansion.
    With lam (rationals, one per variable) the sector is contour-deformed:
    z_j = t_j - i lam_j t_j (1 - t_j) dF/dt_j, rho_j = z_j / t_j, J = dz/dt, and
    G = det J prod_{singular} rho_j^{a_j + b_j eps} prod_{regular} z_j^{a_j + b_j eps}
        U(z)^{u0 + u1 eps} F(z)^{f0 + f1 eps} (principal branches)."""
    ts = sp.symbols(f"t0:{d}")
    e = sp.Symbol("eps")
    R = sp.Rational

    def poly(terms, x):
        return sum(R(c) * sp.Mul(*[x[j] ** k for j, k in enumerate(ex)]) for ex, c in terms.items())

    if lam is None:
        x, G = ts, sp.Integer(1)
        fac = [ts[j] for j in range(d)]
    else:
        Ft = poly(Fterms, ts)
        x = [ts[j] - sp.I * R(lam[j]) * ts[j] * (1 - ts[j]) * sp.diff(Ft, ts[j]) for j in range(d)]
        G = sp.Matrix(d, d, lambda j, l: sp.diff(x[j], ts[l])).det()
        fac = [1 - sp.I * R(lam[j]) * (1 - ts[j]) * sp.diff(Ft, ts[j]) for j in range(d)]
    G = G * poly(Uterms, x) ** (R(u0) + R(u1) * e) * poly(Fterms, x) ** (R(f0) + R(f1) * e)
    sing = []
    for j in range(d):
        if a[j] <= -1:
            sing.append(j)
            if lam is not None:
                G = G * fac[j] ** (a[j] + R(b[j]) * e)
        elif a[j] != 0 or R(b[j]) != 0:
            G = G * (x[j] if lam is not None else ts[j]) ** (a[j] + R(b[j]) * e)
    f = G
    for j in reversed(sing):
        p, bj, tv = -a[j], R(b[j]), ts[j]
        out = tv ** (-p + bj * e) * f
        for k in range(p):
            gk = sp.diff(f, tv, k).subs(tv, 0) / sp.factorial(k)
            out += gk * (1 / (k - p + 1 + bj * e) - tv ** (k - p + bj * e))
        f = out
    f = f.subs({ts[j]: R(tpoint[j]) for j in range(d)})
    ns = len(sing)
    # eps^ns f is analytic in |eps| < min |m / b_j| >= 1/2 (the poles of
    # 1/(m + b_j eps), m != 0); its Taylor coefficients by the trapezoid rule
    # on the circle |eps| = 1/10 (Cauchy's formula; error ~ 5^-64)
    hi = lo + norders - 1
    with mpmath.workdps(60):
        fn = sp.lambdify(e, f * e ** ns, "mpmath")
        N, r = 64, mpmath.mpf(1) / 10
        vals = [fn(r * mpmath.expjpi(mpmath.mpf(2 * j) / N)) for j in range(N)]
        out = []
        for o in range(lo, hi + 1):
            k = o + ns
            if k < 0:
                out.append(0.0)
                continue
            c = sum(v * mpmath.expjpi(-mpmath.mpf(2 * j * k) / N) for j, v in enumerate(vals)) / (N * r ** k)
            out.append(complex(c))
        return np.array(out)


def _oracle_integrand(d, a, b, Uterms, u0, u1, Fterms, f0, f1, tpoint, lo, norders, lam=None):
    I = _toy_integral(d, a, b, Uterms, u0=u0, u1=u1, Fterms=Fterms, f0=f0, f1=f1)
    if lam is not None:
        I.sectors[0].deform = True
    v = oracle.SectorView(I, 0, [], None if lam is None else [float(Fraction(x)) for x in lam])
    val = oracle.integrand_at(v, np.array([float(Fraction(x)) for x in tpoint]), lo, norders)
    return val[:, 0] + 1j * val[:, 1]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_subtracted_integrand_matches_symbolic(case):
    d, a, b, U, u0, u1, F, f0, f1, lo, no, points = CASES[case]
    for tp in points:
        got = _oracle_integrand(d, a, b, U, u0, u1, F, f0, f1, tp, lo, no)
        exact = _exact_integrand(d, a, b, U, u0, u1, F, f0, f1, tp, lo, no)
        scale = np.max(np.abs(exact))
        assert np.max(np.abs(got - exact)) <= 1e-12 * scale, (tp, got, exact)


@pytest.mark.parametrize("case", range(len(DEFORMED_CASES)))
def test_deformed_subtracted_integrand_matches_symbolic(case):
    # contour-deformed sectors: the Taylor coefficients pass through z(t),
    # rho(t), det J and U(z), F(z)
    d, a, b, U, u0, u1, F, f0, f1, lo, no, points, lam = DEFORMED_CASES[case]
    for tp in points:
        got = _oracle_integrand(d, a, b, U, u0, u1, F, f0, f1, tp, lo, no, lam)
        exact = _exact_integrand(d, a, b, U, u0, u1, F, f0, f1, tp, lo, no, lam)
        scale = np.max(np.abs(exact))
        assert np.max(np.abs(got - exact)) <= 1e-12 * scale, (tp, got, exact)


def test_symbolic_check_detects_a_dropped_taylor_term():
    # the symbolic reference is sharp: dropping the k = p - 1 boundary term of
    # one variable (the eps^-1 pole of the integrand) moves the result far
    # outside the tolerance of the test above
    d, a, b, U, u0, u1, F, f0, f1, lo, no, points = CASES[3]
    exact = _exact_integrand(d, a, b, U, u0, u1, F, f0, f1, points[0], lo, no)
    wrong = _exact_integrand(d, [-2, -1], b, U, u0, u1, F, f0, f1, points[0], lo, no)
    assert np.max(np.abs(wrong - exact)) > 1e-3 * np.max(np.abs(exact))


# ---------------------------------------------------------------- integrated
def _baker_integral(I, n, m, lo, norders, seed=1):
    d = I.dmax
    z = cbc_fast(n, d)
    slo = -I.max_poles
    sno = lo + norders - 1 - slo + 1
    acc = np.zeros((m, sno), dtype=complex)
    for si in range(len(I.sectors)):
        v = oracle.SectorView(I, si, [], transform=1)
        out, _, _ = oracle.shift_sums(v, n, z[:I.sectors[si].d], oracle.shifts(seed, si, m, I.sectors[si].d),
                                      slo, sno)
        acc += out[..., 0] + 1j * out[..., 1]
    res = np.array([combine.laurent_product(0, np.array([1.0]), slo, acc[s], lo, norders) for s in range(m)])
    mean, var = combine.shift_stats(res)
    return mean, np.sqrt(var.real + var.imag)


def _exact_poly_sum(coefs, a, b, lo, norders):
    """sum_k c_k prod_j 1/(k_j + a_j + 1 + b_j eps) for polynomial G (all variables
    singular or with b_j = 0)."""
    exact = np.zeros(norders, dtype=complex)
    for ks, c in coefs.items():
        ser_lo, ser = 0, np.array([1.0 + 0j])
        for j, k in enumerate(ks):
            m_ = k + a[j] + 1
            if b[j] == 0:
                ser = ser / m_
                continue
            flo = -1 if m_ == 0 else 0
            ser = combine.laurent_product(ser_lo, ser, flo, _series_of_inverse_linear(m_, b[j], flo, norders + 8),
                                          ser_lo + flo, norders + 8)
            ser_lo += flo
        exact += c * combine.laurent_product(ser_lo, ser, 0, np.array([1.0]), lo, norders)
    return exact


@pytest.mark.parametrize("d,a,b,coefs,n,lo,no,sig", [
    (1, [-3], [1.25], {(0,): 1.0, (1,): 2.0, (2,): 3.0, (3,): -1.0, (4,): 0.5}, 100003, -1, 3, 1e-4),
    (2, [-2, -2], [-1.5, 0.75], {(0, 0): 1.0, (1, 0): -2.0, (0, 1): 0.5, (1, 1): 3.0, (2, 1): -2.0,
                                  (3, 0): 1.5, (2, 2): 1.0}, 40009, -2, 3, 1e-4),
    (4, [-2, -1, -2, 0], [1.5, -1.0, 0.75, 0.0], {(0, 0, 0, 0): 1.0, (1, 0, 1, 0): 2.0, (2, 1, 0, 1): -1.0,
                                                   (1, 1, 2, 0): 0.5, (0, 0, 0, 2): 3.0}, 20011, -3, 4, 1e-3),
])
def test_higher_subtraction_exact_series_baker(d, a, b, coefs, n, lo, no, sig):
    I = _toy_integral(d, a, b, coefs)
    mean, sd = _baker_integral(I, n, 8, lo, no)
    exact = _exact_poly_sum(coefs, a, b, lo, no)
    scale = np.max(np.abs(exact))
    for o in range(no):
        assert abs(mean[o] - exact[o]) <= 3.0 * sd[o] + 1e-12 * scale, (o, mean[o], exact[o], sd[o])
    # not an empty check: the spread is small against the values
    assert np.max(sd) <= sig * scale, (sd, scale)
