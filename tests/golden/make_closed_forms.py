"""Write ``closed_forms.txt``: Laurent coefficients of one-loop integrals from
their textbook closed forms, evaluated with mpmath at 30 digits.

Convention (standard Feynman-parameter normalisation, measure
d^D l / (i pi^{D/2}), D = 4 - 2 eps, no exp(gamma_E eps) factor):
    I = (-1)^N Gamma(N - D/2) Int delta(1 - sum x) U^{N - D} (F - i0)^{-(N - D/2)}.

Sources of the closed forms (not the oracle, not the CUDA path):
* triangle_m1_pm1: the defining Feynman integral of the finite massive
  triangle on the simplex, -Int dx / (1 + x1 x2 + x2 x3 + x3 x1), by
  two-dimensional adaptive quadrature;
* box1L_massless: r_Gamma/(s t) {2/eps^2 [(-s)^-eps + (-t)^-eps] - ln^2(s/t)
  - pi^2} + O(eps) (Bern, Dixon & Kosower; Ellis & Zanderighi, JHEP 02 (2008)
  002, box 1), r_Gamma = Gamma(1+eps) Gamma(1-eps)^2 / Gamma(1-2eps);
* bubble_m0: Gamma(eps) Gamma(1-eps)^2 / Gamma(2-2eps) (-s-i0)^-eps (Dirichlet
  integral over the simplex);
* bubble_m1: Gamma(eps) Int_0^1 (m^2 - x(1-x) s - i0)^-eps dx, whose eps^0
  term is 1/eps - gamma_E - [ln m^2 - 2 + beta ln((beta+1)/(beta-1))],
  beta = sqrt(1 - 4 m^2/s), continued with s -> s + i0;
* triangle_m0 (one off-shell leg p^2 = s, massless lines):
  -r_Gamma (-s-i0)^{-1-eps} / eps^2 (Dirichlet integral).

Usage: python tests/golden/make_closed_forms.py  (rewrites closed_forms.txt)
"""
import os

import mpmath as mp

mp.mp.dps = 30
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.txt")


def series(f, orders, lo):
    """Laurent coefficients eps^lo..eps^(lo+orders-1) of f(eps) via mpmath.taylor
    of eps^(-lo) f(eps)."""
    g = lambda e: f(e) * e ** (-lo)
    # Taylor coefficients at 0 of a function with a removable singularity there,
    # by the Cauchy integral on a circle of radius 0.05 (trapezoidal rule, 256
    # nodes: exponentially accurate for an analytic integrand).
    res = []
    r = mp.mpf("0.05")
    npts = 256
    for k in range(orders):
        acc = mp.mpc(0)
        for j in range(npts):
            th = 2 * mp.pi * j / npts
            e = r * mp.expj(th)
            acc += g(e) * mp.expj(-k * th)
        res.append(acc / npts / r ** k)
    return res


def rgamma(e):
    return mp.gamma(1 + e) * mp.gamma(1 - e) ** 2 / mp.gamma(1 - 2 * e)


def lnm(x):
    """ln(x - i0) for real x."""
    x = mp.mpf(x)
    return mp.log(x) if x > 0 else mp.log(-x) - 1j * mp.pi


def main():
    rows = []
    # triangle_m1_pm1
    f = lambda x1, x2: 1 / (1 + x1 * x2 + x2 * (1 - x1 - x2) + (1 - x1 - x2) * x1)
    val = -mp.quad(lambda x1: mp.quad(lambda x2: f(x1, x2), [0, 1 - x1]), [0, 1])
    rows.append(("triangle_m1_pm1", "", 0, val, "Feynman integral on the simplex, 2-D quadrature"))

    # massless box, expanded analytically in eps via the Cauchy integral
    for s, t in ((-3, -2), (-5, -1)):
        s_, t_ = mp.mpf(s), mp.mpf(t)
        def box(e):
            return rgamma(e) / (s_ * t_) * (2 / e ** 2 * (mp.exp(-e * lnm(-s_)) + mp.exp(-e * lnm(-t_)))
                                             - (lnm(-s_) - lnm(-t_)) ** 2 - mp.pi ** 2)
        cs = series(box, 3, -2)
        for k, c in enumerate(cs):
            rows.append(("box1L_massless", f"s={s},t={t}", -2 + k, c, "BDK / Ellis-Zanderighi box 1"))

    # massless bubble at s (Euclidean and physical)
    for s in (-3, 10):
        s_ = mp.mpf(s)
        bub = lambda e: mp.gamma(e) * mp.gamma(1 - e) ** 2 / mp.gamma(2 - 2 * e) * mp.exp(-e * lnm(-s_))
        for k, c in enumerate(series(bub, 2, -1)):
            rows.append(("bubble_m0", f"s={s}", -1 + k, c, "Dirichlet integral"))

    # massive bubble m^2 = 1: eps^-1 = 1, eps^0 from the closed form of the Feynman integral
    for s in (-3, 10):
        s_ = mp.mpf(s)
        beta = mp.sqrt(1 - 4 / s_ + 0j)
        if s_ > 4:
            L = mp.log((1 + beta) / (1 - beta)) - 1j * mp.pi
        else:
            L = mp.log((beta + 1) / (beta - 1))
        c0 = -mp.euler - (0 - 2 + beta * L)
        rows.append(("bubble_m1", f"s={s}", -1, mp.mpf(1), "Gamma(eps) pole"))
        rows.append(("bubble_m1", f"s={s}", 0, c0, "B0 closed form (ln m^2 - 2 + beta ln)"))

    # one-mass massless triangle
    for s in (-3, 10):
        s_ = mp.mpf(s)
        tri = lambda e: -rgamma(e) * mp.exp((-1 - e) * lnm(-s_)) / e ** 2
        for k, c in enumerate(series(tri, 3, -2)):
            rows.append(("triangle_m0", f"s={s}", -2 + k, c, "Dirichlet integral"))

    with open(OUT, "w") as fh:
        fh.write("# name kinematics order re im  -- textbook closed forms (make_closed_forms.py)\n")
        for name, kin, order, c, src in rows:
            c = mp.mpc(c)
            fh.write(f"{name} {kin or '-'} {order} {mp.nstr(c.real, 22)} {mp.nstr(c.imag, 22)}  # {src}\n")


if __name__ == "__main__":
    main()
