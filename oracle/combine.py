"""Host-side oracle steps (test infrastructure only): shift statistics,
Laurent products of prefactor/coefficient series with sector series, error
propagation, and the variance-driven lattice allocation.

Citations are to arXiv:2305.19768, section "Adaptive weighted sum
evaluation" (Eqs. varscaling and adaptive-solution) and the timings section
(relative error definition).

Readings where the paper is silent or garbled:
* shift variance uses 1/(m-1), separately for Re and Im; sigma = sqrt(var/m);
* var(A^(o)) = sum_i sum_p |C_i^(p)|^2 (var Re + var Im)(I_i^(o-p))
  (sectors have independent shifts, so their errors add in quadrature);
* in Eq. adaptive-solution the sum inside lambda runs over the integrals i and
  C_{jk}, C_{ji} both stand for C_{ki}; for several sums the formula is
  applied sum by sum and n_i keeps the largest value asked for.
"""
from __future__ import annotations

import numpy as np


def shift_stats(Q: np.ndarray):
    """Q: complex [m, norders] per-shift estimates.

    Returns (mean [norders] complex, var_of_mean [norders] as complex
    (var Re / m) + 1j (var Im / m))."""
    m = Q.shape[0]
    mean = Q.mean(axis=0)
    if m < 2:
        return mean, np.full(Q.shape[1], complex(np.inf, np.inf))   # no spread estimate from one shift
    vr = ((Q.real - mean.real) ** 2).sum(axis=0) / (m - 1)
    vi = ((Q.imag - mean.imag) ** 2).sum(axis=0) / (m - 1)
    return mean, vr / m + 1j * vi / m


def laurent_product(a_lo: int, a: np.ndarray, b_lo: int, b: np.ndarray, lo: int, norders: int):
    """Coefficients eps^lo..eps^(lo+norders-1) of (sum a_i eps^(a_lo+i))(sum b_j eps^(b_lo+j))."""
    out = np.zeros(norders, dtype=complex)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            o = a_lo + i + b_lo + j - lo
            if 0 <= o < norders:
                out[o] += ai * bj
    return out


def laurent_variance(c_lo: int, c: np.ndarray, v_lo: int, v: np.ndarray, lo: int, norders: int):
    """Variance propagated through the product with a fixed series c:
    var(out^(o)) = sum_p |c^(p)|^2 (var_re + var_im)(in^(o-p)); v is complex
    var_re + 1j var_im per order."""
    tot = v.real + v.imag
    out = np.zeros(norders)
    for i, ci in enumerate(c):
        for j, vj in enumerate(tot):
            o = c_lo + i + v_lo + j - lo
            if 0 <= o < norders:
                out[o] += abs(ci) ** 2 * vj
    return out


def relative_error(value: complex, variance: float) -> float:
    """sqrt(dR^2 + dI^2) / sqrt(R^2 + I^2) (timings section)."""
    den = abs(value)
    return float(np.sqrt(variance) / den) if den > 0 else float("inf")


def allocate_one_sum(W: np.ndarray, tau: np.ndarray, V: float, alpha: float = 2.0):
    """Eq. adaptive-solution for one sum: minimise sum tau_i n_i subject to
    sum W_i n_i^-alpha = V, with W_i = |C_i|^2 w_i. Returns (n_i, lambda)."""
    W = np.asarray(W, dtype=float)
    tau = np.asarray(tau, dtype=float)
    lam = (1.0 / alpha) * ((1.0 / V) * np.sum((W * tau ** alpha) ** (1.0 / (alpha + 1.0)))) ** (
        (alpha + 1.0) / alpha)
    n = (alpha * W / tau * lam) ** (1.0 / (alpha + 1.0))
    return n, lam


def allocate(Ws, taus, Vs, n_min, alpha: float = 2.0):
    """Several sums in sequence: n_i = max(n_min, max over sums of the one-sum solution)."""
    n = np.full(len(taus), float(n_min))
    for W, V in zip(Ws, Vs):
        if V <= 0 or not np.any(np.asarray(W) > 0):
            continue
        nk, _ = allocate_one_sum(W, taus, V, alpha)
        n = np.maximum(n, nk)
    return n
