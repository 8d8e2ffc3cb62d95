"""Pins of the oracle's host-side steps: Laurent products, shift statistics
and the allocation of Eq. adaptive-solution (no GPU)."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import combine


def test_laurent_product_matches_polynomial_product():
    rng = np.random.default_rng(1)
    a = rng.normal(size=4) + 1j * rng.normal(size=4)
    b = rng.normal(size=3) + 1j * rng.normal(size=3)
    full = np.polynomial.polynomial.polymul(a, b)  # coefficient of x^k
    # a starts at eps^-1, b at eps^-2 -> product starts at eps^-3
    got = combine.laurent_product(-1, a, -2, b, -3, 6)
    assert np.allclose(got, full, rtol=0, atol=1e-14)
    got = combine.laurent_product(-1, a, -2, b, -1, 2)
    assert np.allclose(got, full[2:4], rtol=0, atol=1e-14)


def test_shift_stats_unbiased_variance_of_mean():
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(32, 3)) + 1j * rng.normal(size=(32, 3)) * 2
    mean, var = combine.shift_stats(Q)
    assert np.allclose(mean, Q.mean(0))
    assert np.allclose(var.real, np.var(Q.real, axis=0, ddof=1) / 32)
    assert np.allclose(var.imag, np.var(Q.imag, axis=0, ddof=1) / 32)


def test_shift_stats_hand_computed_cases():
    # two shifts Q = 1 + 2i and 3 - 2i: mean 2 + 0i; the unbiased variances
    # are ((1-2)^2 + (3-2)^2)/1 = 2 and ((2-0)^2 + (-2-0)^2)/1 = 8, so the
    # variances of the mean are 2/2 = 1 and 8/2 = 4
    mean, var = combine.shift_stats(np.array([[1 + 2j], [3 - 2j]]))
    assert mean[0] == 2 + 0j and var[0] == 1 + 4j
    # three shifts 0, 3, 6 (real): mean 3, unbiased variance (9 + 0 + 9)/2 = 9,
    # variance of the mean 9/3 = 3; the imaginary part has zero spread
    mean, var = combine.shift_stats(np.array([[0.0 + 5j], [3.0 + 5j], [6.0 + 5j]]))
    assert mean[0] == 3 + 5j and var[0] == 3 + 0j
    # orders are independent columns
    mean, var = combine.shift_stats(np.array([[1.0, 10.0], [3.0, 10.0]], dtype=complex))
    assert np.array_equal(mean, [2.0, 10.0]) and np.array_equal(var.real, [1.0, 0.0])
    # one shift: no variance estimate
    _, var = combine.shift_stats(np.array([[1.0 + 1j]]))
    assert np.isinf(var[0].real) and np.isinf(var[0].imag)


def test_relative_error_definition():
    # sqrt(dR^2 + dI^2) / sqrt(R^2 + I^2) with variance = dR^2 + dI^2:
    # value 3 + 4i (modulus 5), dR = 0.3, dI = 0.4 -> 0.5 / 5 = 0.1
    assert abs(combine.relative_error(3 + 4j, 0.3 ** 2 + 0.4 ** 2) - 0.1) < 1e-15
    assert combine.relative_error(-2.0, 1e-8) == pytest.approx(5e-5, rel=1e-14)
    assert combine.relative_error(0.0, 1.0) == float("inf")
    assert combine.relative_error(1j, 0.0) == 0.0


def test_variance_propagation_through_coefficients():
    # var(c * I) for a deterministic Laurent c: sum_p |c_p|^2 var(I^(o-p))
    c = np.array([2.0, -1.0 + 1j])
    v = np.array([1.0 + 2.0j, 3.0 + 0.5j])  # var_re + i var_im per order
    out = combine.laurent_variance(0, c, 0, v, 0, 2)
    assert np.allclose(out, [4 * 3.0, 4 * 3.5 + 2 * 3.0])


@pytest.mark.parametrize("alpha", [2.0, 3.0])
def test_allocation_satisfies_constraint_and_is_optimal(alpha):
    rng = np.random.default_rng(3)
    W = rng.uniform(0.1, 10.0, size=5) * 1e-3
    tau = rng.uniform(0.5, 4.0, size=5)
    V = 1e-9
    n, lam = combine.allocate_one_sum(W, tau, V, alpha)
    assert abs(np.sum(W * n ** -alpha) - V) <= 1e-10 * V
    # independent numerical optimisation in log n
    obj = lambda y: np.sum(tau * np.exp(y)) / np.sum(tau * n)
    cons = {"type": "eq", "fun": lambda y: np.log(np.sum(W * np.exp(-alpha * y)) / V)}
    r = minimize(obj, np.log(n) + 0.3, constraints=[cons], method="SLSQP", options={"ftol": 1e-14,
                                                                                     "maxiter": 500})
    assert r.success
    assert np.allclose(np.exp(r.x), n, rtol=1e-4)
    # KKT: tau_i = lam * alpha * W_i n_i^(-alpha-1)
    assert np.allclose(tau, lam * alpha * W * n ** (-alpha - 1), rtol=1e-10)


def test_allocation_several_sums_takes_max_and_floor():
    W1 = np.array([1.0, 0.0, 2.0])
    W2 = np.array([0.0, 5.0, 0.1])
    tau = np.ones(3)
    n = combine.allocate([W1, W2], tau, [1e-6, 1e-6], n_min=1e4)
    n1, _ = combine.allocate_one_sum(W1[[0, 2]], tau[[0, 2]], 1e-6)
    assert n[0] >= n1[0] - 1e-9 and n[2] >= 1e4
    assert np.all(n >= 1e4)
