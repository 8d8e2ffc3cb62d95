"""The C-ABI's host arithmetic (shift statistics, Laurent products, variance
propagation, Eq. adaptive-solution) against the oracle's numpy restatement
(no GPU: these entry points need none)."""
import numpy as np
import pytest

from oracle import combine
from paper_2305_19768_gb300 import qmc


def test_shift_stats_matches_oracle():
    rng = np.random.default_rng(7)
    sums = rng.normal(size=(32, 4, 2))
    mean, var = qmc.qmc_shift_stats(sums)
    Q = sums[..., 0] + 1j * sums[..., 1]
    om, ov = combine.shift_stats(Q)
    assert np.allclose(mean[:, 0] + 1j * mean[:, 1], om, rtol=1e-15, atol=1e-15)
    assert np.allclose(var[:, 0], ov.real, rtol=1e-13) and np.allclose(var[:, 1], ov.imag, rtol=1e-13)
    m1, v1 = qmc.qmc_shift_stats(sums[:1])
    assert np.all(np.isinf(v1))


@pytest.mark.parametrize("alo,blo,lo,n", [(-1, -2, -3, 6), (0, -1, -1, 2), (-2, 0, -4, 3)])
def test_series_mul_and_var_match_oracle(alo, blo, lo, n):
    rng = np.random.default_rng(8)
    a = rng.normal(size=4) + 1j * rng.normal(size=4)
    b = rng.normal(size=3) + 1j * rng.normal(size=3)
    got = qmc.qmc_series_mul(a, alo, b, blo, lo, n)
    assert np.allclose(got, combine.laurent_product(alo, a, blo, b, lo, n), rtol=1e-14, atol=1e-14)
    v = rng.uniform(size=3)
    gotv = qmc.qmc_series_var(a, alo, v, blo, lo, n)
    ov = combine.laurent_variance(alo, a, blo, v + 0j, lo, n)
    assert np.allclose(gotv, ov, rtol=1e-14, atol=1e-14)


def test_allocate_matches_oracle_one_and_several_sums():
    rng = np.random.default_rng(9)
    W = rng.uniform(1e-6, 1e-3, size=(3, 7))
    W[1, 2] = 0.0
    tau = rng.uniform(0.5, 3.0, size=7)
    V = np.array([1e-10, 3e-11, 0.0])
    got = qmc.qmc_allocate(W, tau, V, 2.0, 1e4)
    want = combine.allocate(list(W), tau, list(V), 1e4)
    assert np.allclose(got, want, rtol=1e-12)
    one = qmc.qmc_allocate(W[:1], tau, V[:1], 2.0, 0.0)
    n, _ = combine.allocate_one_sum(W[0], tau, V[0])
    assert np.allclose(one, n, rtol=1e-12)
    assert abs(np.sum(W[0] * one ** -2.0) - V[0]) <= 1e-10 * V[0]


def test_median_candidates_match_the_input_generator():
    from math import gcd

    from paper_2305_19768_gb300.inputs.lattice import median_candidates

    for n, d, r, seed in ((1000003, 3, 11, 42), (20011, 6, 5, 7), (1024, 2, 7, 1)):
        z = qmc.qmc_median_candidates(n, d, r, seed)
        assert np.array_equal(z[:, :d], median_candidates(n, d, r, seed))
        assert np.all(z[:, d:] == 1)
        assert all(gcd(int(c), n) == 1 and 1 <= c < n for c in z[:, :d].ravel())


def test_host_arithmetic_edge_cases():
    """Documented edge behaviour of the host entry points: no shifts is an
    error; empty series and orders outside the window give zeros; a sum with
    no positive weight or no positive variance target leaves the lattices at
    n_min; tau <= 0 and alpha <= 0 are errors."""
    with pytest.raises(qmc.QmcError):
        qmc.qmc_shift_stats(np.zeros((0, 2, 2)))
    a = np.array([1.0 + 2.0j, 3.0 - 1.0j])
    assert qmc.qmc_series_mul(a, -1, a, -1, -2, 0).size == 0
    assert np.all(qmc.qmc_series_mul(a, -1, np.zeros(0, complex), 0, -2, 3) == 0)
    assert np.all(qmc.qmc_series_mul(a, -1, a, -1, 5, 3) == 0)          # window above the product
    assert np.all(qmc.qmc_series_var(a, 0, np.zeros(0), 0, 0, 2) == 0)
    W = np.array([[0.0, 0.0], [1.0, 4.0], [2.0, 1.0]])
    V = np.array([1e-6, -1.0, 1e-6])                                    # the second target is not > 0
    n = qmc.qmc_allocate(W, np.ones(2), V, 2.0, 1000.0)
    n_third = qmc.qmc_allocate(W[2:], np.ones(2), V[2:], 2.0, 1000.0)
    assert np.array_equal(n, n_third)
    assert np.array_equal(qmc.qmc_allocate(W[:1], np.ones(2), V[:1], 2.0, 1000.0), [1000.0, 1000.0])
    with pytest.raises(qmc.QmcError):
        qmc.qmc_allocate(W, np.array([1.0, 0.0]), V)
    with pytest.raises(qmc.QmcError):
        qmc.qmc_allocate(W, np.ones(2), V, alpha=0.0)
