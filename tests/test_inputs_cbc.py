"""Input preparation: the fast CBC construction (Nuyens & Cools, FFT over the
multiplicative group) chooses, at every component, a vector minimising the
squared worst-case error e^2 of the Korobov space with smoothness 2 and unit
product weights -- checked by brute force over all candidates on small prime
n, with e^2 summed directly from its definition (written out here, not taken
from the module under test):

    e^2(z) = -1 + (1/n) sum_k prod_j (1 + 2 pi^2 B_2({k z_j / n})),
    B_2(x) = x^2 - x + 1/6.

Ties (z and its inverse give the same point set in two dimensions) are
compared by value, not by index."""
import math

import numpy as np
import pytest

from paper_2305_19768_gb300.inputs.lattice import cbc_fast, load_table


def e2_direct(n, z):
    tot = 0.0
    for k in range(n):
        p = 1.0
        for zj in z:
            x = (k * zj % n) / n
            p *= 1.0 + 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0)
        tot += p
    return tot / n - 1.0


@pytest.mark.parametrize("n,d", [(11, 3), (31, 3), (53, 3), (101, 3), (13, 4)])
def test_fast_cbc_takes_the_brute_force_minimum_at_every_component(n, d):
    z = cbc_fast(n, d)
    assert z[0] == 1 and len(z) == d
    for s in range(1, d):
        cands = [e2_direct(n, z[:s] + [c]) for c in range(1, n)]
        best = min(cands)
        got = e2_direct(n, z[:s + 1])
        assert got <= best * (1 + 1e-12) + 1e-15, (s, z, got, best)
        assert 1 <= z[s] <= (n - 1) // 2


def test_committed_table_is_prime_sizes_with_units():
    rows = load_table()
    sizes = [r[0] for r in rows]
    assert sizes == sorted(sizes) and sizes[0] == 1009
    for n, z in rows[:12]:
        assert all(math.gcd(int(c), n) == 1 for c in z)
        assert len(z) == 6
