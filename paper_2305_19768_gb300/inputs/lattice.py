"""Rank-1 lattice generating vectors (input preparation).

The paper's integrator uses pre-computed component-by-component (CBC)
generating vectors that minimise the worst-case error in a Korobov space of
smoothness alpha = 2 with product weights (Section on median QMC rules), and,
optionally, median QMC rules whose candidate vectors are drawn uniformly
from U_n = {1 <= z <= n-1, gcd(z, n) = 1}. Neither the tables nor the
weights are printed, so this module builds its own table:

* ``cbc_fast``: fast CBC of Nuyens & Cools (2006) for prime n. With weights
  gamma_j = 1 and omega(x) = 2 pi^2 (x^2 - x + 1/6) (the Korobov kernel for
  sum_h |h|^-2), the squared worst-case error is
      e^2(z) = -1 + (1/n) sum_{k=0}^{n-1} prod_j (1 + gamma_j omega({k z_j / n})).
  Component s is the z in 1..(n-1)/2 minimising e^2 given z_1..z_{s-1}
  (z and n - z are equivalent because omega(x) = omega(1-x)); ties go to the
  smaller z. The sum over k != 0 for all candidates is a circulant product in
  the ordering k = g^b (g a primitive root mod n), done by FFT in O(n log n).
* ``load_table`` / ``lattice_for``: the committed table of (n, z_1..z_6),
  written by ``make_cbc_table.py``; ``lattice_for(n_min)`` gives the smallest
  tabulated n >= n_min (the "round up to an available lattice" rule).
* ``median_candidates``: r random vectors with components in U_n (median
  rules), drawn with splitmix64 from a seed.
"""
from __future__ import annotations

import math
import os
from functools import lru_cache
from typing import List, Tuple

import numpy as np

TABLE_PATH = os.path.join(os.path.dirname(__file__), "cbc_table.txt")
DMAX_TABLE = 6


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:  # deterministic for n < 3.3e24
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def next_prime(n: int) -> int:
    n = max(2, int(n))
    while not is_prime(n):
        n += 1
    return n


def _factor(n: int) -> List[int]:
    fs, p = [], 2
    while p * p <= n:
        if n % p == 0:
            fs.append(p)
            while n % p == 0:
                n //= p
        p += 1 if p == 2 else 2
    if n > 1:
        fs.append(n)
    return fs


def primitive_root(n: int) -> int:
    """Smallest generator of the multiplicative group mod prime n."""
    if n == 2:
        return 1
    fs = _factor(n - 1)
    for g in range(2, n):
        if all(pow(g, (n - 1) // q, n) != 1 for q in fs):
            return g
    raise ValueError("no primitive root")


def _powers(g: int, n: int, M: int) -> np.ndarray:
    """perm[i] = g^i mod n for i < M (blockwise, int64 exact for n < 2^31)."""
    assert n < (1 << 31)
    B = max(1, min(M, int(math.isqrt(M)) + 1))
    base = np.empty(B, dtype=np.int64)
    x = 1
    for i in range(B):
        base[i] = x
        x = x * g % n
    step = x  # g^B
    out = np.empty(M, dtype=np.int64)
    cur = 1
    for i0 in range(0, M, B):
        m = min(B, M - i0)
        out[i0:i0 + m] = (cur * base[:m]) % n
        cur = cur * step % n
    return out


def omega(x):
    return 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0)


def cbc_fast(n: int, d: int, gamma: float = 1.0) -> List[int]:
    """Fast CBC generating vector of length d for prime n (see module doc)."""
    if not is_prime(n):
        raise ValueError("fast CBC needs prime n")
    if n < 5:
        return [1] * d
    M = n - 1
    g = primitive_root(n)
    perm = _powers(g, n, M)                       # k = perm[b]
    om = omega(perm.astype(np.float64) / n)       # omega(g^i / n)
    Om = np.fft.rfft(om)
    q = np.ones(M, dtype=np.float64)              # prod over chosen components, k = g^b
    z = [1]
    q *= 1.0 + gamma * om                          # z_1 = 1: omega(g^b/n)
    half = (n - 1) // 2
    for _s in range(1, d):
        c = np.fft.irfft(Om * np.conj(np.fft.rfft(q)), n=M)   # c[a] = sum_b q[b] om[a+b]
        cz = np.empty(n, dtype=np.float64)
        cz[perm] = c                              # cz[z] for z = g^a
        zs = 1 + int(np.argmin(cz[1:half + 1]))
        z.append(zs)
        # a* with g^a* = zs: shift index
        a_star = int(np.nonzero(perm == zs)[0][0])
        q *= 1.0 + gamma * np.roll(om, -a_star)   # om[(a*+b) mod M]
    return z


def worst_case_error_sq(n: int, z, gamma: float = 1.0) -> float:
    """e^2(z) by direct summation (used by tests and the table checker)."""
    k = np.arange(n, dtype=np.int64)
    prod = np.ones(n)
    for zj in z:
        x = (k * int(zj) % n) / n
        prod *= 1.0 + gamma * omega(x)
    return float(-1.0 + prod.sum() / n)


@lru_cache(maxsize=1)
def load_table() -> Tuple[Tuple[int, Tuple[int, ...]], ...]:
    rows = []
    with open(TABLE_PATH) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(x) for x in line.split()]
            rows.append((v[0], tuple(v[1:])))
    rows.sort()
    return tuple(rows)


def lattice_for(n_min: int, d: int) -> Tuple[int, Tuple[int, ...]]:
    """Smallest tabulated (n, z[:d]) with n >= n_min."""
    if d > DMAX_TABLE:
        raise ValueError(f"table holds vectors up to dimension {DMAX_TABLE}")
    for n, z in load_table():
        if n >= n_min:
            return n, z[:d]
    raise ValueError(f"no tabulated lattice with n >= {n_min}")


def lattice_sizes() -> List[int]:
    return [n for n, _ in load_table()]


def median_candidates(n: int, d: int, r: int, seed: int) -> np.ndarray:
    """r candidate vectors, components uniform in U_n (rejection on gcd)."""
    from .workloads import splitmix64_next

    st = seed & ((1 << 64) - 1)
    out = np.zeros((r, d), dtype=np.int64)
    for i in range(r):
        for j in range(d):
            while True:
                st, v = splitmix64_next(st)
                zc = 1 + v % (n - 1)
                if math.gcd(zc, n) == 1:
                    out[i, j] = zc
                    break
    return out
