"""Synthetic workloads: the integrals and kinematic points the integrator runs on.

The paper's own examples need pySecDec-generated sector files that do not
exist here, so these one- and two-loop integrals stand in for them (same
structure: sector-decomposed, eps-expanded Feynman-parameter integrands, with
and without contour deformation, combined with coefficients into sums).

* ``triangle_massive``: one-loop triangle, three internal masses m^2 = 1,
  p_i^2 = -1 (Euclidean), D = 4: finite, three primary sectors in d = 2.
* ``box_massless``: one-loop box, p_i^2 = 0, D = 4 - 2 eps, invariants s, t:
  poles up to 1/eps^2, twelve sectors in d = 3 after iterative decomposition.
* ``box_massive``: one-loop box with four internal masses m^2 = 1, p_i^2 = 0;
  physical region (s > 4 m^2) needs contour deformation; four sectors, d = 3.
* ``double_box_massless``: two-loop planar double box, seven massless
  propagators, poles up to 1/eps^4, d = 6.
Builders take method="iterative" (primary sectors, then iterative
decomposition) or "geometric" (inputs.geometric).
* ``bubble``/``triangle`` families used in the 10-integral amplitude.

Kinematic points are drawn with splitmix64 (Steele, Lea & Flood 2014) from a
seed, so every workload is reproducible on any machine.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Tuple

import numpy as np

from .feynman import (Graph, exponents, kin_2pt, kin_3pt_one_offshell, kin_massless_4pt,
                      kin_numeric_3pt, prefactor_series, symanzik)
from .integral import Integral
from .secdec import decompose

MASK64 = (1 << 64) - 1


def splitmix64_next(state: int) -> Tuple[int, int]:
    """One splitmix64 step: returns (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def uniform_stream(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0,1): (splitmix64 output >> 11) * 2^-53."""
    st = seed & MASK64
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        st, z = splitmix64_next(st)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def _integral_from_graph(g: Graph, D0: int, *, deform: bool, pref_order: int = 6,
                         method: str = "iterative") -> Integral:
    U, F = symanzik(g)
    N = len(g.edges)
    L = g.nloops
    u0, u1, f0, f1 = exponents(N, L, D0)
    if method == "geometric":
        from .geometric import decompose_geometric

        secs = decompose_geometric(U, F, u0, u1, f0, f1, deform=deform)
    elif method == "iterative":
        secs = decompose(U, F, u0, u1, f0, f1, deform=deform)
    else:
        raise ValueError(f"unknown decomposition method {method!r}")
    lo, pc = prefactor_series(N, L, D0, pref_order)
    return Integral(g.name, L, N, D0, list(g.kin.invariants), lo, [complex(c) for c in pc], secs)


def triangle_massive(msq=1, psq=-1, method: str = "iterative") -> Integral:
    g = Graph(edges=[(0, 1), (1, 2), (2, 0)], masses_sq=[Fraction(msq)] * 3, legs=[0, 1, 2],
              kin=kin_numeric_3pt(psq, psq, psq), name="triangle_m1_pm1")
    return _integral_from_graph(g, 4, deform=False, method=method)


def box_massless(deform: bool = False, method: str = "iterative") -> Integral:
    g = Graph(edges=[(0, 1), (1, 2), (2, 3), (3, 0)], masses_sq=[Fraction(0)] * 4,
              legs=[0, 1, 2, 3], kin=kin_massless_4pt(), name="box1L_massless")
    return _integral_from_graph(g, 4, deform=deform, method=method)


def box_massless_d2(deform: bool = False, method: str = "iterative") -> Integral:
    """The one-loop massless box in D = 2 - 2 eps: U^{2 + 2 eps} F^{-3 - eps};
    12 sectors, each with one or two exponents a_j = -2 (Taylor subtraction of
    degree 1 in one or two variables); deform: contour deformation for
    physical (s, t)."""
    g = Graph(edges=[(0, 1), (1, 2), (2, 3), (3, 0)], masses_sq=[Fraction(0)] * 4,
              legs=[0, 1, 2, 3], kin=kin_massless_4pt(), name="box1L_massless_d2")
    return _integral_from_graph(g, 2, deform=deform, method=method)


def box_massive(msq=1, deform: bool = True) -> Integral:
    g = Graph(edges=[(0, 1), (1, 2), (2, 3), (3, 0)], masses_sq=[Fraction(msq)] * 4,
              legs=[0, 1, 2, 3], kin=kin_massless_4pt(), name="box1L_massive")
    return _integral_from_graph(g, 4, deform=deform)


def double_box_massless_d2(method: str = "iterative") -> Integral:
    """The two-loop planar massless double box in D = 2 - 2 eps: 282 sectors
    with exponents down to a_j = -4 (Taylor subtraction up to degree 3 in up
    to four variables)."""
    g = Graph(edges=[(0, 1), (1, 2), (2, 5), (5, 4), (4, 3), (3, 0), (1, 4)],
              masses_sq=[Fraction(0)] * 7, legs=[3, 0, 2, 5], kin=kin_massless_4pt(),
              name="box2L_planar_massless_d2")
    return _integral_from_graph(g, 2, deform=False, method=method)


def double_box_massless(method: str = "iterative") -> Integral:
    # vertices: 0-1-2 top row, 3-4-5 bottom row; rung 1-4
    # legs: p0 at 3 (bottom left), p1 at 0 (top left), p2 at 2 (top right), p3 at 5
    g = Graph(edges=[(0, 1), (1, 2), (2, 5), (5, 4), (4, 3), (3, 0), (1, 4)],
              masses_sq=[Fraction(0)] * 7, legs=[3, 0, 2, 5], kin=kin_massless_4pt(),
              name="box2L_planar_massless")
    return _integral_from_graph(g, 4, deform=False, method=method)


def bubble(msq=0, inv="s", deform: bool = True, names=None) -> Integral:
    g = Graph(edges=[(0, 1), (1, 0)], masses_sq=[Fraction(msq)] * 2, legs=[0, 1],
              kin=kin_2pt(inv, names), name=f"bubble_m{msq}_{inv}")
    return _integral_from_graph(g, 4, deform=deform)


def triangle_one_offshell(msq=0, inv="s", deform: bool = True, names=None) -> Integral:
    g = Graph(edges=[(0, 1), (1, 2), (2, 0)], masses_sq=[Fraction(msq)] * 3, legs=[0, 1, 2],
              kin=kin_3pt_one_offshell(inv, names), name=f"triangle_m{msq}_{inv}")
    return _integral_from_graph(g, 4, deform=deform)


def massive_box_points(count: int = 1024, seed: int = 3) -> np.ndarray:
    """(s, t) pairs: s ~ U[5, 20], t ~ U[-8, -1], drawn s then t per point."""
    u = uniform_stream(seed, 2 * count).reshape(count, 2)
    return np.stack([5.0 + 15.0 * u[:, 0], -8.0 + 7.0 * u[:, 1]], axis=1)


def amplitude_grid(ns: int = 100, nt: int = 100, t_offset: float = 0.137) -> np.ndarray:
    """Row-major (s, t) grid over s in [5, 20], t in [-8, -1]: s at cell centres,
    t at cell centres moved by ``t_offset`` of a cell, so that no point lies on
    u = -s - t = 0 (on that line the massless box's sector polynomials vanish
    along a line through a sector corner, where the deformation vanishes too,
    and the sector integrands are not integrable)."""
    s = 5.0 + 15.0 * (np.arange(ns) + 0.5) / ns
    t = -8.0 + 7.0 * (np.arange(nt) + 0.5 + t_offset) / nt
    S, T = np.meshgrid(s, t, indexing="ij")
    return np.stack([S.ravel(), T.ravel()], axis=1)


def amplitude_integrals():
    """The ten one-loop integrals of the synthetic amplitude, all over the
    invariants (s, t): massless and massive (m^2 = 1) bubbles and one-mass
    triangles in s (physical, deformed) and in t (Euclidean), and the massless
    and massive boxes in (s, t) (physical, deformed)."""
    st = ["s", "t"]
    out = []
    for msq in (0, 1):
        out.append(bubble(msq, "s", deform=True, names=st))
        out.append(bubble(msq, "t", deform=False, names=st))
    for msq in (0, 1):
        out.append(triangle_one_offshell(msq, "s", deform=True, names=st))
        out.append(triangle_one_offshell(msq, "t", deform=False, names=st))
    out.append(box_massless(deform=True))
    out.append(box_massive(deform=True))
    return out


def amplitude_coefficients(nint: int = 10, seed: int = 5):
    """Coefficient polynomials C_i(s, t) = sum_{a+b<=2} c_iab s^a t^b with
    c = p/q, p uniform in [-9, 9], q in [1, 9] (splitmix64 from ``seed``;
    drawn integral by integral, monomials in the order 1, s, t, s^2, s t, t^2).
    Returns an array [nint][6] of Fractions."""
    st = seed & MASK64
    rows = []
    for _ in range(nint):
        row = []
        for _m in range(6):
            st, a = splitmix64_next(st)
            st, b = splitmix64_next(st)
            row.append(Fraction(int(a % 19) - 9, int(b % 9) + 1))
        rows.append(row)
    return rows


def amplitude_coefficient_values(points: np.ndarray, coefs) -> np.ndarray:
    """C_i at each (s, t): float64 [npoints][nint]."""
    s, t = points[:, 0], points[:, 1]
    mons = np.stack([np.ones_like(s), s, t, s * s, s * t, t * t], axis=1)
    C = np.array([[float(c) for c in row] for row in coefs])
    return mons @ C.T
