"""Geometric sector decomposition (inputs.geometric) checked through the
oracle: a one-dimensional toy with a known integral, the closed forms of the
massive triangle and the massless box, the double box's leading pole, fewer
sectors than the iterative method for the double box, and the text format's
sector weight."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_values import closed_form
from paper_2305_19768_gb300.inputs import geometric
from paper_2305_19768_gb300.inputs import workloads as w
from paper_2305_19768_gb300.inputs.integral import Integral
from paper_2305_19768_gb300.inputs.lattice import cbc_fast, next_prime
from paper_2305_19768_gb300.inputs.polynomial import LinPoly

from test_oracle_pins import assert_within, rqmc_integral


def test_one_dimensional_toy():
    # projective (x1 + x2)^-2 over the simplex = int_0^inf (1 + x)^-2 dx = 1: two cones
    U = LinPoly(2, 1, {(1, 0): (1,), (0, 1): (1,)})
    F = LinPoly(2, 1, {(0, 0): (1,)})
    secs = geometric.decompose_geometric(U, F, -2, 0, 0, 0)
    assert len(secs) == 2 and all(s.weight == 1 for s in secs)
    I = Integral("toy", 1, 2, 4, [], 0, [1.0], secs)
    mean, var = rqmc_integral(I, [], next_prime(4000), 8, 0, 1)
    assert_within(mean, var, [1.0], rel=1e-12)


def test_triangle_closed_form_geometric():
    I = w.triangle_massive(method="geometric")
    assert len(I.sectors) == 3
    mean, var = rqmc_integral(I, [], next_prime(10000), 8, 0, 1)
    assert_within(mean, var, [closed_form("triangle_m1_pm1")[0]])


@pytest.mark.parametrize("s,t", [(-3, -2), (-5, -1)])
def test_massless_box_closed_form_geometric(s, t):
    I = w.box_massless(method="geometric")
    assert I.max_poles == 2
    ex = closed_form("box1L_massless", f"s={s},t={t}")
    mean, var = rqmc_integral(I, [float(s), float(t)], next_prime(20000), 8, -2, 3)
    assert_within(mean, var, [ex[-2], ex[-1], ex[0]], rel=1e-9)


def test_double_box_geometric_fewer_sectors_and_leading_pole():
    Ig = w.double_box_massless(method="geometric")
    Ii = w.double_box_massless()
    assert len(Ig.sectors) < len(Ii.sectors) and Ig.max_poles == 4
    sel = [i for i, s in enumerate(Ig.sectors) if len(s.singular) == 4]
    s_, t_ = -2.0, -5.0
    n, m = 4001, 8
    z = cbc_fast(n, 6)
    acc = np.zeros(m, dtype=complex)
    for si in sel:
        v = oracle.SectorView(Ig, si, [s_, t_])
        out, _, _ = oracle.shift_sums(v, n, z, oracle.shifts(1, si, m, 6), -4, 1)
        acc += out[:, 0, 0] + 1j * out[:, 0, 1]
    c = Ig.prefactor[0] * acc * s_ * s_ * t_
    mean, err = c.mean().real, c.real.std(ddof=1) / np.sqrt(m)
    assert abs(mean - 4.0) <= 4 * err + 1e-6, (mean, err)


def test_weight_round_trips_and_scales_the_sector():
    I = w.triangle_massive(method="geometric")
    I.sectors[1].weight = 3
    J = Integral.from_text(I.to_text())
    assert [s.weight for s in J.sectors] == [1, 3, 1]
    a = oracle.SectorView(I, 1, [])
    z = cbc_fast(1009, 2)
    o3, _, _ = oracle.shift_sums(a, 1009, z, oracle.shifts(1, 1, 2, 2), 0, 1)
    I.sectors[1].weight = 1
    o1, _, _ = oracle.shift_sums(oracle.SectorView(I, 1, []), 1009, z, oracle.shifts(1, 1, 2, 2), 0, 1)
    assert np.allclose(o3, 3 * o1, rtol=1e-15, atol=0)


def test_simplicial_cones_cover_every_direction_once():
    # the triangulated normal fan of the double box's Newton polytope: every
    # (generic) direction lies in exactly one simplicial cone
    from paper_2305_19768_gb300.inputs.feynman import exponents, symanzik

    g = w.Graph(edges=[(0, 1), (1, 2), (2, 5), (5, 4), (4, 3), (3, 0), (1, 4)], masses_sq=[Fraction(0)] * 7,
                legs=[3, 0, 2, 5], kin=w.kin_massless_4pt(), name="dbox")
    U, F = symanzik(g)
    secs = geometric.decompose_geometric(U, F, *exponents(7, 2, 4))
    import ast

    cones = [np.array(ast.literal_eval(s.origin[len("cone "):]), dtype=float) for s in secs]
    assert all(abs(round(np.linalg.det(C))) == s.weight for C, s in zip(cones, secs))
    Y = np.random.default_rng(7).normal(size=(20000, 6))
    counts = np.zeros(len(Y), int)
    for C in cones:
        counts += np.all(np.linalg.solve(C.T, Y.T) >= -1e-12, axis=0)
    assert np.all(counts == 1), np.bincount(counts)
