"""Host side of the Taylor subtraction (exponents a_j <= -2), without a GPU:
the sector loader's limits in a host-only context, and qmc_integrate with the
oracle as its evaluator on sectors whose integral is an exact finite sum."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

from oracle_eval import make_evaluator
from test_oracle_pins import _series_of_inverse_linear, _toy_integral


def _host(**opts):
    ctx = qmc.qmc_create(qmc.QMC_DEVICE_NONE, **opts)
    qmc.load_lattice_table(ctx)
    return ctx


def test_loader_accepts_every_degree_and_rejects_the_rest():
    ctx = _host()
    try:
        qmc.qmc_load_sectors_mem(ctx, w.box_massless_d2().to_text())          # two a = -2, d = 3
        qmc.qmc_load_sectors_mem(ctx, w.double_box_massless_d2().to_text())   # down to -4, boxes <= 72
        toy = lambda a, b: _toy_integral(len(a), a, b, {tuple([0] * len(a)): 1, tuple([1] * len(a)): 2})
        qmc.qmc_load_sectors_mem(ctx, toy([-4], [1]).to_text())
        qmc.qmc_load_sectors_mem(ctx, toy([-2, -2, 0, -1], [1, -1, 0, 2]).to_text())
        rejects = [toy([-5], [1]),                        # beyond degree 3
                   toy([-4, -4, -4, -2], [1, 1, 1, 1]),   # box 128 > 72
                   toy([-2, -1], [0, 1])]                 # unregulated
        deformed = toy([-2, -1], [1, 1])
        deformed.sectors[0].deform = True                 # a = -2 in a deformed d = 2 sector: accepted
        qmc.qmc_load_sectors_mem(ctx, deformed.to_text())
        qmc.qmc_load_sectors_mem(ctx, w.box_massless_d2(deform=True).to_text())
        wide = toy([-2, -2, 0, -1], [1, -1, 0, 2])
        wide.sectors[0].deform = True                     # deformed with d = 4: rejected
        rejects.append(wide)
        for I in rejects:
            with pytest.raises(qmc.QmcError) as e:
                qmc.qmc_load_sectors_mem(ctx, I.to_text())
            assert e.value.code == -1
    finally:
        qmc.qmc_destroy(ctx)


def test_integrate_with_degree2_subtraction_reaches_the_exact_sum():
    # int t^{-3 + b eps} (1 + 2 t + 3 t^2 - t^3 + t^4/2) dt = sum_k c_k / (k - 2 + b eps),
    # through qmc_integrate (baker transform, oracle evaluator): the value per eps
    # order within the reported error and the reported error below the request.
    # (The remainder's border cancellation, about 2^-53 (2u)^-3 per point, keeps
    # this sector from converging much below 1e-5 at any lattice size.)
    b = 1.25
    coefs = {(0,): 1.0, (1,): 2.0, (2,): 3.0, (3,): -1.0, (4,): 0.5}
    I = _toy_integral(1, [-3], [b], coefs)
    lo, no = -1, 3
    exact = sum(c * _series_of_inverse_linear(e[0] - 2, b, lo, no) for e, c in coefs.items())
    ctx = _host(transform=1, max_growth=4)
    try:
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_evaluator(ctx, make_evaluator({iid: I}, [], transform=1))
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-4, lowest_order=lo, norders=no, timeout=60)
        assert rc == 0
        v, e = val[0, 0], err[0, 0]
        for o in range(no):
            sig = abs(e[o].real) + abs(e[o].imag)
            assert abs(v[o] - exact[o]) <= 4 * sig + 1e-12 * abs(exact[o]), (o, v[o], exact[o], sig)
            assert sig <= 1e-4 * np.max(np.abs(exact))
    finally:
        qmc.qmc_destroy(ctx)
