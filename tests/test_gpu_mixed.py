"""The mixed-precision evaluator (FP32 monomial products, FP64 elsewhere)
against the FP64 oracle, per eps order, for real and deformed sectors, and
the double box through the d <= 6 evaluator against its leading pole.

Tolerance of the mixed path: the FP32 group sums carry a relative error of a
few 2^-24; it reaches the result through the logs and powers of U and F and
is amplified where the subtraction corners cancel, so the bound is
MIX_RTOL * max(|Q|, A) + MIX_CTOL * C with the oracle's absolute mass A and
corner mass C (see tests/parity.py): MIX_RTOL = 1e-6, MIX_CTOL = 2e-7."""
import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

from parity import oracle_sums

pytestmark = pytest.mark.gpu

MIX_RTOL = 1e-6
MIX_CTOL = 2e-7


def _errors(I, inv, sectors, n, m, lo, norders, precision, lam=None):
    ctx = qmc.qmc_create(0, precision=precision)
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([inv]))
        specs = [dict(integral_id=iid, sector=s, point=0, shifts=m, n=n, seed=1, stream=s,
                      **({"lambda": lam} if lam is not None else {})) for s in sectors]
        jobs, nj = qmc.make_jobs(specs)
        out = qmc.qmc_eval_jobs(ctx, jobs, nj, lo, norders, nj * m * norders * 2).reshape(nj, m, norders, 2)
    finally:
        qmc.qmc_destroy(ctx)
    worst = np.zeros(norders)
    for i, s in enumerate(sectors):
        o, a, c = oracle_sums(I, s, inv, n, m, 1, s, lo, norders, lam)
        err = np.abs(out[i] - o).max(axis=(0, 2))
        allow = (MIX_RTOL * np.maximum(np.abs(o).max(axis=(0, 2)), a.max(axis=0)) + MIX_CTOL * c.max(axis=0))
        assert np.all(err <= allow), (s, err, allow)
        worst = np.maximum(worst, err / np.maximum(a.max(axis=0), 1e-300))
    return worst


def test_mixed_box_per_order_error():
    I = w.box_massless()
    worst = _errors(I, [-3.0, -2.0], list(range(12)), 10007, 4, -2, 3, qmc.QMC_PRECISION_MIXED)
    print("mixed massless box, max |err| / A per order eps^-2..eps^0:", worst)


def test_mixed_deformed_per_order_error():
    # deformed sectors: derivatives of F and U, F at z from FP32 monomial
    # products; det J, logs and powers of U and F, assembly in FP64
    worst = _errors(w.box_massive(), [10.0, -3.0], list(range(4)), 10007, 4, 0, 1, qmc.QMC_PRECISION_MIXED,
                    lam=0.8)
    print("mixed massive box (physical), max |err| / A:", worst)
    I = w.box_massless(deform=True)
    worst = _errors(I, [7.0, -2.5], list(range(12)), 4001, 4, -2, 3, qmc.QMC_PRECISION_MIXED, lam=1.0)
    print("mixed massless box (physical), max |err| / A per order eps^-2..eps^0:", worst)


def test_mixed_double_box_per_order_error():
    I = w.double_box_massless()
    by_ns = {}
    for i, s in enumerate(I.sectors):
        by_ns.setdefault(len(s.singular), i)
    worst = _errors(I, [-3.0, -1.0], [by_ns[k] for k in sorted(by_ns)], 1009, 2, -4, 5,
                    qmc.QMC_PRECISION_MIXED)
    print("mixed double box, max |err| / A per order eps^-4..eps^0:", worst)


def test_double_box_leading_pole_on_gpu():
    I = w.double_box_massless()
    ctx = qmc.qmc_create(0)
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        s_, t_ = -3.0, -1.0
        qmc.qmc_set_kinematics(ctx, np.array([[s_, t_]]))
        m, n = 16, 100003
        specs = qmc.jobs_for_integral(iid, len(I.sectors), 1, n, m)
        jobs, nj = qmc.make_jobs(specs)
        out = qmc.qmc_eval_jobs(ctx, jobs, nj, -4, 5, nj * m * 5 * 2).reshape(nj, m, 5, 2)
    finally:
        qmc.qmc_destroy(ctx)
    sec = (out[..., 0] + 1j * out[..., 1]).sum(axis=0)       # [m][5] sum over sectors
    c = (I.prefactor[0] * sec[:, 0]).real * s_ * s_ * t_
    mean, err = c.mean(), c.std(ddof=1) / np.sqrt(m)
    assert abs(mean - 4.0) <= 4 * err + 1e-9, (mean, err)
    assert err < 1e-4
