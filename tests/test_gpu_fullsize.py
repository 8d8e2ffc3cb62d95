"""The bench workloads other than the default one at their full sizes and in
the launch configuration bench.py times (context defaults, one plan for all
jobs): sampled outputs recomputed by the oracle one by one, plus a property
that holds at any size."""
import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

from parity import Gpu, assert_close, oracle_sums

pytestmark = pytest.mark.gpu


def test_double_box_full_size_sampled_outputs():
    g = Gpu()
    try:
        I = w.double_box_massless()
        iid = g.load(I)
        s_, t_ = -3.0, -1.0
        qmc.qmc_set_kinematics(g.ctx, np.array([[s_, t_]]))
        n, m, nsec = 1000003, 32, len(I.sectors)
        specs = qmc.jobs_for_integral(iid, nsec, 1, n, m)
        out, _, rc = g.eval(iid, specs, -4, 5)
        assert rc == 0
        out = out.reshape(nsec, m, 5, 2)
        by_ns = {}
        for i, sec in enumerate(I.sectors):
            by_ns.setdefault(len(sec.singular), i)
        for k, (ns, sector) in enumerate(sorted(by_ns.items())):
            shift = (7 * k + 3) % m
            o, a, c = oracle_sums(I, sector, [s_, t_], n, m, 1, sector, -4, 5, shift_rows=[shift])
            assert_close(out[sector, shift][None], o, a, c, lo=-4,
                         what=f"box2L_planar_massless n={n} sector {sector} (ns={ns}) shift {shift}")
        # leading pole of the sum: (prefactor x sectors) at eps^-4 equals 4 / (s^2 t)
        tot = (out[..., 0, 0] + 1j * out[..., 0, 1]).sum(axis=0)       # [m]
        c4 = (I.prefactor[0] * tot).real * s_ * s_ * t_
        assert abs(c4.mean() - 4.0) <= 4 * c4.std(ddof=1) / np.sqrt(m) + 1e-9
    finally:
        g.close()


@pytest.mark.parametrize("name", ["box1L_massive_batch", "box1L_massless_physical"])
def test_deformed_batches_full_size_sampled_outputs(name):
    g = Gpu()
    try:
        if name == "box1L_massive_batch":
            I, lo, nord = w.box_massive(), 0, 1
        else:
            I, lo, nord = w.box_massless(deform=True), -2, 3
        pts = w.massive_box_points(1024, seed=3)
        iid = g.load(I)
        qmc.qmc_set_kinematics(g.ctx, pts)
        n, m, nsec = 10007, 32, len(I.sectors)
        specs = qmc.jobs_for_integral(iid, nsec, len(pts), n, m)
        jobs, nj = qmc.make_jobs(specs)
        lam, rc = qmc.qmc_presample_lambda(g.ctx, jobs, nj, lo, nord, lambda_max=1.0, ncand=16)
        assert rc == 0
        for sp, L in zip(specs, lam):
            sp["lambda"] = float(L)
        out, fails, rc = g.eval(iid, specs, lo, nord)
        assert rc == 0 and fails == 0
        out = out.reshape(nj, m, nord, 2)
        for j, shift in ((0, 0), (nsec * 517 + 1, 13), (nj - 1, 31)):
            sp = specs[j]
            o, a, c = oracle_sums(I, sp["sector"], list(pts[sp["point"]]), n, m, 1, sp["stream"], lo, nord,
                                  lam=sp["lambda"], shift_rows=[shift])
            assert_close(out[j, shift][None], o, a, c, lo=lo, what=f"{name} n={n} job {j} shift {shift}")
    finally:
        g.close()


def test_double_box_every_class_on_the_large_tile_path():
    """Two sectors of each singular-variable count (the REAL6S, REAL6T and
    REAL6 classes) at n = 100003, where plans use 2048-point tiles, every
    shift compared element by element with the oracle."""
    g = Gpu()
    try:
        I = w.double_box_massless()
        iid = g.load(I)
        s_, t_ = -3.0, -1.0
        qmc.qmc_set_kinematics(g.ctx, np.array([[s_, t_]]))
        by_ns = {}
        for i, sec in enumerate(I.sectors):
            by_ns.setdefault(len(sec.singular), []).append(i)
        sectors = [i for ns in sorted(by_ns) for i in (by_ns[ns][0], by_ns[ns][-1])]
        n, m = 100003, 3
        specs = [dict(integral_id=iid, sector=s, point=0, shifts=m, n=n, seed=1, stream=s) for s in sectors]
        out, _, rc = g.eval(iid, specs, -4, 5)
        assert rc == 0
        out = out.reshape(len(sectors), m, 5, 2)
        for k, s in enumerate(sectors):
            o, a, c = oracle_sums(I, s, [s_, t_], n, m, 1, s, -4, 5)
            assert_close(out[k], o, a, c, lo=-4,
                         what=f"box2L_planar_massless n={n} sector {s} (ns={len(I.sectors[s].singular)})")
    finally:
        g.close()


MIX_RTOL, MIX_CTOL = 1e-6, 2e-7


def _mixed_vs_oracle(I, inv, sectors, n, m, lo, norders, lam=None, sample_shifts=None):
    ctx = qmc.qmc_create(0, precision=qmc.QMC_PRECISION_MIXED)
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
    for k, s in enumerate(sectors):
        rows = list(range(m)) if sample_shifts is None else [sample_shifts[k % len(sample_shifts)]]
        o, a, c = oracle_sums(I, s, inv, n, m, 1, s, lo, norders, lam, shift_rows=rows)
        assert_close(out[k][rows], o, a, c, rtol=MIX_RTOL, ctol=MIX_CTOL, lo=lo,
                     what=f"{I.name} mixed n={n} sector {s}")


def test_mixed_classes_on_the_large_tile_path():
    """Every mixed-precision class (FP32 monomial products) against the FP64
    oracle at n = 20011 (2048-point tiles): REAL3M on the massless box,
    CPLX3M on the deformed massive box, REAL6SM/REAL6TM/REAL6M on the double
    box."""
    _mixed_vs_oracle(w.box_massless(), [-3.0, -2.0], list(range(12)), 20011, 4, -2, 3)
    _mixed_vs_oracle(w.box_massive(), [10.0, -3.0], list(range(4)), 20011, 4, 0, 1, lam=0.8)
    I = w.double_box_massless()
    by_ns = {}
    for i, sec in enumerate(I.sectors):
        by_ns.setdefault(len(sec.singular), i)
    _mixed_vs_oracle(I, [-3.0, -1.0], [by_ns[k] for k in sorted(by_ns)], 20011, 2, -4, 5)


def test_mixed_box_full_size_sampled_outputs():
    """The bench's mixed-precision pass at full size (massless box, n =
    1000003, 32 shifts, all 12 sectors in one plan): sampled (sector, shift)
    outputs against the FP64 oracle."""
    _mixed_vs_oracle(w.box_massless(), [-3.0, -2.0], list(range(12)), 1000003, 32, -2, 3,
                     sample_shifts=[0, 17, 31, 5])
