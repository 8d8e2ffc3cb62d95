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
            assert_close(out[sector, shift][None], o, a, c, what=f"double box sector {sector} (ns={ns}) shift {shift}")
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
            assert_close(out[j, shift][None], o, a, c, what=f"{name} job {j} shift {shift}")
    finally:
        g.close()
