"""The physical-region batch: massive box at seeded (s, t) points, lambda
chosen per (point, sector) by presampling, all jobs in one persistent launch,
CUDA-graph replay and the autotuner; sampled jobs checked against the oracle."""
import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

from parity import assert_close, oracle_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    ctx = qmc.qmc_create(0, presamples=4000)
    qmc.load_lattice_table(ctx)
    I = w.box_massive()
    iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
    pts = w.massive_box_points(1024, seed=3)
    qmc.qmc_set_kinematics(ctx, pts)
    yield ctx, I, iid, pts
    qmc.qmc_destroy(ctx)


def test_presampled_batch_of_1024_points_matches_oracle(batch):
    ctx, I, iid, pts = batch
    specs = qmc.jobs_for_integral(iid, 4, 1024, 10007, 4, seed=11)
    jobs, nj = qmc.make_jobs(specs)
    lam, rc = qmc.qmc_presample_lambda(ctx, jobs, nj, 0, 1, lambda_max=1.0, ncand=10)
    assert rc == 0 and np.all(lam > 0) and np.all(lam <= 1.0)
    plan = qmc.qmc_plan_create(ctx, jobs, nj, 0, 1)
    try:
        qmc.qmc_plan_run(ctx, plan)
        out, fails, rc = qmc.qmc_plan_results(ctx, plan, check=False)
        assert rc == 0 and fails == 0
        assert np.all(qmc.qmc_plan_job_failures(ctx, plan, nj) == 0)
        ms, ms_eval, nl = qmc.qmc_plan_last_time(ctx, plan)
        assert nl == 2  # one evaluator launch for all 4096 jobs, one finish
        out = out.reshape(nj, 4, 1, 2)
        for j in (0, 1, 2051, 4095):
            sp = specs[j]
            o, a, c = oracle_sums(I, sp["sector"], list(pts[sp["point"]]), 10007, 4, 11, sp["stream"], 0, 1,
                                  lam=lam[j])
            assert_close(out[j], o, a, c, what=f"job {j}")
        # graph replay: identical results
        qmc.qmc_plan_use_graph(ctx, plan, True)
        for _ in range(2):
            qmc.qmc_plan_run(ctx, plan)
            out2, _, _ = qmc.qmc_plan_results(ctx, plan)
            assert np.array_equal(out2.reshape(out.shape), out)
            ms_g, ms_eval_g, nl_g = qmc.qmc_plan_last_time(ctx, plan)
            assert nl_g == 2 and 0 < ms_eval_g <= ms_g
    finally:
        qmc.qmc_plan_destroy(plan)


def test_presampling_keeps_the_largest_lambda_for_quadratic_F(batch):
    # one-loop F is quadratic in the Feynman parameters, so along the deformed
    # contour Im F(z) = -lambda sum_k t_k (1 - t_k) (dF/dt_k)^2 <= 0 for every
    # lambda > 0: no candidate can fail the sign check and the search keeps the
    # first (largest) one. (A lambda of the wrong sign is caught by the sign
    # check; qmc_integrate then presamples again -- test_gpu_integrate.)
    ctx, I, iid, pts = batch
    specs = qmc.jobs_for_integral(iid, 4, 4, 1009, 2, seed=2)
    jobs, nj = qmc.make_jobs(specs)
    lam, rc = qmc.qmc_presample_lambda(ctx, jobs, nj, 0, 1, lambda_max=8.0, ncand=16)
    assert rc == 0 and np.all(lam == 8.0)
    plan = qmc.qmc_plan_create(ctx, jobs, nj, 0, 1)
    try:
        qmc.qmc_plan_run(ctx, plan)
        _, fails, rc = qmc.qmc_plan_results(ctx, plan, check=False)
        assert rc == 0 and fails == 0
    finally:
        qmc.qmc_plan_destroy(plan)


def test_autotune_keeps_results(batch):
    ctx, I, iid, pts = batch
    specs = qmc.jobs_for_integral(iid, 4, 8, 20011, 4, seed=5, lam=0.3)
    jobs, nj = qmc.make_jobs(specs)
    ref = qmc.qmc_eval_jobs(ctx, jobs, nj, 0, 1, nj * 4 * 2)
    bb, bp = qmc.qmc_autotune(ctx, jobs, nj, 0, 1)
    assert bb[1] in (128, 256) and bp[1] in (1, 2, 4, 8, 16, 32)
    got = qmc.qmc_eval_jobs(ctx, jobs, nj, 0, 1, nj * 4 * 2)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale
