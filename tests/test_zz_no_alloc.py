"""The no-allocation entry point against the allocating one (GPU).

qmc_eval_jobs_noalloc serves callers that cannot allocate device memory at
evaluation time (a real-time loop that must not meet cudaMalloc's implicit
synchronisation, a host whose device memory belongs to a fixed-budget
allocator): it keeps its scratch in a fixed array in device memory instead
of calling cudaMalloc. Here it must reproduce qmc_eval_jobs,
within the parity tolerance of the other GPU tests, on two calls in a row
(the second call sees the array the first one left behind). This file is
collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _close(a, b):
    scale = np.maximum(np.abs(b), np.abs(b).max())
    assert np.all(np.abs(a - b) <= RTOL * scale), float(np.max(np.abs(a - b) / scale))


def test_noalloc_matches_allocating_entry_point_twice():
    import torch

    ctx = qmc.qmc_create(0)
    try:
        qmc.load_lattice_table(ctx)
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0], [-5.0, -1.0]]))
        specs = qmc.jobs_for_integral(iid, len(I.sectors), 2, 20011, 8, seed=3)
        jobs, nj = qmc.make_jobs(specs)
        size = nj * 8 * 3 * 2
        ref = qmc.qmc_eval_jobs(ctx, jobs, nj, -2, 3, size)
        out = torch.full((size,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            qmc.qmc_eval_jobs_noalloc(ctx, jobs, nj, -2, 3, out.data_ptr())
            _close(out.cpu().numpy(), ref)
            out.fill_(float("nan"))
        # a second workload through the same array: deformed sectors
        Im = w.box_massive()
        iid2 = qmc.qmc_load_sectors_mem(ctx, Im.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[12.0, -3.0], [7.5, -1.5]]))
        specs2 = qmc.jobs_for_integral(iid2, len(Im.sectors), 2, 4001, 4, seed=5, lam=0.3)
        jobs2, nj2 = qmc.make_jobs(specs2)
        size2 = nj2 * 4 * 1 * 2
        ref2 = qmc.qmc_eval_jobs(ctx, jobs2, nj2, 0, 1, size2)
        out2 = torch.empty(size2, dtype=torch.float64, device="cuda")
        for _ in range(2):
            qmc.qmc_eval_jobs_noalloc(ctx, jobs2, nj2, 0, 1, out2.data_ptr())
            _close(out2.cpu().numpy(), ref2)
        # beyond the fixed scratch: rejected with a clear error, nothing run
        big = qmc.jobs_for_integral(iid, len(I.sectors), 1, 1000003, 32)
        jb, nb = qmc.make_jobs(big)
        with pytest.raises(qmc.QmcError) as e:
            qmc.qmc_eval_jobs_noalloc(ctx, jb, nb, -2, 3, out.data_ptr())
        assert e.value.code == -1 and "fixed scratch" in str(e.value)
    finally:
        qmc.qmc_destroy(ctx)


def test_noalloc_on_a_caller_stream_and_in_mixed_precision():
    import torch

    ctx = qmc.qmc_create(0, precision=qmc.QMC_PRECISION_MIXED)
    try:
        qmc.load_lattice_table(ctx)
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        specs = qmc.jobs_for_integral(iid, len(I.sectors), 1, 10007, 4, seed=9)
        jobs, nj = qmc.make_jobs(specs)
        size = nj * 4 * 3 * 2
        ref = qmc.qmc_eval_jobs(ctx, jobs, nj, -2, 3, size)   # the mixed-precision class
        st = torch.cuda.Stream()
        out = torch.full((size,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):
            qmc.qmc_eval_jobs_noalloc(ctx, jobs, nj, -2, 3, out.data_ptr(), st.cuda_stream)
            _close(out.cpu().numpy(), ref)
    finally:
        qmc.qmc_destroy(ctx)


def test_noalloc_rejections():
    import torch

    ctx = qmc.qmc_create(0)
    try:
        qmc.load_lattice_table(ctx)
        I = w.box_massless()
        Im = w.box_massive()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        iid2 = qmc.qmc_load_sectors_mem(ctx, Im.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        out = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")

        def expect_inval(specs, what):
            jobs, nj = qmc.make_jobs(specs)
            with pytest.raises(qmc.QmcError) as e:
                qmc.qmc_eval_jobs_noalloc(ctx, jobs, nj, -2, 3, out.data_ptr())
            assert e.value.code == -1, what
            return str(e.value)

        one = dict(integral_id=iid, sector=0, point=0, shifts=1, n=1009, seed=1, stream=0)
        msg = expect_inval([dict(one, stream=i) for i in range(257)], "257 jobs")
        assert "256" in msg
        msg = expect_inval([one, dict(one, integral_id=iid2, **{"lambda": 0.5})], "two classes")
        assert "one evaluator class" in msg
        msg = expect_inval([dict(one, z=[1, 3, 5])], "explicit z")
        assert "qmc_eval_jobs" in msg
        # three invariants per point for an integral that has two
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0, 1.0]]))
        msg = expect_inval([one], "invariant count")
        assert "invariants" in msg
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        # a stream being captured into a graph is refused before any work
        jobs, nj = qmc.make_jobs([one])
        st = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        x = torch.zeros(4, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            g.capture_begin()
            try:
                with pytest.raises(qmc.QmcError) as e:
                    qmc.qmc_eval_jobs_noalloc(ctx, jobs, nj, -2, 3, out.data_ptr(), st.cuda_stream)
                x.add_(1.0)
            finally:
                g.capture_end()
        assert e.value.code == -1 and "captured" in str(e.value)
        g.replay()
        torch.cuda.synchronize()
        assert float(x.sum()) == 4.0
        # the context still evaluates afterwards
        qmc.qmc_eval_jobs_noalloc(ctx, jobs, nj, -2, 3, out.data_ptr())
        ref = qmc.qmc_eval_jobs(ctx, jobs, nj, -2, 3, 6)
        _close(out[:6].cpu().numpy(), ref)
    finally:
        qmc.qmc_destroy(ctx)
