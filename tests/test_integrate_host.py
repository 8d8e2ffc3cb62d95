"""The integration driver's host logic in host-only contexts (no GPU): the
library's qmc_integrate with the CPU oracle installed as its evaluator.
Covers the weighted sums of qmc_set_coefficients, the per-integral results,
the kept per-shift sums, the context statistics, median QMC rules
(lattice_candidates), the unbatched mode, and the rank-partitioned
integration with world size 2 over gloo, which must return the one-rank
result bit for bit."""
import os

import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

from golden_values import closed_form
from oracle_eval import make_evaluator

KIN = [[-3.0, -2.0], [-5.0, -1.0]]


def _host_ctx(integrals, kin, **opts):
    ctx = qmc.qmc_create(qmc.QMC_DEVICE_NONE, **opts)
    qmc.load_lattice_table(ctx)
    ids = {}
    for I in integrals:
        ids[qmc.qmc_load_sectors_mem(ctx, I.to_text())] = I
    if kin is not None:
        qmc.qmc_set_kinematics(ctx, np.array(kin))
    qmc.qmc_set_evaluator(ctx, make_evaluator(ids, kin if kin is not None else []))
    return ctx, list(ids)


def test_host_only_context_refuses_gpu_work():
    ctx = qmc.qmc_create(qmc.QMC_DEVICE_NONE)
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, w.box_massless().to_text())
        qmc.qmc_set_kinematics(ctx, np.array(KIN[:1]))
        jobs, nj = qmc.make_jobs(qmc.jobs_for_integral(iid, 12, 1, 1009, 2))
        with pytest.raises(qmc.QmcError) as e:
            qmc.qmc_eval_jobs(ctx, jobs, nj, -2, 3, 12 * 2 * 3 * 2)
        assert e.value.code == -3
        with pytest.raises(qmc.QmcError) as e:    # no evaluator installed
            qmc.qmc_integrate(ctx, [iid], epsrel=1e-2, lowest_order=-2, norders=3)
        assert e.value.code == -3
    finally:
        qmc.qmc_destroy(ctx)


def test_coefficients_integral_results_kept_sums_and_stats():
    # the same integral by two decompositions, combined with Laurent
    # coefficients into two amplitudes per kinematic point
    Ia, Ib = w.box_massless(), w.box_massless(method="geometric")
    ctx, ids = _host_ctx([Ia, Ib], KIN, shifts=6, min_points=1009, max_points=20011, keep_shift_sums=1)
    try:
        rng = np.random.default_rng(4)
        C = rng.integers(-3, 4, size=(2, 2, 2, 2)) + 1j * rng.integers(-3, 4, size=(2, 2, 2, 2))
        qmc.qmc_set_coefficients(ctx, C, coef_lo=0)
        e0, _ = qmc.qmc_stats(ctx)
        val, err, info, rc = qmc.qmc_integrate(ctx, None, epsrel=3e-3, lowest_order=-2, norders=3, npoints=2,
                                               namp=2, check=False)
        assert rc in (0, -5)
        e1, secs = qmc.qmc_stats(ctx)
        assert e1 - e0 == info["evaluations"] and secs > 0
        res = [qmc.qmc_integral_results(ctx, i, 2, 3) for i in ids]
        # the amplitudes are the coefficient series times the integrals' series
        for p in range(2):
            for k in range(2):
                for o in range(3):
                    ref = sum(C[p, k, i, c] * res[i][0][p, o - c] for i in range(2) for c in range(2) if o - c >= 0)
                    assert abs(val[p, k, o] - ref) <= 1e-12 * (1 + abs(ref))
        # both decompositions give the closed form within their errors
        for p, pt in enumerate(("s=-3,t=-2", "s=-5,t=-1")):
            ex = closed_form("box1L_massless", pt)
            for i in range(2):
                v, e = res[i]
                for o, order in enumerate((-2, -1, 0)):
                    assert abs(v[p, o].real - ex[order]) <= 5 * e[p, o].real + 1e-12
        # the kept per-shift sums reproduce each integral's value
        for i, I in zip(ids, (Ia, Ib)):
            sums, slo, nfin = qmc.qmc_per_shift_sums(ctx, i)
            assert sums.shape[:3] == (2, len(I.sectors), 6) and slo == -2 and nfin.min() >= 1009
            sec = (sums[..., 0] + 1j * sums[..., 1]).mean(axis=2).sum(axis=1)     # [p][sector orders]
            pref = np.array(I.prefactor)
            for p in range(2):
                for o in range(3):
                    ref = sum(pref[q] * sec[p, o - q] for q in range(len(pref)) if o - q >= 0)
                    assert abs(res[ids.index(i)][0][p, o] - ref) <= 1e-12 * (1 + abs(ref))
    finally:
        qmc.qmc_destroy(ctx)


def test_median_rule_integration_reaches_the_closed_form():
    # lattice_candidates = r: every sector's generating vector is the median of
    # r unshifted candidate rules, on lattices of any prime size
    I = w.triangle_massive()
    ctx, ids = _host_ctx([I], None, shifts=8, min_points=1500, lattice_candidates=11)
    try:
        val, err, info, rc, wq, nq = qmc.qmc_integrate(ctx, ids, epsrel=2e-5, lowest_order=0, norders=1,
                                                       nslots=3)
        assert rc == 0
        ex = closed_form("triangle_m1_pm1", "-")[0].real
        assert abs(val[0, 0, 0].real - ex) <= 5 * err[0, 0, 0].real
        assert info["median_evaluations"] >= 11 * 3 * 1511
        from paper_2305_19768_gb300.inputs.lattice import load_table
        table = {r[0] for r in load_table()}
        for n in nq:
            n = int(n)
            assert all(n % q for q in range(2, int(n ** 0.5) + 1))   # prime
        assert any(int(n) not in table for n in nq)
        with pytest.raises(qmc.QmcError):
            qmc.qmc_create(qmc.QMC_DEVICE_NONE, lattice_candidates=10)   # r must be odd
    finally:
        qmc.qmc_destroy(ctx)


def test_unbatched_mode_agrees_with_batched():
    I = w.box_massless()
    out = {}
    for batched in (0, -1):
        ctx, ids = _host_ctx([I], KIN, shifts=6, min_points=1009, max_points=20011, batched=batched)
        try:
            out[batched] = qmc.qmc_integrate(ctx, ids, epsrel=5e-3, lowest_order=-2, norders=3, npoints=2,
                                             check=False)
        finally:
            qmc.qmc_destroy(ctx)
    (v0, e0, _, _), (v1, e1, _, _) = out[0], out[-1]
    comb = np.sqrt(e0.real ** 2 + e1.real ** 2)
    assert np.all(np.abs(v0.real - v1.real) <= 5 * comb + 1e-12)


def _rank_worker(rank, port, world, result_dir):
    import torch.distributed as dist

    from paper_2305_19768_gb300 import dist as qdist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ctx, ids = _host_ctx([w.box_massless()], KIN, shifts=4, min_points=1009, max_points=20011,
                             keep_shift_sums=1)
        try:
            if world > 1:
                qdist.set_ranks(ctx)
            val, err, info, rc = qmc.qmc_integrate(ctx, [ids[0]], epsrel=1e-9, lowest_order=-2, norders=3,
                                                   npoints=2, check=False)
            sums, _, n = qmc.qmc_per_shift_sums(ctx, ids[0])
            if rank == 0:
                np.savez(os.path.join(result_dir, f"w{world}.npz"), val=val, err=err, sums=sums, n=n,
                         rc=rc, evals=info["evaluations"], iters=info["iterations"])
        finally:
            qmc.qmc_destroy(ctx)
    finally:
        dist.destroy_process_group()


def test_two_rank_integration_equals_one_rank(tmp_path):
    import socket

    import torch.multiprocessing as mp

    res = {}
    for world in (1, 2):
        with socket.socket() as s:
            s.bind(("127.0.0.1", 0))
            port = s.getsockname()[1]
        mp.start_processes(_rank_worker, args=(port, world, str(tmp_path)), nprocs=world, start_method="spawn")
        res[world] = np.load(tmp_path / f"w{world}.npz")
    a, b = res[1], res[2]
    assert int(a["iters"]) >= 2                      # at least one allocation pass ran
    for k in ("val", "err", "sums", "n", "rc", "evals", "iters"):
        assert np.array_equal(a[k], b[k]), k


def test_failed_exchange_or_evaluator_ends_the_integration_with_an_error():
    # failure detection on the host: a rank exchange that reports failure (a
    # peer that left) and an evaluator that fails both end qmc_integrate with
    # an error status, nothing hangs
    I = w.box_massless()
    ctx, ids = _host_ctx([I], KIN[:1], shifts=4, min_points=1009, max_points=20011)
    try:
        def broken(buf):
            raise RuntimeError("peer left")

        qmc.qmc_set_ranks(ctx, 0, 2, broken)
        with pytest.raises(qmc.QmcError) as e:
            qmc.qmc_integrate(ctx, ids, epsrel=1e-9, lowest_order=-2, norders=3)
        assert e.value.code == -1 and "exchange" in str(e.value)
        qmc.qmc_set_ranks(ctx, 0, 1, None)

        def failing(jobs, lo, norders):
            raise RuntimeError("device lost")

        qmc.qmc_set_evaluator(ctx, failing)
        with pytest.raises(qmc.QmcError) as e:
            qmc.qmc_integrate(ctx, ids, epsrel=1e-9, lowest_order=-2, norders=3)
        assert "evaluator failed" in str(e.value)
    finally:
        qmc.qmc_destroy(ctx)
