"""The adaptive driver qmc_integrate on the GPU: the requested accuracy is
reached and the values agree with the closed forms within their errors;
amplitudes with coefficient series; timeout and lattice-limit statuses."""
import numpy as np
import pytest

from golden_values import closed_form
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w

pytestmark = pytest.mark.gpu


def _ctx(**opts):
    ctx = qmc.qmc_create(0, **opts)
    qmc.load_lattice_table(ctx)
    return ctx


def _within(val, err, exact, nsig=4.0):
    sig = np.hypot(err.real, err.imag)
    assert abs(val - exact) <= nsig * sig + 1e-13 * abs(exact), (val, exact, sig)


def test_massless_box_to_1e_6():
    ctx = _ctx()
    try:
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-6, lowest_order=-2, norders=3)
        assert rc == 0
        ex = closed_form("box1L_massless", "s=-3,t=-2")
        for o, order in enumerate((-2, -1, 0)):
            _within(val[0, 0, o], err[0, 0, o], ex[order])
            assert np.hypot(err[0, 0, o].real, err[0, 0, o].imag) <= 1e-6 * abs(val[0, 0, o]) * 1.0000001
        assert info["iterations"] >= 1 and info["evaluations"] > 0
    finally:
        qmc.qmc_destroy(ctx)


def test_amplitude_with_coefficient_series():
    # A = (2 - eps) box(s,t) + 3 triangle: coefficients as Laurent series
    ctx = _ctx()
    try:
        box = w.box_massless()
        tri = w.triangle_massive()
        ib = qmc.qmc_load_sectors_mem(ctx, box.to_text())
        it = qmc.qmc_load_sectors_mem(ctx, tri.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        coef = np.zeros((1, 1, 2, 2), dtype=complex)
        coef[0, 0, 0] = [2.0, -1.0]
        coef[0, 0, 1] = [3.0, 0.0]
        val, err, info, rc = qmc.qmc_integrate(ctx, [ib, it], coef=coef, coef_lo=0, epsrel=1e-7,
                                               lowest_order=-2, norders=3)
        assert rc == 0
        b = closed_form("box1L_massless", "s=-3,t=-2")
        t0 = closed_form("triangle_m1_pm1")[0]
        exact = [2 * b[-2], 2 * b[-1] - b[-2], 2 * b[0] - b[-1] + 3 * t0]
        for o in range(3):
            _within(val[0, 0, o], err[0, 0, o], exact[o])
    finally:
        qmc.qmc_destroy(ctx)


def test_several_points_and_physical_deformed_bubble():
    ctx = _ctx(**{"lambda": 0.5})
    try:
        I = w.bubble(1, "s")
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[10.0], [-3.0]]))
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-9, lowest_order=-1, norders=2,
                                               npoints=2)
        assert rc == 0
        for p, s in enumerate((10, -3)):
            ex = closed_form("bubble_m1", f"s={s}")
            _within(val[p, 0, 0], err[p, 0, 0], ex[-1])
            _within(val[p, 0, 1], err[p, 0, 1], ex[0])
    finally:
        qmc.qmc_destroy(ctx)


def test_lattice_limit_and_timeout_statuses():
    ctx = _ctx(max_points=20011)
    try:
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-13, lowest_order=-2, norders=3,
                                               check=False)
        assert rc == -5 and info["max_lattice"] <= 20011
        assert np.all(np.isfinite(val))
    finally:
        qmc.qmc_destroy(ctx)
    ctx = _ctx()
    try:
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-14, timeout=1e-9, lowest_order=-2,
                                               norders=3, check=False)
        assert rc == -4 and info["iterations"] == 1
    finally:
        qmc.qmc_destroy(ctx)


def test_sign_check_failure_is_presampled_again():
    # a deformation parameter of the wrong sign, handed in per slot, puts F(z) on
    # the wrong side of the cut at every point: the driver must presample that
    # slot again, evaluate it once more and agree with the presampled run
    I = w.box_massive()
    vals = []
    for lam_in in (None, -0.5):
        ctx = _ctx()
        try:
            iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
            qmc.qmc_set_kinematics(ctx, np.array([[10.0, -3.0]]))
            lam = None if lam_in is None else np.full(len(I.sectors), lam_in)
            val, err, info, rc, wv, nv = qmc.qmc_integrate(ctx, [iid], epsrel=1e-5, lowest_order=0, norders=1,
                                                           nslots=len(I.sectors), lambda_io=lam, check=False)
            assert rc == 0, qmc.qmc_last_error(ctx)
            if lam is not None:
                assert np.all(lam > 0)
            vals.append((val[0, 0, 0], err[0, 0, 0]))
        finally:
            qmc.qmc_destroy(ctx)
    (a, ea), (b, eb) = vals
    sig = np.hypot(abs(ea), abs(eb))
    assert abs(a - b) <= 5 * sig


def test_mixed_precision_escalates_to_fp64_at_the_lattice_cap():
    # with the lattice capped at the pilot size and a request the pilot cannot
    # meet, every mixed-precision sector is evaluated again in FP64; an FP64
    # context never escalates
    I = w.box_massless()
    for precision, expect in ((qmc.QMC_PRECISION_MIXED, True), (qmc.QMC_PRECISION_FP64, False)):
        ctx = _ctx(precision=precision, max_points=1009, min_points=1009)
        try:
            iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
            qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
            val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-10, lowest_order=-2, norders=3,
                                                   check=False)
            assert rc == -5
            assert (info["fp64_escalations"] > 0) == expect, info
            if expect:
                assert info["fp64_escalations"] == len(I.sectors)
        finally:
            qmc.qmc_destroy(ctx)


def test_amplitude_with_coefficient_strings():
    # the coefficient-series amplitude of test_amplitude_with_coefficient_series,
    # given as strings: parsed, expanded exactly, handed to the same call
    from paper_2305_19768_gb300.inputs.coefficients import coefficient_series

    coef, coef_lo = coefficient_series([["(4 - eps^2)/(2 + eps)", "6/2"]], 2, [{"s": -3.0, "t": -2.0}], 1)
    assert coef_lo == 0 and coef.shape == (1, 1, 2, 2)
    assert np.array_equal(coef[0, 0], np.array([[2.0, -1.0], [3.0, 0.0]]))
    ctx = _ctx()
    try:
        ib = qmc.qmc_load_sectors_mem(ctx, w.box_massless().to_text())
        it = qmc.qmc_load_sectors_mem(ctx, w.triangle_massive().to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        val, err, info, rc = qmc.qmc_integrate(ctx, [ib, it], coef=coef, coef_lo=coef_lo, epsrel=1e-7,
                                               lowest_order=-2, norders=3)
        assert rc == 0
        b = closed_form("box1L_massless", "s=-3,t=-2")
        t0 = closed_form("triangle_m1_pm1")[0]
        exact = [2 * b[-2], 2 * b[-1] - b[-2], 2 * b[0] - b[-1] + 3 * t0]
        for o in range(3):
            _within(val[0, 0, o], err[0, 0, o], exact[o])
    finally:
        qmc.qmc_destroy(ctx)


def test_median_rules_inside_integrate_match_the_closed_form():
    # lattice_candidates = 11: per (point, sector) and lattice size the median
    # of 11 unshifted candidate rules (Eq. (median)), lattices of any prime size
    ctx = _ctx(lattice_candidates=11, min_points=30000)
    try:
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0]]))
        val, err, info, rc, _, nq = qmc.qmc_integrate(ctx, [iid], epsrel=1e-8, lowest_order=-2, norders=3,
                                                      nslots=12)
        assert rc == 0
        ex = closed_form("box1L_massless", "s=-3,t=-2")
        for o, order in enumerate((-2, -1, 0)):
            _within(val[0, 0, o], err[0, 0, o], ex[order], nsig=5.0)
            assert np.hypot(err[0, 0, o].real, err[0, 0, o].imag) <= 1e-8 * abs(val[0, 0, o]) * 1.0000001
        assert info["median_evaluations"] >= 11 * 12 * 30011
        assert all(int(n) >= 30011 for n in nq)
    finally:
        qmc.qmc_destroy(ctx)


def test_weighted_sums_of_set_coefficients_and_per_integral_results():
    ctx = _ctx(keep_shift_sums=1, shifts=16)
    try:
        box = w.box_massless()
        geo = w.box_massless(method="geometric")
        ib = qmc.qmc_load_sectors_mem(ctx, box.to_text())
        ig = qmc.qmc_load_sectors_mem(ctx, geo.to_text())
        kin = np.array([[-3.0, -2.0], [-5.0, -1.0]])
        qmc.qmc_set_kinematics(ctx, kin)
        C = np.zeros((2, 1, 2, 1), dtype=complex)
        C[:, 0, 0, 0], C[:, 0, 1, 0] = 1.0, -1.0          # box minus the same box decomposed differently
        qmc.qmc_set_coefficients(ctx, C)
        val, err, info, rc = qmc.qmc_integrate(ctx, None, epsrel=0.0, epsabs=1e-7, lowest_order=-2, norders=3,
                                               npoints=2)
        assert rc == 0
        for p, pt in enumerate(("s=-3,t=-2", "s=-5,t=-1")):
            ex = closed_form("box1L_massless", pt)
            for o in range(3):
                _within(val[p, 0, o], err[p, 0, o], 0.0, nsig=5.0)     # the difference vanishes
            for iid in (ib, ig):
                v, e = qmc.qmc_integral_results(ctx, iid, 2, 3)
                for o, order in enumerate((-2, -1, 0)):
                    _within(v[p, o], e[p, o], ex[order], nsig=5.0)
        sums, slo, n = qmc.qmc_per_shift_sums(ctx, ib)
        assert sums.shape == (2, 12, 16, 3, 2) and slo == -2
        ev, secs = qmc.qmc_stats(ctx)
        assert ev >= info["evaluations"] and secs >= info["seconds"]
    finally:
        qmc.qmc_destroy(ctx)


def _gpu_rank_worker(rank, port, world, result_dir):
    import os

    import torch.distributed as dist

    from paper_2305_19768_gb300 import dist as qdist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ctx = _ctx(keep_shift_sums=1, shifts=8, max_points=200003)
    try:
        I = w.box_massless()
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array([[-3.0, -2.0], [-5.0, -1.0], [-2.0, -7.0]]))
        if world > 1:
            qdist.set_ranks(ctx)
        val, err, info, rc = qmc.qmc_integrate(ctx, [iid], epsrel=1e-14, lowest_order=-2, norders=3, npoints=3,
                                               check=False)
        sums, _, n = qmc.qmc_per_shift_sums(ctx, iid)
        if rank == 0:
            np.savez(os.path.join(result_dir, f"g{world}.npz"), val=val, err=err, sums=sums, n=n, rc=rc,
                     evals=info["evaluations"], iters=info["iterations"])
    finally:
        qmc.qmc_destroy(ctx)
        dist.destroy_process_group()


def test_two_ranks_partition_the_integration_and_equal_one_rank(tmp_path):
    """Two processes (gloo exchange on the host), each evaluating its share of
    the (point, sector) slots on the GPU: the result equals one process bit
    for bit. The ranks' kernels never wait on each other; the exchange runs on
    the host between passes."""
    import socket

    import torch.multiprocessing as mp

    res = {}
    for world in (1, 2):
        with socket.socket() as s:
            s.bind(("127.0.0.1", 0))
            port = s.getsockname()[1]
        mp.start_processes(_gpu_rank_worker, args=(port, world, str(tmp_path)), nprocs=world, start_method="spawn")
        res[world] = np.load(tmp_path / f"g{world}.npz")
    a, b = res[1], res[2]
    assert int(a["iters"]) >= 2
    for k in ("val", "err", "sums", "n", "rc", "evals", "iters"):
        assert np.array_equal(a[k], b[k]), k
