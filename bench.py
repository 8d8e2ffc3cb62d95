"""Benchmark: randomized rank-1 lattice QMC over the sector-decomposed
two-loop planar massless double box (s = -3, t = -1, D = 4 - 2 eps, orders
eps^-4 .. eps^0; 282 sectors from iterated decomposition in six Feynman
parameters, up to four singular variables), lattice n = 1000003 with a CBC
vector, 32 random shifts per sector: 9.02e9 integrand evaluations per step.

A step is one full evaluation pass: every sector on its lattice with every
shift (lattice point, shift, korobov3, eps-expanded integrand with
subtraction, per-shift reduction), computed by the CUDA kernels behind the
C-ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload box2L_planar_massless|box1L_massless|triangle_massive|
                                box1L_massive_batch|box1L_massless_physical]
                    [--precision fp64|mixed] [--decomposition iterative|geometric]
                    [--gemm M,N,K]

The default line is the double box in FP64; its `extra` holds the one-loop
massless box (s = -3, t = -2, n = 1000003, m = 32) with its time to 1e-4
through qmc_integrate, the mixed-precision (FP32 monomial products) pass of
the double box with its error per eps order against the FP64 oracle, and
the amplitude scan of the learned, batched, mixed-precision form against the
plain FP64 method. The other workloads measure the same metric on the
massless box, the finite massive triangle and the 1024-point deformed
massive-box batches, without extras.

Prints one JSON line (rank 0). Under torchrun each rank evaluates its own
independent batch (its own shift streams): weak scaling, no data-path
collective. ``--impl reference`` times the CPU FP64 oracle on bounded samples
of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "integrand evals/s"
DEFAULT_WORKLOAD = "box2L_planar_massless"
SCAN_TRAIN_STEPS = 600   # Adam steps of the amplitude scan's network
UNIT = "evals/s"
JOB_RECORD_BYTES = 136   # device job record (QmcJobDev) copied per job


def _workloads():
    from paper_2305_19768_gb300.inputs import workloads as w

    return {
        # one-loop massless box, Euclidean point
        "box1L_massless": dict(
            make=lambda method="iterative": w.box_massless(method=method), kin=[[-3.0, -2.0]], lo=-2, nord=3, n=1000003, m=32, deform=False,
            desc="box1L_massless s=-3 t=-2, 12 sectors d=3, eps^-2..eps^0, n={n} CBC, m={m} shifts"),
        # finite massive triangle, p_i^2 = -1, m^2 = 1
        "triangle_massive": dict(
            make=lambda method="iterative": w.triangle_massive(method=method), kin=[[]], lo=0, nord=1, n=100003, m=16, deform=False,
            desc="triangle m^2=1 p_i^2=-1, 3 sectors d=2, eps^0, n={n} CBC, m={m} shifts"),
        # massive box in the physical region: 1024 seeded (s, t), contour deformation
        # with lambda presampled per (point, sector), all jobs in one persistent launch
        "box1L_massive_batch": dict(
            make=w.box_massive, kin=w.massive_box_points(1024, seed=3).tolist(), lo=0, nord=1, n=10007,
            m=32, deform=True,
            desc="box1L_massive m^2=1, 1024 (s,t) s~U[5,20] t~U[-8,-1] seed 3, 4 sectors d=3 deformed, "
                 "eps^0, n={n} CBC, m={m} shifts"),
        # massless box in the physical region at the same 1024 points: deformed
        # sectors with subtraction corners (the amplitude scan's costliest class)
        "box1L_massless_physical": dict(
            make=lambda: w.box_massless(deform=True), kin=w.massive_box_points(1024, seed=3).tolist(), lo=-2,
            nord=3, n=10007, m=32, deform=True,
            desc="box1L_massless deformed, 1024 (s,t) s~U[5,20] t~U[-8,-1] seed 3, 12 sectors d=3, "
                 "eps^-2..eps^0, n={n} CBC, m={m} shifts"),
        # one-loop massless box in D = 2 - 2 eps: every sector has one or two
        # exponents a_j = -2 (Taylor subtraction of degree 1); the baker transform,
        # under which the subtracted remainder keeps its accuracy near the border
        "box1L_massless_d2": dict(
            make=lambda: w.box_massless_d2(), kin=[[-3.0, -2.0]], lo=-2, nord=3, n=100003, m=32, deform=False,
            transform=1,
            desc="box1L_massless in D=2-2eps s=-3 t=-2, 12 sectors d=3 with a_j=-2 (Taylor subtraction), "
                 "eps^-2..eps^0, n={n} CBC, m={m} shifts, baker transform"),
        # the same box at 64 physical points: deformed sectors with a_j = -2
        "box1L_massless_d2_physical": dict(
            make=lambda: w.box_massless_d2(deform=True), kin=w.massive_box_points(64, seed=3).tolist(), lo=-2,
            nord=3, n=10007, m=32, deform=True, transform=1,
            desc="box1L_massless in D=2-2eps deformed, 64 (s,t) s~U[5,20] t~U[-8,-1] seed 3, 12 sectors d=3 "
                 "with a_j=-2 (Taylor subtraction), eps^-2..eps^0, n={n} CBC, m={m} shifts, baker transform"),
        # the default: two-loop planar massless double box, Euclidean point
        "box2L_planar_massless": dict(
            make=lambda method="iterative": w.double_box_massless(method=method), kin=[[-3.0, -1.0]], lo=-4, nord=5, n=1000003, m=32, deform=False,
            desc="box2L_planar_massless s=-3 t=-1, 282 sectors d=6, eps^-4..eps^0, n={n} CBC, m={m} shifts"),
    }

# Figures of one ncu capture of the evaluator for the kernel source with this
# SHA-1 and this workload (any other source or workload reports null):
# traffic = dram__bytes_read.sum + dram__bytes_write.sum per launch;
# fp64_executed_flops_per_eval = (2 DFMA + DMUL + DADD thread instructions)
# per evaluation; fp64_pipe_busy = sm__pipe_fp64_cycles_active of peak;
# warp_inst_per_eval = smsp__inst_executed.sum per evaluation (the issue
# roofline's numerator); issue_busy = smsp__issue_active of peak.
PROFILED = {
    # double box, n = 1000003, m = 32 (the default line): traffic from a 1-pass
    # capture of one full launch; instruction counts and pipe activity from the
    # full capture of the same kernel at n = 20011 (per evaluation, the same code)
    ("76aa350fe61515433bc16a2675f5d037ffad47af", "box2L_planar_massless", "fp64", "iterative", 1000003): {
        "traffic": 1628160 + 3601233152, "fp64_executed_flops_per_eval": 290.7, "fp64_pipe_busy": 0.419,
        "warp_inst_per_eval": 445.4, "issue_busy": 0.364},
}

def kernel_sha1():
    import hashlib

    path = os.path.join(ROOT, "paper_2305_19768_gb300", "csrc", "qmc_kernels.cu")
    with open(path, "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def clock_sampler_start(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        fh = open(path, "w")
        return subprocess.Popen(cmd, stdout=fh, stderr=subprocess.DEVNULL), fh
    except (OSError, FileNotFoundError):
        return None, None


def clock_sampler_stop(proc, fh, path, device_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    fh.close()
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(device_index):
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
    except OSError:
        return None
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_sample(I, inv, n, m, seed, ks, lo, nord, lam=None, transform=0):
    """Oracle per-shift sums of every sector at one kinematic point over lattice
    indices [0, ks): returns (evaluations, seconds, threads)."""
    import oracle
    from paper_2305_19768_gb300.inputs.lattice import lattice_for

    t0 = time.perf_counter()
    evals = 0
    for s in range(len(I.sectors)):
        sec = I.sectors[s]
        _, z = lattice_for(n, sec.d)
        dl = oracle.shifts(seed, s, m, sec.d)
        view = oracle.SectorView(I, s, inv, lam=None if lam is None else lam[s], transform=transform)
        oracle.shift_sums(view, n, z, dl, lo, nord, k0=0, k1=ks)
        evals += m * ks
    return evals, time.perf_counter() - t0, oracle.max_threads()


def oracle_ks(W, nsec):
    """Lattice indices per (sector, shift) of the oracle sample: about 6e5
    evaluations of a d = 3 sector, fewer where sectors are many or wide."""
    return max(64, int(1500 * 12 * 32 / (nsec * W["m"]) * (3.0 / max(3, W.get("d", 3)))))


def run_reference(args):
    """CPU FP64 oracle on bounded samples of the bench workload."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    W = _workloads()[args.workload]
    I = W["make"]()
    n, m = args.n or W["n"], args.shifts or W["m"]
    W = dict(W, m=m, d=max(sec.d for sec in I.sectors))
    nsec = len(I.sectors)
    ks = oracle_ks(W, nsec)
    inv = W["kin"][0]
    lam = [1.0] * nsec if W["deform"] else None
    tr = W.get("transform", 0)
    for _ in range(args.warmup):
        oracle_sample(I, inv, n, m, 1, ks, W["lo"], W["nord"], lam, tr)
    tot_e, tot_t, thr = 0, 0.0, 1
    for _ in range(args.steps):
        e, t, thr = oracle_sample(I, inv, n, m, 1, ks, W["lo"], W["nord"], lam, tr)
        tot_e += e
        tot_t += t
    val = tot_e / tot_t
    sample = f"all {nsec} sectors x {m} shifts x lattice indices [0,{ks}) of n={n} at the first kinematic point"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": W["desc"].format(n=n, m=m), "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_plan(qmc, ctx, plan, out_ptr, sptr, flush, steps, warmup=3):
    """CUDA-event times of the evaluator kernels (ms) over `steps` runs of a
    plan after `warmup` runs, L2 flushed before each timed run."""
    import torch

    for _ in range(warmup):
        qmc.qmc_plan_run(ctx, plan, out_ptr, sptr)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        qmc.qmc_plan_run(ctx, plan, out_ptr, sptr)
        ms.append(qmc.qmc_plan_last_time(ctx, plan)[1])
    return ms


def box_extra(device, opts, sptr, flush, peak_gflops, seed):
    """The one-loop massless box (s = -3, t = -2, 12 sectors, n = 1000003,
    m = 32): throughput with its FP64 roofline, and the time to 1e-4 relative
    error per eps coefficient through qmc_integrate (FP64 and mixed)."""
    import torch

    from paper_2305_19768_gb300 import flops as flopmod
    from paper_2305_19768_gb300 import qmc

    W = _workloads()["box1L_massless"]
    I = W["make"]()
    ctx = qmc.qmc_create(device, **opts)
    out = {}
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, np.array(W["kin"]))
        jobs, nj = qmc.make_jobs(qmc.jobs_for_integral(iid, len(I.sectors), 1, W["n"], W["m"], seed=seed))
        plan = qmc.qmc_plan_create(ctx, jobs, nj, W["lo"], W["nord"])
        o = torch.empty(qmc.qmc_plan_output_size(plan), dtype=torch.float64, device="cuda")
        ms = timed_plan(qmc, ctx, plan, o.data_ptr(), sptr, flush, 10)
        qmc.qmc_plan_destroy(plan)
        evals = nj * W["m"] * W["n"]
        fl = flopmod.workload_work(I, W["lo"], W["nord"]).fp64
        rate = evals / (float(np.mean(ms)) * 1e-3)
        out["box1L_massless"] = {
            "workload": W["desc"].format(n=W["n"], m=W["m"]), "evals_per_s": rate, "eval_ms": float(np.mean(ms)),
            "roofline": {"achieved": fl * rate / 1e9, "peak": peak_gflops, "frac": fl * rate / 1e9 / peak_gflops,
                         "flops_per_eval": fl, "unit": "GFLOP/s (fp64)"}}
        for prec, key in ((qmc.QMC_PRECISION_FP64, "fp64"), (qmc.QMC_PRECISION_MIXED, "mixed")):
            c2 = qmc.qmc_create(device, precision=prec, **opts)
            try:
                qmc.load_lattice_table(c2)
                i2 = qmc.qmc_load_sectors_mem(c2, I.to_text())
                qmc.qmc_set_kinematics(c2, np.array(W["kin"]))
                t0 = time.perf_counter()
                _, _, info, rc = qmc.qmc_integrate(c2, [i2], epsrel=1e-4, lowest_order=W["lo"], norders=W["nord"],
                                                   check=False)
                out["box1L_massless"][f"time_to_1e-4_{key}_s"] = time.perf_counter() - t0
                out["box1L_massless"][f"time_to_1e-4_{key}_rc"] = rc
            finally:
                qmc.qmc_destroy(c2)
    finally:
        qmc.qmc_destroy(ctx)
    return out


def batch_extra(device, opts, sptr, flush, peak_gflops, seed, n=100003, m=32):
    """The massive box in the physical region at 1024 seeded (s, t) points
    (C3: contour deformation with lambda presampled per point and sector, all
    4096 jobs in one persistent launch) at a lattice of n points: throughput
    and FP64 roofline."""
    import torch

    from paper_2305_19768_gb300 import flops as flopmod
    from paper_2305_19768_gb300 import qmc

    W = _workloads()["box1L_massive_batch"]
    I = W["make"]()
    ctx = qmc.qmc_create(device, **opts)
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        kin = np.array(W["kin"])
        qmc.qmc_set_kinematics(ctx, kin)
        specs = qmc.jobs_for_integral(iid, len(I.sectors), len(kin), n, m, seed=seed)
        jobs, nj = qmc.make_jobs(specs)
        lam, _ = qmc.qmc_presample_lambda(ctx, jobs, nj, W["lo"], W["nord"], lambda_max=1.0, ncand=16)
        for sp, L in zip(specs, lam):
            sp["lambda"] = float(L)
        jobs, nj = qmc.make_jobs(specs)
        plan = qmc.qmc_plan_create(ctx, jobs, nj, W["lo"], W["nord"])
        o = torch.empty(qmc.qmc_plan_output_size(plan), dtype=torch.float64, device="cuda")
        ms = timed_plan(qmc, ctx, plan, o.data_ptr(), sptr, flush, 2, warmup=1)
        qmc.qmc_plan_destroy(plan)
    finally:
        qmc.qmc_destroy(ctx)
    evals = nj * m * n
    fl = flopmod.workload_work(I, W["lo"], W["nord"]).fp64
    rate = evals / (float(np.mean(ms)) * 1e-3)
    return {"box1L_massive_batch": {
        "workload": W["desc"].format(n=n, m=m), "evals_per_s": rate, "eval_ms": float(np.mean(ms)),
        "roofline": {"achieved": fl * rate / 1e9, "peak": peak_gflops, "frac": fl * rate / 1e9 / peak_gflops,
                     "flops_per_eval": fl, "unit": "GFLOP/s (fp64)"}}}


def mixed_extra(device, opts, I, W, kin, jobs, nj, evals_per_step, out_dev, sptr, seed, skip_oracle):
    """The double box's mixed-precision pass (FP32 monomial products): its
    throughput, its largest difference from the FP64 GPU pass, and its error
    per eps order against the FP64 oracle on sampled (sector, shift) outputs,
    one sector per number of singular variables."""
    from paper_2305_19768_gb300 import qmc

    ctx = qmc.qmc_create(device, precision=qmc.QMC_PRECISION_MIXED, **opts)
    out = {}
    try:
        qmc.load_lattice_table(ctx)
        iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
        qmc.qmc_set_kinematics(ctx, kin)
        jm, njm = qmc.make_jobs(qmc.jobs_for_integral(iid, len(I.sectors), 1, W["n"], W["m"], seed=seed))
        plan = qmc.qmc_plan_create(ctx, jm, njm, W["lo"], W["nord"])
        ms = []
        for i in range(3):
            qmc.qmc_plan_run(ctx, plan, None, sptr)
            _, me, _ = qmc.qmc_plan_last_time(ctx, plan)
            if i:
                ms.append(me)
        res, _, _ = qmc.qmc_plan_results(ctx, plan, check=False)
        qmc.qmc_plan_destroy(plan)
    finally:
        qmc.qmc_destroy(ctx)
    ref = out_dev.cpu().numpy()
    d = {"evals_per_s": evals_per_step / (float(np.mean(ms)) * 1e-3),
         "max_abs_diff_vs_fp64_gpu": float(np.max(np.abs(res - ref)))}
    if not skip_oracle:
        import oracle
        from paper_2305_19768_gb300.inputs.lattice import lattice_for

        m, nord = W["m"], W["nord"]
        res = res.reshape(nj, m, nord, 2)
        by_ns = {}
        for i, sec in enumerate(I.sectors):
            by_ns.setdefault(len(sec.singular), i)
        err_q = np.zeros(nord)
        err_a = np.zeros(nord)
        for k, (ns, sector) in enumerate(sorted(by_ns.items())):
            shift = (11 * k + 5) % m
            sec = I.sectors[sector]
            _, z = lattice_for(W["n"], sec.d)
            dl = oracle.shifts(seed, sector, m, sec.d)[[shift]]
            o, a, _ = oracle.shift_sums(oracle.SectorView(I, sector, W["kin"][0]), W["n"], z, dl, W["lo"], nord)
            e = np.abs(res[sector, shift] - o[0]).max(axis=-1)
            err_q = np.maximum(err_q, e / np.maximum(np.hypot(o[0, :, 0], o[0, :, 1]), 1e-300))
            err_a = np.maximum(err_a, e / np.maximum(a[0], 1e-300))
        d["error_vs_fp64_oracle"] = {
            "orders": list(range(W["lo"], W["lo"] + nord)), "max_err_over_abs_value": err_q.tolist(),
            "max_err_over_abs_mass": err_a.tolist(),
            "sample": f"one sector per number of singular variables ({sorted(by_ns.values())}), one shift each"}
    return {"box2L_planar_massless_mixed": d}


def run_gemm(args):
    """The learned model's BF16 GEMM C = A B^T on device buffers: milliseconds
    per call (CUDA events on the launching stream after the warm-up calls) and
    TFLOP/s = 2 M N K / time. One JSON line."""
    import torch

    from paper_2305_19768_gb300 import qmc

    M, N, K = (int(v) for v in args.gemm.split(","))
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda", dtype=torch.float32)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    stream = torch.cuda.current_stream()

    def call():
        qmc.qmc_gemm_bf16_device(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, err.data_ptr(),
                                 stream.cuda_stream)

    for _ in range(max(3, args.warmup)):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"metric": "bf16 GEMM throughput", "value": 2.0 * M * N * K / (ms * 1e-3) / 1e12,
                      "unit": "TFLOP/s", "ms_per_call": ms, "shape": [M, N, K], "steps": args.steps,
                      "wait_errors": int(err.item())}), flush=True)
    return 0 if int(err.item()) == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["box1L_massless", "triangle_massive", "box1L_massive_batch", "box1L_massless_physical",
                             "box1L_massless_d2", "box1L_massless_d2_physical",
                             "box2L_planar_massless"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--decomposition", default="iterative", choices=["iterative", "geometric"],
                    help="sector decomposition of the box and double-box workloads")
    ap.add_argument("--n", type=int, default=0, help="lattice size (default: the workload's)")
    ap.add_argument("--shifts", type=int, default=0, help="random shifts (default: the workload's)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ppt", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-scan", action="store_true", help="skip the amplitude-scan comparison")
    ap.add_argument("--gemm", default="", metavar="M,N,K",
                    help="time only the learned model's tensor-core BF16 GEMM at this shape")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.gemm:
        return run_gemm(args)

    import torch

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2305_19768_gb300 import dist as qdist
    from paper_2305_19768_gb300 import flops as flopmod
    from paper_2305_19768_gb300 import qmc
    from paper_2305_19768_gb300.inputs import workloads as w

    W = _workloads()[args.workload]
    I = W["make"](method=args.decomposition) if args.decomposition != "iterative" else W["make"]()
    args.n, args.shifts = args.n or W["n"], args.shifts or W["m"]
    LO, NORD = W["lo"], W["nord"]
    default = (args.workload == DEFAULT_WORKLOAD and args.precision == "fp64" and args.decomposition == "iterative"
               and args.n == W["n"] and args.shifts == W["m"])
    opts = {}
    if args.block:
        opts["block"] = args.block
    if args.ppt:
        opts["ppt"] = args.ppt
    if args.precision == "mixed":
        opts["precision"] = qmc.QMC_PRECISION_MIXED
    if W.get("transform", 0):
        opts["transform"] = W["transform"]
    ctx = qmc.qmc_create(local, **opts)
    qmc.load_lattice_table(ctx)
    iid = qmc.qmc_load_sectors_mem(ctx, I.to_text())
    kin = np.array(W["kin"], dtype=np.float64).reshape(len(W["kin"]), -1)
    qmc.qmc_set_kinematics(ctx, kin if kin.shape[1] else np.zeros((0, 0)))
    npts = len(W["kin"])
    nsec = len(I.sectors)
    seed = qdist.rank_seed(1, rank)  # independent shift streams per rank
    specs = qmc.jobs_for_integral(iid, nsec, npts, args.n, args.shifts, seed=seed)
    jobs, nj = qmc.make_jobs(specs)
    lam0 = None
    if W["deform"]:
        # contour-deformation parameter per (point, sector) by presampling (untimed setup)
        lam, _ = qmc.qmc_presample_lambda(ctx, jobs, nj, LO, NORD, lambda_max=1.0, ncand=16)
        for sp, L in zip(specs, lam):
            sp["lambda"] = float(L)
        jobs, nj = qmc.make_jobs(specs)
        lam0 = [float(L) for L in lam[:nsec]]
    plan = qmc.qmc_plan_create(ctx, jobs, nj, LO, NORD)
    out_n = qmc.qmc_plan_output_size(plan)
    out_dev = torch.empty(out_n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()           # a real stream handle: the plan runs on it
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    evals_per_step = nj * args.shifts * args.n

    for _ in range(max(3, args.warmup)):
        qmc.qmc_plan_run(ctx, plan, out_dev.data_ptr(), sptr)
    torch.cuda.synchronize()

    peak_gflops = qmc.qmc_fp64_peak(ctx)
    clk_dir = os.environ.get("QMC_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, f"bench_clocks_r{rank}.csv")
    proc, fh = clock_sampler_start(clk_path)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    eval_ms = []
    launches = 0
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                          # evict L2 between timed steps (untimed)
        ev[i][0].record(stream)
        qmc.qmc_plan_run(ctx, plan, out_dev.data_ptr(), sptr)
        ev[i][1].record(stream)
        _, ms_eval, nl = qmc.qmc_plan_last_time(ctx, plan)
        eval_ms.append(ms_eval)
        launches += nl
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = clock_sampler_stop(proc, fh, clk_path, local)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(sum(step_ms))
    if dist:
        total_ms = qdist.max_over_ranks(total_ms, device="cuda")
    value = evals_per_step * args.steps * world / (total_ms * 1e-3)

    # end to end through the public API with host buffers: kinematics and the
    # job table in, per-shift sums out, every step
    e2e_val = None
    h2d = kin.nbytes + nj * JOB_RECORD_BYTES
    d2h = out_n * 8
    host_out = np.zeros(out_n)
    t_e2e = 0.0
    n_e2e = max(2, args.steps // 10)
    for i in range(n_e2e):
        t0 = time.perf_counter()
        qmc.qmc_set_kinematics(ctx, kin)
        host_out = qmc.qmc_eval_jobs(ctx, jobs, nj, LO, NORD, out_n)
        t_e2e += time.perf_counter() - t0
    e2e_val = evals_per_step * n_e2e * world / t_e2e

    # roofline of the evaluator kernels: FP64 flops of the formulation (no
    # credit for the steps on the integer pipe) / their event time, against
    # the DFMA peak measured in this run; FP32 work of the mixed classes
    # against the FFMA peak; transcendentals per evaluation beside them
    work = flopmod.workload_work(I, LO, NORD, mixed=args.precision == "mixed")
    avg_eval_ms = float(np.mean(eval_ms))
    rate = evals_per_step / (avg_eval_ms * 1e-3)
    achieved = work.fp64 * rate / 1e9
    sha = kernel_sha1()
    prof = PROFILED.get((sha, args.workload, args.precision, args.decomposition, args.n), {})
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_gflops, "unit": "GFLOP/s (fp64)",
            "frac": achieved / peak_gflops, "traffic": prof.get("traffic"),
            "flops_per_eval": work.fp64, "peak_source": "DFMA probe in this run (of measured)",
            "transcendentals_per_eval": {k: getattr(work, k) for k in ("log", "atan2", "rcp", "exp", "rcp_int")},
            "fp64_executed_flops_per_eval": prof.get("fp64_executed_flops_per_eval"),
            "fp64_pipe_busy": prof.get("fp64_pipe_busy"),
            "evals_per_launch": evals_per_step, "eval_ms_per_step": avg_eval_ms,
            "kernel_sha1": sha}
    # the same formulation counted as if all of it ran in FP64 (the corner stage
    # that the d <= 6 kernel runs on the integer pipe included): algorithmic,
    # not FP64-pipe work
    eq = flopmod.workload_work(I, LO, NORD, mixed=args.precision == "mixed", fp64_corners=True).fp64
    if eq != work.fp64:
        roof["algorithmic_fp64_equivalent"] = {"flops_per_eval": eq, "achieved": eq * rate / 1e9,
                                               "frac": eq * rate / 1e9 / peak_gflops}
    # the issue roofline: warp instructions per evaluation (ncu, this source)
    # at the measured rate, against 4 warp instructions per SM per clock
    if prof.get("warp_inst_per_eval") and clocks and clocks.get("sm_mhz"):
        ipeak = 4.0 * torch.cuda.get_device_properties(local).multi_processor_count * clocks["sm_mhz"] * 1e6
        roof["issue"] = {"warp_inst_per_eval": prof["warp_inst_per_eval"],
                         "achieved": prof["warp_inst_per_eval"] * rate, "peak": ipeak,
                         "frac": prof["warp_inst_per_eval"] * rate / ipeak, "unit": "warp instructions/s",
                         "ncu_issue_busy": prof.get("issue_busy")}
    if work.fp32 > 0:
        peak32 = qmc.qmc_fp32_peak(ctx)
        a32 = work.fp32 * evals_per_step / (avg_eval_ms * 1e-3) / 1e9
        roof["fp32"] = {"flops_per_eval": work.fp32, "achieved": a32, "peak": peak32,
                        "frac": a32 / peak32, "peak_source": "FFMA probe in this run (of measured)"}

    extra = {}
    if not args.no_extra and default:
        extra.update(box_extra(local, opts, sptr, flush, peak_gflops, seed))
        extra.update(batch_extra(local, opts, sptr, flush, peak_gflops, seed))
        extra.update(mixed_extra(local, opts, I, W, kin, jobs, nj, evals_per_step, out_dev, sptr, seed,
                                 args.no_cpu_baseline or rank != 0))

    # the amplitude scan (time to 1e-4 relative amplitude error on the 10^4-point
    # (s, t) grid of a ten-integral amplitude): the learned, batched,
    # mixed-precision form against the plain FP64 method (timed on every 50th
    # point and scaled to the grid) and against the same QMC without the network
    if not args.no_extra and not args.no_scan and world == 1 and default:
        from paper_2305_19768_gb300 import scan

        modes = ("plain", "unsized", "learned", "learned_variance")
        sc = scan.compare(10000, 1e-4, ",".join(modes), 2000, plain_sample=10, steps=SCAN_TRAIN_STEPS)
        keep = ("seconds", "evaluations", "presample_evaluations", "max_rel_error", "rc", "iterations",
                "sampled_points", "accepted", "train_seconds", "model_seconds", "sized_seconds",
                "sized_evaluations", "fit_rel_error", "logn_fit_median_abs", "logw_fit_median_abs",
                "vs_plain_max_rel_diff", "vs_plain_max_diff_over_combined_sigma")
        extra["amplitude_scan"] = {
            "grid": "100 x 100 (s, t), s in [5, 20], t in [-8, -1]; 10 one-loop integrals, 36 sectors",
            "train_steps": SCAN_TRAIN_STEPS,
            **{k: v for k, v in sc.items() if k.startswith("speedup")},
            **{m: {k: v for k, v in sc[m].items() if k in keep} for m in modes}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ks = oracle_ks(dict(W, m=args.shifts, d=max(sec.d for sec in I.sectors)), nsec)
        e, t, thr = oracle_sample(I, W["kin"][0], args.n, args.shifts, 1, ks, LO, NORD, lam0, W.get("transform", 0))
        cpu = {"value": e / t, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"all {nsec} sectors x {args.shifts} shifts x lattice indices [0,{ks}) of n={args.n}"
                         " at the first kinematic point"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": W["desc"].format(n=args.n, m=args.shifts), "evals_per_step": evals_per_step,
                       "precision": args.precision, "decomposition": args.decomposition, "sectors": nsec,
                       "l2": "flushed between timed steps (256 MB write)", "wall_s": wall},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "extra": extra}
    if rank == 0:
        print(json.dumps(line), flush=True)
    qmc.qmc_plan_destroy(plan)
    qmc.qmc_destroy(ctx)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
