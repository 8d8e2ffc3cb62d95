"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
and the CPU oracle on the same seeded inputs, and compare.

Tolerance (FP64 per-shift sums): |gpu - oracle| <= RTOL * max(|oracle|, A)
with A = (1/n) sum_k |Re f_k| + |Im f_k| the absolute mass of the sum (the
oracle reports it). Both sides evaluate every point in FP64 with library
transcendentals (<= 1 ulp apart); the GPU sums in a different order (PPT
points per thread, a 5-level warp tree, warps in order, Neumaier over tiles),
whose worst-case relative error is ~ (PPT + 12) u A / |Q| << 1e-12, and the
subtraction terms' cancellation near t = 0 is damped by the korobov3 weight
(W / t ~ 4 / u), adding ~ u ln(n) per singular variable. RTOL = 1e-12.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs.lattice import lattice_for

RTOL = 1e-12


class Gpu:
    def __init__(self, **opts):
        self.ctx = qmc.qmc_create(0, **opts)
        qmc.load_lattice_table(self.ctx)

    def close(self):
        qmc.qmc_destroy(self.ctx)

    def load(self, integral):
        return qmc.qmc_load_sectors_mem(self.ctx, integral.to_text())

    def eval(self, iid, specs, lo, norders):
        jobs, nj = qmc.make_jobs(specs)
        plan = qmc.qmc_plan_create(self.ctx, jobs, nj, lo, norders)
        try:
            qmc.qmc_plan_run(self.ctx, plan)
            out, fails, rc = qmc.qmc_plan_results(self.ctx, plan, check=False)
        finally:
            qmc.qmc_plan_destroy(plan)
        return out, fails, rc


def oracle_sums(integral, sector, inv, n, m, seed, stream, lo, norders, lam=None, shift_rows=None,
                nthreads=0):
    """Oracle per-shift sums [m][norders][2] and absolute masses [m][norders]."""
    s = integral.sectors[sector]
    _, z = lattice_for(n, s.d)
    dl = oracle.shifts(seed, stream, m, s.d)
    if shift_rows is not None:
        dl = dl[list(shift_rows)]
    view = oracle.SectorView(integral, sector, inv, lam)
    out, absm, fails = oracle.shift_sums(view, n, z, dl, lo, norders, nthreads=nthreads)
    return out, absm, fails


def assert_close(gpu, orc, absm, rtol=RTOL, what=""):
    gpu = np.asarray(gpu).reshape(orc.shape)
    scale = np.maximum(np.abs(orc), absm[..., None])
    err = np.abs(gpu - orc)
    bad = err > rtol * scale + 1e-300
    if bad.any():
        idx = np.argwhere(bad)[:5]
        rel = (err / np.maximum(scale, 1e-300)).max()
        raise AssertionError(f"{what}: {bad.sum()} mismatches, worst rel {rel:.3e}, first {idx.tolist()}")
    return float((err / np.maximum(scale, 1e-300)).max())
