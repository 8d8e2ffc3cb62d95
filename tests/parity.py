"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
and the CPU oracle on the same seeded inputs, and compare.

Tolerance (FP64 per-shift sums):
    |gpu - oracle| <= RTOL * max(|oracle|, A) + CTOL * C
with A = (1/n) sum_k |Re f_k| + |Im f_k| the absolute mass of the sum and
C = (1/n) sum_k W_k sum_V |term_V| the mass of the subtraction-corner terms
before they cancel (the oracle reports both).
* RTOL = 1e-12 is the relative bar the method's FP64 sums are held to. Where
  the corner terms do not cancel (C about |Q|) the measured differences stay
  below 1e-13 |Q|: 1e-16 for real sectors, up to 3e-14 A for deformed
  sectors, whose complex logs, arctangents and det J carry a few ulp on each
  side.
* CTOL covers the orders where the plus-distribution subtraction cancels:
  each corner term carries a few roundings on each side, so the two FP64
  evaluations of a sum whose terms cancel from C down to |Q| differ by a few
  u C. C / |Q| reaches 1e3 to 1e8 at eps^-1 .. eps^0 of the double box
  (1e4 to 3e5 at eps^0 of the one-loop boxes), so 1e-12 |Q| is not
  reachable there by any FP64 evaluation of this formula, the oracle's
  included. Measured over every parity case: |gpu - oracle| <= 0.3 u C on
  those orders; CTOL = 3e-16 (2.7 u) leaves a margin of about 10.
* CTOL_TAYLOR is CTOL for sectors with exponents a_j <= -2 (Taylor
  subtraction). There C also holds, per Taylor state, the magnitudes of the
  binomial-series terms that the oracle sums into each Taylor coefficient.
  The kernel forms the same coefficients through ln(1 + x) and exp of
  truncated power series by Horner's rule (2K + 4 rounded steps for a box of
  total degree K <= 7), and U0^{u0} F0^{f0} through exp(e ln P) where the
  exponent is not a small integer (relative error about |e ln P| u: 5 ln F
  with f0 = -5 in the two-loop D = 2 - 2 eps sectors). Worst case about
  40 u C. Measured on every GPU parity case of these sectors: up to 18 u C
  under korobov3 (the two-loop sectors, where both sums are rounding noise
  near the border), 5.4 u C under baker. CTOL_TAYLOR = 1e-14 (45 u), the
  worst case.
"""
import json
import os

import numpy as np

import oracle
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs.lattice import lattice_for

RTOL = 1e-12
CTOL = 3e-16
CTOL_TAYLOR = 1e-14


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
    """Oracle per-shift sums [m][norders][2], absolute masses [m][norders] and
    corner-term masses [m][norders]."""
    s = integral.sectors[sector]
    _, z = lattice_for(n, s.d)
    dl = oracle.shifts(seed, stream, m, s.d)
    if shift_rows is not None:
        dl = dl[list(shift_rows)]
    view = oracle.SectorView(integral, sector, inv, lam)
    out, absm, fails, cond = oracle.shift_sums(view, n, z, dl, lo, norders, nthreads=nthreads,
                                               with_cond=True)
    return out, absm, cond


def achieved(gpu, orc, absm, cond=None):
    """Per eps order (axis -2 of [shifts][orders][2]): the worst |gpu - oracle|
    relative to |Q| (the complex modulus of the oracle's per-shift sum), to
    the absolute mass A, and to the corner mass C."""
    gpu = np.asarray(gpu).reshape(orc.shape)
    err = np.abs(gpu - orc).max(axis=-1)                      # [shifts][orders]
    q = np.hypot(orc[..., 0], orc[..., 1])
    out = {"err_over_Q": (err / np.maximum(q, 1e-300)).max(axis=0).tolist(),
           "err_over_A": (err / np.maximum(absm, 1e-300)).max(axis=0).tolist()}
    if cond is not None:
        out["err_over_C"] = (err / np.maximum(cond, 1e-300)).max(axis=0).tolist()
        out["C_over_Q"] = (cond / np.maximum(q, 1e-300)).max(axis=0).tolist()
    return out


def record(what, lo, stats, bound="fp64"):
    """Append one parity measurement to the JSON-lines file named by the
    QMC_PARITY_LOG environment variable (nothing if unset)."""
    path = os.environ.get("QMC_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"what": what, "lo": lo, "bound": bound, **stats}) + "\n")


def assert_close(gpu, orc, absm, cond=None, rtol=RTOL, what="", lo=None, ctol=None):
    gpu = np.asarray(gpu).reshape(orc.shape)
    scale = np.maximum(np.abs(orc), absm[..., None])
    err = np.abs(gpu - orc)
    allow = rtol * scale + 1e-300
    if cond is not None:
        allow = allow + (CTOL if ctol is None else ctol) * cond[..., None]
    if orc.ndim == 3:
        stats = achieved(gpu, orc, absm, cond)
        stats["worst_over_bound"] = float((err / allow).max())
        record(what, lo, stats, "fp64" if rtol == RTOL else f"rtol={rtol:g}")
    bad = err > allow
    if bad.any():
        idx = np.argwhere(bad)[:5]
        rel = (err / np.maximum(scale, 1e-300)).max()
        raise AssertionError(f"{what}: {bad.sum()} mismatches, worst rel {rel:.3e}, first {idx.tolist()}")
    return float((err / np.maximum(scale, 1e-300)).max())
