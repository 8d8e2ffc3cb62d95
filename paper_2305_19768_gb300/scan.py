"""The amplitude scan over a grid of kinematic points, three ways.

The sum is A(s, t) = sum_i C_i(s, t) I_i(s, t) over ten one-loop integrals
(inputs.workloads.amplitude_integrals) with seeded rational polynomial
coefficients, eps orders -2..0, requested to a relative error `epsrel`:
every eps coefficient's error sqrt(dR^2 + dI^2) within epsrel times the
largest coefficient of the amplitude at that point (QMC_TARGET_AMPLITUDE;
single coefficients of this amplitude cross zero inside the grid, where the
per-coefficient relative error of the paper's timings section is not
reachable).

* ``plain``: one kinematic point at a time, FP64, each with the 10^4-point
  pilot pass and the adaptive allocation (qmc_integrate) — no batching, no
  model.
* ``batched``: all points in one adaptive qmc_integrate (one evaluator
  launch per pass for every point, sector and shift).
* ``learned``: the spec learned form. QMC on the first `ntrain`
  points (batched) gives per-slot convergence constants w and amplitude
  values; a tensor-core MLP (qmc_mlp_*) learns (s, t) -> (log w per
  sector slot, Re/Im of each eps coefficient); for the other points it
  predicts w, from which Eq. (adaptive-solution) (qmc_allocate) sizes every
  lattice up front instead of the pilot pass. A small-lattice spot check
  runs first; a point takes the surrogate value only where the spot check's
  own error is within the request and the surrogate agrees with it to
  within that error, and everything else runs the sized, batched QMC, which
  still refines adaptively where the prediction was short.

All arithmetic of the method runs behind the C-ABI; this module marshals
arrays and keeps the books.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import qmc
from .inputs import workloads as w

LO, NORD = -2, 3


class Problem:
    def __init__(self, npoints: int = 10000, grid=(100, 100)):
        self.integrals = w.amplitude_integrals()
        self.points = w.amplitude_grid(*grid)[:npoints]
        self.coef_poly = w.amplitude_coefficients(len(self.integrals))
        self.C = w.amplitude_coefficient_values(self.points, self.coef_poly)  # [np][nint]
        self.nsec = [len(I.sectors) for I in self.integrals]
        self.nslot = sum(self.nsec)

    def context(self, precision=qmc.QMC_PRECISION_FP64, shifts=32, max_points=0, min_points=10000):
        # lambda chosen per (point, sector) by presampling; epsrel against each
        # amplitude's largest eps coefficient (QMC_TARGET_AMPLITUDE)
        ctx = qmc.qmc_create(0, precision=precision, shifts=shifts, target_mode=qmc.QMC_TARGET_AMPLITUDE,
                             max_points=max_points, min_points=min_points)
        qmc.load_lattice_table(ctx)
        ids = [qmc.qmc_load_sectors_mem(ctx, I.to_text()) for I in self.integrals]
        return ctx, ids

    def coef(self, sel):
        return self.C[sel].reshape(len(sel), 1, len(self.integrals), 1).astype(np.complex128)


def run_plain(P: Problem, epsrel: float, sel=None):
    """One point at a time, FP64, pilot pass + adaptive allocation."""
    sel = np.arange(len(P.points)) if sel is None else np.asarray(sel)
    ctx, ids = P.context()
    vals = np.zeros((len(sel), NORD), complex)
    errs = np.zeros((len(sel), NORD), complex)
    evals, rcs = 0.0, []
    t0 = time.perf_counter()
    try:
        for k, p in enumerate(sel):
            qmc.qmc_set_kinematics(ctx, P.points[p:p + 1])
            v, e, info, rc = qmc.qmc_integrate(ctx, ids, coef=P.coef([p]), epsrel=epsrel, lowest_order=LO,
                                               norders=NORD, check=False)
            vals[k], errs[k] = v[0, 0], e[0, 0]
            evals += info["evaluations"]
            rcs.append(rc)
    finally:
        qmc.qmc_destroy(ctx)
    return dict(seconds=time.perf_counter() - t0, values=vals, errors=errs, evaluations=evals,
                failures=int(sum(1 for r in rcs if r != 0)))


def run_batched(P: Problem, epsrel: float, sel=None, precision=qmc.QMC_PRECISION_FP64, n_init=None,
                shifts=0, want_slots=False, max_points=0, min_points=10000, lambdas=None):
    """All points of `sel` in one adaptive qmc_integrate_ex. `lambdas` (float64
    [len(sel) * nslot], in/out) carries the deformation parameters: positive
    entries are used, the rest presampled and written back."""
    sel = np.arange(len(P.points)) if sel is None else np.asarray(sel)
    ctx, ids = P.context(precision, max_points=max_points, min_points=min_points)
    t0 = time.perf_counter()
    try:
        qmc.qmc_set_kinematics(ctx, P.points[sel])
        res = qmc.qmc_integrate(ctx, ids, coef=P.coef(sel), epsrel=epsrel, lowest_order=LO, norders=NORD,
                                npoints=len(sel), check=False, n_init=n_init, shifts=shifts,
                                nslots=len(sel) * P.nslot if want_slots else 0, lambda_io=lambdas)
    finally:
        qmc.qmc_destroy(ctx)
    out = dict(seconds=time.perf_counter() - t0, values=res[0][:, 0], errors=res[1][:, 0],
               evaluations=res[2]["evaluations"], rc=res[3], iterations=res[2]["iterations"])
    if want_slots:
        out["w"], out["n"] = res[4].reshape(len(sel), P.nslot), res[5].reshape(len(sel), P.nslot)
    return out


def _features(points):
    s, t = points[:, 0], points[:, 1]
    return np.stack([(s - 12.5) / 7.5, (t + 4.5) / 3.5], axis=1).astype(np.float32)


def _log(msg):
    print(f"[scan] {msg}", file=sys.stderr, flush=True)


def run_learned(P: Problem, epsrel: float, ntrain: int = 2000, precision=qmc.QMC_PRECISION_MIXED,
                steps: int = 1500, spot_n: int = 1009, spot_shifts: int = 8, shifts: int = 16,
                max_points: int = 1000003):
    """Learned sizing + spot-checked surrogate + batched QMC (see module doc).
    Lattices are capped at `max_points` (sizes beyond it come from a model error)."""
    t0 = time.perf_counter()
    train = np.arange(min(ntrain, len(P.points)))
    rest = np.arange(len(train), len(P.points))
    # 1. the method's own outputs on the training points: batched, adaptive,
    #    from a small pilot (n = spot_n, `shifts` shifts) instead of 10^4 x 32
    tr = run_batched(P, epsrel, train, precision, want_slots=True, shifts=shifts, min_points=spot_n,
                     max_points=max_points)
    _log(f"training QMC: {tr['seconds']:.2f} s, {tr['evaluations']:.3g} evals, rc {tr['rc']}, "
         f"{tr['iterations']} passes, n quartiles {np.percentile(tr['n'], [50, 90, 99, 100]).tolist()}")
    # 2. the model: (s, t) -> log w per slot, Re/Im per eps coefficient
    x = _features(P.points[train])
    logw = np.log(np.maximum(tr["w"], 1e-300))
    amp = np.concatenate([tr["values"].real, tr["values"].imag], axis=1)
    Y = np.concatenate([logw, amp], axis=1)
    mu, sd = Y.mean(axis=0), Y.std(axis=0) + 1e-12
    net = qmc.Mlp(2, 256, 4, Y.shape[1], seed=5)
    wt = np.ones(Y.shape[1], dtype=np.float32)
    wt[P.nslot:] = 4.0   # the amplitude coefficients weigh more than the sizing outputs
    try:
        losses = net.train(x, ((Y - mu) / sd).astype(np.float32), steps, 1e-3, wt=wt)
        pred = net.forward(_features(P.points[rest])) * sd + mu
    finally:
        net.close()
    t_model = time.perf_counter() - t0
    _log(f"model trained and evaluated: {t_model:.2f} s since start, final loss {losses[-1]:.4g}")
    res_vals = np.zeros((len(P.points), NORD), complex)
    res_errs = np.zeros((len(P.points), NORD), complex)
    res_vals[train], res_errs[train] = tr["values"], tr["errors"]
    if len(rest) == 0:
        return dict(seconds=time.perf_counter() - t0, values=res_vals, errors=res_errs, accepted=0)
    w_pred = np.exp(pred[:, :P.nslot])
    a_pred = pred[:, P.nslot:P.nslot + NORD] + 1j * pred[:, P.nslot + NORD:]
    # 3. spot check: one small-lattice pass for every remaining point
    lam_rest = np.zeros(len(rest) * P.nslot)      # presampled once, reused by the sized run
    sp = run_batched(P, 1e9, rest, precision, n_init=np.full(len(rest) * P.nslot, spot_n), shifts=spot_shifts,
                     min_points=spot_n, lambdas=lam_rest)
    _log(f"spot check: {sp['seconds']:.2f} s, {sp['evaluations']:.3g} evals")
    target = epsrel * np.abs(sp["values"]).max(axis=1, keepdims=True)
    sig = np.abs(sp["errors"])
    accept = np.all((sig <= target) & (np.abs(a_pred - sp["values"]) <= target), axis=1)
    res_vals[rest[accept]] = a_pred[accept]
    res_errs[rest[accept]] = target[accept]
    # 4. predicted lattice sizes (Eq. adaptive-solution) for the others, then batched QMC
    todo = rest[~accept]
    evals = tr["evaluations"] + sp["evaluations"]
    if len(todo):
        wp = w_pred[~accept]
        ap = a_pred[~accept]
        # per point: W_slot = |C_i|^2 w_slot (prefactor series folded into w by training),
        # V = (epsrel * min over orders |A|)^2, tau from the sector's lattice dimension cost
        n_init = np.zeros((len(todo), P.nslot))
        slot_int = np.repeat(np.arange(len(P.integrals)), P.nsec)
        for k, p in enumerate(todo):
            W = (np.abs(P.C[p, slot_int]) ** 2 * wp[k])[None, :]
            V = np.array([(epsrel * max(np.max(np.abs(ap[k])), 1e-12)) ** 2])
            n_init[k] = qmc.qmc_allocate(W, np.ones(P.nslot), V, 2.0, float(spot_n))
        n_init = np.minimum(n_init, max_points)
        _log(f"sized lattices: quartiles {np.percentile(n_init, [50, 90, 99, 100]).tolist()}")
        lam_todo = lam_rest.reshape(len(rest), P.nslot)[~accept].ravel().copy()
        run = run_batched(P, epsrel, todo, precision, n_init=n_init.ravel(), shifts=shifts, min_points=spot_n,
                          max_points=max_points, lambdas=lam_todo)
        _log(f"sized QMC: {run['seconds']:.2f} s, {run['evaluations']:.3g} evals, rc {run['rc']}, "
             f"{run['iterations']} passes")
        res_vals[todo], res_errs[todo] = run["values"], run["errors"]
        evals += run["evaluations"]
    return dict(seconds=time.perf_counter() - t0, values=res_vals, errors=res_errs, evaluations=evals,
                accepted=int(accept.sum()), model_seconds=t_model, final_loss=float(losses[-1]),
                train_seconds=tr["seconds"], spot_seconds=sp["seconds"],
                train_n_quartiles=np.percentile(tr["n"], [25, 50, 75, 95]).tolist(),
                sized_n_quartiles=np.percentile(n_init, [25, 50, 75, 95]).tolist() if len(todo) else [],
                sized_seconds=run["seconds"] if len(todo) else 0.0,
                sized_iterations=run["iterations"] if len(todo) else 0)


def relative_errors(values, errors):
    """Error of each coefficient over the largest coefficient of its amplitude."""
    return np.abs(errors) / np.maximum(np.abs(values).max(axis=-1, keepdims=True), 1e-300)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=10000)
    ap.add_argument("--epsrel", type=float, default=1e-4)
    ap.add_argument("--modes", default="plain,batched,learned")
    ap.add_argument("--ntrain", type=int, default=2000)
    ap.add_argument("--plain-sample", type=int, default=0, help="time plain on every k-th point only")
    args = ap.parse_args()
    P = Problem(args.points)
    out = {"points": len(P.points), "epsrel": args.epsrel, "slots_per_point": P.nslot}
    ref = None
    for mode in args.modes.split(","):
        if mode == "plain":
            sel = np.arange(0, len(P.points), args.plain_sample) if args.plain_sample else None
            r = run_plain(P, args.epsrel, sel)
            scale = len(P.points) / (len(sel) if sel is not None else len(P.points))
            out["plain"] = dict(seconds=r["seconds"] * scale, measured_seconds=r["seconds"],
                                sampled_points=int(len(sel)) if sel is not None else len(P.points),
                                evaluations=r["evaluations"] * scale, failures=r["failures"])
        elif mode == "batched":
            r = run_batched(P, args.epsrel)
            ref = r
            out["batched"] = dict(seconds=r["seconds"], evaluations=r["evaluations"], rc=r["rc"],
                                  iterations=r["iterations"],
                                  max_rel_error=float(relative_errors(r["values"], r["errors"]).max()))
        elif mode == "learned":
            r = run_learned(P, args.epsrel, args.ntrain)
            d = {k: v for k, v in r.items() if k not in ("values", "errors")}
            d["max_rel_error"] = float(relative_errors(r["values"], r["errors"]).max())
            if ref is not None:
                diff = np.abs(r["values"] - ref["values"])
                comb = np.hypot(np.abs(r["errors"]), np.abs(ref["errors"]))
                d["max_diff_over_combined_sigma"] = float(np.max(diff / np.maximum(comb, 1e-300)))
            out["learned"] = d
    if "plain" in out and "learned" in out:
        out["speedup_learned_vs_plain"] = out["plain"]["seconds"] / out["learned"]["seconds"]
    if "plain" in out and "batched" in out:
        out["speedup_batched_vs_plain"] = out["plain"]["seconds"] / out["batched"]["seconds"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
