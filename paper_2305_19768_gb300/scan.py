"""The amplitude scan over a grid of kinematic points, four ways.

The sum is A(s, t) = sum_i C_i(s, t) I_i(s, t) over ten one-loop integrals
(inputs.workloads.amplitude_integrals) with seeded rational polynomial
coefficients, eps orders -2..0, requested to a relative error `epsrel`:
every eps coefficient's error sqrt(dR^2 + dI^2) within epsrel times the
largest coefficient of the amplitude at that point (QMC_TARGET_AMPLITUDE;
single coefficients of this amplitude cross zero inside the grid, where the
per-coefficient relative error of the paper's timings section is not
reachable).

* ``plain``: one kinematic point at a time, FP64, each with the 10^4-point
  pilot pass and the adaptive allocation (qmc_integrate) -- no batching, no
  model.
* ``batched``: the same, all points in one adaptive qmc_integrate (one
  evaluator launch per pass for every point, sector and shift).
* ``learned``: the production form. Batched, mixed-precision QMC on the
  first `ntrain` points, started from the smallest lattice and with the
  per-pass lattice growth limited (options.max_growth), gives every slot's
  converged lattice size and the amplitude values; a tensor-core MLP
  (qmc_mlp_*) learns (s, t) -> (log n per sector slot, log lambda per
  deformed slot, Re/Im of each eps coefficient); for the other points it
  predicts the lattice sizes, which replace the pilot pass, and the
  deformation parameters, which replace the presampling (the QMC's sign
  check verifies them and presamples where one fails). A small-lattice spot check decides where the
  surrogate amplitude may stand in for QMC (its own error and the
  surrogate's distance to it both within the request); it is skipped when
  the model does not fit its own training points that well. Everything else
  runs the sized, batched QMC, which still refines adaptively where the
  prediction was short.
* ``unsized``: the learned form's QMC without the network (pilot pass on the
  smallest lattice), which isolates what the network contributes.

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

    def context(self, precision=qmc.QMC_PRECISION_FP64, shifts=32, max_points=0, min_points=10000,
                max_growth=0):
        # lambda chosen per (point, sector) by presampling; epsrel against each
        # amplitude's largest eps coefficient (QMC_TARGET_AMPLITUDE)
        ctx = qmc.qmc_create(0, precision=precision, shifts=shifts, target_mode=qmc.QMC_TARGET_AMPLITUDE,
                             max_points=max_points, min_points=min_points, max_growth=max_growth)
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
                shifts=0, want_slots=False, max_points=0, min_points=10000, lambdas=None, max_growth=0):
    """All points of `sel` in one adaptive qmc_integrate_ex. `lambdas` (float64
    [len(sel) * nslot], in/out) carries the deformation parameters: positive
    entries are used, the rest presampled and written back."""
    sel = np.arange(len(P.points)) if sel is None else np.asarray(sel)
    ctx, ids = P.context(precision, max_points=max_points, min_points=min_points, max_growth=max_growth)
    t0 = time.perf_counter()
    try:
        qmc.qmc_set_kinematics(ctx, P.points[sel])
        res = qmc.qmc_integrate(ctx, ids, coef=P.coef(sel), epsrel=epsrel, lowest_order=LO, norders=NORD,
                                npoints=len(sel), check=False, n_init=n_init, shifts=shifts,
                                nslots=len(sel) * P.nslot if want_slots else 0, lambda_io=lambdas)
    finally:
        qmc.qmc_destroy(ctx)
    out = dict(seconds=time.perf_counter() - t0, values=res[0][:, 0], errors=res[1][:, 0],
               evaluations=res[2]["evaluations"], rc=res[3], iterations=res[2]["iterations"],
               kernel_seconds=res[2]["kernel_seconds"], presample_evaluations=res[2]["presample_evaluations"])
    if want_slots:
        out["w"], out["n"] = res[4].reshape(len(sel), P.nslot), res[5].reshape(len(sel), P.nslot)
        if lambdas is not None:
            out["lam"] = np.asarray(lambdas).reshape(len(sel), P.nslot)
    return out


def snap_to_table(n):
    """Each size to the tabulated lattice nearest to it in log n (qmc_integrate_ex
    rounds up, which would lift a prediction of 1009.000001 to the next size)."""
    from .inputs.lattice import load_table

    sizes = np.array([r[0] for r in load_table()], dtype=np.float64)
    k = np.abs(np.log(np.asarray(n, dtype=np.float64))[..., None] - np.log(sizes)).argmin(axis=-1)
    return sizes[k]


def run_unsized(P: Problem, epsrel: float, sel=None, precision=qmc.QMC_PRECISION_MIXED, spot_n: int = 1009,
                shifts: int = 16, max_points: int = 1000003, max_growth: int = 4):
    """The learned form's QMC without the network: the same batched, mixed,
    growth-limited integration, started from the smallest lattice (a pilot pass
    at `spot_n`) instead of from predicted sizes."""
    return run_batched(P, epsrel, sel, precision, shifts=shifts, min_points=spot_n, max_points=max_points,
                       max_growth=max_growth, want_slots=True)


def _features(points):
    s, t = points[:, 0], points[:, 1]
    return np.stack([(s - 12.5) / 7.5, (t + 4.5) / 3.5], axis=1).astype(np.float32)


def _log(msg):
    print(f"[scan] {msg}", file=sys.stderr, flush=True)


def allocate_from_variances(P: Problem, w_pred, amax_pred, epsrel, sel, alpha=2.0):
    """Lattice sizes of Eq. (adaptive-solution) from predicted convergence
    constants: at each point, the sum's variance target (epsrel times the
    amplitude's largest coefficient)^2 is shared over its slots with weights
    W_i = |C_i|^2 w_i and costs tau_i (the evaluator's FP64 work per
    evaluation of the sector, from the flop model)."""
    from . import flops as flopmod

    tau = np.array([flopmod.sector_work(s, LO, NORD).fp64 + 20.0 * flopmod.sector_work(s, LO, NORD).log
                     for I in P.integrals for s in I.sectors])
    cidx = np.concatenate([np.full(n, i) for i, n in enumerate(P.nsec)])
    W = (P.C[sel][:, cidx] ** 2) * w_pred                       # [points][slots]
    V = (epsrel * amax_pred) ** 2                                 # [points]
    q = 1.0 / (alpha + 1.0)
    lam = (1.0 / alpha) * (((W * tau ** alpha) ** q).sum(axis=1) / V) ** ((alpha + 1.0) / alpha)
    return (alpha * lam[:, None] * W / tau) ** q


def run_learned(P: Problem, epsrel: float, ntrain: int = 2000, precision=qmc.QMC_PRECISION_MIXED,
                steps: int = 1500, spot_n: int = 1009, spot_shifts: int = 8, shifts: int = 16,
                max_points: int = 1000003, max_growth: int = 4, sizing: str = "logn"):
    """Learned sizing + spot-checked surrogate + batched QMC (see module doc).
    Every QMC pass here grows a lattice by at most `max_growth` per pass and
    caps it at `max_points`. `sizing`: how the network sizes the lattices of
    the points it has not seen -- "logn" from the log-lattice-size head,
    "variance" by the allocation of Eq. (adaptive-solution) from the
    per-sector log-variance head, "both" the larger of the two."""
    t0 = time.perf_counter()
    train = np.arange(min(ntrain, len(P.points)))
    rest = np.arange(len(train), len(P.points))
    # 1. the method's own outputs on the training points: batched, adaptive,
    #    from the smallest lattice (n = spot_n, `shifts` shifts)
    tr = run_batched(P, epsrel, train, precision, want_slots=True, shifts=shifts, min_points=spot_n,
                     max_points=max_points, max_growth=max_growth, lambdas=np.zeros(len(train) * P.nslot))
    _log(f"training QMC: {tr['seconds']:.2f} s, {tr['evaluations']:.3g} evals, rc {tr['rc']}, "
         f"{tr['iterations']} passes, n percentiles 50/90/99/100 "
         f"{np.percentile(tr['n'], [50, 90, 99, 100]).tolist()}")
    # 2. the model: (s, t) -> log n per slot (the lattice the slot converged on),
    #    Re/Im per eps coefficient. The lattice size itself is learned rather than
    #    w = var n^2: w is far from constant over the lattices used here (the
    #    sector integrands converge much faster than n^-2 under korobov3), so a
    #    size extrapolated from w with alpha = 2 overshoots.
    #    Beside them, the per-sector log-variance: log w with w = var n^2 at the
    #    converged lattice (the convergence constant of Eq. (varscaling) that the
    #    allocation of Eq. (adaptive-solution) takes).
    x = _features(P.points[train])
    logn = np.log(tr["n"].astype(np.float64))
    deformed = tr["lam"][0] > 0                     # slots with a contour deformation
    loglam = np.log(tr["lam"][:, deformed])
    logw = np.log(np.maximum(tr["w"], 1e-300))
    amp = np.concatenate([tr["values"].real, tr["values"].imag], axis=1)
    Y = np.concatenate([logn, loglam, logw, amp], axis=1)
    nw = P.nslot + int(deformed.sum())              # first log-variance output
    na = nw + P.nslot                               # first amplitude output
    mu, sd = Y.mean(axis=0), Y.std(axis=0) + 1e-12
    net = qmc.Mlp(2, 256, 4, Y.shape[1], seed=5)
    wt = np.ones(Y.shape[1], dtype=np.float32)
    wt[na:] = 4.0   # the amplitude coefficients weigh more than the sizing outputs
    try:
        losses = net.train(x, ((Y - mu) / sd).astype(np.float32), steps, 1e-3, wt=wt)
        fit = net.forward(x) * sd + mu
        pred = net.forward(_features(P.points[rest])) * sd + mu if len(rest) else None
    finally:
        net.close()
    a_fit = fit[:, na:na + NORD] + 1j * fit[:, na + NORD:]
    fit_err = float(np.max(np.abs(a_fit - tr["values"]) / np.abs(tr["values"]).max(axis=1, keepdims=True)))
    logn_fit_err = float(np.median(np.abs(fit[:, :P.nslot] - logn)))
    logw_fit_err = float(np.median(np.abs(fit[:, nw:na] - logw)))
    t_model = time.perf_counter() - t0
    _log(f"model trained and evaluated: {t_model:.2f} s since start, final loss {losses[-1]:.4g}, "
         f"largest relative amplitude error on its training points {fit_err:.3g}")
    res_vals = np.zeros((len(P.points), NORD), complex)
    res_errs = np.zeros((len(P.points), NORD), complex)
    res_vals[train], res_errs[train] = tr["values"], tr["errors"]
    base = dict(model_seconds=t_model, final_loss=float(losses[-1]), fit_rel_error=fit_err,
                logn_fit_median_abs=logn_fit_err, logw_fit_median_abs=logw_fit_err, sizing=sizing,
                train_seconds=tr["seconds"], train_evaluations=tr["evaluations"],
                train_n_percentiles=np.percentile(tr["n"], [50, 90, 99, 100]).tolist())
    if len(rest) == 0:
        return dict(seconds=time.perf_counter() - t0, values=res_vals, errors=res_errs, accepted=0,
                    evaluations=tr["evaluations"], spot_seconds=0.0, sized_seconds=0.0, **base)
    n_logn = np.exp(pred[:, :P.nslot])
    a_pred = pred[:, na:na + NORD] + 1j * pred[:, na + NORD:]
    if sizing == "logn":
        n_pred = n_logn
    else:
        n_var = allocate_from_variances(P, np.exp(pred[:, nw:na]), np.abs(a_pred).max(axis=1), epsrel, rest)
        n_pred = n_var if sizing == "variance" else np.maximum(n_var, n_logn)
    # deformation parameters: the prediction snapped to the presampling grid 0.7^c
    # (c = 0..15); the QMC's own sign check verifies it and presamples where it fails
    c = np.clip(np.round(-pred[:, P.nslot:nw] / np.log(1 / 0.7)), 0, 15)
    lam_pred = np.zeros((len(rest), P.nslot))
    lam_pred[:, deformed] = 0.7 ** c
    # 3. spot check, one small-lattice pass for every remaining point -- run only
    #    when the model fits its own training points within the request (a model
    #    that does not cannot have a guess accepted anywhere)
    lam_rest = lam_pred.ravel().copy()
    accept = np.zeros(len(rest), bool)
    evals = tr["evaluations"]
    spot_s = 0.0
    if fit_err <= epsrel:
        sp = run_batched(P, 1e9, rest, precision, n_init=np.full(len(rest) * P.nslot, spot_n),
                         shifts=spot_shifts, min_points=spot_n, lambdas=lam_rest)
        spot_s = sp["seconds"]
        _log(f"spot check: {sp['seconds']:.2f} s, {sp['evaluations']:.3g} evals")
        target = epsrel * np.abs(sp["values"]).max(axis=1, keepdims=True)
        sig = np.abs(sp["errors"])
        accept = np.all((sig <= target) & (np.abs(a_pred - sp["values"]) <= target), axis=1)
        res_vals[rest[accept]] = a_pred[accept]
        res_errs[rest[accept]] = np.broadcast_to(target, sig.shape)[accept]
        evals += sp["evaluations"]
    else:
        _log("spot check skipped: the model misses its own training points by more than the request")
    # 4. the predicted lattice sizes for the others, then batched QMC from there
    todo = rest[~accept]
    n_init = np.zeros((0, P.nslot))
    if len(todo):
        n_init = snap_to_table(np.clip(n_pred[~accept], spot_n, max_points))
        _log(f"sized lattices: percentiles 50/90/99/100 {np.percentile(n_init, [50, 90, 99, 100]).tolist()}")
        lam_todo = lam_rest.reshape(len(rest), P.nslot)[~accept].ravel().copy()
        run = run_batched(P, epsrel, todo, precision, n_init=n_init.ravel(), shifts=shifts, min_points=spot_n,
                          max_points=max_points, lambdas=lam_todo, max_growth=max_growth, want_slots=True)
        _log(f"sized QMC: {run['seconds']:.2f} s ({run['kernel_seconds']:.2f} s in the evaluator), "
             f"{run['evaluations']:.3g} evals, rc {run['rc']}, {run['iterations']} passes, final n "
             f"percentiles 50/90/99/100 {np.percentile(run['n'], [50, 90, 99, 100]).tolist()}")
        res_vals[todo], res_errs[todo] = run["values"], run["errors"]
        evals += run["evaluations"]
    return dict(seconds=time.perf_counter() - t0, values=res_vals, errors=res_errs, evaluations=evals,
                accepted=int(accept.sum()), spot_seconds=spot_s,
                sized_n_percentiles=np.percentile(n_init, [50, 90, 99, 100]).tolist() if len(todo) else [],
                sized_seconds=run["seconds"] if len(todo) else 0.0,
                sized_evaluations=run["evaluations"] if len(todo) else 0.0,
                sized_presample_evaluations=run["presample_evaluations"] if len(todo) else 0.0,
                sized_iterations=run["iterations"] if len(todo) else 0, **base)


def relative_errors(values, errors):
    """Error of each coefficient over the largest coefficient of its amplitude."""
    return np.abs(errors) / np.maximum(np.abs(values).max(axis=-1, keepdims=True), 1e-300)


def compare(points: int = 10000, epsrel: float = 1e-4, modes="plain,unsized,learned", ntrain: int = 2000,
            plain_sample: int = 0, steps: int = 1500):
    """Run the requested modes on the first `points` grid points and return the
    timings, evaluation counts and errors (plain may run on every
    `plain_sample`-th point only; its time is then scaled to the whole grid).
    Modes: plain, batched, unsized, learned (lattices from the log-n head),
    learned_variance (lattices from the log-variance head through Eq.
    (adaptive-solution)); `steps` Adam steps train the network."""
    P = Problem(points)
    out = {"points": len(P.points), "epsrel": epsrel, "slots_per_point": P.nslot}
    ref = None
    plain_sel = None
    for mode in modes.split(",") if isinstance(modes, str) else modes:
        if mode == "plain":
            sel = np.arange(0, len(P.points), plain_sample) if plain_sample else None
            r = run_plain(P, epsrel, sel)
            plain_sel = sel if sel is not None else np.arange(len(P.points))
            plain_vals, plain_errs = r["values"], r["errors"]
            scale = len(P.points) / len(plain_sel)
            out["plain"] = dict(seconds=r["seconds"] * scale, measured_seconds=r["seconds"],
                                sampled_points=int(len(plain_sel)), evaluations=r["evaluations"] * scale,
                                failures=r["failures"],
                                max_rel_error=float(relative_errors(r["values"], r["errors"]).max()))
        elif mode == "batched":
            r = run_batched(P, epsrel)
            ref = r
            out["batched"] = dict(seconds=r["seconds"], evaluations=r["evaluations"], rc=r["rc"],
                                  iterations=r["iterations"],
                                  max_rel_error=float(relative_errors(r["values"], r["errors"]).max()))
        elif mode == "unsized":
            r = run_unsized(P, epsrel)
            out["unsized"] = dict(seconds=r["seconds"], evaluations=r["evaluations"], rc=r["rc"],
                                  presample_evaluations=r["presample_evaluations"],
                                  iterations=r["iterations"], kernel_seconds=r["kernel_seconds"],
                                  max_rel_error=float(relative_errors(r["values"], r["errors"]).max()))
        elif mode in ("learned", "learned_variance"):
            r = run_learned(P, epsrel, ntrain, steps=steps, sizing="logn" if mode == "learned" else "variance")
            d = {k: v for k, v in r.items() if k not in ("values", "errors")}
            d["max_rel_error"] = float(relative_errors(r["values"], r["errors"]).max())
            if ref is not None:
                diff = np.abs(r["values"] - ref["values"])
                comb = np.hypot(np.abs(r["errors"]), np.abs(ref["errors"]))
                d["max_diff_over_combined_sigma"] = float(np.max(diff / np.maximum(comb, 1e-300)))
            if plain_sel is not None:
                # the learned answers against the plain FP64 answers on the points plain ran
                diff = np.abs(r["values"][plain_sel] - plain_vals)
                amax = np.abs(plain_vals).max(axis=1, keepdims=True)
                comb = np.hypot(np.abs(r["errors"][plain_sel]), np.abs(plain_errs))
                d["vs_plain_max_rel_diff"] = float(np.max(diff / amax))
                d["vs_plain_max_diff_over_combined_sigma"] = float(np.max(diff / np.maximum(comb, 1e-300)))
            out[mode] = d
    for mode in ("learned", "learned_variance", "unsized", "batched"):
        if "plain" in out and mode in out:
            out[f"speedup_{mode}_vs_plain"] = out["plain"]["seconds"] / out[mode]["seconds"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=10000)
    ap.add_argument("--epsrel", type=float, default=1e-4)
    ap.add_argument("--modes", default="plain,unsized,learned")
    ap.add_argument("--ntrain", type=int, default=2000)
    ap.add_argument("--plain-sample", type=int, default=0, help="time plain on every k-th point only")
    ap.add_argument("--steps", type=int, default=1500, help="Adam steps of the network's training")
    args = ap.parse_args()
    print(json.dumps(compare(args.points, args.epsrel, args.modes, args.ntrain, args.plain_sample, args.steps)))


if __name__ == "__main__":
    main()
