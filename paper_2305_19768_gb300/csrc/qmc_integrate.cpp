// Combination and adaptive allocation (host side of the C-ABI):
// per-shift statistics, Laurent products of coefficient/prefactor series with
// sector series, variance propagation, the lattice-size allocation of
// Eq. (adaptive-solution), and the iterative driver qmc_integrate
// (section "Adaptive weighted sum evaluation" of arXiv:2305.19768).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "qmc_ctx.h"

static_assert(QMC_NCLASS == QMC_NUM_CLASSES, "evaluator class count of the C-ABI");

#define fail qmc_fail

namespace {

// Relative evaluation cost of a sector (FP64 operations of the evaluator's
// formulation, up to a constant): used to split a class's measured time per
// evaluation between its sectors (the online tau_i estimate).
double sector_cost(const QmcHostSector &S) {
    return 20.0 * S.d + 3.0 * (double)(S.U.size() + S.F.size()) + 30.0 * (double)(1 << S.ns) +
           15.0 * S.ns + (S.deform ? 300.0 : 0.0);
}

}  // namespace

extern "C" {

int qmc_shift_stats(const double *sums, int m, int norders, double *mean, double *var) {
    if (!sums || !mean || !var || m < 1 || norders < 1) return QMC_E_INVAL;
    for (int o = 0; o < norders; ++o) {
        for (int c = 0; c < 2; ++c) {
            double s = 0.0;
            for (int k = 0; k < m; ++k) s += sums[((size_t)k * norders + o) * 2 + c];
            const double mu = s / m;
            double v = 0.0;
            for (int k = 0; k < m; ++k) {
                const double dlt = sums[((size_t)k * norders + o) * 2 + c] - mu;
                v += dlt * dlt;
            }
            mean[o * 2 + c] = mu;
            var[o * 2 + c] = m > 1 ? v / (m - 1) / m : INFINITY;
        }
    }
    return QMC_OK;
}

int qmc_series_mul(const qmc_c64 *a, int a_lo, int na, const qmc_c64 *b, int b_lo, int nb, int lo, int n,
                   qmc_c64 *out) {
    if ((na && !a) || (nb && !b) || !out || n < 0) return QMC_E_INVAL;
    for (int o = 0; o < n; ++o) out[o].re = out[o].im = 0.0;
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
            const int o = a_lo + i + b_lo + j - lo;
            if (o < 0 || o >= n) continue;
            out[o].re += a[i].re * b[j].re - a[i].im * b[j].im;
            out[o].im += a[i].re * b[j].im + a[i].im * b[j].re;
        }
    return QMC_OK;
}

int qmc_series_var(const qmc_c64 *c, int c_lo, int nc, const double *v, int v_lo, int nv, int lo, int n,
                   double *out) {
    if ((nc && !c) || (nv && !v) || !out || n < 0) return QMC_E_INVAL;
    for (int o = 0; o < n; ++o) out[o] = 0.0;
    for (int i = 0; i < nc; ++i) {
        const double c2 = c[i].re * c[i].re + c[i].im * c[i].im;
        for (int j = 0; j < nv; ++j) {
            const int o = c_lo + i + v_lo + j - lo;
            if (o < 0 || o >= n) continue;
            out[o] += c2 * v[j];
        }
    }
    return QMC_OK;
}

int qmc_allocate(const double *W, const double *tau, const double *V, int nsums, int nint, double alpha,
                 double n_min, double *n_out) {
    if (!W || !tau || !V || !n_out || nsums < 0 || nint < 1 || !(alpha > 0)) return QMC_E_INVAL;
    for (int i = 0; i < nint; ++i) {
        if (!(tau[i] > 0)) return QMC_E_INVAL;
        n_out[i] = n_min;
    }
    const double p = 1.0 / (alpha + 1.0);
    for (int k = 0; k < nsums; ++k) {
        const double *Wk = W + (size_t)k * nint;
        if (!(V[k] > 0)) continue;
        double s = 0.0;
        for (int i = 0; i < nint; ++i)
            if (Wk[i] > 0) s += std::pow(Wk[i] * std::pow(tau[i], alpha), p);
        if (!(s > 0)) continue;
        const double lam = (1.0 / alpha) * std::pow(s / V[k], (alpha + 1.0) / alpha);
        for (int i = 0; i < nint; ++i)
            if (Wk[i] > 0) n_out[i] = std::max(n_out[i], std::pow(alpha * lam * Wk[i] / tau[i], p));
    }
    return QMC_OK;
}

int qmc_integrate_ex(qmc_ctx *ctx, const qmc_sum_spec *spec, double epsrel, double epsabs, double timeout_s,
                     int lowest_order, int norders, qmc_c64 *value, qmc_c64 *error, qmc_integrate_info *info,
                     const uint64_t *n_init, int shifts, double *w_out, uint64_t *n_out, double *lambda_io);

int qmc_integrate(qmc_ctx *ctx, const qmc_sum_spec *spec, double epsrel, double epsabs, double timeout_s,
                  int lowest_order, int norders, qmc_c64 *value, qmc_c64 *error, qmc_integrate_info *info) {
    return qmc_integrate_ex(ctx, spec, epsrel, epsabs, timeout_s, lowest_order, norders, value, error, info,
                            nullptr, 0, nullptr, nullptr, nullptr);
}

int qmc_integrate_ex(qmc_ctx *ctx, const qmc_sum_spec *spec, double epsrel, double epsabs, double timeout_s,
                     int lowest_order, int norders, qmc_c64 *value, qmc_c64 *error, qmc_integrate_info *info,
                     const uint64_t *n_init, int shifts, double *w_out, uint64_t *n_out, double *lambda_io) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    if (!ctx || !value || !error || norders < 1 || norders > 16 || !(epsrel >= 0) || !(epsabs >= 0))
        return fail(ctx, QMC_E_INVAL, "qmc_integrate: bad arguments");
    const double presample_evals0 = ctx->presample_evals;
    if (ctx->lattices.empty()) return fail(ctx, QMC_E_INVAL, "qmc_integrate: no lattice table");
    // --- what to sum
    std::vector<int> ids;
    int namp = 1, coef_lo = 0, ncoef = 1;
    const qmc_c64 *coef = nullptr;
    if (spec && spec->nint > 0) {
        ids.assign(spec->integral_ids, spec->integral_ids + spec->nint);
        namp = spec->namp > 0 ? spec->namp : 1;
        coef = spec->coef;
        if (coef) {
            coef_lo = spec->coef_lo;
            ncoef = spec->ncoef;
        }
    } else {
        for (size_t i = 0; i < ctx->integrals.size(); ++i) ids.push_back((int)i);
    }
    if (ids.empty()) return fail(ctx, QMC_E_INVAL, "qmc_integrate: nothing to integrate");
    for (int id : ids)
        if (id < 0 || id >= (int)ctx->integrals.size()) return fail(ctx, QMC_E_INVAL, "bad integral id %d", id);
    const int nint = (int)ids.size();
    bool any_inv = false;
    for (int id : ids) any_inv |= !ctx->integrals[id].invariants.empty();
    const int npts = any_inv ? ctx->npoints : std::max(1, ctx->npoints);
    if (npts < 1) return fail(ctx, QMC_E_INVAL, "qmc_integrate: no kinematic points");
    // --- sector order window
    const int hiA = lowest_order + norders - 1;
    int slo = 0, shi = -1000;
    for (int id : ids) {
        const QmcHostIntegral &I = ctx->integrals[id];
        slo = std::min(slo, -I.max_poles);
        shi = std::max(shi, hiA - coef_lo - I.pref_lo);
    }
    if (shi < slo) return fail(ctx, QMC_E_INVAL, "qmc_integrate: requested orders below every integral's series");
    const int sn = shi - slo + 1;
    // --- combined coefficient series G[p][k][i] = C_ki(p) (x) prefactor_i, orders glo..
    int glo = 1 << 20, ghi = -(1 << 20);
    for (int id : ids) {
        glo = std::min(glo, coef_lo + ctx->integrals[id].pref_lo);
        ghi = std::max(ghi, coef_lo + ncoef - 1 + ctx->integrals[id].pref_lo + (int)ctx->integrals[id].pref.size() - 1);
    }
    const int gn = ghi - glo + 1;
    std::vector<qmc_c64> G((size_t)npts * namp * nint * gn);
    for (int p = 0; p < npts; ++p)
        for (int k = 0; k < namp; ++k)
            for (int i = 0; i < nint; ++i) {
                const QmcHostIntegral &I = ctx->integrals[ids[i]];
                std::vector<qmc_c64> one(1, qmc_c64{1.0, 0.0});
                const qmc_c64 *c = coef ? coef + (((size_t)p * namp + k) * nint + i) * ncoef : one.data();
                qmc_series_mul(c, coef ? coef_lo : 0, coef ? ncoef : 1, I.pref.data(), I.pref_lo, (int)I.pref.size(),
                               glo, gn, &G[(((size_t)p * namp + k) * nint + i) * gn]);
            }
    // --- slots (point, integral, sector)
    struct Slot {
        int p, i, s;
        uint64_t n = 0;
        bool have = false, dirty = true;
        bool fp64 = false;   // escalated to FP64 in a mixed-precision context
        double mean[2 * 8], var[2 * 8];
        double cost = 1.0;
        double lambda = 0.3;
    };
    std::vector<Slot> slots;
    std::vector<uint64_t> sizes;
    for (auto &kv : ctx->lattices) sizes.push_back(kv.first);
    const uint64_t nmax_cap = ctx->opt.max_points ? ctx->opt.max_points : sizes.back();
    auto round_up = [&](double n) -> uint64_t {
        for (uint64_t v : sizes)
            if ((double)v >= n && v <= nmax_cap) return v;
        uint64_t best = sizes.front();
        for (uint64_t v : sizes)
            if (v <= nmax_cap) best = v;
        return best;
    };
    auto round_down = [&](double n) -> uint64_t {   // largest tabulated size <= n (<= the cap)
        uint64_t best = sizes.front();
        for (uint64_t v : sizes)
            if ((double)v <= n && v <= nmax_cap) best = v;
        return best;
    };
    const uint64_t n0 = round_up((double)ctx->opt.min_points);
    if (sn > 8) return fail(ctx, QMC_E_INVAL, "qmc_integrate: %d sector orders exceed 8", sn);
    for (int p = 0; p < npts; ++p)
        for (int i = 0; i < nint; ++i) {
            const QmcHostIntegral &I = ctx->integrals[ids[i]];
            for (int s = 0; s < (int)I.sectors.size(); ++s) {
                Slot sl;
                sl.p = p;
                sl.i = i;
                sl.s = s;
                sl.n = n_init ? round_up((double)n_init[slots.size()]) : n0;
                sl.cost = sector_cost(I.sectors[s]);
                slots.push_back(sl);
            }
        }
    const int m = shifts > 1 ? shifts : ctx->opt.shifts;
    const double alpha = 2.0;
    std::vector<size_t> pbegin(npts + 1, slots.size());   // slots of point p: [pbegin[p], pbegin[p+1])
    for (size_t q = slots.size(); q-- > 0;) pbegin[slots[q].p] = q;
    for (int p = npts - 1; p >= 0; --p) pbegin[p] = std::min(pbegin[p], pbegin[p + 1]);
    // contour-deformation parameter per deformed slot: fixed by the options, or
    // chosen by presampling (number_of_presamples points per candidate)
    {
        std::vector<qmc_job> pre;
        std::vector<size_t> pre_slot;
        for (size_t q = 0; q < slots.size(); ++q) {
            Slot &sl = slots[q];
            const QmcHostIntegral &I = ctx->integrals[ids[sl.i]];
            if (!I.sectors[sl.s].deform) continue;
            if (lambda_io && lambda_io[q] > 0) {
                sl.lambda = lambda_io[q];
                continue;
            }
            if (ctx->opt.lambda > 0) {
                sl.lambda = ctx->opt.lambda;
                continue;
            }
            qmc_job J;
            memset(&J, 0, sizeof J);
            J.integral_id = ids[sl.i];
            J.sector = sl.s;
            J.point = I.invariants.empty() ? 0 : sl.p;
            J.shifts = 2;
            J.n = sizes.front();
            J.seed = ctx->opt.seed;
            J.stream = q;
            pre.push_back(J);
            pre_slot.push_back(q);
        }
        if (!pre.empty()) {
            const int rc = qmc_presample_lambda(ctx, pre.data(), (int)pre.size(), slo, sn, 1.0, 16);
            if (rc && rc != QMC_E_SIGN_CHECK) return rc;
            for (size_t j = 0; j < pre.size(); ++j) slots[pre_slot[j]].lambda = pre[j].lambda[0];
        }
    }
    double evals = 0.0, kernel_s = 0.0;
    int iter = 0, rc_final = QMC_OK;
    std::vector<double> tau(slots.size(), 1.0);
    std::vector<double> amp_val((size_t)npts * namp * norders * 2), amp_var((size_t)npts * namp * norders);
    std::vector<double> amp_vre((size_t)npts * namp * norders), amp_vim((size_t)npts * namp * norders);
    std::vector<size_t> resample;   // slots to presample again after a sign-check failure
    int resample_rounds = 0;
    for (;;) {
        // ---- evaluate dirty slots in one plan
        std::vector<qmc_job> jobs;
        std::vector<size_t> jslot;
        for (size_t q = 0; q < slots.size(); ++q) {
            Slot &sl = slots[q];
            if (!sl.dirty) continue;
            const QmcHostIntegral &I = ctx->integrals[ids[sl.i]];
            qmc_job J;
            memset(&J, 0, sizeof J);
            J.integral_id = ids[sl.i];
            J.sector = sl.s;
            J.point = I.invariants.empty() ? 0 : sl.p;
            J.shifts = m;
            J.n = sl.n;
            J.seed = ctx->opt.seed;
            J.stream = ((uint64_t)iter << 40) | q;
            J.flags = sl.fp64 ? QMC_JOB_FP64 : 0;
            for (int j = 0; j < 6; ++j) J.lambda[j] = sl.lambda;
            jobs.push_back(J);
            jslot.push_back(q);
        }
        if (!jobs.empty()) {
            qmc_plan *plan = nullptr;
            int rc = qmc_plan_create(ctx, jobs.data(), (int)jobs.size(), slo, sn, &plan);
            if (rc) return rc;
            std::vector<double> out(qmc_plan_output_size(plan));
            rc = qmc_plan_run(plan, nullptr, nullptr);
            uint64_t sf = 0;
            if (!rc) rc = qmc_plan_results(plan, out.data(), &sf);
            if (rc && rc != QMC_E_SIGN_CHECK) {
                qmc_plan_destroy(plan);
                return rc;
            }
            if (rc == QMC_E_SIGN_CHECK) {
                // a deformed slot whose contour crossed to Im F > 0 on this lattice:
                // presample again below its lambda and evaluate it once more
                std::vector<uint32_t> fails(jobs.size(), 0);
                rc = qmc_plan_job_failures(plan, fails.data());
                if (rc) {
                    qmc_plan_destroy(plan);
                    return rc;
                }
                for (size_t j = 0; j < jobs.size(); ++j)
                    if (fails[j]) resample.push_back(jslot[j]);
            }
            // per-class time per evaluation -> tau of each slot (cost-weighted)
            for (size_t c = 0; c < plan->launches.size(); ++c) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, plan->kev[2 * c], plan->kev[2 * c + 1]);
                kernel_s += ms * 1e-3;
                double ev = 0.0, cw = 0.0;
                auto eff = [&](const qmc_job &J) {
                    const QmcHostSector &S = ctx->integrals[J.integral_id].sectors[J.sector];
                    return ctx->opt.precision == QMC_PRECISION_MIXED && !(J.flags & QMC_JOB_FP64)
                               ? qmc_class_mixed(S.cls) : S.cls;
                };
                for (size_t j = 0; j < jobs.size(); ++j) {
                    if (eff(jobs[j]) != plan->launches[c].cls) continue;
                    ev += (double)jobs[j].n * m;
                    cw += (double)jobs[j].n * m * slots[jslot[j]].cost;
                }
                const double per_cost = cw > 0 ? ms * 1e-3 / cw : 1e-9;
                for (size_t j = 0; j < jobs.size(); ++j)
                    if (eff(jobs[j]) == plan->launches[c].cls) tau[jslot[j]] = per_cost * slots[jslot[j]].cost;
                evals += ev;
            }
            qmc_plan_destroy(plan);
            for (size_t j = 0; j < jobs.size(); ++j) {
                Slot &sl = slots[jslot[j]];
                qmc_shift_stats(&out[j * (size_t)m * sn * 2], m, sn, sl.mean, sl.var);
                sl.have = true;
                sl.dirty = false;
            }
        }
        ++iter;
        if (!resample.empty() && ++resample_rounds > 8) {
            rc_final = QMC_E_SIGN_CHECK;   // lambda keeps failing: keep the results, report it
            resample.clear();
        }
        if (!resample.empty()) {
            std::vector<qmc_job> pre;
            for (size_t q : resample) {
                const Slot &sl = slots[q];
                qmc_job J;
                memset(&J, 0, sizeof J);
                J.integral_id = ids[sl.i];
                J.sector = sl.s;
                J.point = ctx->integrals[ids[sl.i]].invariants.empty() ? 0 : sl.p;
                J.seed = ctx->opt.seed;
                J.stream = ((uint64_t)iter << 40) | q;
                pre.push_back(J);
            }
            // candidates below the smallest failing lambda (all failing slots in one search)
            double lmax = 1.0;   // (a failing lambda <= 0 restarts from 1)
            for (size_t q : resample)
                if (slots[q].lambda > 0) lmax = std::min(lmax, 0.7 * slots[q].lambda);
            const int prc = qmc_presample_lambda(ctx, pre.data(), (int)pre.size(), slo, sn, lmax, 16);
            if (prc && prc != QMC_E_SIGN_CHECK) return prc;
            for (size_t u = 0; u < resample.size(); ++u) {
                Slot &sl = slots[resample[u]];
                sl.lambda = pre[u].lambda[0];   // the largest passing candidate, else the smallest tried
                sl.dirty = true;
            }
            resample.clear();
            if (std::any_of(slots.begin(), slots.end(), [](const Slot &s) { return s.dirty; })) continue;
        }
        // ---- combine into the sums and check the requested accuracy
        bool all_ok = true;
        std::vector<char> sum_ok((size_t)npts * namp * norders, 1);
        std::vector<double> target((size_t)npts * namp * norders, 0.0);
        std::fill(amp_val.begin(), amp_val.end(), 0.0);
        std::fill(amp_var.begin(), amp_var.end(), 0.0);
        std::fill(amp_vre.begin(), amp_vre.end(), 0.0);
        std::fill(amp_vim.begin(), amp_vim.end(), 0.0);
        for (const Slot &sl : slots) {
            qmc_c64 mu[8];
            double vv[8];
            for (int o = 0; o < sn; ++o) {
                mu[o].re = sl.mean[2 * o];
                mu[o].im = sl.mean[2 * o + 1];
                vv[o] = sl.var[2 * o] + sl.var[2 * o + 1];
            }
            for (int k = 0; k < namp; ++k) {
                const qmc_c64 *g = &G[(((size_t)sl.p * namp + k) * nint + sl.i) * gn];
                qmc_c64 a[64];
                double v[64];
                qmc_series_mul(g, glo, gn, mu, slo, sn, lowest_order, norders, a);
                qmc_series_var(g, glo, gn, vv, slo, sn, lowest_order, norders, v);
                for (int o = 0; o < norders; ++o) {
                    const size_t idx = ((size_t)sl.p * namp + k) * norders + o;
                    amp_val[2 * idx] += a[o].re;
                    amp_val[2 * idx + 1] += a[o].im;
                    amp_var[idx] += v[o];
                    // Re and Im separately: Re(g x) has variance g_r^2 v_r + g_i^2 v_i
                    for (int so = 0; so < sn; ++so) {
                        const int gi = (lowest_order + o) - (slo + so) - glo;
                        if (gi < 0 || gi >= gn) continue;
                        const double gr2 = g[gi].re * g[gi].re, gi2 = g[gi].im * g[gi].im;
                        amp_vre[idx] += gr2 * sl.var[2 * so] + gi2 * sl.var[2 * so + 1];
                        amp_vim[idx] += gi2 * sl.var[2 * so] + gr2 * sl.var[2 * so + 1];
                    }
                }
            }
        }
        for (size_t idx = 0; idx < sum_ok.size(); ++idx) {
            double mag = std::hypot(amp_val[2 * idx], amp_val[2 * idx + 1]);
            if (ctx->opt.target_mode == QMC_TARGET_AMPLITUDE) {
                // relative to the largest coefficient of this amplitude at this point
                const size_t base = idx - idx % norders;
                for (int o = 0; o < norders; ++o)
                    mag = std::max(mag, std::hypot(amp_val[2 * (base + o)], amp_val[2 * (base + o) + 1]));
            }
            const double tgt = std::max(epsrel * mag, epsabs);
            target[idx] = tgt;
            if (!(std::sqrt(amp_var[idx]) <= tgt)) {
                sum_ok[idx] = 0;
                all_ok = false;
            }
        }
        const double elapsed = std::chrono::duration<double>(clk::now() - t_start).count();
        if (all_ok) break;
        if (timeout_s > 0 && elapsed > timeout_s) {
            rc_final = QMC_E_TIMEOUT;
            break;
        }
        // ---- allocation (Eq. adaptive-solution), one sum at a time, keeping the largest n
        bool grew = false;
        for (int p = 0; p < npts; ++p)
            for (int k = 0; k < namp; ++k)
                for (int o = 0; o < norders; ++o) {
                    const size_t idx = ((size_t)p * namp + k) * norders + o;
                    if (sum_ok[idx] || !(target[idx] > 0)) continue;
                    std::vector<size_t> members;
                    std::vector<double> W, tv;
                    for (size_t q = pbegin[p]; q < pbegin[p + 1]; ++q) {
                        const Slot &sl = slots[q];
                        const qmc_c64 *g = &G[(((size_t)p * namp + k) * nint + sl.i) * gn];
                        // W = sum_{o'} |g^{(o - o')}|^2 w^{(o')},  w = var n^alpha
                        double wsum = 0.0;
                        for (int so = 0; so < sn; ++so) {
                            const int gi = (lowest_order + o) - (slo + so) - glo;
                            if (gi < 0 || gi >= gn) continue;
                            const double c2 = g[gi].re * g[gi].re + g[gi].im * g[gi].im;
                            const double w = (sl.var[2 * so] + sl.var[2 * so + 1]) * std::pow((double)sl.n, alpha);
                            wsum += c2 * w;
                        }
                        if (wsum > 0) {
                            members.push_back(q);
                            W.push_back(wsum);
                            tv.push_back(tau[q]);
                        }
                    }
                    if (members.empty()) continue;
                    const double V = target[idx] * target[idx];
                    std::vector<double> nn(members.size());
                    qmc_allocate(W.data(), tv.data(), &V, 1, (int)members.size(), alpha, 0.0, nn.data());
                    for (size_t u = 0; u < members.size(); ++u) {
                        Slot &sl = slots[members[u]];
                        if (ctx->opt.precision == QMC_PRECISION_MIXED && !sl.fp64 &&
                            (nn[u] > (double)nmax_cap || sl.n >= nmax_cap)) {
                            // beyond the lattice cap in mixed precision: the FP32 products'
                            // error floor, not the lattice, limits this sector -- FP64 from here
                            sl.fp64 = true;
                            sl.dirty = true;
                            grew = true;
                        }
                        uint64_t want = round_up(nn[u]);
                        if (ctx->opt.max_growth > 1 && (double)want > (double)sl.n * ctx->opt.max_growth)
                            want = std::max(round_down((double)sl.n * ctx->opt.max_growth), round_up((double)sl.n + 1));
                        if (want > sl.n) {
                            sl.n = want;
                            sl.dirty = true;
                            grew = true;
                        }
                    }
                }
        if (!grew) {
            rc_final = QMC_E_NOT_CONVERGED;
            break;
        }
    }
    for (size_t idx = 0; idx < (size_t)npts * namp * norders; ++idx) {
        value[idx].re = amp_val[2 * idx];
        value[idx].im = amp_val[2 * idx + 1];
        error[idx].re = std::sqrt(amp_vre[idx]);
        error[idx].im = std::sqrt(amp_vim[idx]);
    }
    for (size_t q = 0; q < slots.size(); ++q) {
        const Slot &sl = slots[q];
        if (lambda_io) lambda_io[q] = ctx->integrals[ids[sl.i]].sectors[sl.s].deform ? sl.lambda : 0.0;
        if (n_out) n_out[q] = sl.n;
        if (w_out) {
            double v = 0.0;
            for (int so = 0; so < sn; ++so) v += sl.var[2 * so] + sl.var[2 * so + 1];
            w_out[q] = v * std::pow((double)sl.n, alpha);
        }
    }
    if (info) {
        memset(info, 0, sizeof *info);
        info->evaluations = evals;
        info->seconds = std::chrono::duration<double>(clk::now() - t_start).count();
        info->kernel_seconds = kernel_s;
        info->iterations = iter;
        uint64_t mx = 0;
        for (const Slot &sl : slots) mx = std::max(mx, sl.n);
        info->max_lattice = mx;
        info->presample_evaluations = ctx->presample_evals - presample_evals0;
        int esc = 0;
        for (const Slot &sl : slots) esc += sl.fp64 ? 1 : 0;
        info->fp64_escalations = esc;
    }
    if (rc_final == QMC_E_TIMEOUT) return fail(ctx, QMC_E_TIMEOUT, "qmc_integrate: timeout after %d iterations", iter);
    if (rc_final == QMC_E_NOT_CONVERGED)
        return fail(ctx, QMC_E_NOT_CONVERGED, "qmc_integrate: largest lattice reached before the requested accuracy");
    if (rc_final == QMC_E_SIGN_CHECK)
        return fail(ctx, QMC_E_SIGN_CHECK, "qmc_integrate: deformed points had Im F > 0 (lambda too large)");
    return QMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- presampling and autotuning
extern "C" int qmc_presample_lambda(qmc_ctx *ctx, qmc_job *jobs, int njobs, int lo, int norders,
                                    double lambda_max, int ncand) {
    if (!ctx || !jobs || njobs < 0 || norders < 1 || !(lambda_max > 0) || ncand < 1 || ncand > 32)
        return fail(ctx, QMC_E_INVAL, "qmc_presample_lambda: bad arguments");
    std::vector<uint64_t> sizes;
    for (auto &kv : ctx->lattices) sizes.push_back(kv.first);
    if (sizes.empty()) return fail(ctx, QMC_E_INVAL, "qmc_presample_lambda: no lattice table");
    const int m_pre = 2;
    const double want = std::max(2.0, (double)ctx->opt.presamples / m_pre);
    uint64_t n_pre = sizes.back();
    for (uint64_t v : sizes)
        if ((double)v >= want) {
            n_pre = v;
            break;
        }
    // decreasing-lambda search: round c evaluates candidate lambda_max * 0.7^c for
    // the jobs that have not passed yet; a job takes the first candidate with no
    // sign-check failure and finite estimates
    std::vector<int> pending;
    for (int i = 0; i < njobs; ++i) {
        const qmc_job &J = jobs[i];
        if (J.integral_id < 0 || J.integral_id >= (int)ctx->integrals.size())
            return fail(ctx, QMC_E_INVAL, "job %d: bad integral id", i);
        const QmcHostIntegral &I = ctx->integrals[J.integral_id];
        if (J.sector < 0 || J.sector >= (int)I.sectors.size()) return fail(ctx, QMC_E_INVAL, "job %d: bad sector", i);
        if (I.sectors[J.sector].deform) pending.push_back(i);
    }
    double l = lambda_max;
    for (int c = 0; c < ncand && !pending.empty(); ++c, l *= 0.7) {
        std::vector<qmc_job> cand;
        for (int i : pending) {
            qmc_job C = jobs[i];
            C.shifts = m_pre;
            C.n = n_pre;
            C.stream = jobs[i].stream * 64 + (uint64_t)c + 0x7000000000000000ULL;
            for (int j = 0; j < 6; ++j) C.lambda[j] = l;
            cand.push_back(C);
        }
        qmc_plan *plan = nullptr;
        int rc = qmc_plan_create(ctx, cand.data(), (int)cand.size(), lo, norders, &plan);
        if (rc) return rc;
        ctx->presample_evals += (double)cand.size() * (double)n_pre * m_pre;
        std::vector<double> out(qmc_plan_output_size(plan));
        std::vector<uint32_t> fails(cand.size(), 0);
        rc = qmc_plan_run(plan, nullptr, nullptr);
        if (!rc) {
            rc = qmc_plan_results(plan, out.data(), nullptr);
            if (rc == QMC_E_SIGN_CHECK || rc == QMC_E_NONFINITE) rc = QMC_OK;
        }
        if (!rc) rc = qmc_plan_job_failures(plan, fails.data());
        qmc_plan_destroy(plan);
        if (rc) return rc;
        std::vector<int> still;
        for (size_t k = 0; k < cand.size(); ++k) {
            bool ok = fails[k] == 0;
            const double *q = &out[k * (size_t)m_pre * norders * 2];
            for (int u = 0; u < m_pre * norders * 2; ++u) ok &= std::isfinite(q[u]) != 0;
            const int i = pending[k];
            for (int j = 0; j < 6; ++j) jobs[i].lambda[j] = l;   // the last tried stays if none passes
            if (!ok) still.push_back(i);
        }
        pending.swap(still);
    }
    if (!pending.empty())
        return fail(ctx, QMC_E_SIGN_CHECK, "qmc_presample_lambda: %zu jobs fail the sign check for every candidate",
                    pending.size());
    return QMC_OK;
}

extern "C" int qmc_autotune(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders, int *best_block,
                            int *best_ppt) {
    if (!ctx || !jobs || njobs < 1 || norders < 1) return fail(ctx, QMC_E_INVAL, "qmc_autotune: bad arguments");
    // a sample of up to 32 jobs per kernel class, at most 8 shifts each
    std::vector<std::vector<qmc_job>> per(QMC_NCLASS);
    for (int i = 0; i < njobs; ++i) {
        const qmc_job &J = jobs[i];
        if (J.integral_id < 0 || J.integral_id >= (int)ctx->integrals.size()) continue;
        const QmcHostIntegral &I = ctx->integrals[J.integral_id];
        if (J.sector < 0 || J.sector >= (int)I.sectors.size()) continue;
        const int base = I.sectors[J.sector].cls;
        const int cls = ctx->opt.precision == QMC_PRECISION_MIXED ? qmc_class_mixed(base) : base;
        if (per[cls].size() < 32) {
            qmc_job C = J;
            C.shifts = std::min(C.shifts, 8);
            per[cls].push_back(C);
        }
    }
    const int blocks[2] = {128, 256};
    const int ppts[4] = {4, 8, 16, 32};
    const qmc_options saved = ctx->opt;
    for (int cls = 0; cls < QMC_NCLASS; ++cls) {
        if (per[cls].empty()) continue;
        double best = INFINITY;
        int bb = 128, bp = 16;
        for (int b : blocks)
            for (int p : ppts) {
                if (b == 256 && qmc_class_dmax(cls) > 3) continue;   // 128-thread blocks only
                ctx->opt.block = b;
                ctx->opt.ppt = p;
                qmc_plan *plan = nullptr;
                int rc = qmc_plan_create(ctx, per[cls].data(), (int)per[cls].size(), lo, norders, &plan);
                if (rc) {
                    ctx->opt = saved;
                    return rc;
                }
                float ms = 0.f, best_ms = INFINITY;
                for (int rep = 0; rep < 3 && !rc; ++rep) {
                    rc = qmc_plan_run(plan, nullptr, nullptr);
                    if (!rc) rc = qmc_plan_last_time(plan, nullptr, &ms, nullptr);
                    if (rep > 0) best_ms = std::min(best_ms, ms);
                }
                qmc_plan_destroy(plan);
                if (rc) {
                    ctx->opt = saved;
                    return rc;
                }
                if (best_ms < best) {
                    best = best_ms;
                    bb = b;
                    bp = p;
                }
            }
        ctx->tuned_block[cls] = bb;
        ctx->tuned_ppt[cls] = bp;
    }
    ctx->opt = saved;
    for (int cls = 0; cls < QMC_NCLASS; ++cls) {
        if (best_block) best_block[cls] = ctx->tuned_block[cls];
        if (best_ppt) best_ppt[cls] = ctx->tuned_ppt[cls];
    }
    return QMC_OK;
}

// ---------------------------------------------------------------- median QMC rules
namespace {
uint64_t sm64_next(uint64_t &state) {
    uint64_t z = (state += kQmcGamma);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}
}  // namespace

extern "C" int qmc_median_candidates(uint64_t n, int d, int r, uint64_t seed, uint32_t *z) {
    if (!z || n < 2 || n >= (1ULL << 32) || d < 1 || d > 6 || r < 1) return QMC_E_INVAL;
    uint64_t st = seed;
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < 6; ++j) {
            if (j >= d) {
                z[i * 6 + j] = 1;
                continue;
            }
            for (;;) {
                const uint64_t c = 1 + sm64_next(st) % (n - 1);
                if (gcd64(c, n) == 1) {
                    z[i * 6 + j] = (uint32_t)c;
                    break;
                }
            }
        }
    return QMC_OK;
}

extern "C" int qmc_median_lattice(qmc_ctx *ctx, const qmc_job *job, int lo, int norders, int r, uint64_t seed,
                                  uint32_t *z_out, double *estimates) {
    if (!ctx || !job || !z_out || r < 1 || r > 1024 || !(r & 1) || norders < 1)
        return fail(ctx, QMC_E_INVAL, "qmc_median_lattice: bad arguments (r must be odd)");
    if (job->integral_id < 0 || job->integral_id >= (int)ctx->integrals.size() || job->sector < 0 ||
        job->sector >= (int)ctx->integrals[job->integral_id].sectors.size())
        return fail(ctx, QMC_E_INVAL, "qmc_median_lattice: bad job");
    const int d = ctx->integrals[job->integral_id].sectors[job->sector].d;
    std::vector<uint32_t> cand((size_t)r * 6);
    int rc = qmc_median_candidates(job->n, d, r, seed, cand.data());
    if (rc) return fail(ctx, rc, "qmc_median_lattice: bad lattice size");
    std::vector<qmc_job> jobs((size_t)r, *job);
    for (int i = 0; i < r; ++i) {
        memcpy(jobs[i].z, &cand[(size_t)i * 6], sizeof jobs[i].z);
        jobs[i].shifts = 1;
        jobs[i].flags |= QMC_JOB_UNSHIFTED;
    }
    qmc_plan *plan = nullptr;
    rc = qmc_plan_create(ctx, jobs.data(), r, lo, norders, &plan);
    if (rc) return rc;
    std::vector<double> out(qmc_plan_output_size(plan));
    rc = qmc_plan_run(plan, nullptr, nullptr);
    if (!rc) rc = qmc_plan_results(plan, out.data(), nullptr);
    qmc_plan_destroy(plan);
    if (rc) return rc;
    // Eq. (median): the candidate whose estimate (Re of the highest order) is the median
    std::vector<int> idx((size_t)r);
    for (int i = 0; i < r; ++i) idx[i] = i;
    const int o = norders - 1;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return out[(size_t)a * norders * 2 + 2 * o] <
                                                                         out[(size_t)b * norders * 2 + 2 * o]; });
    const int med = idx[r / 2];
    memcpy(z_out, &cand[(size_t)med * 6], 6 * sizeof(uint32_t));
    if (estimates) memcpy(estimates, out.data(), out.size() * sizeof(double));
    return QMC_OK;
}
