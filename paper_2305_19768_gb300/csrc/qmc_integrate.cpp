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

// Primality of n < 2^32 by Miller-Rabin with the bases 2, 7 and 61, which
// decide every n below 4759123141 (Jaeschke 1993).
uint64_t mulmod(uint64_t a, uint64_t b, uint64_t n) { return (uint64_t)((unsigned __int128)a * b % n); }
uint64_t powmod(uint64_t a, uint64_t e, uint64_t n) {
    uint64_t r = 1;
    a %= n;
    while (e) {
        if (e & 1) r = mulmod(r, a, n);
        a = mulmod(a, a, n);
        e >>= 1;
    }
    return r;
}
bool is_prime32(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t p : {2ULL, 3ULL, 5ULL, 7ULL, 61ULL})
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    for (uint64_t a : {2ULL, 7ULL, 61ULL}) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}
constexpr uint64_t kLargestPrime32 = 4294967291ULL;   // the largest prime below 2^32
uint64_t next_prime(uint64_t n) {
    if (n <= 2) return 2;
    if (n > kLargestPrime32) return kLargestPrime32;
    while (!is_prime32(n)) ++n;
    return n;
}
uint64_t prev_prime(uint64_t n) {
    if (n > kLargestPrime32) return kLargestPrime32;
    while (n > 2 && !is_prime32(n)) --n;
    return n < 2 ? 2 : n;
}
// splitmix64's output function: decorrelated seeds for the median candidates
uint64_t mix64(uint64_t z) {
    z += kQmcGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
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
    if (ctx->lattices.empty() && ctx->opt.lattice_candidates == 0)
        return fail(ctx, QMC_E_INVAL, "qmc_integrate: no lattice table");
    if (ctx->host_only && !ctx->eval_hook)
        return fail(ctx, QMC_E_CUDA, "qmc_integrate: host-only context without an evaluator");
    const int world = (ctx->allreduce && ctx->world > 1) ? ctx->world : 1;
    const int rank = world > 1 ? ctx->rank : 0;
    // --- what to sum: the spec, the coefficients of qmc_set_coefficients, or all integrals with C = 1
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
        if (ctx->coef_namp > 0) {
            if (ctx->coef_nint != (int)ctx->integrals.size())
                return fail(ctx, QMC_E_INVAL, "qmc_integrate: coefficients were set for %d integrals, %zu are loaded",
                            ctx->coef_nint, ctx->integrals.size());
            namp = ctx->coef_namp;
            coef = ctx->coef.data();
            coef_lo = ctx->coef_lo;
            ncoef = ctx->coef_n;
        }
    }
    if (ids.empty()) return fail(ctx, QMC_E_INVAL, "qmc_integrate: nothing to integrate");
    for (int id : ids)
        if (id < 0 || id >= (int)ctx->integrals.size()) return fail(ctx, QMC_E_INVAL, "bad integral id %d", id);
    const int nint = (int)ids.size();
    bool any_inv = false;
    for (int id : ids) any_inv |= !ctx->integrals[id].invariants.empty();
    const int npts = any_inv ? ctx->npoints : std::max(1, ctx->npoints);
    if (npts < 1) return fail(ctx, QMC_E_INVAL, "qmc_integrate: no kinematic points");
    if (!(spec && spec->nint > 0) && ctx->coef_namp > 0 && ctx->coef_npoints != npts)
        return fail(ctx, QMC_E_INVAL, "qmc_integrate: coefficients were set for %d points, the kinematics have %d",
                    ctx->coef_npoints, npts);
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
    if (sn > 8) return fail(ctx, QMC_E_INVAL, "qmc_integrate: %d sector orders exceed 8", sn);
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
                const qmc_c64 one{1.0, 0.0};
                const qmc_c64 *c = coef ? coef + (((size_t)p * namp + k) * nint + i) * ncoef : &one;
                qmc_series_mul(c, coef ? coef_lo : 0, coef ? ncoef : 1, I.pref.data(), I.pref_lo, (int)I.pref.size(),
                               glo, gn, &G[(((size_t)p * namp + k) * nint + i) * gn]);
            }
    // --- lattice sizes: the CBC table, or any prime for median rules
    const bool median = ctx->opt.lattice_candidates > 0;
    const int rcand = ctx->opt.lattice_candidates;
    std::vector<uint64_t> sizes;
    for (auto &kv : ctx->lattices) sizes.push_back(kv.first);
    const uint64_t nmax_cap = ctx->opt.max_points ? ctx->opt.max_points
                                                  : (median ? kLargestPrime32 : sizes.back());
    auto round_up = [&](double n) -> uint64_t {
        if (median) {
            const uint64_t want = n < 2.0 ? 2 : (n >= (double)nmax_cap ? nmax_cap : (uint64_t)std::ceil(n));
            const uint64_t v = next_prime(want);
            return v <= nmax_cap ? v : prev_prime(nmax_cap);
        }
        for (uint64_t v : sizes)
            if ((double)v >= n && v <= nmax_cap) return v;
        uint64_t best = sizes.front();
        for (uint64_t v : sizes)
            if (v <= nmax_cap) best = v;
        return best;
    };
    auto round_down = [&](double n) -> uint64_t {   // largest available size <= n (<= the cap)
        if (median) return prev_prime((uint64_t)std::min<double>(std::max(n, 2.0), (double)nmax_cap));
        uint64_t best = sizes.front();
        for (uint64_t v : sizes)
            if ((double)v <= n && v <= nmax_cap) best = v;
        return best;
    };
    // --- slots (point, integral, sector)
    struct Slot {
        int p, i, s;
        uint64_t n = 0;
        bool have = false, dirty = true;
        bool fp64 = false;   // escalated to FP64 in a mixed-precision context
        double mean[2 * 8], var[2 * 8];
        double cost = 1.0;
        double lambda = 0.3;
        uint64_t zn = 0;     // lattice size the median vector z was chosen for
        uint32_t z[6] = {0, 0, 0, 0, 0, 0};
        std::vector<double> sums;   // last per-shift sums [m][sn][2] (keep_shift_sums)
    };
    std::vector<Slot> slots;
    const uint64_t n0 = round_up((double)ctx->opt.min_points);
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
    auto job_for = [&](size_t q) {
        const Slot &sl = slots[q];
        const QmcHostIntegral &I = ctx->integrals[ids[sl.i]];
        qmc_job J;
        memset(&J, 0, sizeof J);
        J.integral_id = ids[sl.i];
        J.sector = sl.s;
        J.point = I.invariants.empty() ? 0 : sl.p;
        J.seed = ctx->opt.seed;
        return J;
    };
    // split items (with costs) over the ranks: largest first, each to the least-loaded rank
    auto partition = [&](const std::vector<double> &cost) {
        std::vector<int> owner(cost.size(), 0);
        if (world == 1) return owner;
        std::vector<size_t> order(cost.size());
        for (size_t u = 0; u < order.size(); ++u) order[u] = u;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
        std::vector<double> load(world, 0.0);
        for (size_t u : order) {
            int best = 0;
            for (int r = 1; r < world; ++r)
                if (load[r] < load[best]) best = r;
            owner[u] = best;
            load[best] += cost[u];
        }
        return owner;
    };
    auto exchange = [&](std::vector<double> &buf) -> int {
        if (world == 1 || buf.empty()) return QMC_OK;
        if (ctx->allreduce(ctx->allreduce_user, buf.data(), buf.size()) != 0)
            return fail(ctx, QMC_E_INVAL, "qmc_integrate: the rank exchange failed");
        return QMC_OK;
    };
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
            qmc_job J = job_for(q);
            J.shifts = 2;
            J.n = sizes.empty() ? n0 : sizes.front();
            J.stream = q;
            pre.push_back(J);
            pre_slot.push_back(q);
        }
        if (!pre.empty()) {
            std::vector<double> pc(pre.size());
            for (size_t u = 0; u < pre.size(); ++u) pc[u] = slots[pre_slot[u]].cost;
            const std::vector<int> owner = partition(pc);
            std::vector<qmc_job> mine;
            std::vector<size_t> mine_idx;
            for (size_t u = 0; u < pre.size(); ++u)
                if (owner[u] == rank) {
                    mine.push_back(pre[u]);
                    mine_idx.push_back(u);
                }
            const double pe0 = ctx->presample_evals;
            if (!mine.empty()) {
                const int rc = qmc_presample_lambda(ctx, mine.data(), (int)mine.size(), slo, sn, 1.0, 16);
                if (rc && rc != QMC_E_SIGN_CHECK) return rc;
            }
            std::vector<double> buf(pre.size() + 1, 0.0);
            for (size_t u = 0; u < mine.size(); ++u) buf[mine_idx[u]] = mine[u].lambda[0];
            buf[pre.size()] = ctx->presample_evals - pe0;
            int rc = exchange(buf);
            if (rc) return rc;
            for (size_t u = 0; u < pre.size(); ++u) slots[pre_slot[u]].lambda = buf[u];
            ctx->presample_evals = pe0 + buf[pre.size()];
        }
    }
    double evals = 0.0, kernel_s = 0.0, median_evals = 0.0;
    int iter = 0, rc_final = QMC_OK;
    std::vector<double> tau(slots.size(), 1.0);
    std::vector<double> amp_val((size_t)npts * namp * norders * 2), amp_var((size_t)npts * namp * norders);
    std::vector<double> amp_vre((size_t)npts * namp * norders), amp_vim((size_t)npts * namp * norders);
    // evaluate host jobs (this rank's share): the caller's evaluator or one GPU
    // plan; per-shift sums, per-job sign-check failures, evaluator seconds per
    // class (slot QMC_NCLASS: one figure for all classes, from an evaluator
    // that is not timed per class)
    auto eval_jobs = [&](const std::vector<qmc_job> &jobs, std::vector<double> &out, std::vector<uint32_t> &fails,
                         std::vector<double> &cls_s) -> int {
        out.assign(jobs.size() * (size_t)m * sn * 2, 0.0);
        fails.assign(jobs.size(), 0);
        cls_s.assign(QMC_NCLASS + 1, 0.0);
        if (jobs.empty()) return QMC_OK;
        if (ctx->eval_hook) {
            const auto t0 = clk::now();
            int rc = ctx->eval_hook(ctx->eval_user, jobs.data(), (int)jobs.size(), slo, sn, out.data(), fails.data());
            cls_s[QMC_NCLASS] = std::chrono::duration<double>(clk::now() - t0).count();
            if (rc && rc != QMC_E_SIGN_CHECK) return fail(ctx, rc, "qmc_integrate: the evaluator failed (%d)", rc);
            if (rc != QMC_E_SIGN_CHECK) std::fill(fails.begin(), fails.end(), 0u);
            for (const qmc_job &J : jobs) ctx->stat_evals += (double)J.n * J.shifts;
            return QMC_OK;
        }
        qmc_plan *plan = nullptr;
        int rc = qmc_plan_create(ctx, jobs.data(), (int)jobs.size(), slo, sn, &plan);
        if (rc) return rc;
        rc = qmc_plan_run(plan, nullptr, nullptr);
        uint64_t sf = 0;
        if (!rc) rc = qmc_plan_results(plan, out.data(), &sf);
        if (rc && rc != QMC_E_SIGN_CHECK) {
            qmc_plan_destroy(plan);
            return rc;
        }
        if (rc == QMC_E_SIGN_CHECK) {
            rc = qmc_plan_job_failures(plan, fails.data());
            if (rc) {
                qmc_plan_destroy(plan);
                return rc;
            }
        }
        for (size_t c = 0; c < plan->launches.size(); ++c) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, plan->kev[2 * c], plan->kev[2 * c + 1]);
            cls_s[plan->launches[c].cls] += ms * 1e-3;
        }
        qmc_plan_destroy(plan);
        return QMC_OK;
    };
    auto eff_class = [&](const qmc_job &J) {
        const QmcHostSector &S = ctx->integrals[J.integral_id].sectors[J.sector];
        return ctx->opt.precision == QMC_PRECISION_MIXED && !(J.flags & QMC_JOB_FP64) ? qmc_class_mixed(S.cls)
                                                                                         : S.cls;
    };
    // median rules: for every slot in `todo` choose the generating vector of its
    // lattice as the median of r unshifted candidate rules (Eq. (median))
    auto choose_median = [&](const std::vector<size_t> &todo) -> int {
        if (todo.empty()) return QMC_OK;
        std::vector<double> cost(todo.size());
        for (size_t u = 0; u < todo.size(); ++u) cost[u] = (double)slots[todo[u]].n * slots[todo[u]].cost;
        const std::vector<int> owner = partition(cost);
        std::vector<qmc_job> jobs;
        std::vector<size_t> mine;
        std::vector<uint32_t> cand;
        for (size_t u = 0; u < todo.size(); ++u) {
            if (owner[u] != rank) continue;
            const size_t q = todo[u];
            const Slot &sl = slots[q];
            const int d = ctx->integrals[ids[sl.i]].sectors[sl.s].d;
            std::vector<uint32_t> zc((size_t)rcand * 6);
            const uint64_t seed = ctx->opt.seed ^ mix64(((uint64_t)q << 32) ^ sl.n);
            if (qmc_median_candidates(sl.n, d, rcand, seed, zc.data()))
                return fail(ctx, QMC_E_INVAL, "qmc_integrate: no median candidates for n=%llu",
                            (unsigned long long)sl.n);
            for (int c = 0; c < rcand; ++c) {
                qmc_job J = job_for(q);
                J.shifts = 1;
                J.n = sl.n;
                J.stream = q;
                J.flags = QMC_JOB_UNSHIFTED | (sl.fp64 ? QMC_JOB_FP64 : 0);
                for (int j = 0; j < 6; ++j) {
                    J.lambda[j] = sl.lambda;
                    J.z[j] = zc[(size_t)c * 6 + j];
                }
                jobs.push_back(J);
            }
            mine.push_back(u);
            cand.insert(cand.end(), zc.begin(), zc.end());
        }
        // the candidates' estimates in one evaluation (one unshifted rule each)
        std::vector<double> est;
        if (!jobs.empty()) {
            est.assign(jobs.size() * (size_t)sn * 2, 0.0);
            if (ctx->eval_hook) {
                std::vector<uint32_t> fails(jobs.size(), 0);
                int rc = ctx->eval_hook(ctx->eval_user, jobs.data(), (int)jobs.size(), slo, sn, est.data(),
                                        fails.data());
                for (const qmc_job &J : jobs) ctx->stat_evals += (double)J.n;
                if (rc && rc != QMC_E_SIGN_CHECK) return fail(ctx, rc, "qmc_integrate: the evaluator failed (%d)", rc);
            } else {
                qmc_plan *plan = nullptr;
                int rc = qmc_plan_create(ctx, jobs.data(), (int)jobs.size(), slo, sn, &plan);
                if (rc) return rc;
                rc = qmc_plan_run(plan, nullptr, nullptr);
                if (!rc) rc = qmc_plan_results(plan, est.data(), nullptr);
                qmc_plan_destroy(plan);
                if (rc && rc != QMC_E_SIGN_CHECK && rc != QMC_E_NONFINITE) return rc;
            }
        }
        std::vector<double> buf(todo.size() * 6 + 1, 0.0);
        double mev = 0.0;
        for (size_t v = 0; v < mine.size(); ++v) {
            // the candidate whose estimate (Re of the highest sector order) is the median; ties keep the lower index
            std::vector<int> idx(rcand);
            for (int c = 0; c < rcand; ++c) idx[c] = c;
            const double *e = &est[v * (size_t)rcand * sn * 2];
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
                return e[(size_t)a * sn * 2 + 2 * (sn - 1)] < e[(size_t)b * sn * 2 + 2 * (sn - 1)];
            });
            const int med = idx[rcand / 2];
            for (int j = 0; j < 6; ++j) buf[mine[v] * 6 + j] = (double)cand[(v * rcand + med) * 6 + j];
            mev += (double)slots[todo[mine[v]]].n * rcand;
        }
        buf[todo.size() * 6] = mev;
        int rc = exchange(buf);
        if (rc) return rc;
        for (size_t u = 0; u < todo.size(); ++u) {
            Slot &sl = slots[todo[u]];
            for (int j = 0; j < 6; ++j) sl.z[j] = (uint32_t)buf[u * 6 + j];
            sl.zn = sl.n;
        }
        median_evals += buf[todo.size() * 6];
        return QMC_OK;
    };
    // one adaptive run over the slots [q0, q1) of the points [p0, p1)
    auto run = [&](size_t q0, size_t q1, int p0, int p1) -> int {
        std::vector<size_t> resample;   // slots to presample again after a sign-check failure
        int resample_rounds = 0;
        for (;;) {
            // ---- median vectors for slots whose lattice changed
            if (median) {
                std::vector<size_t> todo;
                for (size_t q = q0; q < q1; ++q)
                    if (slots[q].dirty && slots[q].zn != slots[q].n) todo.push_back(q);
                int rc = choose_median(todo);
                if (rc) return rc;
            }
            // ---- evaluate the dirty slots: each rank its share, in one plan
            std::vector<size_t> dirty;
            for (size_t q = q0; q < q1; ++q)
                if (slots[q].dirty) dirty.push_back(q);
            if (!dirty.empty()) {
                std::vector<double> cost(dirty.size());
                for (size_t u = 0; u < dirty.size(); ++u) cost[u] = (double)slots[dirty[u]].n * slots[dirty[u]].cost;
                const std::vector<int> owner = partition(cost);
                std::vector<qmc_job> jobs;
                std::vector<size_t> mine;
                for (size_t u = 0; u < dirty.size(); ++u) {
                    if (owner[u] != rank) continue;
                    const size_t q = dirty[u];
                    Slot &sl = slots[q];
                    qmc_job J = job_for(q);
                    J.shifts = m;
                    J.n = sl.n;
                    J.stream = ((uint64_t)iter << 40) | q;
                    J.flags = sl.fp64 ? QMC_JOB_FP64 : 0;
                    for (int j = 0; j < 6; ++j) {
                        J.lambda[j] = sl.lambda;
                        J.z[j] = median ? sl.z[j] : 0;
                    }
                    jobs.push_back(J);
                    mine.push_back(u);
                }
                std::vector<double> out, cls_s;
                std::vector<uint32_t> fails;
                int rc = eval_jobs(jobs, out, fails, cls_s);
                if (rc) return rc;
                double own_evals = 0.0;
                for (const qmc_job &J : jobs) own_evals += (double)J.n * J.shifts;
                // exchange: per dirty slot its sums and failure flag, per class the
                // evaluator seconds and the cost-weighted evaluations, the evaluations
                const size_t per = (size_t)m * sn * 2 + 1;
                const size_t cls_off = dirty.size() * per;
                std::vector<double> buf(cls_off + 2 * (QMC_NCLASS + 1) + 1, 0.0);
                for (size_t v = 0; v < mine.size(); ++v) {
                    memcpy(&buf[mine[v] * per], &out[v * (size_t)m * sn * 2], (size_t)m * sn * 2 * sizeof(double));
                    buf[mine[v] * per + per - 1] = fails[v] ? 1.0 : 0.0;
                }
                for (int c = 0; c <= QMC_NCLASS; ++c) buf[cls_off + 2 * c] = cls_s[c];
                for (size_t v = 0; v < jobs.size(); ++v) {
                    const double w = (double)jobs[v].n * m;
                    const int c = cls_s[QMC_NCLASS] > 0 ? QMC_NCLASS : eff_class(jobs[v]);
                    buf[cls_off + 2 * c + 1] += w * slots[dirty[mine[v]]].cost;
                    buf[buf.size() - 1] += w;
                }
                rc = exchange(buf);
                if (rc) return rc;
                for (int c = 0; c <= QMC_NCLASS; ++c) kernel_s += buf[cls_off + 2 * c];
                evals += buf[buf.size() - 1];
                ctx->stat_evals += buf[buf.size() - 1] - own_evals;   // the other ranks' evaluations
                // per-class time per cost unit -> tau of each slot
                for (size_t u = 0; u < dirty.size(); ++u) {
                    const size_t q = dirty[u];
                    Slot &sl = slots[q];
                    qmc_job J = job_for(q);
                    J.flags = sl.fp64 ? QMC_JOB_FP64 : 0;
                    const int c = buf[cls_off + 2 * QMC_NCLASS + 1] > 0 ? QMC_NCLASS : eff_class(J);
                    const double cw = buf[cls_off + 2 * c + 1];
                    const double per_cost = cw > 0 ? buf[cls_off + 2 * c] / cw : 1e-9;
                    tau[q] = std::max(per_cost, 1e-15) * sl.cost;
                    const double *qs = &buf[u * per];
                    qmc_shift_stats(qs, m, sn, sl.mean, sl.var);
                    if (ctx->opt.keep_shift_sums) sl.sums.assign(qs, qs + (size_t)m * sn * 2);
                    sl.have = true;
                    sl.dirty = false;
                    if (qs[per - 1] != 0.0) resample.push_back(q);
                }
            }
            ++iter;
            if (!resample.empty() && ++resample_rounds > 8) {
                rc_final = QMC_E_SIGN_CHECK;   // lambda keeps failing: keep the results, report it
                resample.clear();
            }
            if (!resample.empty()) {
                // a deformed slot whose contour crossed to Im F > 0 on its lattice: presample
                // again below its lambda (candidates below the smallest failing lambda, all
                // failing slots in one search) and evaluate it once more
                std::vector<qmc_job> pre;
                for (size_t q : resample) {
                    qmc_job J = job_for(q);
                    J.stream = ((uint64_t)iter << 40) | q;
                    pre.push_back(J);
                }
                double lmax = 1.0;   // (a failing lambda <= 0 restarts from 1)
                for (size_t q : resample)
                    if (slots[q].lambda > 0) lmax = std::min(lmax, 0.7 * slots[q].lambda);
                std::vector<double> pc(pre.size());
                for (size_t u = 0; u < pre.size(); ++u) pc[u] = slots[resample[u]].cost;
                const std::vector<int> owner = partition(pc);
                std::vector<qmc_job> mine;
                std::vector<size_t> mine_idx;
                for (size_t u = 0; u < pre.size(); ++u)
                    if (owner[u] == rank) {
                        mine.push_back(pre[u]);
                        mine_idx.push_back(u);
                    }
                if (!mine.empty()) {
                    const int prc = qmc_presample_lambda(ctx, mine.data(), (int)mine.size(), slo, sn, lmax, 16);
                    if (prc && prc != QMC_E_SIGN_CHECK) return prc;
                }
                std::vector<double> buf(pre.size(), 0.0);
                for (size_t u = 0; u < mine.size(); ++u) buf[mine_idx[u]] = mine[u].lambda[0];
                int rc = exchange(buf);
                if (rc) return rc;
                for (size_t u = 0; u < resample.size(); ++u) {
                    Slot &sl = slots[resample[u]];
                    sl.lambda = buf[u];   // the largest passing candidate, else the smallest tried
                    sl.dirty = true;
                }
                resample.clear();
                continue;
            }
            // ---- combine into the sums of the points [p0, p1) and check the requested accuracy
            bool all_ok = true;
            const size_t a0 = (size_t)p0 * namp * norders, a1 = (size_t)p1 * namp * norders;
            std::vector<char> sum_ok(a1, 1);
            std::vector<double> target(a1, 0.0);
            std::fill(amp_val.begin() + 2 * a0, amp_val.begin() + 2 * a1, 0.0);
            std::fill(amp_var.begin() + a0, amp_var.begin() + a1, 0.0);
            std::fill(amp_vre.begin() + a0, amp_vre.begin() + a1, 0.0);
            std::fill(amp_vim.begin() + a0, amp_vim.begin() + a1, 0.0);
            for (size_t q = q0; q < q1; ++q) {
                const Slot &sl = slots[q];
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
            for (size_t idx = a0; idx < a1; ++idx) {
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
            if (all_ok) return QMC_OK;
            // the same decision on every rank (the wall clocks differ)
            std::vector<double> tbuf(1, timeout_s > 0 && elapsed > timeout_s ? 1.0 : 0.0);
            int rc = exchange(tbuf);
            if (rc) return rc;
            if (tbuf[0] > 0) {
                rc_final = QMC_E_TIMEOUT;
                return QMC_OK;
            }
            // ---- allocation (Eq. adaptive-solution), one sum at a time, keeping the largest n
            bool grew = false;
            for (int p = p0; p < p1; ++p)
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
                                want = std::max(round_down((double)sl.n * ctx->opt.max_growth),
                                                round_up((double)sl.n + 1));
                            if (want > sl.n) {
                                sl.n = want;
                                sl.dirty = true;
                                grew = true;
                            }
                        }
                    }
            if (!grew) {
                rc_final = QMC_E_NOT_CONVERGED;
                return QMC_OK;
            }
        }
    };
    if (ctx->opt.batched == -1) {
        for (int p = 0; p < npts && rc_final != QMC_E_TIMEOUT; ++p) {
            const int rc0 = rc_final;
            rc_final = QMC_OK;
            const int rc = run(pbegin[p], pbegin[p + 1], p, p + 1);
            if (rc) return rc;
            if (rc_final == QMC_OK) rc_final = rc0;
        }
    } else {
        const int rc = run(0, slots.size(), 0, npts);
        if (rc) return rc;
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
    // per-integral results of this call (qmc_integral_results, qmc_per_shift_sums)
    ctx->last.clear();
    for (int i = 0; i < nint; ++i) {
        const QmcHostIntegral &I = ctx->integrals[ids[i]];
        QmcLastIntegral &L = ctx->last[ids[i]];
        const int nsec = (int)I.sectors.size();
        L.lowest_order = lowest_order;
        L.norders = norders;
        L.npoints = npts;
        L.value.assign((size_t)npts * norders, qmc_c64{0.0, 0.0});
        L.error.assign((size_t)npts * norders, qmc_c64{0.0, 0.0});
        L.nsectors = nsec;
        L.shifts = m;
        L.sector_lo = slo;
        L.sector_orders = sn;
        L.have_sums = ctx->opt.keep_shift_sums != 0;
        L.n.assign((size_t)npts * nsec, 0);
        if (L.have_sums) L.sums.assign((size_t)npts * nsec * m * sn * 2, 0.0);
        std::vector<double> vre((size_t)npts * norders, 0.0), vim((size_t)npts * norders, 0.0);
        for (size_t q = 0; q < slots.size(); ++q) {
            const Slot &sl = slots[q];
            if (sl.i != i) continue;
            L.n[(size_t)sl.p * nsec + sl.s] = sl.n;
            if (L.have_sums && !sl.sums.empty())
                memcpy(&L.sums[((size_t)sl.p * nsec + sl.s) * m * sn * 2], sl.sums.data(),
                       sl.sums.size() * sizeof(double));
            qmc_c64 mu[8], a[64];
            for (int o = 0; o < sn; ++o) {
                mu[o].re = sl.mean[2 * o];
                mu[o].im = sl.mean[2 * o + 1];
            }
            qmc_series_mul(I.pref.data(), I.pref_lo, (int)I.pref.size(), mu, slo, sn, lowest_order, norders, a);
            for (int o = 0; o < norders; ++o) {
                L.value[(size_t)sl.p * norders + o].re += a[o].re;
                L.value[(size_t)sl.p * norders + o].im += a[o].im;
                for (int so = 0; so < sn; ++so) {
                    const int gi = (lowest_order + o) - (slo + so) - I.pref_lo;
                    if (gi < 0 || gi >= (int)I.pref.size()) continue;
                    const double gr2 = I.pref[gi].re * I.pref[gi].re, gi2 = I.pref[gi].im * I.pref[gi].im;
                    vre[(size_t)sl.p * norders + o] += gr2 * sl.var[2 * so] + gi2 * sl.var[2 * so + 1];
                    vim[(size_t)sl.p * norders + o] += gi2 * sl.var[2 * so] + gr2 * sl.var[2 * so + 1];
                }
            }
        }
        for (size_t u = 0; u < vre.size(); ++u) {
            L.error[u].re = std::sqrt(vre[u]);
            L.error[u].im = std::sqrt(vim[u]);
        }
    }
    const double seconds = std::chrono::duration<double>(clk::now() - t_start).count();
    ctx->stat_seconds += seconds;
    if (info) {
        memset(info, 0, sizeof *info);
        info->evaluations = evals;
        info->seconds = seconds;
        info->kernel_seconds = kernel_s;
        info->iterations = iter;
        uint64_t mx = 0;
        for (const Slot &sl : slots) mx = std::max(mx, sl.n);
        info->max_lattice = mx;
        info->presample_evaluations = ctx->presample_evals - presample_evals0;
        int esc = 0;
        for (const Slot &sl : slots) esc += sl.fp64 ? 1 : 0;
        info->fp64_escalations = esc;
        info->median_evaluations = median_evals;
    }
    if (rc_final == QMC_E_TIMEOUT) return fail(ctx, QMC_E_TIMEOUT, "qmc_integrate: timeout after %d iterations", iter);
    if (rc_final == QMC_E_NOT_CONVERGED)
        return fail(ctx, QMC_E_NOT_CONVERGED, "qmc_integrate: largest lattice reached before the requested accuracy");
    if (rc_final == QMC_E_SIGN_CHECK)
        return fail(ctx, QMC_E_SIGN_CHECK, "qmc_integrate: deformed points had Im F > 0 (lambda too large)");
    return QMC_OK;
}

int qmc_set_coefficients(qmc_ctx *ctx, int namp, const qmc_c64 *C, int npoints, int nint, int lowest_coef_order,
                         int ncoef_orders) {
    if (!ctx) return QMC_E_INVAL;
    if (namp == 0) {
        ctx->coef_namp = 0;
        ctx->coef.clear();
        return QMC_OK;
    }
    if (namp < 0 || !C || npoints < 1 || nint < 1 || ncoef_orders < 1 || ncoef_orders > 32)
        return fail(ctx, QMC_E_INVAL, "qmc_set_coefficients: bad arguments");
    if (nint != (int)ctx->integrals.size())
        return fail(ctx, QMC_E_INVAL, "qmc_set_coefficients: %d integrals given, %zu loaded", nint,
                    ctx->integrals.size());
    const size_t count = (size_t)npoints * namp * nint * ncoef_orders;
    for (size_t u = 0; u < count; ++u)
        if (!std::isfinite(C[u].re) || !std::isfinite(C[u].im))
            return fail(ctx, QMC_E_INVAL, "qmc_set_coefficients: coefficient %zu is not finite", u);
    ctx->coef.assign(C, C + count);
    ctx->coef_namp = namp;
    ctx->coef_npoints = npoints;
    ctx->coef_nint = nint;
    ctx->coef_lo = lowest_coef_order;
    ctx->coef_n = ncoef_orders;
    return QMC_OK;
}

int qmc_integral_results(qmc_ctx *ctx, int integral_id, qmc_c64 *value, qmc_c64 *error) {
    if (!ctx || !value || !error) return fail(ctx, QMC_E_INVAL, "qmc_integral_results: bad arguments");
    auto it = ctx->last.find(integral_id);
    if (it == ctx->last.end())
        return fail(ctx, QMC_E_INVAL, "qmc_integral_results: integral %d took no part in the last qmc_integrate",
                    integral_id);
    std::copy(it->second.value.begin(), it->second.value.end(), value);
    std::copy(it->second.error.begin(), it->second.error.end(), error);
    return QMC_OK;
}

int qmc_per_shift_sums(qmc_ctx *ctx, int integral_id, double *out, size_t cap, qmc_shift_layout *layout,
                       uint64_t *n_out) {
    if (!ctx) return QMC_E_INVAL;
    auto it = ctx->last.find(integral_id);
    if (it == ctx->last.end())
        return fail(ctx, QMC_E_INVAL, "qmc_per_shift_sums: integral %d took no part in the last qmc_integrate",
                    integral_id);
    const QmcLastIntegral &L = it->second;
    if (layout) {
        layout->npoints = L.npoints;
        layout->nsectors = L.nsectors;
        layout->shifts = L.shifts;
        layout->sector_lo = L.sector_lo;
        layout->sector_orders = L.sector_orders;
        layout->count = (size_t)L.npoints * L.nsectors * L.shifts * L.sector_orders * 2;
    }
    if (n_out) std::copy(L.n.begin(), L.n.end(), n_out);
    if (!out) return QMC_OK;
    if (!L.have_sums)
        return fail(ctx, QMC_E_INVAL, "qmc_per_shift_sums: set options.keep_shift_sums before qmc_integrate");
    if (cap < L.sums.size())
        return fail(ctx, QMC_E_INVAL, "qmc_per_shift_sums: %zu doubles needed, %zu given", L.sums.size(), cap);
    std::copy(L.sums.begin(), L.sums.end(), out);
    return QMC_OK;
}

int qmc_stats(qmc_ctx *ctx, double *evaluations, double *seconds) {
    if (!ctx) return QMC_E_INVAL;
    if (evaluations) *evaluations = ctx->stat_evals;
    if (seconds) *seconds = ctx->stat_seconds;
    return QMC_OK;
}

int qmc_set_ranks(qmc_ctx *ctx, int rank, int world, qmc_allreduce_fn allreduce, void *user) {
    if (!ctx || world < 1 || rank < 0 || rank >= world || (world > 1 && !allreduce))
        return fail(ctx, QMC_E_INVAL, "qmc_set_ranks: bad arguments");
    ctx->rank = rank;
    ctx->world = world;
    ctx->allreduce = allreduce;
    ctx->allreduce_user = user;
    return QMC_OK;
}

int qmc_set_evaluator(qmc_ctx *ctx, qmc_eval_fn eval, void *user) {
    if (!ctx) return QMC_E_INVAL;
    ctx->eval_hook = eval;
    ctx->eval_user = user;
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
    const int ppts[6] = {1, 2, 4, 8, 16, 32};
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
