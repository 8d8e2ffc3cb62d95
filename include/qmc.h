/*
 * qmc.h -- C-ABI of the GB300 randomized-lattice QMC integrator for
 * sector-decomposed, eps-expanded Feynman-parameter integrals.
 *
 * What the library computes follows arXiv:2305.19768 (pySecDec 1.6,
 * "Numerical scattering amplitudes with pySecDec"):
 *   - the randomized rank-1 shifted lattice rule of the Disteval integrator
 *     (section "The new Quasi-Monte-Carlo evaluator Disteval"): for each
 *     sector and random shift Delta_s, Q_s = (1/n) sum_{k<n} f(frac(k z/n + Delta_s)),
 *     value = mean over shifts, error = sqrt(var/m);
 *   - the korobov3 transform (timings section), contour deformation with its
 *     Jacobian determinant (number_of_presamples in the usage section), and the
 *     eps-expansion of the sector integrands;
 *   - weighted sums A_k = sum_i C_ki I_i with the variance-driven lattice
 *     allocation of Eq. (adaptive-solution), alpha = 2, minimum lattice 10^4
 *     (section "Adaptive weighted sum evaluation");
 *   - the per-coefficient relative error sqrt(dR^2 + dI^2) / sqrt(R^2 + I^2)
 *     (timings section).
 *
 * Conventions for every entry point:
 *   - Return 0 on success, a negative QMC_E_* code on failure; the message of
 *     the last failure on a context is available from qmc_last_error().
 *   - Input buffers are borrowed for the duration of the call only (copied).
 *     Output buffers are owned by the caller and must hold the stated size.
 *   - Pointers documented as "host" are ordinary host memory (pinned or not);
 *     "device" pointers are CUDA device memory of the context's device.
 *   - A context is used by one host thread at a time. All GPU work of a
 *     context is issued on its own CUDA stream unless a stream is passed.
 *   - Nothing falls back to the CPU: without a usable CUDA device every call
 *     that needs one returns QMC_E_CUDA.
 */
#ifndef QMC_H
#define QMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QMC_OK 0
#define QMC_E_INVAL (-1)          /* bad argument or unsupported sector shape */
#define QMC_E_PARSE (-2)          /* malformed sector description */
#define QMC_E_CUDA (-3)           /* CUDA runtime error (message has the detail) */
#define QMC_E_TIMEOUT (-4)        /* qmc_integrate ran past timeout_s */
#define QMC_E_NOT_CONVERGED (-5)  /* max_points reached before the requested accuracy */
#define QMC_E_SIGN_CHECK (-6)     /* contour deformation put F on the wrong side of the cut */
#define QMC_E_NONFINITE (-7)      /* a partial sum was NaN or Inf */
#define QMC_E_NOMEM (-8)          /* allocation failed */

typedef struct qmc_ctx qmc_ctx;
typedef struct qmc_plan qmc_plan;

typedef struct {
    double re, im;
} qmc_c64;

/* Options of a context. Zero-initialise and set what you need; zero fields
 * take the defaults in brackets, which mirror the paper's call arguments
 * (points = 1e4, number_of_presamples, timeout, lattice_candidates). */
typedef struct {
    int shifts;            /* m random shifts per lattice [32] */
    uint64_t seed;         /* seed of the shift streams [1] */
    int block;             /* threads per block of the evaluator, 128 or 256 [autotuned] */
    int ppt;               /* lattice points per thread [autotuned] */
    uint64_t min_points;   /* smallest lattice (pilot pass) [10000] */
    uint64_t max_points;   /* largest lattice qmc_integrate may use [largest tabulated] */
    int presamples;        /* points per lambda candidate in the deformation presampling [10000] */
    double lambda;         /* deformation parameter of qmc_integrate for deformed sectors; 0 = choose
                              per (point, sector) by presampling (qmc_presample_lambda,
                              lambda_max 1, 16 candidates) [0] */
    int precision;         /* QMC_PRECISION_FP64 [default] or QMC_PRECISION_MIXED */
    int transform;         /* QMC_TRANSFORM_KOROBOV3 [default], _BAKER or _NONE */
    int target_mode;       /* QMC_TARGET_COEFFICIENT [default] or QMC_TARGET_AMPLITUDE */
    int max_growth;        /* largest factor by which one pass of qmc_integrate may enlarge a
                              sector's lattice (the next pass re-measures before growing
                              further); 0 = no limit, the allocation rule alone [0] */
    int lattice;           /* QMC_LATTICE_CBC [default]: the installed table of generating
                              vectors; QMC_LATTICE_MEDIAN: median QMC rules in qmc_integrate */
    int lattice_candidates;/* r of the median rule (odd); r > 0 selects median rules as in the
                              paper's lattice_candidates option [0 = CBC; 11 with QMC_LATTICE_MEDIAN] */
    int batched;           /* qmc_integrate: -1 = one kinematic point at a time (the unbatched
                              method); 0 or 1 = all points in one adaptive run [default] */
    int keep_shift_sums;   /* qmc_integrate keeps every slot's last per-shift sums for
                              qmc_per_shift_sums [0 = no] */
    int reserved[4];
} qmc_options;

/* Generating vectors of qmc_integrate (section "Median Quasi-Monte Carlo
 * rules"). CBC: the installed table, lattice sizes rounded up to tabulated
 * sizes. MEDIAN: lattice sizes are any prime (rounded up to the next prime),
 * and for every (kinematic point, sector) and size the generating vector is
 * the median of r candidates drawn from U_n (Eq. (median); qmc_median_lattice),
 * which costs r extra unshifted evaluations of the sector on that lattice. */
#define QMC_LATTICE_CBC 0
#define QMC_LATTICE_MEDIAN 1

/* Device argument of qmc_create for a host-only context: no GPU is used and
 * every call that would need one returns QMC_E_CUDA; qmc_integrate then
 * evaluates through an evaluator installed with qmc_set_evaluator. */
#define QMC_DEVICE_NONE (-1)

/* What epsrel refers to in qmc_integrate. COEFFICIENT: each eps coefficient
 * A^(o) separately, sqrt(dR^2 + dI^2) <= epsrel |A^(o)| (the paper's
 * definition, timings section). AMPLITUDE: every coefficient of an amplitude
 * at a point against the amplitude's largest coefficient there,
 * sqrt(dR^2 + dI^2) <= epsrel max_o |A^(o)| (reachable where one coefficient
 * passes through zero). */
#define QMC_TARGET_COEFFICIENT 0
#define QMC_TARGET_AMPLITUDE 1

/* Periodizing transforms (timings section: korobov3 by default, baker for
 * some examples): korobov3 t = u^4 (35 - 84u + 70u^2 - 20u^3) with weight
 * 140 u^3 (1-u)^3; baker t = 1 - |2u - 1| with weight 1; none t = u. */
#define QMC_TRANSFORM_KOROBOV3 0
#define QMC_TRANSFORM_BAKER 1
#define QMC_TRANSFORM_NONE 2

/* Arithmetic of the evaluator. FP64: everything in FP64. MIXED: the
 * monomial products of U and F and their group sums in FP32 (for deformed
 * sectors also the first and second derivatives of F at the real point and
 * U and F at the complex point z); the korobov3 weight, the deformation
 * matrix and det J, logs and powers of U and F, the series assembly and all
 * reductions in FP64. */
#define QMC_PRECISION_FP64 0
#define QMC_PRECISION_MIXED 1

/* One evaluation job: one sector of one loaded integral at one kinematic
 * point, on one lattice, with `shifts` random shifts. */
typedef struct {
    int32_t integral_id;   /* from qmc_load_sectors_mem */
    int32_t sector;        /* sector index within the integral */
    int32_t point;         /* kinematic point index (qmc_set_kinematics) */
    int32_t shifts;        /* m >= 1 */
    uint64_t n;            /* lattice size; must be in the lattice table */
    uint64_t seed;         /* shift seed */
    uint64_t stream;       /* shift stream id: Delta[s][j] is output s*d+j of
                              splitmix64 started at seed ^ (0x9E3779B97F4A7C15 * (stream + 1)),
                              as (out >> 11) * 2^-53 */
    double lambda[6];      /* deformation parameter per variable (deformed sectors) */
    uint32_t z[6];         /* explicit generating vector, each z_j in U_n (z[0] = 0: the table's) */
    int32_t flags;         /* QMC_JOB_UNSHIFTED: evaluate the unshifted rule (Delta = 0);
                              QMC_JOB_FP64: FP64 arithmetic even in a mixed-precision context */
    int32_t pad;
} qmc_job;

#define QMC_JOB_UNSHIFTED 1
#define QMC_JOB_FP64 2

/* Create a context on CUDA device `device` (or a host-only context with
 * QMC_DEVICE_NONE). `opt` may be NULL (defaults). On success *out owns all
 * device memory the context allocates; free with qmc_destroy.
 * Errors: QMC_E_CUDA (no device), QMC_E_NOMEM, QMC_E_INVAL (options). */
int qmc_create(qmc_ctx **out, int device, const qmc_options *opt);

/* Destroy a context and everything it owns (plans included). NULL is a no-op. */
void qmc_destroy(qmc_ctx *ctx);

/* Message of the last failure on this context ("" if none). The string is
 * owned by the context and valid until the next call on it. */
const char *qmc_last_error(const qmc_ctx *ctx);

/* Install the table of rank-1 lattices: count rows of (n[i], z[i][0..5]),
 * host buffers. Generating vectors are an input: the paper uses
 * pre-computed component-by-component vectors (section on median QMC
 * rules). n must be < 2^32 and every z component coprime to n.
 * Errors: QMC_E_INVAL. */
int qmc_set_lattices(qmc_ctx *ctx, const uint64_t *n, const uint32_t *z, int count);

/* Parse one integral's sector description (text, `len` bytes, host) and
 * upload its monomial tables to the device. The format (one integral: name,
 * loop and propagator counts, D0, invariant names, prefactor Laurent series,
 * then per sector the dimension, deformation flag, monomial prefactor
 * exponents a_j + b_j eps, and the monomial tables of U^{u0+u1 eps} and
 * F^{f0+f1 eps}) is the one written by the Python input generators. Sector
 * limits: d <= 6, at most 4 singular variables (a_j <= -1), a_j >= -4,
 * exponents <= 4 per variable, <= 3 invariants; deformed sectors d <= 3 with
 * at most 2 singular variables. A variable with
 * a_j = -p, p >= 2, takes the Taylor subtraction of degree p - 1 (the
 * integrand gains the boundary terms g_k / (k - p + 1 + b_j eps), k < p, of
 * int_0^1 t^{-p + b_j eps} g(t) dt); prod_j p_j over the singular variables
 * must stay <= 16 (d <= 3, <= 2 singular variables, and every deformed
 * sector) or <= 72 (otherwise).
 * Sectors with d <= 3 and <= 2 singular variables run in the compact
 * evaluators (series of <= 4 eps orders, i.e. highest requested order +
 * singular variables + 1 <= 4), the others in the d <= 6 evaluators (<= 6).
 * *integral_id receives the new id.
 * Errors: QMC_E_PARSE, QMC_E_INVAL (limits), QMC_E_CUDA. */
int qmc_load_sectors_mem(qmc_ctx *ctx, const char *text, size_t len, int *integral_id);

/* Same as qmc_load_sectors_mem, reading the description from a file. */
int qmc_load_sectors(qmc_ctx *ctx, const char *path, int *integral_id);

/* Sector count, maximal number of singular variables and prefactor series
 * (lowest order and up to `cap` complex coefficients) of a loaded integral.
 * Any output pointer may be NULL. */
int qmc_integral_info(qmc_ctx *ctx, int integral_id, int *nsectors, int *max_poles,
                      int *prefactor_lo, qmc_c64 *prefactor, int cap, int *prefactor_len);

/* Set the kinematic points: inv is a host array [npoints][ninv] of the
 * invariants in the order of the sector description. Replaces earlier points.
 * Errors: QMC_E_INVAL, QMC_E_CUDA. */
int qmc_set_kinematics(qmc_ctx *ctx, const double *inv, int npoints, int ninv);

/* Build an evaluation plan for `njobs` jobs (host array): uploads the job
 * table, sizes the tile queue and partial-sum scratch, and picks the kernel
 * class of every job. Each job yields per-shift estimates of the eps orders
 * lo .. lo+norders-1 of its sector integral (orders below the sector's
 * leading pole are 0). *out owns its device buffers; destroy with
 * qmc_plan_destroy (or with the context). Errors: QMC_E_INVAL, QMC_E_CUDA. */
int qmc_plan_create(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders,
                    qmc_plan **out);

/* Number of doubles the plan writes: sum over jobs of shifts * norders * 2. */
size_t qmc_plan_output_size(const qmc_plan *plan);

/* Enqueue one evaluation of the plan on `stream` (a cudaStream_t; NULL =
 * the context's stream) writing per-shift sums to `out_dev` (device, layout
 * [job][shift][order][re, im], qmc_plan_output_size doubles; NULL = the
 * plan's own buffer). Asynchronous: returns after the launches are queued.
 * Errors: QMC_E_CUDA. */
int qmc_plan_run(qmc_plan *plan, double *out_dev, void *stream);

/* Wait for the plan's last run, then copy its per-shift sums to the host
 * buffer `out` (same layout as qmc_plan_run), and check the device status:
 * QMC_E_NONFINITE if a partial sum was NaN/Inf, QMC_E_SIGN_CHECK if a
 * deformed point had Im F > 0 (the sums are still written).
 * `sign_failures` (may be NULL) receives the count of such points. */
int qmc_plan_results(qmc_plan *plan, double *out, uint64_t *sign_failures);

/* Device time of the plan's last run measured with CUDA events: ms_total for
 * the whole run, ms_eval for the evaluator kernels alone (the span from the
 * first one's start to the last one's end: a plan with several evaluator
 * classes runs them concurrently on side streams forked from and joined back
 * into the run's stream), and the number of kernel launches it issued. Waits
 * for the run to finish. Any output may be NULL. */
int qmc_plan_last_time(qmc_plan *plan, float *ms_total, float *ms_eval, int *launches);

/* Replay the plan's runs as one CUDA graph (enable != 0): the first run
 * after enabling captures the sequence (status reset, per-class evaluator
 * and finishing kernels, timing events) on the run's stream and later runs
 * launch the instantiated graph; a different out_dev recaptures. */
int qmc_plan_use_graph(qmc_plan *plan, int enable);

/* Sign-check failures (deformed points with Im F > 0) of each job of the
 * plan's last run, host array out[njobs] in the caller's job order. Waits. */
int qmc_plan_job_failures(qmc_plan *plan, uint32_t *out);

/* Free a plan. NULL is a no-op. */
void qmc_plan_destroy(qmc_plan *plan);

/* One-shot evaluation through host buffers: plan, run, copy back, free.
 * `out` is a host array of qmc_plan_output_size doubles. */
int qmc_eval_jobs(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders,
                  double *out);

/* The shifted lattice points the evaluator uses (steps "lattice index" and
 * "shifted point"): x[i][j] = frac((k0+i) z_j / n + delta_j) for
 * i < count, as (double)r/(double)n + delta with r = (k z_j) mod n exact,
 * folded once into [0,1). Host buffers: z[d], delta[d], x[count][d],
 * r[count][d] (r may be NULL). Errors: QMC_E_INVAL, QMC_E_CUDA. */
int qmc_lattice_points(qmc_ctx *ctx, uint64_t n, const uint32_t *z, int d,
                       const double *delta, uint64_t k0, uint64_t count, double *x,
                       uint64_t *r);

/* Random shifts the evaluator draws for (seed, stream): Delta[s][j], host
 * array [m][d] (see qmc_job.stream). Computed on the device. */
int qmc_shifts(qmc_ctx *ctx, uint64_t seed, uint64_t stream, int m, int d, double *delta);

/* Choose the contour-deformation parameter of every deformed job by
 * presampling (the paper's number_of_presamples): a decreasing search over
 * lambda_max * 0.7^c, c < ncand (<= 32); round c evaluates candidate c, on
 * the smallest tabulated lattice with >= presamples/2 points and 2 shifts,
 * for the jobs that have not qualified yet, and a job keeps the first
 * candidate with no sample at Im F(z) > 0 and finite estimates (the largest
 * qualifying lambda). Writes jobs[i].lambda[0..5] (host array, in/out);
 * undeformed jobs are untouched. QMC_E_SIGN_CHECK if some job has no
 * qualifying candidate (it gets the smallest one). */
int qmc_presample_lambda(qmc_ctx *ctx, qmc_job *jobs, int njobs, int lo, int norders, double lambda_max,
                         int ncand);

/* Autotune the evaluator's launch shape per kernel class (0: real d <= 3,
 * 1: deformed d <= 3, 2: real d <= 6 with 3 or 4 singular variables, 3 and
 * 4: the mixed-precision variants of 0 and 2, 5: real d <= 6 with at most 2
 * singular variables, 6: its mixed-precision variant, 7: the mixed-precision
 * variant of 1, 8: real d <= 3 with exponents a_j <= -2 (Taylor
 * subtraction), 9: real d <= 6 with 3 singular variables, 10: its
 * mixed-precision variant, 11: real d <= 6 with exponents a_j <= -2, 12:
 * deformed d <= 3 with exponents a_j <= -2; class 2 then holds the d <= 6
 * sectors with 4): on up to 32 of the
 * given jobs per class (at most 8 shifts each) every block size in
 * {128, 256} and points per thread in {1, 2, 4, 8, 16, 32} is timed with CUDA
 * events; the fastest is kept in the context and used by later plans whose
 * options leave block/ppt at 0. best_block/best_ppt (may be NULL) receive
 * QMC_NUM_CLASSES entries (0 = class absent). */
#define QMC_NUM_CLASSES 13
int qmc_autotune(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders, int *best_block,
                 int *best_ppt);

/* Median QMC rule candidates (section "Median Quasi-Monte Carlo rules"):
 * r generating vectors with components uniform in U_n = {1 <= z <= n-1,
 * gcd(z, n) = 1}: component j of candidate i is 1 + (x mod (n-1)) for the
 * next splitmix64 output x (state started at `seed`) that gives a value
 * coprime to n, drawn candidate-major; components d..5 are set to 1.
 * z: host array [r][6]. Pure host arithmetic. */
int qmc_median_candidates(uint64_t n, int d, int r, uint64_t seed, uint32_t *z);

/* Median QMC rule for one job (Eq. (median)): evaluates the unshifted rank-1
 * rule Q_{n,z_i} of the job's sector with each of r (odd) candidates from
 * qmc_median_candidates(job->n, d, r, seed) in one plan and returns in
 * z_out[6] the candidate whose estimate is the median, ranked by the real
 * part of order lo+norders-1 (ties keep the lower candidate index).
 * `estimates` (may be NULL): host [r][norders][2] per-candidate values. The
 * uncertainty then comes from random shifts of this lattice (set job.z). */
int qmc_median_lattice(qmc_ctx *ctx, const qmc_job *job, int lo, int norders, int r, uint64_t seed,
                       uint32_t *z_out, double *estimates);

/* ------------------------------------------------------------------------
 * Combination and allocation (host arithmetic, no GPU needed)
 * ------------------------------------------------------------------------ */

/* Statistics over m random shifts (section "Adaptive weighted sum
 * evaluation": each integral is a normal variable whose variance the m
 * shifts estimate): sums[m][norders][2] -> mean[norders][2] and
 * var[norders][2] = the variance of the mean, (1/(m-1)) sum (Q_s - mean)^2 / m,
 * separately for Re and Im (INFINITY if m = 1). Errors: QMC_E_INVAL. */
int qmc_shift_stats(const double *sums, int m, int norders, double *mean, double *var);

/* Laurent product: out[o] = coefficient of eps^(lo+o) in
 * (sum_i a[i] eps^(a_lo+i)) (sum_j b[j] eps^(b_lo+j)), o < n (complex). */
int qmc_series_mul(const qmc_c64 *a, int a_lo, int na, const qmc_c64 *b, int b_lo, int nb, int lo, int n,
                   qmc_c64 *out);

/* Variance through a fixed Laurent factor: out[o] = sum_{i+j = o'} |c[i]|^2 v[j]
 * with v[j] = var Re + var Im of the eps^(v_lo+j) coefficient (independent
 * shifts per sector, so variances add). */
int qmc_series_var(const qmc_c64 *c, int c_lo, int nc, const double *v, int v_lo, int nv, int lo, int n,
                   double *out);

/* Lattice sizes of Eq. (adaptive-solution): for each of nsums sums k with
 * requested variance V[k] > 0 and weights W[k][i] = |C_ki|^2 w_i (w_i the
 * convergence constant of var(I_i) = w_i / n_i^alpha) minimise
 * sum_i tau_i n_i subject to sum_i W[k][i] n_i^-alpha = V[k]:
 *   lambda = (1/alpha) ((1/V) sum_i (W_i tau_i^alpha)^(1/(alpha+1)))^((alpha+1)/alpha),
 *   n_i = (alpha lambda W_i / tau_i)^(1/(alpha+1)).
 * Several sums are applied in turn and n_out[i] keeps the largest value,
 * at least n_min (the paper's reading of its multiple-sum procedure).
 * Integrals with W[k][i] = 0 do not enter sum k. tau[i] > 0 required. */
int qmc_allocate(const double *W, const double *tau, const double *V, int nsums, int nint, double alpha,
                 double n_min, double *n_out);

/* What qmc_integrate sums: amplitudes A_k = sum_i C_ki I_i over the
 * integrals integral_ids[0..nint-1], with complex Laurent coefficients
 * coef[npoints][namp][nint][ncoef] of orders coef_lo.. (host). coef = NULL
 * means every C_ki = 1. A NULL spec sums all loaded integrals with the
 * coefficients of qmc_set_coefficients, or with C = 1 (namp = 1) if none
 * are set. */
typedef struct {
    const int *integral_ids;
    int nint;
    int namp;
    const qmc_c64 *coef;
    int coef_lo;
    int ncoef;
} qmc_sum_spec;

typedef struct {
    double evaluations;     /* lattice points x shifts evaluated (all ranks) */
    double seconds;         /* wall time of the call */
    double kernel_seconds;  /* device time of the evaluator kernels */
    int iterations;         /* evaluation passes */
    uint64_t max_lattice;   /* largest lattice any sector reached */
    double presample_evaluations;   /* lattice points x shifts of the lambda presampling */
    int fp64_escalations;           /* sectors re-evaluated in FP64 in a mixed-precision context */
    double median_evaluations;      /* lattice points of the median-rule candidate evaluations */
} qmc_integrate_info;

/* Adaptive integration of the sums (section "Adaptive weighted sum
 * evaluation"): every sector at every kinematic point starts on the
 * smallest tabulated lattice >= min_points (the pilot pass) with `shifts`
 * random shifts; each pass evaluates the sectors whose lattice changed,
 * combines prefactor, coefficients and sector means into value and
 * variance per eps order, stops when every requested coefficient has
 * sqrt(dR^2 + dI^2) <= max(epsrel |A|, epsabs), and otherwise re-sizes the
 * lattices with qmc_allocate (alpha = 2, w_i = var_i n_i^2, tau_i from the
 * measured kernel time split by a per-sector cost model), rounding up to
 * tabulated lattices (<= max_points; options.max_growth limits the growth
 * per pass; in a mixed-precision context a sector that would need more than
 * max_points, or has reached it short of its target, is evaluated again in
 * FP64, below the FP32 products' error floor). Deformed sectors use
 * options.lambda, or, when it is 0, a lambda
 * per (point, sector) chosen once by presampling; a sector whose evaluation
 * fails the sign check (a point with Im F > 0) is presampled again with
 * candidates below its lambda and evaluated again (at most 8 such rounds,
 * after which the call returns QMC_E_SIGN_CHECK with the results it has).
 * Outputs (host, caller-owned): value[npoints][namp][norders] for orders
 * lowest_order.., error[..] with re = sigma of Re, im = sigma of Im.
 * Returns QMC_E_TIMEOUT (timeout_s > 0 exceeded), QMC_E_NOT_CONVERGED
 * (largest lattice reached) or QMC_E_SIGN_CHECK with the outputs written. */
int qmc_integrate(qmc_ctx *ctx, const qmc_sum_spec *spec, double epsrel, double epsabs, double timeout_s,
                  int lowest_order, int norders, qmc_c64 *value, qmc_c64 *error, qmc_integrate_info *info);

/* qmc_integrate with control over the start and per-slot outputs. Slots are
 * the (kinematic point, integral, sector) triples in that nesting order.
 * n_init (host [nslots], may be NULL): starting lattice size of every slot,
 * rounded up to a tabulated lattice, replacing the pilot pass (the learned
 * sizing hands its predicted sizes in here). shifts > 1 overrides the
 * context's shift count. w_out (host [nslots], may be NULL) receives each
 * slot's convergence constant w = n^2 sum_orders (var Re + var Im) from its
 * last evaluation (Eq. (varscaling) with alpha = 2), n_out its final lattice
 * size. lambda_io (host [nslots], may be NULL): on input a positive entry
 * fixes the deformation parameter of that (deformed) slot and skips its
 * presampling; on output every deformed slot's lambda (0 for the others).
 * Everything else as qmc_integrate. */
int qmc_integrate_ex(qmc_ctx *ctx, const qmc_sum_spec *spec, double epsrel, double epsabs, double timeout_s,
                     int lowest_order, int norders, qmc_c64 *value, qmc_c64 *error, qmc_integrate_info *info,
                     const uint64_t *n_init, int shifts, double *w_out, uint64_t *n_out, double *lambda_io);

/* Coefficients of the weighted sums A_k = sum_i C_ki I_i that qmc_integrate
 * forms when it is given no qmc_sum_spec (the paper's problem statement:
 * sums of integrals with coefficient series, section "Adaptive weighted sum
 * evaluation"): C is a host array [npoints][namp][nint][ncoef_orders] of
 * complex Laurent coefficients, orders lowest_coef_order.., over the nint
 * integrals loaded so far, in load order, at the npoints kinematic points of
 * qmc_set_kinematics (copied). namp = 0 clears them (qmc_integrate then sums
 * all loaded integrals with C = 1). Errors: QMC_E_INVAL. */
int qmc_set_coefficients(qmc_ctx *ctx, int namp, const qmc_c64 *C, int npoints, int nint, int lowest_coef_order,
                         int ncoef_orders);

/* Value and error per eps order of one integral from the last qmc_integrate
 * call on this context, prefactor included: host arrays value[npoints][norders]
 * and error[npoints][norders] (re = sigma of Re, im = sigma of Im) for that
 * call's orders lowest_order.. and kinematic points. Errors: QMC_E_INVAL if the
 * integral took no part in the last call. */
int qmc_integral_results(qmc_ctx *ctx, int integral_id, qmc_c64 *value, qmc_c64 *error);

/* Layout of qmc_per_shift_sums. */
typedef struct {
    int npoints, nsectors, shifts;
    int sector_lo, sector_orders;   /* sector eps orders sector_lo .. sector_lo + sector_orders - 1 */
    size_t count;                   /* doubles in the full array */
} qmc_shift_layout;

/* Per-shift sums of one integral's sectors from their last evaluation in the
 * last qmc_integrate call (options.keep_shift_sums must have been set): host
 * array out[npoints][nsectors][shifts][sector_orders][re, im] with cap doubles
 * of room (out may be NULL to query the layout only). `layout` (may be NULL)
 * receives the shape, and each slot's lattice size goes to n_out[npoints][nsectors]
 * (may be NULL). Errors: QMC_E_INVAL (not kept, not integrated, cap too small). */
int qmc_per_shift_sums(qmc_ctx *ctx, int integral_id, double *out, size_t cap, qmc_shift_layout *layout,
                       uint64_t *n_out);

/* Cumulative work of the context: lattice points x shifts evaluated by every
 * plan, one-shot evaluation and integration on it (all ranks' evaluations for
 * rank-partitioned integrations), and the wall-clock seconds spent inside
 * qmc_integrate calls. Either output may be NULL. */
int qmc_stats(qmc_ctx *ctx, double *evaluations, double *seconds);

/* Ranks of a distributed qmc_integrate (section on distributed evaluation:
 * independent integrand evaluations spread over workers). Every rank runs the
 * same qmc_integrate call on its own context with the same tables,
 * kinematics, options and seed. Each pass, the (kinematic point, sector) slots
 * to evaluate are split over the ranks by cost (largest first, each to the
 * least-loaded rank); each rank evaluates its share, then `allreduce` sums a
 * buffer of n doubles in place over all ranks (the per-shift sums, sign-check
 * flags and timings of the pass, zeros where another rank evaluated), so that
 * every rank holds the same statistics and takes the same allocation
 * decisions: the results equal a one-rank call bit for bit. The callback
 * returns 0 on success; it is called the same number of times on every rank.
 * world = 1 (or allreduce = NULL) restores single-rank integration. */
typedef int (*qmc_allreduce_fn)(void *user, double *buf, size_t n);
int qmc_set_ranks(qmc_ctx *ctx, int rank, int world, qmc_allreduce_fn allreduce, void *user);

/* Evaluator of qmc_integrate supplied by the caller: fills out[job][shift]
 * [order][re, im] (the layout of qmc_eval_jobs) for the host job array, and
 * returns 0 (QMC_E_SIGN_CHECK with job_fail[njobs] set nonzero for the jobs
 * with sign-check failures). The library has no CPU
 * evaluator of its own; this exists so that the driver's host logic
 * (allocation, combination, rank partition) runs in a host-only context
 * (QMC_DEVICE_NONE) for tests on machines without a GPU. NULL restores the
 * GPU evaluator. */
typedef int (*qmc_eval_fn)(void *user, const qmc_job *jobs, int njobs, int lo, int norders, double *out,
                           uint32_t *job_fail);
int qmc_set_evaluator(qmc_ctx *ctx, qmc_eval_fn eval, void *user);

/* Evaluation that allocates nothing. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * time they evaluate -- hard real-time loops that must not hit cudaMalloc's
 * implicit device synchronisation, or hosts whose device memory is owned by
 * another allocator with a fixed budget. It computes what qmc_eval_jobs
 * computes for the same jobs (per-shift sums, layout
 * [job][shift][order][re, im]) but writes them to the caller's device buffer
 * `out_dev` (qmc_plan_output_size doubles for the same jobs) and keeps its
 * job table, tile counter, status words and tile partial sums in one fixed
 * 4 MiB array in device memory that every GPU loading this library holds
 * until the process exits. Limits: at most 256 jobs per call, all of one
 * evaluator class (all deformed or all undeformed, d <= 3; the context's
 * precision setting picks the FP64 or the mixed-precision class, as in
 * qmc_plan_create), and at most 520160 doubles of tile partials
 * ((4 MiB - 33024 bytes) / 8), counted as the sum over jobs of
 * shifts * ceil(n / (block * ppt)) * 2 * norders with the launch shape fixed
 * by the options (block 128 unless 256 is set, ppt 16 unless set; the
 * autotuned and small-lattice shapes of qmc_plan_create are not used, so the
 * sums agree with qmc_eval_jobs to rounding, not bit for bit); larger requests
 * are rejected with QMC_E_INVAL and a message, before any GPU work. It never
 * calls cudaMalloc, cudaFree or any allocating library routine. The context
 * (qmc_create, qmc_set_lattices, qmc_load_sectors_mem, qmc_set_kinematics)
 * must be set up beforehand; that set-up does allocate. The first call on a
 * device looks up the array's device address (a one-time set-up with that
 * device current). The call copies its job table from host memory, then
 * blocks until the work on `stream` (NULL = the context's stream) has
 * finished; it must not be captured into a CUDA graph, and a stream that is
 * being captured is refused with QMC_E_INVAL. Every call reuses the same
 * array and clears the counter and status words it needs at zero; calls that
 * overlap on the GPU (other threads, other streams) race on it and give wrong
 * results. Returns QMC_E_NONFINITE / QMC_E_SIGN_CHECK as qmc_plan_results,
 * QMC_E_INVAL also when an integral's invariant count differs from the
 * loaded kinematics. */
int qmc_eval_jobs_noalloc(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders,
                          double *out_dev, void *stream);

/* The evaluator's own natural logarithm applied on the device to n doubles
 * (host arrays x[n] -> out[n]), for verification: Tang's table-driven
 * reduction (ACM TOMS 16, 1990) with a 1025-entry table, evaluated in
 * integer fixed point (a 128-bit sum) and rounded once: within 0.51 ulp of
 * the exact logarithm. Zero gives -inf, +inf gives +inf, a negative x or NaN
 * gives NaN, subnormals are accepted. Errors: QMC_E_INVAL for null arrays. */
int qmc_fp64_log(qmc_ctx *ctx, const double *x, size_t n, double *out);

/* The evaluator's korobov3 transform of the d <= 3 integrands (timings
 * section of the paper: the korobov3 periodizing transform) applied on the
 * device to n points u (host arrays u[n] -> out[n][3]): out[i][0] = t =
 * phi(u) = u^4 (35 - 84u + 70u^2 - 20u^3), out[i][1] = 1 - t = phi(1 - u)
 * (with the exact 1 - u), out[i][2] = u (1 - u) (the weight is
 * 140 (u (1 - u))^3 per coordinate). Integer fixed-point products, rounded
 * once: within about 0.53 ulp of the exact values. u = 0 gives (0, 1, 0).
 * Errors: QMC_E_INVAL for null arrays or a u outside {0} and the normal
 * numbers of (0, 1). */
int qmc_korobov3(qmc_ctx *ctx, const double *u, size_t n, double *out);

/* The evaluator's own FP64 reciprocal (two Newton-Raphson steps from the
 * hardware approximation), applied like qmc_fp64_log, for verification:
 * within 1 ulp of the correctly rounded 1/x. Same arguments; QMC_E_INVAL
 * also for a non-positive, subnormal or non-finite x. */
int qmc_fp64_rcp(qmc_ctx *ctx, const double *x, size_t n, double *out);

/* The evaluator's own two-argument arctangent (table-driven reduction by
 * atan(j/64), one division, a degree-7 series; IEEE sign conventions for
 * signed zeros) applied on the device to host arrays y[n], x[n] -> out[n],
 * for verification: within 4 ulp. Errors: QMC_E_INVAL for non-finite
 * input or (0, 0). */
int qmc_fp64_atan2(qmc_ctx *ctx, const double *y, const double *x, size_t n, double *out);

/* Measure the FP64 fused-multiply-add throughput of the device (the
 * roofline denominator of the evaluator): *gflops = 2 * DFMA / s over a
 * dependent-chain-free loop timed with CUDA events. */
int qmc_fp64_peak(qmc_ctx *ctx, double *gflops);

/* The same for FP32 (8 independent FFMA chains per thread): the roofline
 * denominator of the mixed-precision classes' FP32 monomial products. */
int qmc_fp32_peak(qmc_ctx *ctx, double *gflops);

/* ------------------------------------------------------------------------
 * Learned part: tensor-core MLP kernels
 * ------------------------------------------------------------------------ */

/* BF16 GEMM on the tensor cores (TMA-fed tcgen05.mma, FP32 accumulation in
 * tensor memory, split-K over the SMs when the M tiles are few):
 * C[M][N] = sum_k A[M][K] B[N][K] with A, B row-major bf16 (raw 16-bit
 * patterns) and C row-major float, host buffers, current CUDA device.
 * M % 128 == 0, K % 16 == 0, N % 16 == 0 and 16 <= N <= 256.
 * Errors: QMC_E_INVAL (shape), QMC_E_CUDA (launch, or a completion wait
 * that ran out). */
int qmc_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int M, int N, int K);

/* The same GEMM on device buffers (A, B 16-byte aligned), enqueued on
 * `stream` (NULL: the legacy default stream); err_dev (device, one unsigned,
 * caller-zeroed) is incremented by every CTA whose completion wait ran out.
 * Returns at once (no synchronisation). Errors: QMC_E_INVAL (shape,
 * alignment, NULL pointers), QMC_E_CUDA (launch). */
int qmc_gemm_bf16_device(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                         void *stream);

/* qmc_gemm_bf16_device with an explicit limit on the polls of each pipeline
 * wait (TMA stage filled, stage freed by the MMAs, all MMAs complete).
 * qmc_gemm_bf16_device uses 2^26 polls (seconds). A CTA whose wait runs out
 * increments *err_dev, waits with the full limit for the copies and MMAs it
 * has in flight, frees its tensor memory and returns without writing its
 * tile; with wait_limit = 0 every CTA takes that path. This exists to test
 * the timeout path without a hung GPU. Errors as qmc_gemm_bf16_device. */
int qmc_gemm_bf16_device_limit(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                               void *stream, unsigned wait_limit);

/* A multilayer perceptron trained and evaluated on the GPU (the learned
 * sizing/surrogate model): x (nin) -> tanh(W0 x + b0) -> (depth - 1) layers
 * tanh(Wl h + bl) of `width` units -> Wout h + bout (nout). Layer 0 runs on
 * the CUDA cores in FP32; all other layers and all gradient products run on
 * the tensor cores through the BF16 GEMM above (bf16 operands, FP32
 * accumulation); master weights, gradients and Adam moments are FP32.
 * width must be 128 or 256; nin <= 64, nout <= 256, depth 1..16. Weights
 * start uniform in +-1/sqrt(fan_in) from splitmix64(seed), biases 0.
 * Parameters are one flat FP32 vector: for l = 0..depth, W_l [rows][fan_in]
 * row-major then b_l [rows] (rows = width, and nout for l = depth). */
typedef struct qmc_mlp qmc_mlp;
int qmc_mlp_create(qmc_mlp **out, int device, int nin, int width, int depth, int nout, uint64_t seed);
void qmc_mlp_destroy(qmc_mlp *mlp);
int qmc_mlp_num_params(const qmc_mlp *mlp, size_t *n);
/* Copy the FP32 master parameters out of / into the model (host [n]). */
int qmc_mlp_get_params(qmc_mlp *mlp, float *params, size_t n);
int qmc_mlp_set_params(qmc_mlp *mlp, const float *params, size_t n);
/* y[B][nout] = model(x[B][nin]) (host buffers). */
int qmc_mlp_forward(qmc_mlp *mlp, const float *x, int B, float *y);
/* Loss (1/B) sum_b sum_o wt[o] (model(x_b)_o - y_b,o)^2 (wt may be NULL = 1)
 * and its gradient with respect to the parameters (host grad[n], may be NULL). */
int qmc_mlp_grad(qmc_mlp *mlp, const float *x, const float *y, const float *wt, int B, float *loss,
                 float *grad);
/* `steps` full-batch Adam steps (beta 0.9/0.999, eps 1e-8) on the same loss;
 * losses[steps] (may be NULL) receives the loss before each step. */
int qmc_mlp_train(qmc_mlp *mlp, const float *x, const float *y, const float *wt, int B, int steps, float lr,
                  float *losses);

#ifdef __cplusplus
}
#endif
#endif /* QMC_H */
