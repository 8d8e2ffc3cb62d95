// Internal layouts shared by the host library (qmc_host.cpp) and the kernels
// (qmc_kernels.cu). Not part of the public C-ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#define QMC_DMAX 6          // integration variables per sector
#define QMC_SMAX 4          // logarithmically singular variables per sector
#define QMC_NCOEF 4         // 1 + up to 3 kinematic invariants per coefficient
#define QMC_EMAX 4          // largest exponent of one variable in one monomial
#define QMC_MAXMONO 160     // monomials per sector (U, F and, if deformed, dF, d2F)
#define QMC_NGROUP (1 << QMC_SMAX)
#define QMC_PMAX 4          // largest p of an endpoint singularity t^{-p + b eps} (Taylor degree p - 1)
#define QMC_JMAX3 16        // Taylor coefficients per subtraction box, d <= 3 class (prod_q p_q)
#define QMC_JMAX6 72        // the same, d <= 6 class (4 x 3 x 3 x 2)
#define QMC_NHESS (QMC_DMAX * (QMC_DMAX + 1) / 2)

// One monomial c(inv) * prod_j t_j^{e_j}; exponents packed 4 bits per variable.
struct QmcMono {
    uint32_t exps;
    uint32_t pad;
    double coef[QMC_NCOEF];   // c_0 + c_1 inv_1 + ...
};

// Per-sector description as the kernels read it. Monomials of U and F are
// sorted by their mask of singular variables (bit q set if the monomial
// contains t_{sing[q]}); group g of U is monomials [gU[g], gU[g+1]) counted
// from monoU. Deformed sectors also carry dF/dt_j and d2F/dt_j dt_k tables.
struct QmcSectorDev {
    int32_t d, ns, nU, nF;
    int32_t deform, u0_int, f0_int, ninv;   // u0_int/f0_int: 1 if the exponent is an integer
    int32_t monoU, monoF, nmono, pad0;      // offsets into the global monomial array; pad0 = max exponent
    int32_t a[QMC_DMAX];
    int32_t sing[QMC_SMAX];                 // variable index of singular slot q
    int32_t regular_mask;                   // bit j: j not singular and (a_j != 0 or b_j != 0)
    int32_t pad1;                           // bit 0: u1, f1 integers with |.| <= QMC_EMAX (one log per
                                            // corner); bit 1: every b_j too (one complex log per corner)
    int32_t bi[QMC_DMAX];                   // b_j, u1, f1 as integers where bit 1 / bit 0 of pad1 is set
    int32_t u1i, f1i;
    int32_t gU[QMC_NGROUP + 1];
    int32_t gF[QMC_NGROUP + 1];
    int32_t dFoff[QMC_DMAX], dFn[QMC_DMAX];   // relative to monoF + nF
    int32_t Hoff[QMC_NHESS], Hn[QMC_NHESS];   // j <= k packed row-major
    double b[QMC_DMAX];
    double u0, u1, f0, f1;
    double weight;                          // constant factor of the sector
};

// One evaluation job: (sector, kinematic point) with its lattice and shifts.
struct QmcJobDev {
    int32_t sector;        // index into the sector table
    int32_t point;         // kinematic point
    int32_t shifts;        // m
    int32_t tiles_per_shift;
    uint64_t n;            // lattice size
    uint64_t tile_begin;   // first global tile of this job
    uint64_t seed_state;   // splitmix64 state for this job's shifts
    uint64_t out_off;      // offset (in doubles) of [shifts][norders][2] in the output
    uint32_t z[QMC_DMAX];  // generating vector
    double inv_n;          // RN(1/n), for the corrected lattice division
    double lambda[QMC_DMAX];
    int32_t flags;         // bit 0: no random shift (Delta = 0)
    int32_t pad2;
};

struct QmcLaunch {
    const QmcSectorDev *sectors;
    const QmcMono *monos;
    const double *kin;     // [npoints][ninv]
    const QmcJobDev *jobs;
    int32_t njobs;
    int32_t ninv;
    int32_t lo;            // lowest eps order written
    int32_t norders;
    uint64_t ntiles;
    uint32_t tile_k;       // points per tile = block * ppt
    int32_t transform;     // 0 korobov3, 1 baker, 2 none
    int32_t prow;          // power-table rows per variable (x^1..x^prow): the launch's largest exponent, 1..4
    double *partials;      // [ntiles][norders][2]
    unsigned long long *queue;   // tile counter (reset by the finish kernel)
    unsigned long long *status;  // [0]: sign-check failures, [1]: non-finite partials
    double *out;           // per-shift sums
    unsigned int *job_fail;      // per-job sign-check failures (class-local job index) or null
};

// Fixed scratch of the no-allocation entry point (qmc_eval_jobs_noalloc).
#define QMC_NOALLOC_BYTES (4u << 20)   // 4 MiB per device
#define QMC_NOALLOC_MAX_JOBS 256

// Kernel classes (compile-time sizes of the evaluator).
enum QmcClass {
    QMC_CLASS_REAL3 = 0,   // real integrand, d <= 3, <= 2 singular variables
    QMC_CLASS_CPLX3 = 1,   // contour-deformed, d <= 3, <= 2 singular variables
    QMC_CLASS_REAL6 = 2,   // real integrand, d <= 6 or > 2 singular variables (up to 4: 16 corners)
    QMC_CLASS_REAL3M = 3,  // REAL3 with FP32 monomial products
    QMC_CLASS_REAL6M = 4,  // REAL6 with FP32 monomial products
    QMC_CLASS_REAL6S = 5,  // former split of REAL6 (<= 2 singular variables); now the REAL6 kernel
    QMC_CLASS_REAL6SM = 6, // its mixed-precision variant (the REAL6M kernel)
    QMC_CLASS_CPLX3M = 7,  // CPLX3 with FP32 monomial products (derivatives of F, U and F at z)
    QMC_CLASS_REAL3H = 8,  // real, d <= 3, <= 2 singular variables, some with a <= -2 (Taylor subtraction)
    QMC_CLASS_REAL6T = 9,  // former split of REAL6 (3 singular variables); now the REAL6 kernel
    QMC_CLASS_REAL6TM = 10,// its mixed-precision variant (the REAL6M kernel)
    QMC_CLASS_REAL6H = 11, // real, d <= 6, <= 4 singular variables, some with a <= -2 (Taylor subtraction)
    QMC_CLASS_CPLX3H = 12, // contour-deformed, d <= 3, <= 2 singular variables, some with a <= -2
    QMC_NCLASS = 13
};

static inline bool qmc_class_big(int cls) {
    return cls == QMC_CLASS_REAL6 || cls == QMC_CLASS_REAL6M || cls == QMC_CLASS_REAL6S || cls == QMC_CLASS_REAL6SM ||
           cls == QMC_CLASS_REAL6T || cls == QMC_CLASS_REAL6TM || cls == QMC_CLASS_REAL6H;
}
// Series length (orders) each class supports: K + ns + 1 <= class_lmax.
static inline int qmc_class_lmax(int cls) { return qmc_class_big(cls) ? 6 : 4; }
static inline int qmc_class_dmax(int cls) { return qmc_class_big(cls) ? 6 : 3; }
static inline int qmc_class_smax(int cls) { return qmc_class_big(cls) ? 4 : 2; }
// The mixed-precision variant of a class.
static inline int qmc_class_mixed(int cls) {
    switch (cls) {
        case QMC_CLASS_REAL3: return QMC_CLASS_REAL3M;
        case QMC_CLASS_REAL6: return QMC_CLASS_REAL6M;
        case QMC_CLASS_REAL6S: return QMC_CLASS_REAL6SM;
        case QMC_CLASS_CPLX3: return QMC_CLASS_CPLX3M;
        case QMC_CLASS_REAL6T: return QMC_CLASS_REAL6TM;
        default: return cls;
    }
}

extern "C" {
// Launch helpers implemented in qmc_kernels.cu (all asynchronous on `stream`).
int qmc_k_launch_eval(int cls, const QmcLaunch *L, int block, int ppt, int grid, void *stream);
int qmc_k_launch_finish(const QmcLaunch *L, void *stream);
int qmc_k_lattice_points(uint64_t n, const uint32_t *z_dev, int d, const double *delta_dev,
                         uint64_t k0, uint64_t count, double *x_dev, uint64_t *r_dev, void *stream);
int qmc_k_fp64_probe(double *out_dev, int iters, int grid, int block, void *stream);
int qmc_k_fp32_probe(float *out_dev, int iters, int grid, int block, void *stream);
int qmc_k_sm_count(int device);
int qmc_k_occupancy(int cls, int block, int prow);
size_t qmc_k_noalloc_partial_capacity(void);
int qmc_k_noalloc_setup(int device, void **ptr);
int qmc_k_noalloc_eval(int device, int cls, const QmcJobDev *jobs_host, int njobs, const QmcLaunch *tmpl,
                       int block, int ppt, int sm_count, unsigned long long *status_host, void *stream);
}
