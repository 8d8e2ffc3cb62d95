// Host-side state of the C-ABI shared by qmc_host.cpp and qmc_integrate.cpp.
// Not part of the public C-ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/qmc.h"
#include "qmc_internal.h"

constexpr uint64_t kQmcGamma = 0x9E3779B97F4A7C15ULL;

struct QmcTerm {
    int e[QMC_DMAX];
    double c[QMC_NCOEF];
};

struct QmcHostSector {
    int d = 0;
    bool deform = false;
    int a[QMC_DMAX] = {0};
    double b[QMC_DMAX] = {0};
    double u0 = 0, u1 = 0, f0 = 0, f1 = 0;
    std::vector<QmcTerm> U, F;
    int ns = 0;
    int cls = 0;
    int global_index = 0;  // index in the device sector table
    int prow = 4;          // largest exponent of one variable (monomials and t^{a_j}): power-table rows
    double weight = 1.0;   // constant factor of the sector (geometric decomposition: |det N|)
};

struct QmcHostIntegral {
    std::string name;
    int L = 0, N = 0, D0 = 0;
    std::vector<std::string> invariants;
    int pref_lo = 0;
    std::vector<qmc_c64> pref;
    std::vector<QmcHostSector> sectors;
    int max_poles = 0;
};

struct qmc_plan;

// What the last qmc_integrate call left for one integral.
struct QmcLastIntegral {
    int lowest_order = 0, norders = 0, npoints = 0;
    std::vector<qmc_c64> value, error;   // [npoints][norders], prefactor included
    int nsectors = 0, shifts = 0, sector_lo = 0, sector_orders = 0;
    bool have_sums = false;
    std::vector<double> sums;            // [npoints][nsectors][shifts][sector_orders][2]
    std::vector<uint64_t> n;             // [npoints][nsectors] final lattice sizes
};

struct qmc_ctx {
    int device = 0;
    qmc_options opt{};
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    std::map<uint64_t, std::vector<uint32_t>> lattices;
    std::vector<QmcHostIntegral> integrals;
    // device tables (rebuilt when an integral is loaded)
    QmcSectorDev *d_sectors = nullptr;
    QmcMono *d_monos = nullptr;
    int nsectors_dev = 0;
    double *d_kin = nullptr;
    int npoints = 0, ninv = 0;
    std::vector<qmc_plan *> plans;
    int tuned_block[QMC_NCLASS] = {};   // autotuned launch shape per kernel class (0 = default)
    int tuned_ppt[QMC_NCLASS] = {};
    double presample_evals = 0.0;       // lattice points x shifts spent in qmc_presample_lambda
    bool host_only = false;             // QMC_DEVICE_NONE: no GPU, caller-supplied evaluator only
    std::vector<double> h_kin;          // host copy of the kinematics [npoints][ninv]
    // coefficients of qmc_set_coefficients: [npoints][namp][nint][ncoef]
    int coef_namp = 0, coef_npoints = 0, coef_nint = 0, coef_lo = 0, coef_n = 0;
    std::vector<qmc_c64> coef;
    std::map<int, QmcLastIntegral> last;   // by integral id, from the last qmc_integrate
    double stat_evals = 0.0, stat_seconds = 0.0;
    int rank = 0, world = 1;            // qmc_set_ranks
    qmc_allreduce_fn allreduce = nullptr;
    void *allreduce_user = nullptr;
    qmc_eval_fn eval_hook = nullptr;    // qmc_set_evaluator
    void *eval_user = nullptr;
};

struct ClassLaunch {
    int cls = 0;
    QmcLaunch L{};
    QmcJobDev *d_jobs = nullptr;
    double *d_partials = nullptr;
    unsigned long long *d_queue = nullptr;
    unsigned int *d_jobfail = nullptr;   // per-job sign-check failures
    std::vector<int> orig;               // caller's index of each class-local job
    int block = 128, ppt = 16, grid = 0;
};

struct qmc_plan {
    qmc_ctx *ctx = nullptr;
    int lo = 0, norders = 0, njobs = 0;
    double evals = 0.0;                  // lattice points x shifts of one run
    size_t out_size = 0;
    double *d_out = nullptr;
    unsigned long long *d_status = nullptr;
    std::vector<ClassLaunch> launches;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> kev;   // [2 * class launch]: around each evaluator kernel
    // class launches after the first run concurrently on side streams, forked
    // from and joined back into the run's stream
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaStream_t last_stream = nullptr;
    double *last_out = nullptr;
    int last_launches = 0;
    bool use_graph = false;              // replay the run as one CUDA graph
    cudaGraphExec_t gexec = nullptr;
    double *graph_out = nullptr;         // output pointer the graph was captured with
};

// Record `fmt` as the context's last error and return `code`.
int qmc_fail(qmc_ctx *ctx, int code, const char *fmt, ...);
