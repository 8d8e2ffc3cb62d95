// Host side of the C-ABI (include/qmc.h): sector-description parser, packing
// of monomial tables for the kernels, evaluation plans (job tables, tile
// queue, partial-sum scratch), and the adaptive integration driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <vector>

#include "qmc_ctx.h"

extern "C" int qmc_k_shifts(uint64_t state, int m, int d, double *out_dev, void *stream);
extern "C" int qmc_k_log(const double *x_dev, uint64_t n, double *out_dev, void *stream);
extern "C" int qmc_k_rcp(const double *x_dev, uint64_t n, double *out_dev, void *stream);
extern "C" int qmc_k_korobov(const double *x_dev, uint64_t n, double *out_dev, void *stream);
extern "C" int qmc_k_atan2(const double *yx_dev, uint64_t n, double *out_dev, void *stream);
extern "C" int qmc_k_occupancy(int cls, int block, int prow);

namespace {

constexpr uint64_t kGamma = kQmcGamma;
using Term = QmcTerm;
using HostSector = QmcHostSector;
using HostIntegral = QmcHostIntegral;
#define fail qmc_fail

#define CUDA_TRY(ctx, call)                                                                     \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail((ctx), QMC_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                        __FILE__, __LINE__);                                                    \
    } while (0)

// ------------------------------------------------------------------ parsing
struct Tok {
    std::istringstream is;
    bool ok = true;
    explicit Tok(const std::string &s) : is(s) {}
    std::string word() {
        std::string w;
        if (!(is >> w)) ok = false;
        return w;
    }
    bool expect(const char *w) { return word() == w && ok; }
    std::string peek() {
        const auto pos = is.tellg();
        std::string w;
        is >> w;
        is.clear();
        is.seekg(pos);
        return w;
    }
    long long integer() {
        std::string w = word();
        if (!ok) return 0;
        char *end = nullptr;
        long long v = strtoll(w.c_str(), &end, 10);
        if (!end || *end) ok = false;
        return v;
    }
    double real() {
        std::string w = word();
        if (!ok) return 0;
        char *end = nullptr;
        double v = strtod(w.c_str(), &end);
        if (!end || *end) ok = false;
        return v;
    }
};

int parse_integral(qmc_ctx *ctx, const std::string &text, HostIntegral &I) {
    Tok t(text);
    if (!t.expect("qmc-sectors") || t.integer() != 1) return fail(ctx, QMC_E_PARSE, "bad header");
    if (!t.expect("name")) return fail(ctx, QMC_E_PARSE, "expected 'name'");
    I.name = t.word();
    if (!t.expect("loops")) return fail(ctx, QMC_E_PARSE, "expected 'loops'");
    I.L = (int)t.integer();
    if (!t.expect("propagators")) return fail(ctx, QMC_E_PARSE, "expected 'propagators'");
    I.N = (int)t.integer();
    if (!t.expect("dim")) return fail(ctx, QMC_E_PARSE, "expected 'dim'");
    I.D0 = (int)t.integer();
    if (!t.expect("invariants")) return fail(ctx, QMC_E_PARSE, "expected 'invariants'");
    long long k = t.integer();
    if (!t.ok || k < 0 || k > QMC_NCOEF - 1)
        return fail(ctx, QMC_E_INVAL, "invariant count %lld outside 0..%d", k, QMC_NCOEF - 1);
    for (long long i = 0; i < k; ++i) I.invariants.push_back(t.word());
    if (!t.expect("prefactor")) return fail(ctx, QMC_E_PARSE, "expected 'prefactor'");
    I.pref_lo = (int)t.integer();
    long long np = t.integer();
    if (!t.ok || np < 1 || np > 64) return fail(ctx, QMC_E_PARSE, "bad prefactor length");
    for (long long i = 0; i < np; ++i) {
        qmc_c64 c;
        c.re = t.real();
        c.im = t.real();
        I.pref.push_back(c);
    }
    if (!t.expect("nsectors")) return fail(ctx, QMC_E_PARSE, "expected 'nsectors'");
    long long ns = t.integer();
    if (!t.ok || ns < 1 || ns > 1000000) return fail(ctx, QMC_E_PARSE, "bad sector count");
    for (long long si = 0; si < ns; ++si) {
        HostSector S;
        if (!t.expect("sector")) return fail(ctx, QMC_E_PARSE, "sector %lld: expected 'sector'", si);
        t.integer();
        if (!t.expect("d")) return fail(ctx, QMC_E_PARSE, "sector %lld: expected 'd'", si);
        S.d = (int)t.integer();
        if (S.d < 1 || S.d > QMC_DMAX)
            return fail(ctx, QMC_E_INVAL, "sector %lld: d=%d outside 1..%d", si, S.d, QMC_DMAX);
        if (!t.expect("deform")) return fail(ctx, QMC_E_PARSE, "sector %lld: expected 'deform'", si);
        S.deform = t.integer() != 0;
        if (t.peek() == "weight") {   // optional constant factor of the sector
            t.word();
            S.weight = t.real();
            if (!(S.weight > 0) || !std::isfinite(S.weight))
                return fail(ctx, QMC_E_PARSE, "sector %lld: weight must be positive", si);
        }
        if (!t.expect("a")) return fail(ctx, QMC_E_PARSE, "sector %lld: expected 'a'", si);
        for (int j = 0; j < S.d; ++j) S.a[j] = (int)t.integer();
        if (!t.expect("b")) return fail(ctx, QMC_E_PARSE, "sector %lld: expected 'b'", si);
        for (int j = 0; j < S.d; ++j) S.b[j] = t.real();
        for (int which = 0; which < 2; ++which) {
            if (!t.expect(which == 0 ? "U" : "F"))
                return fail(ctx, QMC_E_PARSE, "sector %lld: expected '%s'", si, which ? "F" : "U");
            double e0 = t.real(), e1 = t.real();
            long long nt = t.integer();
            if (!t.ok || nt < 1 || nt > QMC_MAXMONO)
                return fail(ctx, QMC_E_INVAL, "sector %lld: term count out of range", si);
            std::vector<Term> &P = which == 0 ? S.U : S.F;
            for (long long m = 0; m < nt; ++m) {
                Term T{};
                for (int j = 0; j < S.d; ++j) T.e[j] = (int)t.integer();
                for (long long i = 0; i <= k; ++i) T.c[i] = t.real();
                P.push_back(T);
            }
            if (which == 0) {
                S.u0 = e0;
                S.u1 = e1;
            } else {
                S.f0 = e0;
                S.f1 = e1;
            }
        }
        if (!t.ok) return fail(ctx, QMC_E_PARSE, "sector %lld: truncated", si);
        I.sectors.push_back(std::move(S));
    }
    if (!t.expect("end")) return fail(ctx, QMC_E_PARSE, "expected 'end'");
    return QMC_OK;
}

// ------------------------------------------------------------------ packing
uint32_t pack_exps(const int *e, int d) {
    uint32_t v = 0;
    for (int j = 0; j < d; ++j) v |= (uint32_t)e[j] << (4 * j);
    return v;
}

int classify(qmc_ctx *ctx, HostSector &S, int si) {
    S.ns = 0;
    int box = 1;   // Taylor coefficients of the full subtraction box, prod_q p_q
    for (int j = 0; j < S.d; ++j) {
        if (S.a[j] < -QMC_PMAX)
            return fail(ctx, QMC_E_INVAL, "sector %d: a_%d=%d needs Taylor subtraction beyond degree %d", si, j,
                        S.a[j], QMC_PMAX - 1);
        if (S.a[j] <= -1) {
            if (S.b[j] == 0.0) return fail(ctx, QMC_E_INVAL, "sector %d: unregulated 1/t_%d", si, j);
            ++S.ns;
            box *= -S.a[j];
        } else if (S.a[j] > QMC_EMAX) {
            return fail(ctx, QMC_E_INVAL, "sector %d: a_%d=%d above %d", si, j, S.a[j], QMC_EMAX);
        }
    }
    if (S.ns > QMC_SMAX) return fail(ctx, QMC_E_INVAL, "sector %d: %d singular variables > %d", si, S.ns, QMC_SMAX);
    if (box > 1) {
        // some a_j <= -2: Taylor subtraction
        if (S.deform) {
            if (S.d > 3 || S.ns > 2 || box > QMC_JMAX3)
                return fail(ctx, QMC_E_INVAL,
                            "sector %d: a deformed sector with a_j <= -2 needs d <= 3, <= 2 singular variables "
                            "and a Taylor box of <= %d coefficients", si, QMC_JMAX3);
            S.cls = QMC_CLASS_CPLX3H;
            return QMC_OK;
        }
        if (S.d <= 3 && S.ns <= 2 && box <= QMC_JMAX3) {
            S.cls = QMC_CLASS_REAL3H;
        } else if (box <= QMC_JMAX6) {
            S.cls = QMC_CLASS_REAL6H;
        } else {
            return fail(ctx, QMC_E_INVAL, "sector %d: subtraction box of %d Taylor coefficients > %d", si, box,
                        QMC_JMAX6);
        }
        return QMC_OK;
    }
    if (S.deform) {
        if (S.d > 3 || S.ns > 2)
            return fail(ctx, QMC_E_INVAL, "sector %d: deformed sectors need d <= 3 and <= 2 singular variables", si);
        S.cls = QMC_CLASS_CPLX3;
    } else if (S.d <= 3 && S.ns <= 2) {
        S.cls = QMC_CLASS_REAL3;
    } else {
        // one d <= 6 evaluator for 0 to 4 singular variables: it dispatches per
        // tile, so all such sectors share one launch
        S.cls = QMC_CLASS_REAL6;
    }
    return QMC_OK;
}

// Pack one sector: header + monomials appended to `monos`.
int pack_sector(qmc_ctx *ctx, const HostSector &S, int si, int ninv, std::vector<QmcMono> &monos,
                QmcSectorDev &H) {
    memset(&H, 0, sizeof H);
    H.d = S.d;
    H.ns = S.ns;
    H.deform = S.deform ? 1 : 0;
    H.weight = S.weight;
    H.ninv = ninv;
    H.u0 = S.u0;
    H.u1 = S.u1;
    H.f0 = S.f0;
    H.f1 = S.f1;
    H.u0_int = (S.u0 == std::floor(S.u0) && std::fabs(S.u0) <= QMC_EMAX) ? 1 : 0;
    H.f0_int = (S.f0 == std::floor(S.f0) && std::fabs(S.f0) <= QMC_EMAX) ? 1 : 0;
    H.pad1 = (S.u1 == std::floor(S.u1) && std::fabs(S.u1) <= QMC_EMAX && S.f1 == std::floor(S.f1) &&
              std::fabs(S.f1) <= QMC_EMAX) ? 1 : 0;
    bool bint = true;
    for (int j = 0; j < S.d; ++j)
        bint = bint && S.b[j] == std::floor(S.b[j]) && std::fabs(S.b[j]) <= QMC_EMAX;
    if (H.pad1 && bint) H.pad1 |= 2;
    if (H.pad1) {
        H.u1i = (int32_t)S.u1;
        H.f1i = (int32_t)S.f1;
    }
    int q = 0;
    for (int j = 0; j < S.d; ++j) {
        H.a[j] = S.a[j];
        H.b[j] = S.b[j];
        if (bint) H.bi[j] = (int32_t)S.b[j];
        if (S.a[j] <= -1) H.sing[q++] = j;
        else if (S.a[j] != 0 || S.b[j] != 0.0) H.regular_mask |= 1 << j;
    }
    int emax = 0;
    auto mask_of = [&](const Term &T) {
        int m = 0;
        for (int qq = 0; qq < S.ns; ++qq)
            if (T.e[H.sing[qq]] > 0) m |= 1 << qq;
        return m;
    };
    std::vector<QmcMono> local;
    auto push = [&](const Term &T) -> int {
        QmcMono M{};
        for (int j = 0; j < S.d; ++j) {
            if (T.e[j] < 0 || T.e[j] > QMC_EMAX)
                return fail(ctx, QMC_E_INVAL, "sector %d: exponent %d outside 0..%d", si, T.e[j], QMC_EMAX);
            emax = std::max(emax, T.e[j]);
        }
        M.exps = pack_exps(T.e, S.d);
        for (int i = 0; i < QMC_NCOEF; ++i) M.coef[i] = T.c[i];
        local.push_back(M);
        return QMC_OK;
    };
    // U and F sorted by singular mask, with group boundaries
    for (int which = 0; which < 2; ++which) {
        const std::vector<Term> &P = which == 0 ? S.U : S.F;
        int32_t *g = which == 0 ? H.gU : H.gF;
        int count = 0;
        for (int grp = 0; grp < QMC_NGROUP; ++grp) {
            g[grp] = count;
            for (const Term &T : P)
                if (mask_of(T) == grp) {
                    int rc = push(T);
                    if (rc) return rc;
                    ++count;
                }
        }
        g[QMC_NGROUP] = count;
        if (which == 0) H.nU = count;
        else H.nF = count;
    }
    // dP/dt_j as a monomial table, merged by exponent
    auto deriv = [&](const std::vector<Term> &P, int j) {
        std::vector<Term> out;
        for (const Term &T : P) {
            if (T.e[j] == 0) continue;
            Term D = T;
            for (int i = 0; i < QMC_NCOEF; ++i) D.c[i] *= T.e[j];
            D.e[j] -= 1;
            bool merged = false;
            for (Term &O : out)
                if (memcmp(O.e, D.e, sizeof D.e) == 0) {
                    for (int i = 0; i < QMC_NCOEF; ++i) O.c[i] += D.c[i];
                    merged = true;
                    break;
                }
            if (!merged) out.push_back(D);
        }
        return out;
    };
    if (S.deform) {
        // dF/dt_j and d2F/dt_j dt_k (j <= k) as monomial tables, merged by exponent
        int base = (int)local.size();
        for (int j = 0; j < S.d; ++j) {
            std::vector<Term> dj = deriv(S.F, j);
            H.dFoff[j] = (int)local.size() - base;
            H.dFn[j] = (int)dj.size();
            for (const Term &T : dj) {
                int rc = push(T);
                if (rc) return rc;
            }
        }
        for (int j = 0; j < S.d; ++j) {
            std::vector<Term> dj = deriv(S.F, j);
            for (int k = j; k < S.d; ++k) {
                std::vector<Term> hk = deriv(dj, k);
                const int h = j * QMC_DMAX - j * (j - 1) / 2 + (k - j);
                H.Hoff[h] = (int)local.size() - base;
                H.Hn[h] = (int)hk.size();
                for (const Term &T : hk) {
                    int rc = push(T);
                    if (rc) return rc;
                }
            }
        }
    }
    if ((int)local.size() > QMC_MAXMONO)
        return fail(ctx, QMC_E_INVAL, "sector %d: %zu monomials > %d", si, local.size(), QMC_MAXMONO);
    H.pad0 = std::max(emax, 1);
    for (int j = 0; j < S.d; ++j)
        if (S.a[j] > 0) H.pad0 = std::max(H.pad0, S.a[j]);
    H.monoU = (int)monos.size();
    H.monoF = H.monoU + H.nU;
    H.nmono = (int)local.size();
    monos.insert(monos.end(), local.begin(), local.end());
    return QMC_OK;
}

int upload_tables(qmc_ctx *ctx) {
    std::vector<QmcSectorDev> secs;
    std::vector<QmcMono> monos;
    for (HostIntegral &I : ctx->integrals) {
        for (size_t si = 0; si < I.sectors.size(); ++si) {
            HostSector &S = I.sectors[si];
            QmcSectorDev H;
            int rc = pack_sector(ctx, S, (int)si, (int)I.invariants.size(), monos, H);
            if (rc) return rc;
            S.global_index = (int)secs.size();
            S.prow = std::min(std::max(H.pad0, 1), QMC_EMAX);
            secs.push_back(H);
        }
    }
    ctx->nsectors_dev = (int)secs.size();
    if (ctx->host_only) return QMC_OK;   // tables checked and indexed, nothing to upload
    cudaFree(ctx->d_sectors);
    cudaFree(ctx->d_monos);
    ctx->d_sectors = nullptr;
    ctx->d_monos = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_sectors, std::max<size_t>(1, secs.size()) * sizeof(QmcSectorDev)));
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_monos, std::max<size_t>(1, monos.size()) * sizeof(QmcMono)));
    CUDA_TRY(ctx, cudaMemcpy(ctx->d_sectors, secs.data(), secs.size() * sizeof(QmcSectorDev),
                             cudaMemcpyHostToDevice));
    CUDA_TRY(ctx, cudaMemcpy(ctx->d_monos, monos.data(), monos.size() * sizeof(QmcMono),
                             cudaMemcpyHostToDevice));
    ctx->nsectors_dev = (int)secs.size();
    return QMC_OK;
}

void free_plan_buffers(qmc_plan *p) {
    for (ClassLaunch &c : p->launches) {
        cudaFree(c.d_jobs);
        cudaFree(c.d_partials);
        cudaFree(c.d_queue);
        cudaFree(c.d_jobfail);
    }
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->launches.clear();
    cudaFree(p->d_out);
    cudaFree(p->d_status);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    for (cudaEvent_t e : p->kev) cudaEventDestroy(e);
    p->kev.clear();
    for (cudaStream_t st : p->side) cudaStreamDestroy(st);
    p->side.clear();
    for (cudaEvent_t e : p->join) cudaEventDestroy(e);
    p->join.clear();
    if (p->fork) cudaEventDestroy(p->fork);
    p->fork = nullptr;
    p->d_out = nullptr;
    p->d_status = nullptr;
}

}  // namespace

// ====================================================================== C-ABI
int qmc_fail(qmc_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

extern "C" {

int qmc_create(qmc_ctx **out, int device, const qmc_options *opt) {
    if (!out) return QMC_E_INVAL;
    *out = nullptr;
    const bool host_only = device == QMC_DEVICE_NONE;
    if (!host_only) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return QMC_E_CUDA;
        if (device < 0 || device >= ndev) return QMC_E_INVAL;
    }
    qmc_ctx *ctx = new (std::nothrow) qmc_ctx();
    if (!ctx) return QMC_E_NOMEM;
    ctx->device = host_only ? 0 : device;
    ctx->host_only = host_only;
    if (opt) ctx->opt = *opt;
    if (ctx->opt.shifts <= 0) ctx->opt.shifts = 32;
    if (ctx->opt.seed == 0) ctx->opt.seed = 1;
    if (ctx->opt.min_points == 0) ctx->opt.min_points = 10000;
    if (ctx->opt.presamples <= 0) ctx->opt.presamples = 10000;
    if (ctx->opt.transform < 0 || ctx->opt.transform > 2 || ctx->opt.lattice < 0 || ctx->opt.lattice > 1 ||
        ctx->opt.lattice_candidates < 0 || (ctx->opt.lattice_candidates > 0 && !(ctx->opt.lattice_candidates & 1)) ||
        ctx->opt.batched < -1 || ctx->opt.batched > 1) {
        delete ctx;
        return QMC_E_INVAL;
    }
    if (ctx->opt.lattice == QMC_LATTICE_MEDIAN && ctx->opt.lattice_candidates == 0) ctx->opt.lattice_candidates = 11;
    if (host_only) {
        *out = ctx;
        return QMC_OK;
    }
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return QMC_E_CUDA;
    }
    ctx->sm_count = qmc_k_sm_count(device);
    *out = ctx;
    return QMC_OK;
}

void qmc_destroy(qmc_ctx *ctx) {
    if (!ctx) return;
    if (ctx->host_only) {
        delete ctx;
        return;
    }
    cudaSetDevice(ctx->device);
    for (qmc_plan *p : ctx->plans) {
        free_plan_buffers(p);
        delete p;
    }
    ctx->plans.clear();
    cudaFree(ctx->d_sectors);
    cudaFree(ctx->d_monos);
    cudaFree(ctx->d_kin);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *qmc_last_error(const qmc_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int qmc_set_lattices(qmc_ctx *ctx, const uint64_t *n, const uint32_t *z, int count) {
    if (!ctx || !n || !z || count <= 0) return fail(ctx, QMC_E_INVAL, "qmc_set_lattices: bad arguments");
    for (int i = 0; i < count; ++i) {
        if (n[i] < 2 || n[i] >= (1ULL << 32)) return fail(ctx, QMC_E_INVAL, "lattice n=%llu outside 2..2^32-1", (unsigned long long)n[i]);
        std::vector<uint32_t> v(z + (size_t)i * 6, z + (size_t)i * 6 + 6);
        for (uint32_t c : v) {
            uint64_t a = c, b = n[i];
            while (b) { uint64_t r = a % b; a = b; b = r; }
            if (c == 0 || c >= n[i] || a != 1)
                return fail(ctx, QMC_E_INVAL, "lattice n=%llu: component %u not in U_n", (unsigned long long)n[i], c);
        }
        ctx->lattices[n[i]] = v;
    }
    return QMC_OK;
}

int qmc_load_sectors_mem(qmc_ctx *ctx, const char *text, size_t len, int *integral_id) {
    if (!ctx || !text) return fail(ctx, QMC_E_INVAL, "qmc_load_sectors_mem: null argument");
    if (!ctx->host_only) cudaSetDevice(ctx->device);
    HostIntegral I;
    int rc = parse_integral(ctx, std::string(text, len), I);
    if (rc) return rc;
    for (size_t si = 0; si < I.sectors.size(); ++si) {
        rc = classify(ctx, I.sectors[si], (int)si);
        if (rc) return rc;
        I.max_poles = std::max(I.max_poles, I.sectors[si].ns);
    }
    ctx->integrals.push_back(std::move(I));
    rc = upload_tables(ctx);
    if (rc) {
        ctx->integrals.pop_back();
        return rc;
    }
    if (integral_id) *integral_id = (int)ctx->integrals.size() - 1;
    return QMC_OK;
}

int qmc_load_sectors(qmc_ctx *ctx, const char *path, int *integral_id) {
    if (!ctx || !path) return fail(ctx, QMC_E_INVAL, "qmc_load_sectors: null argument");
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(ctx, QMC_E_INVAL, "cannot open %s", path);
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    return qmc_load_sectors_mem(ctx, s.data(), s.size(), integral_id);
}

int qmc_integral_info(qmc_ctx *ctx, int integral_id, int *nsectors, int *max_poles, int *prefactor_lo,
                      qmc_c64 *prefactor, int cap, int *prefactor_len) {
    if (!ctx || integral_id < 0 || integral_id >= (int)ctx->integrals.size())
        return fail(ctx, QMC_E_INVAL, "bad integral id");
    const HostIntegral &I = ctx->integrals[integral_id];
    if (nsectors) *nsectors = (int)I.sectors.size();
    if (max_poles) *max_poles = I.max_poles;
    if (prefactor_lo) *prefactor_lo = I.pref_lo;
    if (prefactor_len) *prefactor_len = (int)I.pref.size();
    if (prefactor)
        for (int i = 0; i < cap && i < (int)I.pref.size(); ++i) prefactor[i] = I.pref[i];
    return QMC_OK;
}

int qmc_set_kinematics(qmc_ctx *ctx, const double *inv, int npoints, int ninv) {
    if (!ctx || npoints < 0 || ninv < 0 || ninv > QMC_NCOEF - 1 || (npoints > 0 && ninv > 0 && !inv))
        return fail(ctx, QMC_E_INVAL, "qmc_set_kinematics: bad arguments");
    for (size_t i = 0; i < (size_t)npoints * ninv; ++i)
        if (!std::isfinite(inv[i])) return fail(ctx, QMC_E_INVAL, "non-finite invariant at %zu", i);
    ctx->h_kin.assign(inv, inv + (size_t)npoints * ninv);
    if (ctx->host_only) {
        ctx->npoints = npoints;
        ctx->ninv = ninv;
        return QMC_OK;
    }
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_kin);
    ctx->d_kin = nullptr;
    size_t bytes = std::max<size_t>(1, (size_t)npoints * ninv) * sizeof(double);
    CUDA_TRY(ctx, cudaMalloc(&ctx->d_kin, bytes));
    if (npoints * ninv > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_kin, inv, (size_t)npoints * ninv * sizeof(double),
                                      cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->npoints = npoints;
    ctx->ninv = ninv;
    return QMC_OK;
}

int qmc_plan_create(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders, qmc_plan **out) {
    if (!ctx || !out || (njobs > 0 && !jobs) || njobs < 0 || norders < 1)
        return fail(ctx, QMC_E_INVAL, "qmc_plan_create: bad arguments");
    *out = nullptr;
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_plan_create: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    const int hi = lo + norders - 1;
    std::vector<std::vector<QmcJobDev>> per(QMC_NCLASS);
    std::vector<std::vector<int>> per_orig(QMC_NCLASS);
    uint64_t out_off = 0;
    double evals = 0.0;
    for (int i = 0; i < njobs; ++i) {
        const qmc_job &J = jobs[i];
        if (J.integral_id < 0 || J.integral_id >= (int)ctx->integrals.size())
            return fail(ctx, QMC_E_INVAL, "job %d: bad integral id %d", i, J.integral_id);
        const HostIntegral &I = ctx->integrals[J.integral_id];
        if (J.sector < 0 || J.sector >= (int)I.sectors.size())
            return fail(ctx, QMC_E_INVAL, "job %d: bad sector %d", i, J.sector);
        const HostSector &S = I.sectors[J.sector];
        if (!I.invariants.empty() && (int)I.invariants.size() != ctx->ninv)
            return fail(ctx, QMC_E_INVAL, "job %d: integral has %zu invariants, kinematics %d", i,
                        I.invariants.size(), ctx->ninv);
        if (J.point < 0 || (J.point >= ctx->npoints && !(I.invariants.empty() && J.point == 0)))
            return fail(ctx, QMC_E_INVAL, "job %d: bad kinematic point %d", i, J.point);
        if (J.shifts < 1) return fail(ctx, QMC_E_INVAL, "job %d: shifts < 1", i);
        std::vector<uint32_t> zvec;
        if (J.z[0] != 0) {
            if (J.n < 2 || J.n >= (1ULL << 32)) return fail(ctx, QMC_E_INVAL, "job %d: n outside 2..2^32-1", i);
            for (int j = 0; j < S.d; ++j) {
                uint64_t a = J.z[j], b = J.n;
                while (b) { uint64_t r = a % b; a = b; b = r; }
                if (J.z[j] == 0 || J.z[j] >= J.n || a != 1)
                    return fail(ctx, QMC_E_INVAL, "job %d: z_%d = %u not in U_n", i, j, J.z[j]);
            }
            zvec.assign(J.z, J.z + 6);
        } else {
            auto it = ctx->lattices.find(J.n);
            if (it == ctx->lattices.end())
                return fail(ctx, QMC_E_INVAL, "job %d: lattice n=%llu not in the table", i, (unsigned long long)J.n);
            zvec = it->second;
        }
        const bool mixed = ctx->opt.precision == QMC_PRECISION_MIXED && !(J.flags & QMC_JOB_FP64);
        const int cls = mixed ? qmc_class_mixed(S.cls) : S.cls;
        if (norders > qmc_class_lmax(cls) || hi + S.ns + 1 > qmc_class_lmax(cls))
            return fail(ctx, QMC_E_INVAL, "job %d: orders %d..%d with %d poles exceed the evaluator's series length %d",
                        i, lo, hi, S.ns, qmc_class_lmax(cls));
        QmcJobDev D{};
        D.sector = S.global_index;
        D.point = I.invariants.empty() ? 0 : J.point;
        D.shifts = J.shifts;
        D.n = J.n;
        D.seed_state = J.seed ^ (kGamma * (J.stream + 1));
        D.inv_n = 1.0 / (double)J.n;
        D.out_off = out_off;
        for (int j = 0; j < QMC_DMAX; ++j) {
            D.z[j] = j < S.d ? zvec[j] : 0;
            D.lambda[j] = (S.deform && j < S.d) ? J.lambda[j] : 0.0;
        }
        D.flags = J.flags & QMC_JOB_UNSHIFTED;
        out_off += (uint64_t)J.shifts * norders * 2;
        evals += (double)J.n * J.shifts;
        per[cls].push_back(D);
        per_orig[cls].push_back(i);
    }
    qmc_plan *p = new qmc_plan();
    p->ctx = ctx;
    p->lo = lo;
    p->norders = norders;
    p->njobs = njobs;
    p->out_size = (size_t)out_off;
    p->evals = evals;
    auto bail = [&](int rc) {
        free_plan_buffers(p);
        delete p;
        return rc;
    };
#define PLAN_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return bail(fail(ctx, QMC_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)));        \
    } while (0)
    PLAN_TRY(cudaMalloc(&p->d_out, std::max<size_t>(1, p->out_size) * sizeof(double)));
    PLAN_TRY(cudaMalloc(&p->d_status, 2 * sizeof(unsigned long long)));
    PLAN_TRY(cudaMemset(p->d_status, 0, 2 * sizeof(unsigned long long)));
    PLAN_TRY(cudaEventCreate(&p->ev0));
    PLAN_TRY(cudaEventCreate(&p->ev1));
    for (int cls = 0; cls < QMC_NCLASS; ++cls) {
        std::vector<QmcJobDev> &v = per[cls];
        if (v.empty()) continue;
        // the tile queue hands out tiles in job order: costly jobs first (more
        // singular variables, larger lattices) shortens the tail of the launch,
        // and jobs of one sector shape run side by side on the SMs
        {
            std::vector<int> ord(v.size());
            for (size_t u = 0; u < ord.size(); ++u) ord[u] = (int)u;
            auto key = [&](int u) {
                const qmc_job &J = jobs[per_orig[cls][u]];
                const int ns = ctx->integrals[J.integral_id].sectors[J.sector].ns;
                return std::make_pair(ns, (double)v[u].n * v[u].shifts);
            };
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return key(a) > key(b); });
            std::vector<QmcJobDev> v2;
            std::vector<int> o2;
            for (int u : ord) {
                v2.push_back(v[u]);
                o2.push_back(per_orig[cls][u]);
            }
            v.swap(v2);
            per_orig[cls].swap(o2);
        }
        ClassLaunch c;
        c.cls = cls;
        c.orig = per_orig[cls];
        c.block = ctx->opt.block == 256 ? 256 : (ctx->opt.block == 128 ? 128 : (ctx->tuned_block[cls] ? ctx->tuned_block[cls] : 128));
        if (qmc_class_dmax(cls) > 3) c.block = 128;   // the d <= 6 classes exist with 128-thread blocks only
        c.ppt = ctx->opt.ppt > 0 ? ctx->opt.ppt : (ctx->tuned_ppt[cls] ? ctx->tuned_ppt[cls] : 16);
        if (ctx->opt.ppt <= 0 && !ctx->tuned_ppt[cls]) {
            // small lattices: tiles of 512 points instead of 2048, so that a
            // lattice of a few thousand points does not leave most threads idle
            uint64_t nmax = 0;
            for (const QmcJobDev &D : v) nmax = std::max<uint64_t>(nmax, D.n);
            if (nmax < 16384) c.ppt = 4;
        }
        const uint64_t tile_k = (uint64_t)c.block * c.ppt;
        uint64_t tiles = 0;
        for (QmcJobDev &D : v) {
            D.tiles_per_shift = (int32_t)((D.n + tile_k - 1) / tile_k);
            D.tile_begin = tiles;
            tiles += (uint64_t)D.tiles_per_shift * D.shifts;
        }
        PLAN_TRY(cudaMalloc(&c.d_jobs, v.size() * sizeof(QmcJobDev)));
        PLAN_TRY(cudaMemcpy(c.d_jobs, v.data(), v.size() * sizeof(QmcJobDev), cudaMemcpyHostToDevice));
        PLAN_TRY(cudaMalloc(&c.d_partials, std::max<uint64_t>(1, tiles) * 2 * norders * sizeof(double)));
        PLAN_TRY(cudaMalloc(&c.d_queue, sizeof(unsigned long long)));
        PLAN_TRY(cudaMemset(c.d_queue, 0, sizeof(unsigned long long)));
        PLAN_TRY(cudaMalloc(&c.d_jobfail, v.size() * sizeof(unsigned int)));
        PLAN_TRY(cudaMemset(c.d_jobfail, 0, v.size() * sizeof(unsigned int)));
        // power-table rows: the largest exponent among the launch's sectors
        // (fewer rows, less shared memory per block, more resident blocks)
        int prow = 1;
        for (int u : c.orig) {
            const qmc_job &J = jobs[u];
            prow = std::max(prow, ctx->integrals[J.integral_id].sectors[J.sector].prow);
        }
        int occ = qmc_k_occupancy(cls, c.block, prow);
        if (occ < 1) occ = 1;
        c.grid = (int)std::min<uint64_t>(tiles, (uint64_t)ctx->sm_count * occ);
        if (c.grid < 1) c.grid = 1;
        QmcLaunch &L = c.L;
        L.sectors = ctx->d_sectors;
        L.monos = ctx->d_monos;
        L.kin = ctx->d_kin;
        L.jobs = c.d_jobs;
        L.njobs = (int)v.size();
        L.ninv = ctx->ninv;
        L.lo = lo;
        L.norders = norders;
        L.ntiles = tiles;
        L.tile_k = (uint32_t)tile_k;
        L.transform = ctx->opt.transform;
        L.prow = prow;
        L.partials = c.d_partials;
        L.queue = c.d_queue;
        L.status = p->d_status;
        L.out = p->d_out;
        L.job_fail = c.d_jobfail;
        p->launches.push_back(c);
    }
    // the largest class first: it sets the length of the run, the others fill its tail
    std::stable_sort(p->launches.begin(), p->launches.end(), [](const ClassLaunch &a, const ClassLaunch &b) {
        return a.L.ntiles * a.L.tile_k > b.L.ntiles * b.L.tile_k;
    });
    for (size_t i = 0; i < 2 * p->launches.size(); ++i) {
        cudaEvent_t e;
        PLAN_TRY(cudaEventCreate(&e));
        p->kev.push_back(e);
    }
    if (p->launches.size() > 1) {
        PLAN_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
        for (size_t i = 1; i < p->launches.size(); ++i) {
            cudaStream_t st;
            cudaEvent_t e;
            PLAN_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            p->side.push_back(st);
            PLAN_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            p->join.push_back(e);
        }
    }
#undef PLAN_TRY
    ctx->plans.push_back(p);
    *out = p;
    return QMC_OK;
}

size_t qmc_plan_output_size(const qmc_plan *plan) { return plan ? plan->out_size : 0; }

}  // extern "C"

namespace {
// Enqueue one evaluation of the plan on `st` writing to `out`. While a graph
// is being captured the timing events become external event-record nodes,
// so that the host can still query them after each replay.
int plan_enqueue(qmc_plan *plan, double *out, cudaStream_t st, bool capturing) {
    qmc_ctx *ctx = plan->ctx;
    const unsigned evflags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    CUDA_TRY(ctx, cudaMemsetAsync(plan->d_status, 0, 2 * sizeof(unsigned long long), st));
    CUDA_TRY(ctx, cudaEventRecordWithFlags(plan->ev0, st, evflags));
    if (plan->fork) CUDA_TRY(ctx, cudaEventRecord(plan->fork, st));
    int launches = 0;
    for (size_t i = 0; i < plan->launches.size(); ++i) {
        ClassLaunch &c = plan->launches[i];
        cudaStream_t cs = i == 0 ? st : plan->side[i - 1];
        if (i > 0) CUDA_TRY(ctx, cudaStreamWaitEvent(cs, plan->fork, 0));
        c.L.out = out;
        c.L.kin = ctx->d_kin;
        CUDA_TRY(ctx, cudaMemsetAsync(c.d_jobfail, 0, c.orig.size() * sizeof(unsigned int), cs));
        CUDA_TRY(ctx, cudaEventRecordWithFlags(plan->kev[2 * i], cs, evflags));
        if (c.L.ntiles > 0) {
            if (qmc_k_launch_eval(c.cls, &c.L, c.block, c.ppt, c.grid, cs))
                return fail(ctx, QMC_E_CUDA, "evaluator launch failed: %s", cudaGetErrorString(cudaGetLastError()));
            ++launches;
        }
        CUDA_TRY(ctx, cudaEventRecordWithFlags(plan->kev[2 * i + 1], cs, evflags));
        if (qmc_k_launch_finish(&c.L, cs))
            return fail(ctx, QMC_E_CUDA, "finish launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        ++launches;
        if (i > 0) {
            CUDA_TRY(ctx, cudaEventRecord(plan->join[i - 1], cs));
            CUDA_TRY(ctx, cudaStreamWaitEvent(st, plan->join[i - 1], 0));
        }
    }
    CUDA_TRY(ctx, cudaEventRecordWithFlags(plan->ev1, st, evflags));
    plan->last_launches = launches;
    return QMC_OK;
}
}  // namespace

extern "C" {

int qmc_plan_run(qmc_plan *plan, double *out_dev, void *stream) {
    if (!plan) return QMC_E_INVAL;
    qmc_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    double *out = out_dev ? out_dev : plan->d_out;
    if (plan->use_graph) {
        if (!plan->gexec || plan->graph_out != out) {
            if (plan->gexec) cudaGraphExecDestroy(plan->gexec);
            plan->gexec = nullptr;
            cudaGraph_t g = nullptr;
            CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            int rc = plan_enqueue(plan, out, st, true);
            cudaError_t e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return fail(ctx, QMC_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&plan->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(ctx, QMC_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            plan->graph_out = out;
        }
        CUDA_TRY(ctx, cudaGraphLaunch(plan->gexec, st));
    } else {
        int rc = plan_enqueue(plan, out, st, false);
        if (rc) return rc;
    }
    plan->last_stream = st;
    plan->last_out = out;
    ctx->stat_evals += plan->evals;
    return QMC_OK;
}

int qmc_plan_use_graph(qmc_plan *plan, int enable) {
    if (!plan) return QMC_E_INVAL;
    plan->use_graph = enable != 0;
    if (!plan->use_graph && plan->gexec) {
        cudaGraphExecDestroy(plan->gexec);
        plan->gexec = nullptr;
    }
    return QMC_OK;
}

int qmc_plan_job_failures(qmc_plan *plan, uint32_t *out) {
    if (!plan || !out) return QMC_E_INVAL;
    qmc_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    CUDA_TRY(ctx, cudaStreamSynchronize(plan->last_stream ? plan->last_stream : ctx->stream));
    for (const ClassLaunch &c : plan->launches) {
        std::vector<uint32_t> v(c.orig.size());
        CUDA_TRY(ctx, cudaMemcpy(v.data(), c.d_jobfail, v.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        for (size_t j = 0; j < v.size(); ++j) out[c.orig[j]] = v[j];
    }
    return QMC_OK;
}

int qmc_plan_results(qmc_plan *plan, double *out, uint64_t *sign_failures) {
    if (!plan) return QMC_E_INVAL;
    qmc_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = plan->last_stream ? plan->last_stream : ctx->stream;
    unsigned long long status[2] = {0, 0};
    if (out && plan->out_size)
        CUDA_TRY(ctx, cudaMemcpyAsync(out, plan->last_out ? plan->last_out : plan->d_out,
                                      plan->out_size * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(status, plan->d_status, sizeof status, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (sign_failures) *sign_failures = status[0];
    if (status[1]) return fail(ctx, QMC_E_NONFINITE, "%llu tile partial sums were not finite", status[1]);
    if (status[0]) return fail(ctx, QMC_E_SIGN_CHECK, "%llu deformed points had Im F > 0", status[0]);
    return QMC_OK;
}

int qmc_plan_last_time(qmc_plan *plan, float *ms_total, float *ms_eval, int *launches) {
    if (!plan) return QMC_E_INVAL;
    qmc_ctx *ctx = plan->ctx;
    CUDA_TRY(ctx, cudaEventSynchronize(plan->ev1));
    // the evaluator kernels run concurrently: their time is the span from the
    // earliest start to the latest end
    float t = 0.f, t0 = 1e30f, t1 = 0.f;
    CUDA_TRY(ctx, cudaEventElapsedTime(&t, plan->ev0, plan->ev1));
    for (size_t i = 0; i < plan->launches.size(); ++i) {
        float a = 0.f, b = 0.f;
        CUDA_TRY(ctx, cudaEventElapsedTime(&a, plan->ev0, plan->kev[2 * i]));
        CUDA_TRY(ctx, cudaEventElapsedTime(&b, plan->ev0, plan->kev[2 * i + 1]));
        t0 = std::min(t0, a);
        t1 = std::max(t1, b);
    }
    const float te = plan->launches.empty() ? 0.f : t1 - t0;
    if (ms_total) *ms_total = t;
    if (ms_eval) *ms_eval = te;
    if (launches) *launches = plan->last_launches;
    return QMC_OK;
}

void qmc_plan_destroy(qmc_plan *plan) {
    if (!plan) return;
    qmc_ctx *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(plan->last_stream ? plan->last_stream : ctx->stream);
    free_plan_buffers(plan);
    ctx->plans.erase(std::remove(ctx->plans.begin(), ctx->plans.end(), plan), ctx->plans.end());
    delete plan;
}

int qmc_eval_jobs(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders, double *out) {
    qmc_plan *p = nullptr;
    int rc = qmc_plan_create(ctx, jobs, njobs, lo, norders, &p);
    if (rc) return rc;
    rc = qmc_plan_run(p, nullptr, nullptr);
    if (!rc) rc = qmc_plan_results(p, out, nullptr);
    qmc_plan_destroy(p);
    return rc;
}

int qmc_lattice_points(qmc_ctx *ctx, uint64_t n, const uint32_t *z, int d, const double *delta,
                       uint64_t k0, uint64_t count, double *x, uint64_t *r) {
    if (!ctx || !z || !delta || !x || d < 1 || d > QMC_DMAX || n < 2 || n >= (1ULL << 32))
        return fail(ctx, QMC_E_INVAL, "qmc_lattice_points: bad arguments");
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_lattice_points: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    uint32_t *dz = nullptr;
    double *dd = nullptr, *dx = nullptr;
    uint64_t *dr = nullptr;
    int rc = QMC_OK;
    do {
        if (cudaMalloc(&dz, d * sizeof(uint32_t)) || cudaMalloc(&dd, d * sizeof(double)) ||
            cudaMalloc(&dx, std::max<uint64_t>(1, count) * d * sizeof(double)) ||
            (r && cudaMalloc(&dr, std::max<uint64_t>(1, count) * d * sizeof(uint64_t)))) {
            rc = fail(ctx, QMC_E_CUDA, "qmc_lattice_points: allocation failed");
            break;
        }
        cudaMemcpyAsync(dz, z, d * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(dd, delta, d * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (qmc_k_lattice_points(n, dz, d, dd, k0, count, dx, dr, ctx->stream)) {
            rc = fail(ctx, QMC_E_CUDA, "lattice kernel launch failed");
            break;
        }
        cudaMemcpyAsync(x, dx, count * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (r) cudaMemcpyAsync(r, dr, count * d * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = fail(ctx, QMC_E_CUDA, "qmc_lattice_points: %s", cudaGetErrorString(e));
    } while (0);
    cudaFree(dz);
    cudaFree(dd);
    cudaFree(dx);
    cudaFree(dr);
    return rc;
}

int qmc_shifts(qmc_ctx *ctx, uint64_t seed, uint64_t stream, int m, int d, double *delta) {
    if (!ctx || !delta || m < 1 || d < 1) return fail(ctx, QMC_E_INVAL, "qmc_shifts: bad arguments");
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_shifts: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    double *dd = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&dd, (size_t)m * d * sizeof(double)));
    int rc = qmc_k_shifts(seed ^ (kGamma * (stream + 1)), m, d, dd, ctx->stream);
    if (!rc) {
        cudaMemcpyAsync(delta, dd, (size_t)m * d * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = QMC_E_CUDA;
    } else {
        rc = QMC_E_CUDA;
    }
    cudaFree(dd);
    return rc ? fail(ctx, rc, "qmc_shifts failed") : QMC_OK;
}

// one device function applied elementwise to host data (verification entry points)
// positive_normal: the function's domain is the positive normal doubles
// (others are rejected); otherwise every double is accepted
static int fp64_apply(qmc_ctx *ctx, const double *x, size_t n, double *out, const char *name,
                      int (*launch)(const double *, uint64_t, double *, void *), bool positive_normal,
                      size_t out_per = 1) {
    if (!ctx || (n && (!x || !out))) return fail(ctx, QMC_E_INVAL, "%s: bad arguments", name);
    for (size_t i = 0; positive_normal && i < n; ++i)
        if (!(x[i] >= 2.2250738585072014e-308) || !std::isfinite(x[i]))
            return fail(ctx, QMC_E_INVAL, "%s: x[%zu] is not a positive normal number", name, i);
    if (n == 0) return QMC_OK;
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "%s: host-only context (no GPU)", name);
    cudaSetDevice(ctx->device);
    double *dx = nullptr, *dy = nullptr;
    int rc = QMC_OK;
    if (cudaMalloc(&dx, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dy, n * out_per * sizeof(double)) != cudaSuccess) {
        rc = fail(ctx, QMC_E_CUDA, "%s: allocation failed", name);
    } else {
        cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (launch(dx, n, dy, ctx->stream)) rc = fail(ctx, QMC_E_CUDA, "%s: kernel launch failed", name);
        cudaMemcpyAsync(out, dy, n * out_per * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (!rc && e != cudaSuccess) rc = fail(ctx, QMC_E_CUDA, "%s: %s", name, cudaGetErrorString(e));
    }
    cudaFree(dx);
    cudaFree(dy);
    return rc;
}

int qmc_fp64_log(qmc_ctx *ctx, const double *x, size_t n, double *out) {
    return fp64_apply(ctx, x, n, out, "qmc_fp64_log", qmc_k_log, false);
}

int qmc_fp64_rcp(qmc_ctx *ctx, const double *x, size_t n, double *out) {
    return fp64_apply(ctx, x, n, out, "qmc_fp64_rcp", qmc_k_rcp, true);
}

int qmc_korobov3(qmc_ctx *ctx, const double *u, size_t n, double *out) {
    if (ctx)
        for (size_t i = 0; u && i < n; ++i)
            if (!(u[i] >= 0.0 && u[i] < 1.0) || (u[i] > 0.0 && u[i] < 2.2250738585072014e-308))
                return fail(ctx, QMC_E_INVAL, "qmc_korobov3: u[%zu] is not 0 or a normal number in (0, 1)", i);
    return fp64_apply(ctx, u, n, out, "qmc_korobov3", qmc_k_korobov, false, 3);
}

int qmc_fp64_atan2(qmc_ctx *ctx, const double *y, const double *x, size_t n, double *out) {
    if (!ctx || (n && (!x || !y || !out))) return fail(ctx, QMC_E_INVAL, "qmc_fp64_atan2: bad arguments");
    std::vector<double> yx(2 * n);
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || (x[i] == 0.0 && y[i] == 0.0))
            return fail(ctx, QMC_E_INVAL, "qmc_fp64_atan2: (y, x)[%zu] is not finite or is (0, 0)", i);
        yx[2 * i] = y[i];
        yx[2 * i + 1] = x[i];
    }
    if (n == 0) return QMC_OK;
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_fp64_atan2: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    double *dyx = nullptr, *dout = nullptr;
    int rc = QMC_OK;
    if (cudaMalloc(&dyx, 2 * n * sizeof(double)) != cudaSuccess || cudaMalloc(&dout, n * sizeof(double)) != cudaSuccess) {
        rc = fail(ctx, QMC_E_CUDA, "qmc_fp64_atan2: allocation failed");
    } else {
        cudaMemcpyAsync(dyx, yx.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (qmc_k_atan2(dyx, n, dout, ctx->stream)) rc = fail(ctx, QMC_E_CUDA, "qmc_fp64_atan2: kernel launch failed");
        cudaMemcpyAsync(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (!rc && e != cudaSuccess) rc = fail(ctx, QMC_E_CUDA, "qmc_fp64_atan2: %s", cudaGetErrorString(e));
    }
    cudaFree(dyx);
    cudaFree(dout);
    return rc;
}

int qmc_fp64_peak(qmc_ctx *ctx, double *gflops) {
    if (!ctx || !gflops) return QMC_E_INVAL;
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_fp64_peak: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    double *d = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&d, 2 * sizeof(double)));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int block = 256, grid = ctx->sm_count * 8, iters = 4096;
    qmc_k_fp64_probe(d, 64, grid, block, ctx->stream);  // warm-up
    cudaEventRecord(a, ctx->stream);
    qmc_k_fp64_probe(d, iters, grid, block, ctx->stream);
    cudaEventRecord(b, ctx->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, QMC_E_CUDA, "fp64 probe: %s", cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * iters * (double)grid * block;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return QMC_OK;
}

int qmc_fp32_peak(qmc_ctx *ctx, double *gflops) {
    if (!ctx || !gflops) return QMC_E_INVAL;
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_fp32_peak: host-only context (no GPU)");
    cudaSetDevice(ctx->device);
    float *d = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&d, 2 * sizeof(float)));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int block = 256, grid = ctx->sm_count * 8, iters = 16384;
    qmc_k_fp32_probe(d, 256, grid, block, ctx->stream);  // warm-up
    cudaEventRecord(a, ctx->stream);
    qmc_k_fp32_probe(d, iters, grid, block, ctx->stream);
    cudaEventRecord(b, ctx->stream);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, QMC_E_CUDA, "fp32 probe: %s", cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * iters * (double)grid * block;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return QMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation entry point
extern "C" int qmc_eval_jobs_noalloc(qmc_ctx *ctx, const qmc_job *jobs, int njobs, int lo, int norders,
                                     double *out_dev, void *stream) {
    if (!ctx || !jobs || !out_dev || njobs < 1 || norders < 1)
        return fail(ctx, QMC_E_INVAL, "qmc_eval_jobs_noalloc: bad arguments");
    if (njobs > QMC_NOALLOC_MAX_JOBS)
        return fail(ctx, QMC_E_INVAL, "qmc_eval_jobs_noalloc: %d jobs exceed the fixed limit of %d", njobs,
                    QMC_NOALLOC_MAX_JOBS);
    if (ctx->host_only) return fail(ctx, QMC_E_CUDA, "qmc_eval_jobs_noalloc: host-only context (no GPU)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, QMC_E_CUDA, "cudaSetDevice failed");
    {
        // the call copies from host stack memory and waits for the stream: neither
        // belongs in a graph, so a capturing stream is refused before any work
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStream_t cst = stream ? (cudaStream_t)stream : ctx->stream;
        if (cudaStreamIsCapturing(cst, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return fail(ctx, QMC_E_INVAL, "qmc_eval_jobs_noalloc: the stream is being captured; this call blocks "
                                          "until its work has finished and cannot be captured");
    }
    QmcJobDev recs[QMC_NOALLOC_MAX_JOBS];
    const int block = ctx->opt.block == 256 ? 256 : 128;
    const int ppt = ctx->opt.ppt > 0 ? ctx->opt.ppt : 16;
    const uint64_t tile_k = (uint64_t)block * ppt;
    const int hi = lo + norders - 1;
    int cls = -1;
    uint64_t tiles = 0, out_off = 0;
    for (int i = 0; i < njobs; ++i) {
        const qmc_job &J = jobs[i];
        if (J.integral_id < 0 || J.integral_id >= (int)ctx->integrals.size())
            return fail(ctx, QMC_E_INVAL, "job %d: bad integral id %d", i, J.integral_id);
        const HostIntegral &I = ctx->integrals[J.integral_id];
        if (J.sector < 0 || J.sector >= (int)I.sectors.size())
            return fail(ctx, QMC_E_INVAL, "job %d: bad sector %d", i, J.sector);
        const HostSector &S = I.sectors[J.sector];
        if (!I.invariants.empty() && (int)I.invariants.size() != ctx->ninv)
            return fail(ctx, QMC_E_INVAL, "job %d: integral has %zu invariants, kinematics %d", i,
                        I.invariants.size(), ctx->ninv);
        if (J.point < 0 || (J.point >= ctx->npoints && !(I.invariants.empty() && J.point == 0)))
            return fail(ctx, QMC_E_INVAL, "job %d: bad kinematic point %d", i, J.point);
        if (J.shifts < 1) return fail(ctx, QMC_E_INVAL, "job %d: shifts < 1", i);
        if (J.z[0] != 0 || J.flags)
            return fail(ctx, QMC_E_INVAL, "job %d: explicit generating vectors and job flags need qmc_eval_jobs", i);
        auto it = ctx->lattices.find(J.n);
        if (it == ctx->lattices.end())
            return fail(ctx, QMC_E_INVAL, "job %d: lattice n=%llu not in the table", i, (unsigned long long)J.n);
        // the context's precision picks the class, as in qmc_plan_create
        const int scls = ctx->opt.precision == QMC_PRECISION_MIXED ? qmc_class_mixed(S.cls) : S.cls;
        if (cls < 0) cls = scls;
        if (scls != cls)
            return fail(ctx, QMC_E_INVAL, "qmc_eval_jobs_noalloc: all jobs must use one evaluator class");
        if (qmc_class_big(cls) || norders > qmc_class_lmax(cls) || hi + S.ns + 1 > qmc_class_lmax(cls))
            return fail(ctx, QMC_E_INVAL, "job %d: orders %d..%d not supported by the evaluator", i, lo, hi);
        QmcJobDev &D = recs[i];
        memset(&D, 0, sizeof D);
        D.sector = S.global_index;
        D.point = I.invariants.empty() ? 0 : J.point;
        D.shifts = J.shifts;
        D.n = J.n;
        D.seed_state = J.seed ^ (kGamma * (J.stream + 1));
        D.inv_n = 1.0 / (double)J.n;
        D.out_off = out_off;
        for (int j = 0; j < QMC_DMAX; ++j) {
            D.z[j] = j < S.d ? it->second[j] : 0;
            D.lambda[j] = (S.deform && j < S.d) ? J.lambda[j] : 0.0;
        }
        D.tiles_per_shift = (int32_t)((D.n + tile_k - 1) / tile_k);
        D.tile_begin = tiles;
        tiles += (uint64_t)D.tiles_per_shift * D.shifts;
        out_off += (uint64_t)J.shifts * norders * 2;
    }
    const uint64_t need = tiles * (uint64_t)(2 * norders);
    const uint64_t cap = qmc_k_noalloc_partial_capacity();
    if (need > cap)
        return fail(ctx, QMC_E_INVAL,
                    "qmc_eval_jobs_noalloc: %llu tile partials exceed the fixed scratch of %llu doubles "
                    "(%u bytes); use fewer points or shifts per call, or qmc_eval_jobs",
                    (unsigned long long)need, (unsigned long long)cap, (unsigned)QMC_NOALLOC_BYTES);
    QmcLaunch L{};
    L.sectors = ctx->d_sectors;
    L.monos = ctx->d_monos;
    L.kin = ctx->d_kin;
    L.ninv = ctx->ninv;
    L.lo = lo;
    L.norders = norders;
    L.ntiles = tiles;
    L.tile_k = (uint32_t)tile_k;
    L.transform = ctx->opt.transform;
    L.prow = QMC_EMAX;   // the fixed launch shape: a table for every exponent
    L.out = out_dev;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    unsigned long long status[2] = {0, 0};
    int rc = qmc_k_noalloc_eval(ctx->device, cls, recs, njobs, &L, block, ppt, ctx->sm_count, status, st);
    if (rc == -2) return fail(ctx, QMC_E_INVAL, "qmc_eval_jobs_noalloc: size beyond the fixed scratch");
    if (rc) return fail(ctx, QMC_E_CUDA, "qmc_eval_jobs_noalloc: %s", cudaGetErrorString(cudaGetLastError()));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int i = 0; i < njobs; ++i) ctx->stat_evals += (double)jobs[i].n * jobs[i].shifts;
    if (status[1]) return fail(ctx, QMC_E_NONFINITE, "%llu tile partial sums were not finite", status[1]);
    if (status[0]) return fail(ctx, QMC_E_SIGN_CHECK, "%llu deformed points had Im F > 0", status[0]);
    return QMC_OK;
}
