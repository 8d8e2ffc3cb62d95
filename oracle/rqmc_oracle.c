/*
 * CPU FP64 ORACLE for randomized rank-1 lattice QMC over sector-decomposed,
 * eps-expanded Feynman-parameter integrands.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code with
 * the CUDA path: it is a plain, slow, literal restatement of the method.
 *
 * What it computes (citations are to arXiv:2305.19768):
 *  - the randomly shifted rank-1 lattice rule of the Disteval integrator
 *    (Section "The new Quasi-Monte-Carlo evaluator Disteval"; median rules,
 *    Eq. (median) and the set U_n): points x_k = frac(k z / n + Delta),
 *    k = 0..n-1, one estimate Q_s = (1/n) sum_k f(x_k) per random shift s;
 *  - the korobov3 periodizing transform named in the timings section;
 *  - contour deformation z = t - i lambda t (1 - t) dF/dt with its Jacobian
 *    determinant (the paper only names the presampling that tunes lambda);
 *  - the eps-expanded sector integrand with subtraction of the endpoint
 *    singularities t_j^{-p + b_j eps}: plus distributions for p = 1, the
 *    Taylor polynomial of degree p - 1 for p >= 2 (in deformed sectors with
 *    every quantity of the deformation formed on truncated power series).
 * The paper is silent on the lattice-point rounding, the transform formula,
 * the deformation formula and the subtraction; the readings used here are:
 *  x = (double)r / (double)n + Delta; if (x >= 1) x -= 1, with r = k z mod n
 *  exact in 64-bit integers; t = u^4 (35 - 84 u + 70 u^2 - 20 u^3),
 *  1 - t = phi(1 - u), weight 140 u^3 (1 - u)^3; a point whose weight is 0 or
 *  whose transformed coordinate underflows to 0 contributes 0.
 *
 * Parity pins (checked by the CPU test suite, not by this file): closed forms
 * of the one-loop massive triangle, massless box and massive bubble,
 * lattice-sum invariants, Korobov moments, subtraction integrals of degree
 * 1 to 3 in one to four variables with polynomial G (exact sums) and with
 * eps-dependent powers of U and F (adaptive quadrature of the remainder),
 * and tensor-product Gauss-Legendre quadrature.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_DMAX 8
#define ORC_LMAX 16      /* series coefficients kept */
#define ORC_SMAX 6       /* singular variables per sector */

typedef double complex cplx;

typedef struct {
    int d;
    int a[ORC_DMAX];
    double b[ORC_DMAX];
    double u0, u1, f0, f1;
    int nU, nF;
    const int *Ue;       /* [nU][d] exponents */
    const double *Uc;    /* [nU] coefficient values at the kinematic point */
    const int *Fe;       /* [nF][d] */
    const double *Fc;    /* [nF] */
    int deform;
    double lambda[ORC_DMAX];
    int transform;       /* 0 korobov3, 1 baker, 2 none */
    double weight;       /* constant factor of the sector (0 is read as 1) */
} orc_sector;

/* ---------------- splitmix64 (Steele, Lea & Flood 2014) ---------------- */
static uint64_t sm64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Random shifts Delta[s][j] in [0,1): 53-bit uniforms, state seeded with
 * seed ^ (golden gamma * (sector id + 1)), drawn shift-major. */
void orc_shifts(uint64_t seed, uint64_t sector_id, int m, int d, double *out) {
    uint64_t st = seed ^ (0x9E3779B97F4A7C15ULL * (sector_id + 1));
    for (int s = 0; s < m; ++s)
        for (int j = 0; j < d; ++j)
            out[s * d + j] = (double)(sm64(&st) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------- lattice ---------------- */
/* r_j = (k z_j) mod n by 128-bit product, then x = r/n + Delta folded to [0,1). */
void orc_lattice_points(uint64_t n, const uint32_t *z, int d, const double *delta,
                        uint64_t k0, uint64_t count, double *x_out, uint64_t *r_out) {
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t k = k0 + i;
        for (int j = 0; j < d; ++j) {
            uint64_t r = (uint64_t)(((unsigned __int128)k * z[j]) % n);
            double x = (double)r / (double)n;
            x = x + delta[j];
            if (x >= 1.0) x -= 1.0;
            if (x_out) x_out[i * d + j] = x;
            if (r_out) r_out[i * d + j] = r;
        }
    }
}

/* ---------------- korobov3 ---------------- */
static double korobov_phi(double u) {
    return u * u * u * u * (35.0 - 84.0 * u + 70.0 * u * u - 20.0 * u * u * u);
}
static double korobov_w(double u) {
    double v = 1.0 - u;
    return 140.0 * u * u * u * v * v * v;
}
void orc_korobov3(double u, double *t, double *omt, double *w) {
    *t = korobov_phi(u);
    *omt = korobov_phi(1.0 - u);
    *w = korobov_w(u);
}

/* baker (tent) transform: t = 1 - |2u - 1|, weight 1 (the map is two-to-one
 * and each branch has |dt/du| = 2); t and 1 - t are formed piecewise so that
 * both are exact for u >= 1/2 and t is exact for u < 1/2. */
void orc_baker(double u, double *t, double *omt, double *w) {
    if (u < 0.5) {
        *t = 2.0 * u;
        *omt = 1.0 - 2.0 * u;
    } else {
        *t = 2.0 * (1.0 - u);
        *omt = 2.0 * u - 1.0;
    }
    *w = 1.0;
}

static void transform_point(int transform, double u, double *t, double *omt, double *w) {
    if (transform == 1) orc_baker(u, t, omt, w);
    else if (transform == 2) { *t = u; *omt = 1.0 - u; *w = 1.0; }
    else orc_korobov3(u, t, omt, w);
}

/* ---------------- truncated Laurent series in eps ---------------- */
typedef struct {
    int lo;               /* order of c[0] */
    int n;                /* number of coefficients */
    cplx c[ORC_LMAX];
} series;

static series s_const(cplx v) {
    series s;
    memset(&s, 0, sizeof s);
    s.lo = 0; s.n = 1; s.c[0] = v;
    return s;
}
/* exp(eps * L) up to eps^hi */
static series s_exp_eps(cplx L, int hi) {
    series s;
    memset(&s, 0, sizeof s);
    s.lo = 0; s.n = hi + 1;
    cplx term = 1.0;
    for (int k = 0; k <= hi; ++k) {
        s.c[k] = term;
        term = term * L / (double)(k + 1);
    }
    return s;
}
static series s_mul(const series *a, const series *b, int hi) {
    series r;
    memset(&r, 0, sizeof r);
    r.lo = a->lo + b->lo;
    r.n = hi - r.lo + 1;
    if (r.n < 0) r.n = 0;
    if (r.n > ORC_LMAX) abort();
    for (int i = 0; i < a->n; ++i)
        for (int j = 0; j < b->n; ++j) {
            int k = i + j;
            if (k < r.n) r.c[k] += a->c[i] * b->c[j];
        }
    return r;
}
static series s_scale(const series *a, cplx v) {
    series r = *a;
    for (int i = 0; i < r.n; ++i) r.c[i] *= v;
    return r;
}
/* a + b (any lo), keep up to eps^hi */
static series s_add(const series *a, const series *b, int hi) {
    series r;
    memset(&r, 0, sizeof r);
    r.lo = a->lo < b->lo ? a->lo : b->lo;
    r.n = hi - r.lo + 1;
    if (r.n > ORC_LMAX) abort();
    for (int i = 0; i < a->n; ++i) {
        int k = a->lo + i - r.lo;
        if (k < r.n) r.c[k] += a->c[i];
    }
    for (int i = 0; i < b->n; ++i) {
        int k = b->lo + i - r.lo;
        if (k < r.n) r.c[k] += b->c[i];
    }
    return r;
}
static cplx s_coef(const series *a, int order) {
    int k = order - a->lo;
    if (k < 0 || k >= a->n) return 0.0;
    return a->c[k];
}
/* |Re| + |Im| of every coefficient: products of such series bound the
 * magnitudes of everything a product of the original series sums */
static series s_mass(const series *a) {
    series r = *a;
    for (int i = 0; i < r.n; ++i) r.c[i] = fabs(creal(a->c[i])) + fabs(cimag(a->c[i]));
    return r;
}

/* ---------------- polynomials ---------------- */
static cplx cipow(cplx x, int e) {
    cplx r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}
/* Mixed partial derivative d^|D| P / prod dt_j^{D_j} at complex/real point x,
 * from the monomial table: each monomial c prod x^e contributes
 * c prod_j e_j (e_j - 1) ... (e_j - D_j + 1) x_j^(e_j - D_j). */
static cplx poly_deriv(int nterms, int d, const int *ex, const double *co, const cplx *x,
                       const int *D) {
    cplx sum = 0.0;
    for (int m = 0; m < nterms; ++m) {
        cplx term = co[m];
        for (int j = 0; j < d; ++j) {
            int e = ex[m * d + j];
            int dj = D ? D[j] : 0;
            if (e < dj) { term = 0.0; break; }
            for (int q = 0; q < dj; ++q) term *= (double)(e - q);
            term *= cipow(x[j], e - dj);
        }
        sum += term;
    }
    return sum;
}

/* ---------------- determinant (Leibniz formula) ---------------- */
static cplx det_leibniz(int d, const cplx *A) {
    int perm[ORC_DMAX];
    for (int i = 0; i < d; ++i) perm[i] = i;
    cplx det = 0.0;
    /* iterate permutations in lexicographic order, tracking the sign by
     * counting inversions */
    for (;;) {
        int inv = 0;
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j)
                if (perm[i] > perm[j]) ++inv;
        cplx p = (inv % 2) ? -1.0 : 1.0;
        for (int i = 0; i < d; ++i) p *= A[i * d + perm[i]];
        det += p;
        int i = d - 2;
        while (i >= 0 && perm[i] > perm[i + 1]) --i;
        if (i < 0) break;
        int j = d - 1;
        while (perm[j] < perm[i]) --j;
        int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        for (int l = i + 1, r = d - 1; l < r; ++l, --r) {
            tmp = perm[l]; perm[l] = perm[r]; perm[r] = tmp;
        }
    }
    return det;
}

/* singular: t_j^{a_j + b_j eps} with a_j <= -1. a_j = -1 is logarithmic;
 * a_j = -p, p >= 2, takes the Taylor subtraction of degree p - 1 (undeformed
 * sectors only) */
static int is_singular(const orc_sector *S, int j) { return S->a[j] <= -1; }

/* G(t', eps): everything in the sector integrand except prod_{j in S}
 * t_j^{-1 + b_j eps}, at the real point tp (omtp = 1 - tp), as a series up
 * to eps^hi. With deformation, z_j = t_j - i lambda_j t_j (1 - t_j) dF/dt_j,
 * rho_j = z_j / t_j, J = dz/dt, and
 *   G = prod_{j not in S} z_j^{a_j + b_j eps} prod_{j in S} rho_j^{-1 + b_j eps}
 *       U(z)^{u0 + u1 eps} F(z)^{f0 + f1 eps} det J.
 * Counts Im F(z) > 0 (wrong side of the F - i0 cut) in *signfail. */
static series G_series(const orc_sector *S, const double *tp, const double *omtp, int hi,
                       int *signfail) {
    int d = S->d;
    cplx t[ORC_DMAX], z[ORC_DMAX], rho[ORC_DMAX], dF[ORC_DMAX];
    cplx J[ORC_DMAX * ORC_DMAX];
    cplx detJ = 1.0;
    for (int j = 0; j < d; ++j) { t[j] = tp[j]; z[j] = tp[j]; rho[j] = 1.0; }
    if (S->deform) {
        int D[ORC_DMAX];
        for (int j = 0; j < d; ++j) {
            memset(D, 0, sizeof D);
            D[j] = 1;
            dF[j] = poly_deriv(S->nF, d, S->Fe, S->Fc, t, D);
        }
        for (int j = 0; j < d; ++j) {
            double tj = tp[j], omt = omtp[j];
            z[j] = tj - I * S->lambda[j] * tj * omt * dF[j];
            rho[j] = 1.0 - I * S->lambda[j] * omt * dF[j];
            for (int l = 0; l < d; ++l) {
                memset(D, 0, sizeof D);
                D[j] += 1;
                D[l] += 1;
                cplx d2 = poly_deriv(S->nF, d, S->Fe, S->Fc, t, D);
                cplx v = -I * S->lambda[j] * (tj * omt * d2 + (j == l ? (omt - tj) * dF[j] : 0.0));
                J[j * d + l] = (j == l ? 1.0 : 0.0) + v;
            }
        }
        detJ = det_leibniz(d, J);
    }
    cplx U = poly_deriv(S->nU, d, S->Ue, S->Uc, z, NULL);
    cplx F = poly_deriv(S->nF, d, S->Fe, S->Fc, z, NULL);
    if (cimag(F) > 0.0) ++*signfail;
    if (cimag(F) == 0.0) F = CMPLX(creal(F), -0.0); /* F - i0 */
    if (cimag(U) == 0.0) U = CMPLX(creal(U), 0.0);

    series G = s_const(detJ);
    for (int j = 0; j < d; ++j) {
        cplx base;
        double a, b;
        if (is_singular(S, j)) { base = rho[j]; a = (double)S->a[j]; b = S->b[j]; }
        else { base = z[j]; a = S->a[j]; b = S->b[j]; }
        if (a == 0.0 && b == 0.0) continue;
        cplx lg = clog(base);
        series f = s_exp_eps(b * lg, hi);
        /* base^a: the monomial factor itself; for a real positive base the
         * library power (within an ulp), since exp(a ln base) would carry the
         * rounding of ln base times |a ln base| */
        cplx pa = (cimag(base) == 0.0 && creal(base) > 0.0) ? pow(creal(base), a) : cexp(a * lg);
        f = s_scale(&f, pa);
        G = s_mul(&G, &f, hi);
    }
    {
        cplx lg = clog(U);
        series f = s_exp_eps(S->u1 * lg, hi);
        f = s_scale(&f, cexp(S->u0 * lg));
        G = s_mul(&G, &f, hi);
    }
    {
        cplx lg = clog(F);
        series f = s_exp_eps(S->f1 * lg, hi);
        f = s_scale(&f, cexp(S->f0 * lg));
        G = s_mul(&G, &f, hi);
    }
    return G;
}

/* ---------------- Taylor coefficients of G in the zeroed variables ---------------- */
/* Truncated multivariate power series ("jets") in the variables t_{V[0..nv-1]}
 * over the box 0 <= k_q < rad[q]; flat index sum_q k_q prod_{r<q} rad[r]. */
#define ORC_JMAX 128
typedef struct {
    int nv;
    int rad[ORC_SMAX];
    int size;
} jbox;

static void jbox_digits(const jbox *B, int idx, int *dig) {
    for (int q = 0; q < B->nv; ++q) {
        dig[q] = idx % B->rad[q];
        idx /= B->rad[q];
    }
}

/* c = a b, every product whose exponents leave the box dropped (c may alias a or b) */
static void jet_mul(const jbox *B, const cplx *a, const cplx *b, cplx *c) {
    cplx r[ORC_JMAX];
    for (int k = 0; k < B->size; ++k) r[k] = 0.0;
    for (int i = 0; i < B->size; ++i) {
        int di[ORC_SMAX];
        jbox_digits(B, i, di);
        for (int j = 0; j < B->size; ++j) {
            int dj[ORC_SMAX];
            jbox_digits(B, j, dj);
            int k = 0, stride = 1, inside = 1;
            for (int q = 0; q < B->nv; ++q) {
                int e = di[q] + dj[q];
                if (e >= B->rad[q]) { inside = 0; break; }
                k += e * stride;
                stride *= B->rad[q];
            }
            if (inside) r[k] += a[i] * b[j];
        }
    }
    for (int k = 0; k < B->size; ++k) c[k] = r[k];
}

/* P^{e0 + e1 eps} over the box for a jet P with P[0] != 0 (Pabs: magnitudes
 * of P's entries), as eps-series up to eps^hi per box entry, by the
 * generalized binomial theorem: with P = P0 + delta (delta without constant
 * term),
 *   P^alpha = sum_k binom(alpha, k) P0^{alpha - k} delta^k,
 * binom(alpha, k) = prod_{i<k} (alpha - i) / k! a polynomial in eps, and
 * P0^{alpha - k} = P0^{e0 - k} exp(e1 eps ln P0) (principal log; m0: on the
 * real axis the argument is taken from below, the F - i0 prescription).
 * delta^k vanishes in the box beyond k = sum_q (rad_q - 1). mass (may be
 * NULL) receives the same sums of the terms' magnitudes. */
static void sjet_pow(const jbox *B, const cplx *P, const cplx *Pabs, double e0, double e1, int m0, int hi,
                     series *out, series *mass) {
    cplx delta[ORC_JMAX], dabs[ORC_JMAX];
    for (int k = 0; k < B->size; ++k) {
        delta[k] = P[k];
        dabs[k] = Pabs[k];
    }
    cplx P0 = delta[0];
    if (cimag(P0) == 0.0) P0 = CMPLX(creal(P0), m0 ? -0.0 : 0.0);
    delta[0] = 0.0;
    dabs[0] = 0.0;
    cplx lg = clog(P0);
    series pe = s_exp_eps(e1 * lg, hi);                /* P0^{e1 eps} */
    series pem = s_mass(&pe);
    int K = 0;
    for (int q = 0; q < B->nv; ++q) K += B->rad[q] - 1;
    for (int i = 0; i < B->size; ++i) {
        memset(&out[i], 0, sizeof(series));
        out[i].lo = 0;
        out[i].n = hi + 1;
        if (mass) mass[i] = out[i];
    }
    cplx dk[ORC_JMAX], dkabs[ORC_JMAX];                 /* delta^k, |delta|^k */
    for (int i = 0; i < B->size; ++i) dk[i] = dkabs[i] = 0.0;
    dk[0] = dkabs[0] = 1.0;
    series binom = s_const(1.0);
    for (int k = 0; k <= K; ++k) {
        if (k > 0) {
            jet_mul(B, dk, delta, dk);
            jet_mul(B, dkabs, dabs, dkabs);
            series lin;                                  /* (e0 - (k - 1) + e1 eps) / k */
            memset(&lin, 0, sizeof lin);
            lin.lo = 0; lin.n = 2;
            lin.c[0] = (e0 - (k - 1)) / (double)k;
            lin.c[1] = e1 / (double)k;
            binom = s_mul(&binom, &lin, hi);
        }
        series c = s_mul(&binom, &pe, hi);
        c = s_scale(&c, cexp((e0 - k) * lg));
        series bm = s_mass(&binom);
        series cm = s_mul(&bm, &pem, hi);
        cm = s_scale(&cm, cabs(cexp((e0 - k) * lg)));
        for (int i = 0; i < B->size; ++i)
            if (dk[i] != 0.0 || dkabs[i] != 0.0) {
                series term = s_scale(&c, dk[i]);
                out[i] = s_add(&out[i], &term, hi);
                if (mass) {
                    series tm = s_scale(&cm, dkabs[i]);
                    mass[i] = s_add(&mass[i], &tm, hi);
                }
            }
    }
}

/* Taylor coefficients of P^{e0 + e1 eps} (P = U or F) in the variables V at
 * t_V = 0, the other variables at t (undeformed sector): P's box entries are
 * read off the monomial table (t_V^e lands at entry e, the other variables
 * multiply in), then sjet_pow. */
static void jet_power(const orc_sector *S, int isF, const double *t, const int *V, const jbox *B,
                      int hi, series *out, series *mass) {
    int d = S->d;
    int nP = isF ? S->nF : S->nU;
    const int *ex = isF ? S->Fe : S->Ue;
    const double *co = isF ? S->Fc : S->Uc;
    double e0 = isF ? S->f0 : S->u0, e1 = isF ? S->f1 : S->u1;
    int inV[ORC_DMAX] = {0};
    for (int q = 0; q < B->nv; ++q) inV[V[q]] = 1;
    cplx P[ORC_JMAX], Pabs[ORC_JMAX];
    for (int k = 0; k < B->size; ++k) P[k] = Pabs[k] = 0.0;
    for (int m = 0; m < nP; ++m) {
        int idx = 0, stride = 1, inside = 1;
        for (int q = 0; q < B->nv; ++q) {
            int e = ex[m * d + V[q]];
            if (e >= B->rad[q]) { inside = 0; break; }
            idx += e * stride;
            stride *= B->rad[q];
        }
        if (!inside) continue;
        cplx v = co[m];
        for (int j = 0; j < d; ++j)
            if (!inV[j]) v *= cipow(t[j], ex[m * d + j]);
        P[idx] += v;
        Pabs[idx] += cabs(v);
    }
    sjet_pow(B, P, Pabs, e0, e1, isF, hi, out, mass);
}

/* Taylor coefficient of G (undeformed sector) of prod_{q} t_{V[q]}^{kap[q]}
 * at t_V = 0, the other variables at t, as an eps-series up to eps^hi. There
 * G = prod_{j regular} t_j^{a_j + b_j eps} U^{u0 + u1 eps} F^{f0 + f1 eps}, and
 * only U and F depend on t_V: the coefficient is the regular factor times
 * sum_{k' <= kap} [U^.]_{k'} [F^.]_{kap - k'}. */
static series taylor_G(const orc_sector *S, const double *t, int nv, const int *V, const int *kap,
                       int hi, series *massout) {
    jbox B;
    B.nv = nv;
    B.size = 1;
    for (int q = 0; q < nv; ++q) {
        B.rad[q] = kap[q] + 1;
        B.size *= B.rad[q];
    }
    if (B.size > ORC_JMAX) abort();
    series PU[ORC_JMAX], PF[ORC_JMAX], MU[ORC_JMAX], MF[ORC_JMAX];
    jet_power(S, 0, t, V, &B, hi, PU, MU);
    jet_power(S, 1, t, V, &B, hi, PF, MF);
    series prod, mass;
    memset(&prod, 0, sizeof prod);
    prod.lo = 0; prod.n = hi + 1;
    mass = prod;
    for (int i = 0; i < B.size; ++i) {
        int di[ORC_SMAX], j = 0, stride = 1;
        jbox_digits(&B, i, di);
        for (int q = 0; q < nv; ++q) {
            j += (kap[q] - di[q]) * stride;
            stride *= B.rad[q];
        }
        series term = s_mul(&PU[i], &PF[j], hi);
        prod = s_add(&prod, &term, hi);
        series tm = s_mul(&MU[i], &MF[j], hi);
        mass = s_add(&mass, &tm, hi);
    }
    for (int j = 0; j < S->d; ++j) {
        if (is_singular(S, j) || (S->a[j] == 0 && S->b[j] == 0.0)) continue;
        cplx lg = clog((cplx)t[j]);
        series f = s_exp_eps(S->b[j] * lg, hi);
        f = s_scale(&f, pow(t[j], (double)S->a[j]));
        prod = s_mul(&prod, &f, hi);
        series fm = s_mass(&f);
        mass = s_mul(&mass, &fm, hi);
    }
    if (massout) *massout = mass;
    return prod;
}

/* ---------------- Taylor coefficients of G in deformed sectors ---------------- */
/* Jets of eps-series: c = a b over the box (every series starts at eps^0). */
static void sjet_mul(const jbox *B, const series *a, const series *b, int hi, series *c) {
    for (int k = 0; k < B->size; ++k) {
        memset(&c[k], 0, sizeof(series));
        c[k].lo = 0;
        c[k].n = hi + 1;
    }
    for (int i = 0; i < B->size; ++i) {
        int di[ORC_SMAX];
        jbox_digits(B, i, di);
        for (int j = 0; j < B->size; ++j) {
            int dj[ORC_SMAX];
            jbox_digits(B, j, dj);
            int k = 0, stride = 1, inside = 1;
            for (int q = 0; q < B->nv; ++q) {
                int e = di[q] + dj[q];
                if (e >= B->rad[q]) { inside = 0; break; }
                k += e * stride;
                stride *= B->rad[q];
            }
            if (!inside) continue;
            series term = s_mul(&a[i], &b[j], hi);
            c[k] = s_add(&c[k], &term, hi);
        }
    }
}

/* A polynomial's mixed partial derivative d^|D| P / prod dt^D (D may be NULL)
 * at jet arguments x_j: sum_m c_m prod_j e(e-1)..(e-D_j+1) x_j^(e - D_j), the
 * powers by repeated jet products. outabs: the sum of the terms' magnitudes. */
static void jet_poly(const jbox *B, int nterms, int d, const int *ex, const double *co, cplx x[][ORC_JMAX],
                     const int *D, cplx *out, cplx *outabs) {
    for (int k = 0; k < B->size; ++k) out[k] = outabs[k] = 0.0;
    for (int m = 0; m < nterms; ++m) {
        cplx term[ORC_JMAX];
        for (int k = 0; k < B->size; ++k) term[k] = 0.0;
        term[0] = co[m];
        int zero = 0;
        for (int j = 0; j < d && !zero; ++j) {
            int e = ex[m * d + j], dj = D ? D[j] : 0;
            if (e < dj) { zero = 1; break; }
            for (int q = 0; q < dj; ++q) term[0] *= (double)(e - q);
            for (int r = 0; r < e - dj; ++r) jet_mul(B, term, x[j], term);
        }
        if (zero) continue;
        for (int k = 0; k < B->size; ++k) {
            out[k] += term[k];
            outabs[k] += cabs(term[k]);
        }
    }
}

/* Taylor coefficient of G of prod_q t_{V[q]}^{kap[q]} at t_V = 0 in a deformed
 * sector, the other variables at t (omt = 1 - t). Every quantity of G_series
 * is formed on jets in t_V: t_j, 1 - t_j, dF/dt_j and d2F/dt_j dt_l, then
 *   z_j = t_j - i lambda_j t_j (1 - t_j) dF_j,  rho_j = 1 - i lambda_j (1 - t_j) dF_j,
 *   J_jl = delta_jl - i lambda_j (t_j (1 - t_j) d2F_jl + delta_jl (1 - 2 t_j) dF_j),
 * det J by the Leibniz formula, U(z) and F(z); each power factor (rho_j or
 * z_j, U, F) by sjet_pow, and G = det J times their product. massout: the
 * coefficient's mass (magnitudes of the binomial terms and of the products). */
static series taylor_G_deformed(const orc_sector *S, const double *t, const double *omt, int nv, const int *V,
                                const int *kap, int hi, series *massout) {
    int d = S->d;
    jbox B;
    B.nv = nv;
    B.size = 1;
    int stride[ORC_SMAX], pos[ORC_DMAX];
    for (int j = 0; j < d; ++j) pos[j] = -1;
    for (int q = 0; q < nv; ++q) {
        B.rad[q] = kap[q] + 1;
        stride[q] = B.size;
        B.size *= B.rad[q];
        pos[V[q]] = q;
    }
    if (B.size > ORC_JMAX) abort();
    static __thread cplx tj[ORC_DMAX][ORC_JMAX], oj[ORC_DMAX][ORC_JMAX], Fj[ORC_DMAX][ORC_JMAX],
        zj[ORC_DMAX][ORC_JMAX], rj[ORC_DMAX][ORC_JMAX], Jm[ORC_DMAX * ORC_DMAX][ORC_JMAX];
    cplx tmp[ORC_JMAX], tabs[ORC_JMAX];
    for (int j = 0; j < d; ++j) {
        for (int k = 0; k < B.size; ++k) tj[j][k] = oj[j][k] = 0.0;
        int q = pos[j];
        if (q >= 0) {                                 /* t_j = 0 + the jet variable */
            oj[j][0] = 1.0;
            if (B.rad[q] > 1) {
                tj[j][stride[q]] = 1.0;
                oj[j][stride[q]] = -1.0;
            }
        } else {
            tj[j][0] = t[j];
            oj[j][0] = omt[j];
        }
    }
    int D[ORC_DMAX];
    for (int j = 0; j < d; ++j) {
        memset(D, 0, sizeof D);
        D[j] = 1;
        jet_poly(&B, S->nF, d, S->Fe, S->Fc, tj, D, Fj[j], tabs);
    }
    for (int j = 0; j < d; ++j) {
        cplx g[ORC_JMAX];                             /* lambda_j (1 - t_j) dF_j */
        jet_mul(&B, oj[j], Fj[j], g);
        for (int k = 0; k < B.size; ++k) {
            g[k] *= S->lambda[j];
            rj[j][k] = (k == 0 ? 1.0 : 0.0) - I * g[k];
        }
        jet_mul(&B, tj[j], rj[j], zj[j]);             /* z_j = t_j rho_j */
        for (int l = 0; l < d; ++l) {
            memset(D, 0, sizeof D);
            D[j] += 1;
            D[l] += 1;
            cplx h[ORC_JMAX], w[ORC_JMAX];
            jet_poly(&B, S->nF, d, S->Fe, S->Fc, tj, D, h, tabs);
            jet_mul(&B, tj[j], oj[j], w);             /* t_j (1 - t_j) d2F_jl */
            jet_mul(&B, w, h, w);
            if (j == l) {                             /* + (1 - 2 t_j) dF_j */
                cplx u[ORC_JMAX];
                for (int k = 0; k < B.size; ++k) u[k] = oj[j][k] - tj[j][k];
                jet_mul(&B, u, Fj[j], u);
                for (int k = 0; k < B.size; ++k) w[k] += u[k];
            }
            for (int k = 0; k < B.size; ++k)
                Jm[j * d + l][k] = (j == l && k == 0 ? 1.0 : 0.0) - I * S->lambda[j] * w[k];
        }
    }
    /* det J = sum over permutations of sign prod_i J[i][perm i] */
    cplx detJ[ORC_JMAX], dabsJ[ORC_JMAX];
    for (int k = 0; k < B.size; ++k) detJ[k] = dabsJ[k] = 0.0;
    {
        int perm[ORC_DMAX];
        for (int i = 0; i < d; ++i) perm[i] = i;
        for (;;) {
            int inv = 0;
            for (int i = 0; i < d; ++i)
                for (int j = i + 1; j < d; ++j)
                    if (perm[i] > perm[j]) ++inv;
            for (int k = 0; k < B.size; ++k) tmp[k] = (k == 0) ? ((inv % 2) ? -1.0 : 1.0) : 0.0;
            for (int i = 0; i < d; ++i) jet_mul(&B, tmp, Jm[i * d + perm[i]], tmp);
            for (int k = 0; k < B.size; ++k) {
                detJ[k] += tmp[k];
                dabsJ[k] += cabs(tmp[k]);
            }
            int i = d - 2;
            while (i >= 0 && perm[i] > perm[i + 1]) --i;
            if (i < 0) break;
            int j = d - 1;
            while (perm[j] < perm[i]) --j;
            int tt = perm[i]; perm[i] = perm[j]; perm[j] = tt;
            for (int l = i + 1, r = d - 1; l < r; ++l, --r) {
                tt = perm[l]; perm[l] = perm[r]; perm[r] = tt;
            }
        }
    }
    /* the product of the power factors, starting from det J (no eps exponent) */
    static __thread series prod[ORC_JMAX], mass[ORC_JMAX], fs[ORC_JMAX], fm[ORC_JMAX], nx[ORC_JMAX];
    for (int k = 0; k < B.size; ++k) {
        prod[k] = s_const(detJ[k]);
        prod[k].n = hi + 1;
        mass[k] = s_const(dabsJ[k]);
        mass[k].n = hi + 1;
    }
    for (int f = 0; f < d + 2; ++f) {
        const cplx *P;
        cplx Pabs[ORC_JMAX], pv[ORC_JMAX];
        double e0, e1;
        int m0 = 0;
        if (f < d) {
            if (is_singular(S, f)) P = rj[f];
            else if (S->a[f] != 0 || S->b[f] != 0.0) P = zj[f];
            else continue;
            e0 = S->a[f];
            e1 = S->b[f];
            for (int k = 0; k < B.size; ++k) Pabs[k] = cabs(P[k]);
        } else {
            int isF = f == d + 1;
            jet_poly(&B, isF ? S->nF : S->nU, d, isF ? S->Fe : S->Ue, isF ? S->Fc : S->Uc, zj, NULL, pv, Pabs);
            P = pv;
            e0 = isF ? S->f0 : S->u0;
            e1 = isF ? S->f1 : S->u1;
            m0 = isF;
        }
        if (e0 == 0.0 && e1 == 0.0) continue;
        sjet_pow(&B, P, Pabs, e0, e1, m0, hi, fs, fm);
        sjet_mul(&B, prod, fs, hi, nx);
        for (int k = 0; k < B.size; ++k) prod[k] = nx[k];
        for (int k = 0; k < B.size; ++k) fm[k] = s_mass(&fm[k]);
        sjet_mul(&B, mass, fm, hi, nx);
        for (int k = 0; k < B.size; ++k) mass[k] = nx[k];
    }
    if (massout) *massout = mass[B.size - 1];
    return prod[B.size - 1];
}

/* The eps-expanded integrand at the transformed point t (omt = 1 - t):
 *   f = sum_{V subset of S} G(t with t_V = 0)
 *         prod_{j in V} (1/(b_j eps) - t_j^{-1+b_j eps}) prod_{j in S\V} t_j^{-1+b_j eps},
 * which integrates over [0,1]^d to the Laurent expansion of the sector
 * integral (each j in S: int t^{-1+b eps} g = g(0)/(b eps) + int t^{-1+b eps}(g - g(0))).
 * A variable with a_j = -p, p >= 2, takes the Taylor subtraction of degree
 * p - 1:
 *   int t^{-p+b eps} g = sum_{k<p} g_k / (k - p + 1 + b eps)
 *                        + int t^{-p+b eps} (g - sum_{k<p} g_k t^k),
 * g_k the k-th Taylor coefficient of g at t = 0, so per singular variable the
 * states are "t kept" (factor t^{-p+b eps}) and k = 0..p-1 (t = 0, Taylor
 * coefficient k of G in that variable, factor 1/(k - p + 1 + b eps) -
 * t^{k-p+b eps}); f sums over all state choices, with the mixed Taylor
 * coefficient in the variables set to 0.
 * Returns coefficients of eps^lo .. eps^hi in out[(o - lo)]. */
static void integrand_series(const orc_sector *S, const double *t, const double *omt, int lo,
                             int hi, cplx *out, double *cond, int *signfail) {
    int d = S->d;
    int sing[ORC_SMAX], ns = 0;
    for (int j = 0; j < d; ++j)
        if (is_singular(S, j)) {
            if (ns == ORC_SMAX) abort();
            sing[ns++] = j;
        }
    int H = hi + ns; /* every factor truncated here is exact up to eps^hi */
    series total;
    memset(&total, 0, sizeof total);
    total.lo = lo; total.n = hi - lo + 1;
    /* state of slot q: 0 = t_q kept, k + 1 = (t_q = 0, k-th derivative), k < p_q */
    int nstates = 1, radix[ORC_SMAX];
    for (int q = 0; q < ns; ++q) {
        radix[q] = 1 - S->a[sing[q]];          /* p_q + 1 */
        nstates *= radix[q];
    }
    for (int st = 0; st < nstates; ++st) {
        int state[ORC_SMAX], rem = st, nv = 0, V[ORC_SMAX], kap[ORC_SMAX], taylor = 0;
        double tp[ORC_DMAX], omtp[ORC_DMAX];
        for (int j = 0; j < d; ++j) { tp[j] = t[j]; omtp[j] = omt[j]; }
        for (int q = 0; q < ns; ++q) {
            state[q] = rem % radix[q];
            rem /= radix[q];
            if (state[q] > 0) {
                tp[sing[q]] = 0.0;
                omtp[sing[q]] = 1.0;
                V[nv] = sing[q];
                kap[nv++] = state[q] - 1;
                if (state[q] > 1) taylor = 1;
            }
        }
        /* every Taylor order 0: G itself at t_V = 0; else the Taylor coefficient */
        series gmass;
        series term = !taylor ? G_series(S, tp, omtp, H, signfail)
                      : S->deform ? taylor_G_deformed(S, t, omt, nv, V, kap, H, &gmass)
                                  : taylor_G(S, t, nv, V, kap, H, &gmass);
        for (int q = 0; q < ns; ++q) {
            int j = sing[q];
            int p = -S->a[j];
            double b = S->b[j];
            int k = state[q] - 1;
            series tpow = s_exp_eps(b * log(t[j]), H);
            tpow = s_scale(&tpow, pow(t[j], state[q] == 0 ? -p : k - p));   /* t^{c + b eps} */
            series fac;
            if (state[q] > 0) {
                int m = k - p + 1;                    /* 1/(m + b eps) */
                series inv;
                memset(&inv, 0, sizeof inv);
                if (m == 0) {
                    inv.lo = -1; inv.n = 1; inv.c[0] = 1.0 / b;
                } else {
                    inv.lo = 0; inv.n = H + 1;
                    cplx c = 1.0 / m;
                    for (int i = 0; i <= H; ++i) { inv.c[i] = c; c *= -b / m; }
                }
                series neg = s_scale(&tpow, -1.0);
                fac = s_add(&inv, &neg, H);
            } else {
                fac = tpow;
            }
            term = s_mul(&term, &fac, H);
            if (taylor) {
                series fm = s_mass(&fac);
                gmass = s_mul(&gmass, &fm, H);
            }
        }
        total = s_add(&total, &term, hi);
        /* the mass of what cancels: |term| per order; for a Taylor state the
         * magnitudes of the binomial-series terms inside its coefficient too */
        if (cond)
            for (int o = lo; o <= hi; ++o) {
                cplx c = s_coef(taylor ? &gmass : &term, o);
                cond[o - lo] += fabs(creal(c)) + fabs(cimag(c));
            }
    }
    for (int o = lo; o <= hi; ++o) out[o - lo] = s_coef(&total, o);
}

/* Integrand times the korobov3 weight at the raw lattice point u[d].
 * out[(o - lo) * 2 + {0,1}] = Re, Im; cond[o - lo] (may be NULL) = W times
 * the sum over subtraction corners of |Re| + |Im| of each corner's term (the
 * size of what cancels). Returns 0 if the point contributes 0. */
static int point_value_cond(const orc_sector *S, const double *u, int lo, int norders,
                            double *out, double *cond, int *signfail) {
    int d = S->d;
    double t[ORC_DMAX], omt[ORC_DMAX], W = 1.0;
    for (int o = 0; o < 2 * norders; ++o) out[o] = 0.0;
    for (int j = 0; j < d; ++j) {
        double w;
        transform_point(S->transform, u[j], &t[j], &omt[j], &w);
        W *= w;
    }
    if (W == 0.0) return 0;
    for (int j = 0; j < d; ++j)
        if (t[j] == 0.0) return 0;
    if (S->weight != 0.0) W *= S->weight;
    cplx vals[ORC_LMAX];
    double cnd[ORC_LMAX] = {0};
    integrand_series(S, t, omt, lo, lo + norders - 1, vals, cnd, signfail);
    for (int o = 0; o < norders; ++o) {
        out[2 * o] = W * creal(vals[o]);
        out[2 * o + 1] = W * cimag(vals[o]);
        if (cond) cond[o] = W * cnd[o];
    }
    return 1;
}

int orc_point_value(const orc_sector *S, const double *u, int lo, int norders, double *out,
                    int *signfail) {
    return point_value_cond(S, u, lo, norders, out, NULL, signfail);
}

/* Integrand (no weight) at a transformed point t in (0,1]^d: used by the
 * quadrature cross-checks. */
void orc_integrand_at(const orc_sector *S, const double *t, int lo, int norders, double *out,
                      int *signfail) {
    double omt[ORC_DMAX];
    cplx vals[ORC_LMAX];
    for (int j = 0; j < S->d; ++j) omt[j] = 1.0 - t[j];
    integrand_series(S, t, omt, lo, lo + norders - 1, vals, NULL, signfail);
    const double wt = S->weight != 0.0 ? S->weight : 1.0;
    for (int o = 0; o < norders; ++o) {
        out[2 * o] = wt * creal(vals[o]);
        out[2 * o + 1] = wt * cimag(vals[o]);
    }
}

/* ---------------- per-shift sums ---------------- */
typedef struct { double s, c; } neum;
static void neum_add(neum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

#define ORC_CHUNK 4096

/* Per-shift estimates Q_s = (1/n) sum_{k=k0}^{k1-1} f(x_k + Delta_s) for each
 * eps order, out[(s * norders + o) * 2 + {re, im}]; absout[s * norders + o] =
 * (1/n) sum |Re f| + |Im f| (the scale for relative comparisons) and
 * absout[(m + s) * norders + o] = (1/n) sum of the corner-term masses
 * (the size of the cancellation inside the subtraction).
 * The k range is cut into fixed chunks of ORC_CHUNK points, each summed
 * left to right with Neumaier compensation, and the chunk sums are combined
 * in index order, so the result does not depend on the thread count.
 * Returns the number of sign-check failures. */
long orc_shift_sums(const orc_sector *S, uint64_t n, const uint32_t *z, int m,
                    const double *delta, uint64_t k0, uint64_t k1, int lo, int norders,
                    double *out, double *absout, int nthreads) {
    int d = S->d;
    uint64_t nk = k1 > k0 ? k1 - k0 : 0;
    uint64_t nchunks = (nk + ORC_CHUNK - 1) / ORC_CHUNK;
    size_t per = (size_t)norders * 2;
    const size_t stride = per * 3 + (size_t)norders;
    double *part = (double *)calloc((size_t)m * nchunks * stride + 1, sizeof(double));
    long fails = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : fails)
    for (long long job = 0; job < (long long)(m * nchunks); ++job) {
        int s = (int)(job / nchunks);
        uint64_t c = job % nchunks;
        uint64_t ka = k0 + c * ORC_CHUNK;
        uint64_t kb = ka + ORC_CHUNK < k1 ? ka + ORC_CHUNK : k1;
        neum acc[ORC_LMAX * 2];
        double aacc[ORC_LMAX], cacc[ORC_LMAX];
        memset(acc, 0, sizeof acc);
        memset(aacc, 0, sizeof aacc);
        memset(cacc, 0, sizeof cacc);
        int sf = 0;
        for (uint64_t k = ka; k < kb; ++k) {
            double u[ORC_DMAX], v[ORC_LMAX * 2], cv[ORC_LMAX];
            orc_lattice_points(n, z, d, delta + (size_t)s * d, k, 1, u, NULL);
            if (!point_value_cond(S, u, lo, norders, v, cv, &sf)) continue;
            for (int q = 0; q < 2 * norders; ++q) neum_add(&acc[q], v[q]);
            for (int o = 0; o < norders; ++o) {
                aacc[o] += fabs(v[2 * o]) + fabs(v[2 * o + 1]);
                cacc[o] += cv[o];
            }
        }
        double *dst = part + ((size_t)s * nchunks + c) * stride;
        for (size_t q = 0; q < per; ++q) { dst[q] = acc[q].s; dst[per + q] = acc[q].c; }
        for (int o = 0; o < norders; ++o) { dst[2 * per + o] = aacc[o]; dst[3 * per + o] = cacc[o]; }
        fails += sf;
    }
    for (int s = 0; s < m; ++s) {
        for (size_t q = 0; q < per; ++q) {
            neum a = {0.0, 0.0};
            for (uint64_t c = 0; c < nchunks; ++c) {
                const double *src = part + ((size_t)s * nchunks + c) * stride;
                neum_add(&a, src[q]);
                neum_add(&a, src[per + q]);
            }
            out[s * per + q] = (a.s + a.c) / (double)n;
        }
        if (absout)
            for (int o = 0; o < norders; ++o) {
                double a = 0.0, cm = 0.0;
                for (uint64_t c = 0; c < nchunks; ++c) {
                    a += part[((size_t)s * nchunks + c) * stride + 2 * per + o];
                    cm += part[((size_t)s * nchunks + c) * stride + 3 * per + o];
                }
                absout[s * norders + o] = a / (double)n;
                absout[((size_t)m + s) * norders + o] = cm / (double)n;
            }
    }
    free(part);
    return fails;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
