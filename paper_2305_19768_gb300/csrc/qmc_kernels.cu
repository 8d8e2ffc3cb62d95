// sm_103a kernels of the randomized rank-1 lattice QMC evaluator.
//
// qmc_eval_kernel: persistent blocks pull tiles (job, shift, chunk of k) from
// an atomic queue. Per tile the block stages the sector's monomial tables,
// with coefficients evaluated at the job's kinematic point, in shared memory
// and draws the shift on the device (splitmix64 is counter based). Each
// thread walks PPT consecutive lattice indices with the exact integer update
// r <- r + z (mod n), maps the point through korobov3, evaluates the
// eps-expanded integrand (optionally on the deformed contour) and
// accumulates; a warp-shuffle + shared-memory reduction writes one partial
// per tile and eps order. qmc_finish_kernel sums a job's tile partials in
// tile order with Neumaier compensation (deterministic), divides by n, and
// re-arms the queue.
//
// Method steps (arXiv:2305.19768): the shifted lattice rule of the Disteval
// integrator and its on-GPU summation (Disteval section), the korobov3
// transform (timings section), contour deformation whose parameter the
// presampling tunes (usage section), the sums of samples per shift and eps
// order that feed Eq. (adaptive-solution).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "qmc_ilog.h"
#include "qmc_internal.h"
#include "qmc_log_table.h"
#include "qmc_xf.h"

#ifndef QMC_PART
#define QMC_PART 0
#endif
// 1: the d <= 6 classes also take korobov3 on the integer pipe (as the d <= 3
// classes do; measured 3 % faster on the double box than FP64 arithmetic
// there); 0: FP64 arithmetic for them
#ifndef QMC_KOROBOV_INT6
#define QMC_KOROBOV_INT6 1
#endif

namespace {

__device__ const uint64_t kLogTable[3 * QMC_LOG_TABLE_ROWS] = QMC_LOG_TABLE_INIT;
__device__ const double kAtanTable[2 * QMC_ATAN_TABLE_ROWS] = QMC_ATAN_TABLE_INIT;

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Output i (0-based) of splitmix64 started at `state`.
__device__ __forceinline__ double splitmix_uniform(uint64_t state, uint64_t i) {
    uint64_t z = splitmix_mix(state + (i + 1) * kGamma);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// x >= 0 finite: compares on the bit pattern (integer pipe) instead of FP64
__device__ __forceinline__ bool nonneg_is_zero(double x) { return __double_as_longlong(x) == 0; }
__device__ __forceinline__ bool nonneg_ge_one(double x) {
    return __double_as_longlong(x) >= 0x3FF0000000000000LL;
}

// Lattice coordinate (steps "lattice index" and "shifted point"): RN(r/n) +
// delta folded into [0,1), every operation correctly rounded and never
// contracted. RN(r/n) comes from Markstein's correction with y = RN(1/n)
// computed on the host: q0 = RN(r y), rho = r - n q0 (exact by FMA: q0 is
// within 1.5 ulp of r/n and n < 2^32), q = RN(q0 + rho y). The corrected sum
// is within 1.5 * 2^-52 ulp of r/n, while r/n (n < 2^32, not a midpoint
// because its odd denominator part does not divide r, or else it is a short
// dyadic) lies at least 1/(2n) > 2^-33 ulp away from any rounding midpoint,
// so q is exactly the correctly rounded quotient.
// Exact doubles from integer operations on the bits (integer pipe):
// u32_to_double(r) = r for r < 2^32; frac_of_one_two(x) = x - 1 for x in [1, 2).
__device__ __forceinline__ double u32_to_double(uint64_t r) {
    if (r == 0) return 0.0;
    const int p = 63 - __clzll((long long)r);                          // leading bit, 0..31
    const uint64_t mant = (r << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
    return __longlong_as_double((long long)(((uint64_t)(1023 + p) << 52) | mant));
}
__device__ __forceinline__ double frac_of_one_two(double x) {
    const uint64_t f = (uint64_t)__double_as_longlong(x) & 0x000FFFFFFFFFFFFFULL;   // (x - 1) 2^52
    if (f == 0) return 0.0;
    const int p = 63 - __clzll((long long)f);                          // 0..51
    const uint64_t mant = (f << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
    return __longlong_as_double((long long)(((uint64_t)(1023 + p - 52) << 52) | mant));
}

__device__ __forceinline__ double lattice_coord(uint64_t r, double nd, double inv_n, double delta) {
    const double rd = u32_to_double(r);
    const double q0 = __dmul_rn(rd, inv_n);
    const double rho = __fma_rn(-q0, nd, rd);
    const double q = __fma_rn(rho, inv_n, q0);
    const double x = __dadd_rn(q, delta);
    return nonneg_ge_one(x) ? frac_of_one_two(x) : x;   // x - 1 is exact for x in [1, 2)
}

// The same coordinate on the integer pipe. One lattice coordinate is walked
// as r = k z mod n together with the exact binary expansion of r/n to 64
// places: Q = floor(r 2^64 / n), R = r 2^64 mod n (n < 2^32). Stepping k by
// one adds (Qz, Rz), the expansion of z/n, with a carry from R into Q;
// modulo 2^64 the wrap of r needs no correction. When r/n >= 2^-12
// (Q >= 2^52) the 53-bit rounding of r/n is read off Q with R as the sticky
// part (r/n is never a rounding midpoint, see above), RN(r/n) is then a
// multiple of 2^-64, and so is delta (the shifts are multiples of 2^-53):
// their sum is exact in 64 bits plus a carry, and its IEEE rounding and the
// fold are integer operations. The rare coordinates with r/n < 2^-12 take
// the FP64 steps. Both give the bits of lattice_coord.
struct LatticeWalk {
    uint64_t Q;
    uint32_t r, R;
};

// floor(a 2^64 / n) and a 2^64 mod n for a < n < 2^32: two long-division
// steps of 32 bits each
__host__ __device__ __forceinline__ void fixdiv64(uint64_t a, uint64_t n, uint64_t &q, uint64_t &rem) {
    const uint64_t h = a << 32;
    const uint64_t q1 = h / n, r1 = h - q1 * n;
    const uint64_t l = r1 << 32;
    const uint64_t q0 = l / n;
    q = (q1 << 32) | q0;
    rem = l - q0 * n;
}

__device__ __forceinline__ void walk_init(LatticeWalk &w, uint64_t r0, uint64_t n) {
    uint64_t R;
    w.r = (uint32_t)r0;
    fixdiv64(r0, n, w.Q, R);
    w.R = (uint32_t)R;
}

// One step k -> k + 1 with z, rz < n < 2^32. A 32-bit sum of two residues
// may wrap; a wrapped sum exceeds n as well, and subtracting n modulo 2^32
// gives the residue either way.
__device__ __forceinline__ void walk_step(LatticeWalk &w, uint32_t z, uint64_t qz, uint32_t rz, uint32_t n) {
    const uint32_t rn = w.r + z;
    w.r = (rn >= n || rn < w.r) ? rn - n : rn;
    const uint32_t R = w.R + rz;
    const bool c = R >= n || R < w.R;
    w.R = c ? R - n : R;
    w.Q += qz + (c ? 1ULL : 0ULL);
}

// RN(s 2^-64) for s < 2^64 (integer operations on the bits)
__device__ __forceinline__ double fix64_to_double_rn(uint64_t s) {
    if (s < (1ULL << 53)) {                     // at most 53 significant bits: exact
        if (s == 0) return 0.0;
        const int p = 63 - __clzll((long long)s);
        const uint64_t mant = (s << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
        return __longlong_as_double((long long)(((uint64_t)(1023 + p - 64) << 52) | mant));
    }
    const int sh = 11 - __clzll((long long)s);   // 1..11 dropped bits
    uint64_t m = s >> sh;
    const uint64_t dropped = s & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
    m += (dropped > half || (dropped == half && (m & 1))) ? 1 : 0;
    // s 2^-64 = m 2^(sh - 64), m in [2^52, 2^53]: a carry moves into the exponent
    return __longlong_as_double((long long)(((uint64_t)(1023 + 52 + sh - 64 - 1) << 52) + m));
}

// delta as a multiple of 2^-64, if it is one (delta in [0, 1))
__device__ __forceinline__ bool delta_fix(double delta, uint64_t &D) {
    const uint64_t b = (uint64_t)__double_as_longlong(delta);
    D = 0;
    if (b == 0) return true;
    const int e = (int)(b >> 52) - 1023;        // delta = 1.f 2^e, e <= -1
    if (e >= 0 || e < -1022) return false;
    const uint64_t mant = (b & 0x000FFFFFFFFFFFFFULL) | (1ULL << 52);
    const int sh = 64 + e - 52;                 // delta 2^64 = mant 2^sh
    if (sh >= 0) {
        D = mant << sh;
        return true;
    }
    if (sh < -52 || (mant & ((1ULL << -sh) - 1))) return false;
    D = mant >> -sh;
    return true;
}

// The coordinate of the walk with shift delta (D = delta 2^64 when dfix_ok)
__device__ __forceinline__ double walk_coord(const LatticeWalk &w, uint32_t n, double nd, double inv_n, double delta,
                                             uint64_t D, bool dfix_ok) {
    const uint64_t Q = w.Q;
    if (!dfix_ok || Q < (1ULL << 52)) return lattice_coord(w.r, nd, inv_n, delta);
    // RN(r/n) 2^64: keep 53 bits of Q, round with the dropped bits and R/n
    const int sh = 11 - __clzll((long long)Q);   // 0..11
    uint64_t m = Q >> sh;
    bool up;
    if (sh == 0) {
        up = 2 * (uint64_t)w.R > n || (2 * (uint64_t)w.R == n && (m & 1));
    } else {
        const uint64_t dropped = Q & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
        up = dropped > half || (dropped == half && (w.R != 0 || (m & 1)));
    }
    const uint64_t q = (m + (up ? 1 : 0)) << sh;   // < 2^64: r/n <= 1 - 1/n
    const uint64_t sum = q + D;
    if (sum >= q) {                                 // q + delta < 1; a sum rounded to 1 folds to 0
        const double x = fix64_to_double_rn(sum);
        return nonneg_ge_one(x) ? 0.0 : x;
    }
    // q + delta in [1, 2): round to the 2^-52 grid (ties to even on bit 12),
    // then subtract 1; a sum rounded up to 2 folds to 0
    uint64_t y = sum >> 12;
    const uint64_t low = sum & 0xFFF;
    y += (low > 0x800 || (low == 0x800 && (y & 1))) ? 1 : 0;
    if (y >= (1ULL << 52)) return 0.0;
    if (y == 0) return 0.0;
    const int p = 63 - __clzll((long long)y);
    const uint64_t mant = (y << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
    return __longlong_as_double((long long)(((uint64_t)(1023 + p - 52) << 52) | mant));
}

// korobov3 on the integer pipe for u in (0, 1): t = phi(u) = u^4 P(u),
// P(u) = 35 - 84u + 70u^2 - 20u^3; 1 - t = phi(1 - u); and ws = u (1 - u)
// (the weight is 140^d prod ws^3).
// phi(x) for x = M 2^(e-63) (M a normalised 64-bit mantissa) with
// X = floor(x 2^64): x^2 and x^4 are mantissa products kept to 64 bits
// (truncated); P runs by Horner on X with nonnegative intermediate values,
// for x < 1/2 as 35 - x(84 - x(70 - 20x)) in Q57 (P >= 8 there), for
// x >= 1/2 in y = 1 - x as 1 + y(4 + y(10 + 20y)) in Q59 (P >= 1), with
// y 2^64 = 2^64 - X. t takes x = u from the mantissa of u; 1 - t takes
// x = 1 - u from V = 2^64 - U, which is exact for u >= 2^-11 (else within
// 2^-64 relative). Each result is one 128-bit product rounded once to
// nearest: within about 0.53 ulp of the exact values for this u.
// RN((a b) 2^x) for a b > 0; 0 where the result would not be normal
__device__ __forceinline__ double round_pack(uint64_t a, uint64_t b, int x) {
    const qmc_u128 r = (qmc_u128)a * b;
    const uint64_t hi = (uint64_t)(r >> 64), lo = (uint64_t)r;
    if ((hi | lo) == 0) return 0.0;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    const int E = 127 - lz + x;                       // leading bit 2^E
    if (E < -1022) return 0.0;
    const qmc_u128 N = r << lz;
    const uint64_t nh = (uint64_t)(N >> 64), nl = (uint64_t)N;
    uint64_t mant = nh >> 11;
    const bool round_bit = ((nh >> 10) & 1) != 0, sticky = (nh & 0x3FF) != 0 || nl != 0;
    mant += (round_bit && (sticky || (mant & 1))) ? 1 : 0;
    return __longlong_as_double((long long)(((uint64_t)(1023 + E - 1) << 52) + mant));
}

__device__ __forceinline__ double korobov_phi_fix(uint64_t M, int e, uint64_t X) {
    uint64_t P;
    int pq;
    if (X < (1ULL << 63)) {
        const uint64_t a1 = (70ULL << 57) - __umul64hi(X, 20ULL << 57);
        const uint64_t a2 = (84ULL << 57) - __umul64hi(X, a1);
        P = (35ULL << 57) - __umul64hi(X, a2);
        pq = 57;
    } else {
        const uint64_t Y = 0 - X;
        const uint64_t a1 = (10ULL << 59) + __umul64hi(Y, 20ULL << 59);
        const uint64_t a2 = (4ULL << 59) + __umul64hi(Y, a1);
        P = (1ULL << 59) + __umul64hi(Y, a2);
        pq = 59;
    }
    const uint64_t p2 = __umul64hi(M, M);             // x^2 = p2 2^(2e - 62)
    const uint64_t p4 = __umul64hi(p2, p2);           // x^4 = p4 2^(4e - 60)
    return round_pack(p4, P, 4 * e - 60 - pq);
}

template <bool OMT>
__device__ __forceinline__ void korobov3_int(double u, double &t, double &omt, double &ws) {
    const uint64_t b = (uint64_t)__double_as_longlong(u);
    const int e = (int)(b >> 52) - 1023;              // -1022 <= e <= -1 for a normal u < 1
    const uint64_t mu = (b & 0x000FFFFFFFFFFFFFULL) | (1ULL << 52);
    const int s = e + 12;                             // u 2^64 = mu 2^s
    const uint64_t U = s >= 0 ? mu << s : (s > -53 ? mu >> -s : 0);
    const uint64_t V = U ? 0 - U : ~0ULL;             // (1 - u) 2^64 (u < 2^-64: 2^64 - 1)
    t = korobov_phi_fix(mu << 11, e, U);
    if (OMT) {
        const int lz = __clzll((long long)V);         // V >= 2^11
        omt = korobov_phi_fix(V << lz, -1 - lz, V);
    }
    ws = round_pack(mu, V, e - 52 - 64);
}

__device__ __noinline__ double walk_coord_call(uint64_t Q, uint32_t r, uint32_t R, uint32_t n, double nd,
                                               double inv_n, double delta, uint64_t D) {
    LatticeWalk w;
    w.Q = Q;
    w.r = r;
    w.R = R;
    return walk_coord(w, n, nd, inv_n, delta, D, true);
}

struct K3 {
    double t, omt, ws;
};
__device__ __noinline__ K3 korobov3_call(double u) {
    K3 r{0.0, 1.0, 0.0};
    korobov3_int<false>(u, r.t, r.omt, r.ws);
    return r;
}

// Natural logarithm: the fixed-point evaluation of qmc_ilog.h on the integer
// pipe (Tang's reduction with a 1025-row table; within 0.501 ulp). `tab` is
// the table of that header, staged in shared memory.
__device__ __forceinline__ double qlog(double x, const uint64_t *tab) { return qmc_ilog(x, tab); }

// The same logarithm as one out-of-line function. The fixed-order d <= 6
// kernel takes up to about twenty logarithms per evaluation; inlined, their
// copies overflow the SM's instruction cache (warps then stall on
// instruction fetch), so that kernel calls this single copy instead.
// QMC_LOG_CALL: bit 0 for the d <= 6 kernel, bit 1 for the d <= 3 kernel.
#ifndef QMC_LOG_CALL
#define QMC_LOG_CALL 1
#endif
// korobov3 out of line in the d <= 6 fixed-order kernel (same reason;
// measured: +7 % on the double box over the inlined form, after the
// logarithm's +18 %; the d <= 3 kernel runs 2 % faster with its logarithm
// inlined)
#ifndef QMC_KOROBOV_CALL
#define QMC_KOROBOV_CALL 1
#endif
// the lattice coordinate out of line as well (+1 % on the double box)
#ifndef QMC_WALK_CALL
#define QMC_WALK_CALL 1
#endif
__device__ __noinline__ double qlog_call(double x, const uint64_t *tab) { return qmc_ilog(x, tab); }

// Reciprocal by Newton-Raphson (y <- y + y (1 - x y), quadratic convergence)
// from the hardware approximation rcp.approx.ftz.f64, two steps: not
// correctly rounded, within about 1 ulp for normal x (checked against
// CUDA's correctly rounded reciprocal).
__device__ __forceinline__ double qrcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// Two-argument arctangent of finite (y, x), not both zero, table-driven:
// with mn <= mx the smaller and larger of |x|, |y| and c = j/64 nearest
// mn/mx (the index from an FP32 estimate), atan(mn/mx) = atan(c) +
// atan(delta), delta = (mn - c mx) / (mx + c mn) (one division, |delta| <=
// 2^-7); atan(delta) by its Taylor series to delta^7 (truncation below
// 2^-58 relative); then the octant: pi/2 - r where |y| > |x|, pi - r where
// x < 0 (sign bit, so -0 counts), and the sign of y. Measured worst case
// about 2 ulp. 19 FP64 operations. `tab` holds rows {atan(j/64) hi, lo}.
__device__ __forceinline__ double qatan2(double y, double x, const double *tab) {
    const long long xb = __double_as_longlong(x), yb = __double_as_longlong(y);
    const long long ab = xb & 0x7FFFFFFFFFFFFFFFLL, bb = yb & 0x7FFFFFFFFFFFFFFFLL;
    const bool swap = bb > ab;
    const long long mnb = swap ? ab : bb, mxb = swap ? bb : ab;
    const double mn = __longlong_as_double(mnb), mx = __longlong_as_double(mxb);
    int j = 0;
    const int de = (int)(mxb >> 52) - (int)(mnb >> 52);
    if (de <= 7 && mnb != 0) {
        const float fmn = __int_as_float(0x3F800000 | (int)((mnb >> 29) & 0x7FFFFF));
        const float fmx = __int_as_float(0x3F800000 | (int)((mxb >> 29) & 0x7FFFFF));
        const float w = __fdividef(fmn, fmx) * __int_as_float((127 - de) << 23);
        j = min(__float2int_rn(w * 64.0f), 64);
    }
    // c = j / 64 from the bits of j
    const double c = j ? __longlong_as_double(__double_as_longlong(u32_to_double((uint64_t)j)) - (6LL << 52)) : 0.0;
    const double num = fma(-c, mx, mn);
    const double den = fma(c, mn, mx);
    const double dl = num * qrcp(den);
    const double s2 = dl * dl;
    const double q = fma(fma(s2, -1.0 / 7.0, 0.2), s2, -1.0 / 3.0);
    double r = tab[2 * j] + (tab[2 * j + 1] + fma(dl * s2, q, dl));
    if (swap) r = (QMC_PIO2_HI - r) + QMC_PIO2_LO;
    if (xb < 0) r = (QMC_PI_HI - r) + QMC_PI_LO;
    return __longlong_as_double(__double_as_longlong(r) ^ (yb & (long long)0x8000000000000000ULL));
}

// ---------------------------------------------------------------- complex
struct dc {
    double re, im;
};
__device__ __forceinline__ dc C(double r, double i = 0.0) { return dc{r, i}; }
__device__ __forceinline__ dc operator+(dc a, dc b) { return dc{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ dc operator-(dc a, dc b) { return dc{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ dc operator*(dc a, dc b) {
    return dc{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ dc operator*(dc a, double s) { return dc{a.re * s, a.im * s}; }
__device__ __forceinline__ dc cinv(dc a) {
    double q = qrcp(fma(a.re, a.re, a.im * a.im));
    return dc{a.re * q, -a.im * q};
}
__device__ __forceinline__ dc conj_(dc a) { return dc{a.re, -a.im}; }
__device__ __forceinline__ double norm_(dc a) { return fma(a.re, a.re, a.im * a.im); }
// FP32 estimate of the principal argument (branch bookkeeping only); `m0`:
// on the negative real axis take -pi (the F - i0 prescription)
__device__ __forceinline__ float arg32(dc a, bool m0) {
    float im = __double2float_rn(a.im);
    if (m0 && (__double_as_longlong(a.im) << 1) == 0) im = -0.0f;
    return atan2f(im, __double2float_rn(a.re));
}
// Principal log; on the real axis the argument is taken from below
// (x - i0), the prescription of F - i0.
__device__ __forceinline__ dc clog_m0(dc a, const uint64_t *tab, const double *atab) {
    double arg = (a.im == 0.0) ? (a.re < 0.0 ? -CUDART_PI : 0.0) : qatan2(a.im, a.re, atab);
    return dc{0.5 * qlog(fma(a.re, a.re, a.im * a.im), tab), arg};
}
__device__ __forceinline__ dc cexp_(dc a) {
    double s, c;
    sincos(a.im, &s, &c);
    double e = exp(a.re);
    return dc{e * c, e * s};
}

// complex FP32 (mixed-precision monomial products of the deformed evaluator)
struct fc {
    float re, im;
};
__device__ __forceinline__ fc operator+(fc a, fc b) { return fc{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ fc operator*(fc a, fc b) {
    return fc{fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ fc to_fc(dc a) { return fc{__double2float_rn(a.re), __double2float_rn(a.im)}; }
__device__ __forceinline__ dc to_dc(fc a) { return dc{(double)a.re, (double)a.im}; }

// scalar-generic helpers
__device__ __forceinline__ float mulsc(float a, float s) { return a * s; }
__device__ __forceinline__ fc mulsc(fc a, float s) { return fc{a.re * s, a.im * s}; }
__device__ __forceinline__ double mulsc(double a, double s) { return a * s; }
__device__ __forceinline__ dc mulsc(dc a, double s) { return a * s; }
template <class T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ dc zero<dc>() { return dc{0.0, 0.0}; }
template <> __device__ __forceinline__ fc zero<fc>() { return fc{0.0f, 0.0f}; }
template <class T> __device__ __forceinline__ T from_real(double);
template <> __device__ __forceinline__ float from_real<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double from_real<double>(double x) { return x; }
template <> __device__ __forceinline__ dc from_real<dc>(double x) { return dc{x, 0.0}; }
template <> __device__ __forceinline__ fc from_real<fc>(double x) { return fc{(float)x, 0.0f}; }
template <class T> __device__ __forceinline__ T one() { return from_real<T>(1.0); }
__device__ __forceinline__ double re_of(double a) { return a; }
__device__ __forceinline__ double re_of(dc a) { return a.re; }
__device__ __forceinline__ double im_of(double) { return 0.0; }
__device__ __forceinline__ double im_of(dc a) { return a.im; }

// x^e for 0 <= e <= QMC_EMAX from the power table p[q] = x^(q+1)
template <class T>
__device__ __forceinline__ T pow_sel(const T (&p)[QMC_EMAX], uint32_t e) {
    T r = p[0];
    if (e == 2) r = p[1];
    if (e == 3) r = p[2];
    if (e == 4) r = p[3];
    return r;
}

// num *= x^e (e > 0) or den *= x^-e (e < 0), integer |e| <= QMC_EMAX
template <class T>
__device__ __forceinline__ void mul_ipow(T x, int e, T &num, T &den) {
    if (e == 0) return;
    int a = e > 0 ? e : -e;
    T p = x;
    for (int q = 1; q < a; ++q) p = p * x;
    if (e > 0) num = num * p;
    else den = den * p;
}

// ---------------------------------------------------------------- shared tile state
template <int LMAX>
struct TileSmem {
    QmcSectorDev sec;
    QmcJobDev job;
    uint32_t exps[QMC_MAXMONO];
    // the monomial as a list of factors t_j^e, decoded once per tile: bits 0..2
    // the factor count k (0..6), then k codes of 5 bits, code = 4 j + e - 1
    // (the row of x_j^e in a thread's power table)
    uint64_t mdesc[QMC_MAXMONO];
    double cval[QMC_MAXMONO];
    float cvalf[QMC_MAXMONO];
    double delta[QMC_DMAX];
    uint64_t dfix[QMC_DMAX];   // delta 2^64
    uint64_t qz[QMC_DMAX];     // floor(z 2^64 / n)
    uint32_t rz[QMC_DMAX];     // z 2^64 mod n
    uint32_t zmod[QMC_DMAX];   // z mod n
    double invb[QMC_SMAX];
    double invb_full;  // prod over the singular slots of 1/b_q (A of the full pole set)
    uint64_t logtab[3 * QMC_LOG_TABLE_ROWS];
    double atantab[2 * QMC_ATAN_TABLE_ROWS];
    double w140d;  // constant factor of the staged sector: its weight, times 140^d for korobov3
    unsigned long long tile;
    int cached_sector, cached_point;
    int job_index;
    double red[32][2 * LMAX];
};

// Polynomial value over monomials [m0, m1) of the staged table at a point given
// by its power table (real or complex).
template <int DMAX, class T, class CT>
__device__ __forceinline__ T poly_sum(const uint32_t *exps, const CT *cval, int m0, int m1,
                                      const T (&tp)[DMAX][QMC_EMAX]) {
    T s = zero<T>();
    for (int m = m0; m < m1; ++m) {
        const uint32_t e = exps[m];
        const CT c = cval[m];
        if (e == 0u) {                      // constant monomial
            s = (m == m0) ? from_real<T>(c) : s + from_real<T>(c);
            continue;
        }
        bool first = true;
        T v = from_real<T>(1.0);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            const uint32_t ej = (e >> (4 * j)) & 15u;
            if (ej) {
                const T p = pow_sel<T>(tp[j], ej);
                v = first ? p : v * p;
                first = false;
            }
        }
        s = (m == m0) ? mulsc(v, c) : s + mulsc(v, c);   // contracted into an FMA
    }
    return s;
}

// Polynomial value over monomials [m0, m1) from the decoded factor lists and
// the thread's power table in shared memory (row r of the thread at pt[r * S],
// S the block size): per factor one shared load and one multiply.
template <class T, class CT>
__device__ __forceinline__ T poly_sum_tab(const uint64_t *desc, const CT *cval, int m0, int m1, const T *pt,
                                          int stride) {
    T s = zero<T>();
    for (int m = m0; m < m1; ++m) {
        const uint64_t dsc = desc[m];
        const int k = (int)(dsc & 7u);
        const CT c = cval[m];
        if (k == 0) {                       // constant monomial
            s = (m == m0) ? from_real<T>(c) : s + from_real<T>(c);
            continue;
        }
        T v = pt[(int)((dsc >> 3) & 31u) * stride];
        for (int i = 1; i < k; ++i) v = v * pt[(int)((dsc >> (3 + 5 * i)) & 31u) * stride];
        s = (m == m0) ? mulsc(v, c) : s + mulsc(v, c);   // contracted into an FMA
    }
    return s;
}

// The thread's power table x_j^e (e = 1 .. emax <= prow) into rows prow j + e - 1
template <int DMAX, class T>
__device__ __forceinline__ void powers_tab(const T (&x)[DMAX], int d, int emax, int prow, T *pt, int stride) {
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            const T x1 = x[j];
            T *r = pt + prow * j * stride;
            r[0] = x1;
            if (emax >= 2) {
                const T x2 = x1 * x1;
                r[stride] = x2;
                if (emax >= 3) r[2 * stride] = x2 * x1;
                if (emax >= 4) r[3 * stride] = x2 * x2;
            }
        }
    }
}

template <int DMAX, class T>
__device__ __forceinline__ void powers(const T (&x)[DMAX], int d, int emax, T (&tp)[DMAX][QMC_EMAX]) {
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        tp[j][0] = x[j];
        tp[j][1] = x[j];
        tp[j][2] = x[j];
        tp[j][3] = x[j];
        if (j < d) {
            if (emax >= 2) tp[j][1] = x[j] * x[j];
            if (emax >= 3) tp[j][2] = tp[j][1] * x[j];
            if (emax >= 4) tp[j][3] = tp[j][1] * tp[j][1];
        }
    }
}

// Assemble the Laurent coefficients from per-corner B_V exp(eps Lambda_V):
//   f = sum_P eps^{-|P|} A_P D_P(eps) exp(eps E_P),
//   D_P = sum_{V superset of P} (-1)^{|V\P|} B_V exp(eps Lambda_V),
//   A_P = prod_{q in P} 1/b_q prod_{q not in P} 1/t_q,  E_P = sum_{q not in P} b_q ln t_q,
// which is the plus-distribution subtraction of every singular variable
// (each int_0^1 t^{-1+b eps} g = g(0)/(b eps) + int t^{-1+b eps}(g - g(0))).
// Only series terms that reach an order <= hi are formed: the corner V needs
// Lambda_V^i for i <= hi + |V|, the pole set P its product terms k <= hi + |P|.
// D_P comes from the corner series by the superset Moebius transform.
// res[o] receives the coefficient of eps^(lo+o).
template <int SMAX, int LMAX, class T>
__device__ __forceinline__ void assemble(int ns, int lo, int hi, int nord, const T (&BV)[1 << SMAX],
                                         const T (&LV)[1 << SMAX], const double (&it)[SMAX],
                                         const double (&lt)[SMAX], const double (&bq)[SMAX],
                                         const double (&invb)[SMAX], double A_empty, double A_full,
                                         T (&res)[LMAX]) {
    constexpr int NG = 1 << SMAX;
    const int full = (1 << ns) - 1;
    T g[NG][LMAX];
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        const int nV = hi + __popc(V) + 1;
#pragma unroll
        for (int i = 0; i < LMAX; ++i) g[V][i] = zero<T>();
        if (V > full || nV < 1) continue;
        g[V][0] = BV[V];
#pragma unroll
        for (int i = 1; i < LMAX; ++i)
            if (i < nV) g[V][i] = mulsc(g[V][i - 1] * LV[V], 1.0 / i);
    }
    // superset Moebius transform over the singular slots
#pragma unroll
    for (int q = 0; q < SMAX; ++q) {
        if (q >= ns) continue;
#pragma unroll
        for (int P = 0; P < NG; ++P) {
            if (P > full || (P & (1 << q))) continue;
            const int nP = hi + __popc(P) + 1;
#pragma unroll
            for (int i = 0; i < LMAX; ++i)
                if (i < nP) g[P][i] = g[P][i] - g[P | (1 << q)][i];
        }
    }
#pragma unroll
    for (int o = 0; o < LMAX; ++o) res[o] = zero<T>();
#pragma unroll
    for (int P = 0; P < NG; ++P) {
        if (P > full) continue;
        const int np = __popc(P);
        const int nP = hi + np + 1;
        if (nP < 1) continue;
        // A_P = prod_{q in P} 1/b_q prod_{q not in P} 1/t_q; the empty and the
        // full pole set come precomputed
        const bool Aknown = (P == 0) || (P == full);
        double A = P == 0 ? A_empty : (P == full ? A_full : 1.0), E = 0.0;
#pragma unroll
        for (int q = 0; q < SMAX; ++q) {
            if (q < ns) {
                if (P & (1 << q)) {
                    if (!Aknown) A *= invb[q];
                } else {
                    if (!Aknown) A *= it[q];
                    if (nP > 1) E = fma(bq[q], lt[q], E);
                }
            }
        }
        T PE[LMAX];
        if (P == full) {
            // every singular variable in the pole set: no exp(eps E_P) factor
#pragma unroll
            for (int k = 0; k < LMAX; ++k) PE[k] = (k < nP && k >= lo + np) ? g[P][k] : zero<T>();
        } else {
            double e[LMAX];
            e[0] = 1.0;
#pragma unroll
            for (int l = 1; l < LMAX; ++l) e[l] = (l < nP) ? e[l - 1] * E * (1.0 / l) : 0.0;
#pragma unroll
            for (int k = 0; k < LMAX; ++k) {
                PE[k] = zero<T>();
                if (k < nP && k >= lo + np) {
                    PE[k] = g[P][k];
#pragma unroll
                    for (int i = 0; i < k; ++i) PE[k] = PE[k] + mulsc(g[P][i], e[k - i]);
                }
            }
        }
        // res[o] += A * PE[lo + o + np] (index selected without local memory)
        const int shift = lo + np;
#pragma unroll
        for (int o = 0; o < LMAX; ++o) {
            if (o >= nord || o + shift < 0) continue;
            T sel = zero<T>();
#pragma unroll
            for (int k = 0; k < LMAX; ++k)
                if (k == o + shift) sel = PE[k];
            res[o] = res[o] + mulsc(sel, A);
        }
    }
}

// x^e for integer |e| <= QMC_EMAX with x^-1 supplied
template <class T>
__device__ __forceinline__ T ipow_signed(T x, T xinv, int e) {
    const T b = e < 0 ? xinv : x;
    const int a = e < 0 ? -e : e;
    T p = b;
    for (int q = 1; q < a; ++q) p = p * b;
    return a == 0 ? from_real<T>(1.0) : p;
}

// ---------------------------------------------------------------- real integrand
// MIXED: the monomial products and their group sums in FP32 (coefficients
// rounded to FP32), converted to FP64 before the subset sums; everything
// else (korobov3 weight, logs and powers of U and F, the series assembly and
// the reductions) stays FP64.
template <int DMAX, int SMAX, int LMAX, bool MIXED, int NS = -1>
__device__ __forceinline__ void eval_real(const TileSmem<LMAX> &S, const double (&t)[DMAX], int lo,
                                          int hi, int nord, double (&res)[LMAX]) {
    constexpr int NG = 1 << SMAX;
    const QmcSectorDev &sec = S.sec;
    // NS >= 0: the number of singular variables fixed at compile time (the
    // caller dispatches per tile), so the corner and pole-set loops are exact
    const int d = sec.d, ns = NS >= 0 ? NS : sec.ns;
    const uint64_t *tab = S.logtab;
    double tp[DMAX][QMC_EMAX];
    powers<DMAX, double>(t, d, sec.pad0, tp);

    // group sums by singular mask, then subset sums h[X] = sum_{M subset X} g[M];
    // the polynomial at corner V (t_V = 0) is h[(NG-1) ^ V].
    double hU[NG], hF[NG];
    if constexpr (MIXED) {
        float tf[DMAX], tpf[DMAX][QMC_EMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) tf[j] = __double2float_rn(t[j]);
        powers<DMAX, float>(tf, d, sec.pad0, tpf);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            hU[g] = 0.0;
            hF[g] = 0.0;
            if (g < (1 << ns)) {
                hU[g] = (double)poly_sum<DMAX, float>(S.exps, S.cvalf, sec.gU[g], sec.gU[g + 1], tpf);
                hF[g] = (double)poly_sum<DMAX, float>(S.exps, S.cvalf, sec.nU + sec.gF[g], sec.nU + sec.gF[g + 1], tpf);
            }
        }
    } else {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            hU[g] = 0.0;
            hF[g] = 0.0;
            if (g < (1 << ns)) {
                hU[g] = poly_sum<DMAX, double>(S.exps, S.cval, sec.gU[g], sec.gU[g + 1], tp);
                hF[g] = poly_sum<DMAX, double>(S.exps, S.cval, sec.nU + sec.gF[g], sec.nU + sec.gF[g + 1], tp);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < SMAX; ++q) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            if (g & (1 << q)) {
                if (q < ns) {
                    if (g < (1 << ns)) {
                        hU[g] += hU[g ^ (1 << q)];
                        hF[g] += hF[g ^ (1 << q)];
                    }
                } else {
                    hU[g] = hU[g ^ (1 << q)];
                    hF[g] = hF[g ^ (1 << q)];
                }
            }
        }
    }
    const bool need_lam = hi + ns >= 1;   // some corner needs its eps exponent

    // factors of the regular variables: prod t^{a_j} and sum b_j ln t_j
    double Cc = 1.0, Lc = 0.0;
    bool hasCc = false;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d && ((sec.regular_mask >> j) & 1)) {
            const int a = sec.a[j];
            if (a > 0) {
                Cc = hasCc ? Cc * pow_sel<double>(tp[j], (uint32_t)a) : pow_sel<double>(tp[j], (uint32_t)a);
                hasCc = true;
            }
            if (need_lam && sec.b[j] != 0.0) Lc = fma(sec.b[j], qlog(t[j], tab), Lc);
        }
    }
    // singular slots: 1/t, ln t (needed when a pole set without q has a term of order >= 1), b
    const bool need_lt = hi + ns - 1 >= 1;
    double it[SMAX], lt[SMAX], bq[SMAX];
#pragma unroll
    for (int q = 0; q < SMAX; ++q) {
        it[q] = 0.0;
        lt[q] = 0.0;
        bq[q] = 0.0;
        if (q < ns) {
            double tq = 1.0, bb = 0.0;
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
                if (j == sec.sing[q]) {
                    tq = t[j];
                    bb = sec.b[j];
                }
            it[q] = tq;   // the reciprocal follows below, in pairs
            bq[q] = bb;
            if (need_lt) lt[q] = qlog(tq, tab);
        }
    }
    // 1/t_q in pairs: 1/a = b / (a b), one reciprocal per pair; for two
    // singular variables that reciprocal is also A of the empty pole set
    double A_empty = 1.0;
    if (ns == 2) {
        const double r = qrcp(it[0] * it[1]);
        const double t0 = it[0];
        it[0] = it[1] * r;
        it[1] = t0 * r;
        A_empty = r;
    } else {
#pragma unroll
        for (int q = 0; q < SMAX; ++q)
            if (q < ns) it[q] = qrcp(it[q]);
        if (ns == 1) A_empty = it[0];
        else if (ns > 2) {
            A_empty = it[0];
#pragma unroll
            for (int q = 1; q < SMAX; ++q)
                if (q < ns) A_empty *= it[q];
        }
    }
    // corners: B_V = Cc U^u0 F^f0, Lambda_V = Lc + ln(U^u1 F^f1) (one log when
    // u1, f1 are small integers, else u1 ln U + f1 ln F)
    const int u0 = (int)sec.u0, f0 = (int)sec.f0, u1 = (int)sec.u1, f1 = (int)sec.f1;
    const bool comb = (sec.pad1 & 1) != 0;
    double BV[NG], LV[NG];
    const int full = (1 << ns) - 1;
    // 1/F at the corners that need it, in pairs of corners (V, V + 1)
    double FiV[NG];
#pragma unroll
    for (int V = 0; V < NG; V += 2) {
        const double Fa = hF[(NG - 1) ^ V], Fb = hF[(NG - 1) ^ (V + 1)];
        const bool na = V <= full && ((sec.f0_int && f0 < 0) || (hi + __popc(V) >= 1 && comb && f1 < 0));
        const bool nb = V + 1 <= full && ((sec.f0_int && f0 < 0) || (hi + __popc(V + 1) >= 1 && comb && f1 < 0));
        FiV[V] = 0.0;
        FiV[V + 1] = 0.0;
        if (na && nb) {
            const double r = qrcp(Fa * Fb);
            FiV[V] = Fb * r;
            FiV[V + 1] = Fa * r;
        } else if (na) {
            FiV[V] = qrcp(Fa);
        } else if (nb) {
            FiV[V + 1] = qrcp(Fb);
        }
    }
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        BV[V] = 0.0;
        LV[V] = 0.0;
        if (V > full) continue;
        const bool lam_here = hi + __popc(V) >= 1;
        const double U = hU[(NG - 1) ^ V];
        const double F = hF[(NG - 1) ^ V];
        const bool needUinv = (sec.u0_int && u0 < 0) || (lam_here && comb && u1 < 0);
        const double Ui = needUinv ? qrcp(U) : 0.0;
        const double Fi = FiV[V];
        // B = Cc U^u0 F^f0 without multiplications by unit factors (the
        // conditions are uniform over the tile's sector)
        double B = 1.0;
        bool unit = true;
        if (hasCc) {
            B = Cc;
            unit = false;
        }
        if (!sec.u0_int || u0 != 0) {
            const double pu = sec.u0_int ? ipow_signed<double>(U, Ui, u0) : exp(sec.u0 * qlog(U, tab));
            B = unit ? pu : B * pu;
            unit = false;
        }
        if (!sec.f0_int || f0 != 0) {
            const double pf = sec.f0_int ? ipow_signed<double>(F, Fi, f0) : exp(sec.f0 * qlog(F, tab));
            B = unit ? pf : B * pf;
        }
        BV[V] = B;
        if (lam_here) {
            double l;
            if (comb) l = qlog(ipow_signed<double>(U, Ui, u1) * ipow_signed<double>(F, Fi, f1), tab);
            else l = sec.u1 * qlog(U, tab) + sec.f1 * qlog(F, tab);
            LV[V] = Lc + l;
        }
    }
    double ib[SMAX];
#pragma unroll
    for (int q = 0; q < SMAX; ++q) ib[q] = S.invb[q];
    assemble<SMAX, LMAX, double>(ns, lo, hi, nord, BV, LV, it, lt, bq, ib, A_empty, S.invb_full, res);
}

// ---------------------------------------------------------------- fixed orders
// The assembly and the real integrand with the number of singular variables
// NS and the highest requested order HI fixed at compile time (the evaluator
// dispatches on them per tile): every series has its exact length, so no
// term beyond the requested orders is formed and no order is selected at run
// time. resN[i] receives the coefficient of eps^(i - NS), i = 0 .. NS + HI
// (the sector's leading pole eps^-NS up to eps^HI).
template <int NS> struct SlotArr {
    static constexpr int N = NS > 0 ? NS : 1;
};

// The real fixed-order kernels' corner stage on the integer pipe (qmc_xf.h)
// or in FP64: bit 0 for the d <= 6 kernel, bit 1 for the d <= 3 kernel.
// Measured (evaluations/s): the double box 9.40e8 -> 1.01e9 at n = 1000003
// with the integer corners; the box 4.28e9 with FP64 corners, 3.86e9 with
// integer ones (its corners are few, and the conversions cost more than the
// FP64 work they replace).
#ifndef QMC_XF_CORNERS
#define QMC_XF_CORNERS 1
#endif
// the pole sets' exponential series by Horner's rule (1) or by its powers (0)
#ifndef QMC_HORNER
#define QMC_HORNER 1
#endif
// the d <= 6 kernel's corner as one out-of-line function (1) or inlined with
// an out-of-line logarithm (0): inlined, its sixteen copies per tile path
// overflowed the instruction cache (8.3e8 evaluations/s on the double box)
#ifndef QMC_CORNER_CALL
#define QMC_CORNER_CALL 1
#endif

// Corner series B_V Lambda_V^i / i! in FP64, i < HI + |V| + 1
template <int NS, int HI>
__device__ __forceinline__ void series_fp64(const double (&BV)[1 << NS], const double (&LV)[1 << NS],
                                            double (&g)[1 << NS][HI + NS + 1]) {
    constexpr int NG = 1 << NS;
    constexpr int LM = HI + NS + 1;   // series length of the full corner
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        const int nV = HI + __popc(V) + 1;
        g[V][0] = BV[V];
#pragma unroll
        for (int i = 1; i < LM; ++i)
            if (i < nV) g[V][i] = i == 1 ? g[V][0] * LV[V] : (g[V][i - 1] * LV[V]) * (1.0 / i);
    }
}

// Superset Moebius transform of the corner series, in place:
// g[P][i] <- D_P coefficient i, D_P = sum_{V >= P} (-1)^|V\P| B_V exp(eps Lambda_V)
template <int NS, int HI>
__device__ __forceinline__ void moebius_fp64(double (&g)[1 << NS][HI + NS + 1]) {
    constexpr int NG = 1 << NS;
    constexpr int LM = HI + NS + 1;
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int P = 0; P < NG; ++P) {
            if (P & (1 << q)) continue;
            const int nP = HI + __popc(P) + 1;
#pragma unroll
            for (int i = 0; i < LM; ++i)
                if (i < nP) g[P][i] = g[P][i] - g[P | (1 << q)][i];
        }
}

// Assemble the Laurent coefficients from the Moebius-transformed corner
// series g[P][i] (above):
//   f = sum_P eps^{-|P|} A_P D_P(eps) exp(eps E_P),
//   A_P = prod_{q in P} 1/b_q prod_{q not in P} 1/t_q,  E_P = sum_{q not in P} b_q ln t_q.
template <int NS, int HI>
__device__ __forceinline__ void pole_sets_fixed(const double (&g)[1 << NS][HI + NS + 1],
                                                const double (&tb)[SlotArr<NS>::N],
                                                const double (&lt)[SlotArr<NS>::N],
                                                const double (&bq)[SlotArr<NS>::N], double A_empty,
                                                double A_full, double (&resN)[NS + HI + 1]) {
    constexpr int NG = 1 << NS;
    constexpr int LM = HI + NS + 1;   // series length of the full corner
    // A_P = prod_{q in P} 1/b_q prod_{q not in P} 1/t_q by the subset
    // recursion A_P = A_{P - q} t_q / b_q (q the lowest slot of P), and
    // E_P = sum_{q not in P} b_q ln t_q by E_P = E_{P + q} + b_q ln t_q (q the
    // lowest slot outside P), from E_full = 0
    double AP[NG], EP[NG], bl[SlotArr<NS>::N];
#pragma unroll
    for (int q = 0; q < NS; ++q) bl[q] = bq[q] * lt[q];
    AP[0] = A_empty;
#pragma unroll
    for (int P = 1; P < NG; ++P) AP[P] = P == NG - 1 ? A_full : AP[P & (P - 1)] * tb[__ffs(P) - 1];
    EP[NG - 1] = 0.0;
#pragma unroll
    for (int P = NG - 2; P >= 0; --P) {
        const int q = __ffs(~P) - 1;           // lowest slot outside P
        const int nP = HI + __popc(P) + 1;
        EP[P] = 0.0;
        if (nP > 1) EP[P] = (P | (1 << q)) == NG - 1 ? bl[q] : EP[P | (1 << q)] + bl[q];
    }
#pragma unroll
    for (int i = 0; i < LM; ++i) resN[i] = 0.0;
#pragma unroll
    for (int P = 0; P < NG; ++P) {
        const int np = __popc(P);
        const int nP = HI + np + 1;
        const double A = AP[P];
        double PE[LM];
        if (P == NG - 1) {
            // every singular variable in the pole set: no exp(eps E_P) factor
#pragma unroll
            for (int k = 0; k < LM; ++k)
                if (k < nP) PE[k] = g[P][k];
        } else {
            const double E = EP[P];
#if QMC_HORNER
            // PE_k = sum_{i <= k} g_i E^{k-i} / (k-i)! by Horner's rule:
            // PE_k = g_k + E (g_{k-1} + E/2 (g_{k-2} + E/3 (...)))
            double Ej[LM + 1];
            Ej[1] = E;
#pragma unroll
            for (int j = 2; j < LM; ++j)
                if (j < nP) Ej[j] = E * (1.0 / j);
#pragma unroll
            for (int k = 0; k < LM; ++k) {
                if (k >= nP) continue;
                double h = g[P][0];
#pragma unroll
                for (int i = 1; i < LM; ++i)
                    if (i <= k) h = fma(Ej[k - i + 1], h, g[P][i]);
                PE[k] = h;
            }
#else
            // the exponential series of E_P
            double e[LM];
            e[0] = 1.0;
#pragma unroll
            for (int l = 1; l < LM; ++l)
                if (l < nP) e[l] = l == 1 ? E : e[l - 1] * (E * (1.0 / l));
#pragma unroll
            for (int k = 0; k < LM; ++k) {
                if (k >= nP) continue;
                PE[k] = g[P][k];
#pragma unroll
                for (int i = 0; i < LM; ++i)
                    if (i < k) PE[k] = fma(g[P][i], e[k - i], PE[k]);
            }
#endif
        }
        // term k of pole set P is the order k - |P|
#pragma unroll
        for (int k = 0; k < LM; ++k)
            if (k < nP) resN[k - np + NS] = fma(PE[k], A, resN[k - np + NS]);
    }
}

// The logarithm of the fixed-order kernels: out of line for d <= 6 (see qlog_call)
template <int DMAX>
__device__ __forceinline__ double qlog_fx(double x, const uint64_t *tab) {
    if constexpr ((DMAX > 3 && (QMC_LOG_CALL & 1)) || (DMAX <= 3 && (QMC_LOG_CALL & 2))) return qlog_call(x, tab);
    else return qmc_ilog(x, tab);
}

// The corner stage in FP64 for sectors whose exponents are not all small
// integers (none of the built-in workloads): subset sums, 1/F in pairs of
// corners, B_V and Lambda_V per corner, the corner series and their Moebius
// transform.
template <int DMAX, int NS, int HI>
__device__ __forceinline__ void corners_fp64(const QmcSectorDev &sec, double (&hU)[1 << NS], double (&hF)[1 << NS],
                                          double Cc, bool hasCc, double Lc, bool hasLc, const uint64_t *tab,
                                          double (&gm)[1 << NS][HI + NS + 1]) {
    constexpr int NG = 1 << NS;
    // subset sums h[X] = sum_{M subset X} g[M]; the polynomial at corner V
    // (t_V = 0) is h[(NG-1) ^ V]
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int g = 0; g < NG; ++g)
            if (g & (1 << q)) {
                hU[g] += hU[g ^ (1 << q)];
                hF[g] += hF[g ^ (1 << q)];
            }
    // corners: B_V = Cc U^u0 F^f0, Lambda_V = Lc + ln(U^u1 F^f1) (one log when
    // u1, f1 are small integers, else u1 ln U + f1 ln F)
    const int u0 = (int)sec.u0, f0 = (int)sec.f0, u1 = (int)sec.u1, f1 = (int)sec.f1;
    const bool comb = (sec.pad1 & 1) != 0;
    double BV[NG], LV[NG];
    // 1/F at the corners that need it, in pairs of corners (V, V + 1)
    double FiV[NG];
#pragma unroll
    for (int V = 0; V < NG; V += 2) {
        const bool lamA = HI + __popc(V) >= 1;
        const double Fa = hF[(NG - 1) ^ V];
        const bool na = (sec.f0_int && f0 < 0) || (lamA && comb && f1 < 0);
        FiV[V] = 0.0;
        if (V + 1 < NG) {
            const bool lamB = HI + __popc(V + 1) >= 1;
            const double Fb = hF[(NG - 1) ^ (V + 1)];
            const bool nb = (sec.f0_int && f0 < 0) || (lamB && comb && f1 < 0);
            FiV[V + 1] = 0.0;
            if (na && nb) {
                const double r = qrcp(Fa * Fb);
                FiV[V] = Fb * r;
                FiV[V + 1] = Fa * r;
            } else if (na) {
                FiV[V] = qrcp(Fa);
            } else if (nb) {
                FiV[V + 1] = qrcp(Fb);
            }
        } else if (na) {
            FiV[V] = qrcp(Fa);
        }
    }
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        const bool lam_here = HI + __popc(V) >= 1;
        const double U = hU[(NG - 1) ^ V];
        const double F = hF[(NG - 1) ^ V];
        const bool needUinv = (sec.u0_int && u0 < 0) || (lam_here && comb && u1 < 0);
        const double Ui = needUinv ? qrcp(U) : 0.0;
        const double Fi = FiV[V];
        double B = 1.0;
        bool unit = true;
        if (hasCc) {
            B = Cc;
            unit = false;
        }
        if (!sec.u0_int || u0 != 0) {
            const double pu = sec.u0_int ? ipow_signed<double>(U, Ui, u0) : exp(sec.u0 * qlog_fx<DMAX>(U, tab));
            B = unit ? pu : B * pu;
            unit = false;
        }
        if (!sec.f0_int || f0 != 0) {
            const double pf = sec.f0_int ? ipow_signed<double>(F, Fi, f0) : exp(sec.f0 * qlog_fx<DMAX>(F, tab));
            B = unit ? pf : B * pf;
        }
        BV[V] = B;
        LV[V] = 0.0;
        if (lam_here) {
            double l;
            if (comb) l = qlog_fx<DMAX>(ipow_signed<double>(U, Ui, u1) * ipow_signed<double>(F, Fi, f1), tab);
            else l = fma(sec.u1, qlog_fx<DMAX>(U, tab), sec.f1 * qlog_fx<DMAX>(F, tab));
            LV[V] = hasLc ? Lc + l : l;
        }
    }
    series_fp64<NS, HI>(BV, LV, gm);
    moebius_fp64<NS, HI>(gm);
}

// One corner on the integer pipe: U, F at the corner (exact in 64-bit
// mantissas), their reciprocals where a negative exponent needs them,
// B = Cc U^u0 F^f0 and, where the corner needs its eps exponent,
// Lambda = Lc + ln(U^u1 F^f1); B rounded once to FP64 (the corner series and
// their Moebius transform stay in FP64 registers: in 64-bit-mantissa form
// they took twice the registers and spilled, -15 % on the double box).
// bad: a reciprocal of zero was needed.
struct XfCorner {
    double B;
    double L;
    int bad;
};
// the logarithm of a 64-bit mantissa: out of line in the d <= 6 kernel (its
// instruction cache; see qlog_call)
__device__ __noinline__ double qlog_xf_call(qmc_xf x, const uint64_t *tab) { return qmc_ilog_xf(x, tab); }
template <int DMAX>
__device__ __forceinline__ XfCorner corner_xf(double Ud, double Fd, double Cc, int u0, int f0, int u1, int f1,
                                              bool lam, bool hasLc, double Lc, const uint64_t *tab) {
    const qmc_xf U = qmc_xf_of(Ud), F = qmc_xf_of(Fd), Ccx = qmc_xf_of(Cc);
    const bool needU = u0 < 0 || (lam && u1 < 0);
    const bool needF = f0 < 0 || (lam && f1 < 0);
    XfCorner r;
    r.bad = (needU && U.m == 0) || (needF && F.m == 0);
    const qmc_xf rU = needU ? qmc_xf_rcp(U) : U;
    const qmc_xf rF = needF ? qmc_xf_rcp(F) : F;
    r.B = qmc_xf_to_double(qmc_xf_mul(Ccx, qmc_xf_mul(qmc_xf_ipow(U, rU, u0), qmc_xf_ipow(F, rF, f0))));
    r.L = 0.0;
    if (lam) {
        const qmc_xf X = qmc_xf_mul(qmc_xf_ipow(U, rU, u1), qmc_xf_ipow(F, rF, f1));
        double l;
        if constexpr (DMAX > 3 && QMC_CORNER_CALL == 0) l = qlog_xf_call(X, tab);
        else l = qmc_ilog_xf(X, tab);
        r.L = hasLc ? Lc + l : l;
    }
    return r;
}
// the whole corner out of line (one copy of its code, the logarithm inlined)
__device__ __noinline__ XfCorner corner_xf_call(double Ud, double Fd, double Cc, int u0, int f0, int u1, int f1,
                                                bool lam, bool hasLc, double Lc, const uint64_t *tab) {
    return corner_xf<6>(Ud, Fd, Cc, u0, f0, u1, f1, lam, hasLc, Lc, tab);
}

// Subset sums h[X] = sum_{M subset X} g[M] of one polynomial's group sums on
// the integer pipe (64-bit mantissas, each sum within 2^-62 of its larger
// operand), rounded once to FP64 in place: the polynomial at corner V
// (t_V = 0) is h[(NG-1) ^ V]
template <int NS>
__device__ __forceinline__ void subset_sums_xf(double (&h)[1 << NS]) {
    constexpr int NG = 1 << NS;
    qmc_xf x[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) x[g] = qmc_xf_of(h[g]);
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int g = 0; g < NG; ++g)
            if (g & (1 << q)) x[g] = qmc_xf_add(x[g], x[g ^ (1 << q)]);
#pragma unroll
    for (int g = 0; g < NG; ++g) h[g] = qmc_xf_to_double(x[g]);
}

// The corner stage on the integer pipe (qmc_xf.h): the subset sums of U and
// F, each corner's B_V and Lambda_V, then the corner series and their Moebius
// transform into gm. Returns true if some corner needed the reciprocal of a
// zero polynomial value.
template <int DMAX, int NS, int HI>
__device__ __forceinline__ bool corners_xf(double (&hU)[1 << NS], double (&hF)[1 << NS], double Cc, bool hasCc,
                                           double Lc, bool hasLc, int u0, int f0, int u1, int f1,
                                           const uint64_t *tab, double (&gm)[1 << NS][HI + NS + 1]) {
    constexpr int NG = 1 << NS;
    subset_sums_xf<NS>(hU);
    subset_sums_xf<NS>(hF);
    const double Cc1 = hasCc ? Cc : 1.0;
    double BV[NG], LV[NG];
    int bad = 0;
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        XfCorner c;
        if constexpr (DMAX > 3 && QMC_CORNER_CALL)
            c = corner_xf_call(hU[(NG - 1) ^ V], hF[(NG - 1) ^ V], Cc1, u0, f0, u1, f1, HI + __popc(V) >= 1, hasLc,
                               Lc, tab);
        else
            c = corner_xf<DMAX>(hU[(NG - 1) ^ V], hF[(NG - 1) ^ V], Cc1, u0, f0, u1, f1, HI + __popc(V) >= 1,
                                hasLc, Lc, tab);
        BV[V] = c.B;
        LV[V] = c.L;
        bad |= c.bad;
    }
    series_fp64<NS, HI>(BV, LV, gm);
    moebius_fp64<NS, HI>(gm);
    return bad != 0;
}

// ptd / ptf: this thread's column of the power table in shared memory (FP64
// and, for the mixed classes, FP32 view of the same storage), row stride
// `ps`, prow rows per variable
template <int DMAX, int NS, int HI, bool MIXED, int LMAX>
__device__ __forceinline__ void eval_real_fx(const TileSmem<LMAX> &S, const double (&t)[DMAX],
                                             double (&resN)[NS + HI + 1], double *ptd, float *ptf, int ps,
                                             int prow) {
    constexpr int NG = 1 << NS;
    constexpr int NSA = SlotArr<NS>::N;
    const QmcSectorDev &sec = S.sec;
    const int d = sec.d;
    const uint64_t *tab = S.logtab;
    // group sums by singular mask, then subset sums h[X] = sum_{M subset X} g[M];
    // the polynomial at corner V (t_V = 0) is h[(NG-1) ^ V]
    double hU[NG], hF[NG];
    if constexpr (MIXED) {
        float tf[DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) tf[j] = __double2float_rn(t[j]);
        powers_tab<DMAX, float>(tf, d, sec.pad0, prow, ptf, ps);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            hU[g] = (double)poly_sum_tab<float>(S.mdesc, S.cvalf, sec.gU[g], sec.gU[g + 1], ptf, ps);
            hF[g] = (double)poly_sum_tab<float>(S.mdesc, S.cvalf, sec.nU + sec.gF[g], sec.nU + sec.gF[g + 1], ptf, ps);
        }
    } else {
        powers_tab<DMAX, double>(t, d, sec.pad0, prow, ptd, ps);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            hU[g] = poly_sum_tab<double>(S.mdesc, S.cval, sec.gU[g], sec.gU[g + 1], ptd, ps);
            hF[g] = poly_sum_tab<double>(S.mdesc, S.cval, sec.nU + sec.gF[g], sec.nU + sec.gF[g + 1], ptd, ps);
        }
    }
    constexpr bool need_lam = HI + NS >= 1;   // some corner needs its eps exponent
    // factors of the regular variables: prod t^{a_j} and sum b_j ln t_j
    double Cc = 1.0, Lc = 0.0;
    bool hasCc = false, hasLc = false;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d && ((sec.regular_mask >> j) & 1)) {
            const int a = sec.a[j];
            if (a > 0) {
                // t_j^a: the FP64 power table, or (mixed classes, whose table is FP32) products
                const double p = MIXED ? ipow_signed<double>(t[j], 1.0, a) : ptd[(prow * j + a - 1) * ps];
                Cc = hasCc ? Cc * p : p;
                hasCc = true;
            }
            if (need_lam && sec.b[j] != 0.0) {
                const double l = qlog_fx<DMAX>(t[j], tab);
                Lc = hasLc ? fma(sec.b[j], l, Lc) : sec.b[j] * l;
                hasLc = true;
            }
        }
    }
    // singular slots: t, ln t (needed when a pole set without q has a term of
    // order >= 1 below HI), b
    constexpr bool need_lt = HI + NS - 1 >= 1;
    double it[NSA], lt[NSA], bq[NSA];
#pragma unroll
    for (int q = 0; q < NSA; ++q) {
        it[q] = 1.0;
        lt[q] = 0.0;
        bq[q] = 0.0;
        if (q < NS) {
            double tq = 1.0, bb = 0.0;
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
                if (j == sec.sing[q]) {
                    tq = t[j];
                    bb = sec.b[j];
                }
            it[q] = tq;
            bq[q] = bb;
            if (need_lt) lt[q] = qlog_fx<DMAX>(tq, tab);
        }
    }
    // t_q / b_q (the factors of the pole-set prefactors A_P), then 1/t_q in
    // pairs: 1/a = b / (a b) with one reciprocal per pair, whose value is also
    // the pair's share of A of the empty pole set prod 1/t_q
    double tb[NSA];
#pragma unroll
    for (int q = 0; q < NSA; ++q) tb[q] = q < NS ? it[q] * S.invb[q] : 0.0;
    double A_empty = 1.0;
#pragma unroll
    for (int q = 0; q + 1 < NS; q += 2) {
        const double r = qrcp(it[q] * it[q + 1]);
        const double t0 = it[q];
        it[q] = it[q + 1] * r;
        it[q + 1] = t0 * r;
        A_empty = q == 0 ? r : A_empty * r;
    }
    if constexpr (NS & 1) {
        it[NS - 1] = qrcp(it[NS - 1]);
        A_empty = NS == 1 ? it[0] : A_empty * it[NS - 1];
    }
    // corners: B_V = Cc U^u0 F^f0 and Lambda_V = Lc + ln(U^u1 F^f1) on the
    // integer pipe where every exponent is a small integer (the corner values
    // of U and F as 64-bit-mantissa subset sums), else in FP64; then the
    // corner series and their Moebius transform, and the pole sets
    double gm[NG][HI + NS + 1];
    constexpr bool xf_corners = (QMC_XF_CORNERS & (DMAX > 3 ? 1 : 2)) != 0;
    if (xf_corners && sec.u0_int && sec.f0_int && (sec.pad1 & 1)) {
        const bool bad = corners_xf<DMAX, NS, HI>(hU, hF, Cc, hasCc, Lc, hasLc, (int)sec.u0, (int)sec.f0, sec.u1i,
                                                  sec.f1i, tab, gm);
        pole_sets_fixed<NS, HI>(gm, tb, lt, bq, A_empty, S.invb_full, resN);
        if (bad) {
#pragma unroll
            for (int i = 0; i < NS + HI + 1; ++i) resN[i] = __longlong_as_double(0x7FF8000000000000LL);
        }
    } else {
        corners_fp64<DMAX, NS, HI>(sec, hU, hF, Cc, hasCc, Lc, hasLc, tab, gm);
        pole_sets_fixed<NS, HI>(gm, tb, lt, bq, A_empty, S.invb_full, resN);
    }
}

// ---------------------------------------------------------------- Taylor subtraction
// Sectors where some singular variables have a_q = -p_q, p_q >= 2 (undeformed).
// Per singular variable the integrand takes
//   t^{-p+b eps} g(t) + sum_{k<p} g_k [1/(k - p + 1 + b eps) - t^{k-p+b eps}],
// g_k the k-th Taylor coefficient of g at t_q = 0, so that its integral over
// [0,1] is that of t^{-p+b eps} g (the boundary terms g_k / (k - p + 1 + b eps)
// plus the integral of the remainder). Grouped by the set V of variables at
// t = 0, the terms of one V need the mixed Taylor coefficients G_kappa,
// kappa_q < p_q, of G = C U^{u0+u1 eps} F^{f0+f1 eps} at t_V = 0 (only U and F
// depend on t_V). Over the box of exponents, with U = U0 (1 + u) (u without
// constant term) and L_U = ln(1 + u) as truncated power series ("jets"),
//   U^{u0 + u1 eps} = U0^{u0} e^{eps u1 ln U0} exp(u0 L_U) exp(eps u1 L_U),
// and the same for F; with A = u0 L_U + f0 L_F and B = u1 L_U + f1 L_F,
//   G_kappa(eps) = C U0^{u0} F0^{f0} e^{eps Lam0} sum_i eps^i [exp(A) B^i / i!]_kappa,
// where B^i vanishes beyond the box's total degree. Then
//   f = sum_V base_V(eps) prod_{q not in V} t_q^{-p_q+b_q eps}
//         sum_kappa G_kappa(eps) prod_{q in V} phi_q(kappa_q; eps),
//   phi_q(k; eps) = 1/(k - p_q + 1 + b_q eps) - t_q^{k-p_q+b_q eps}.
// Plain run-time loops over series and jets in local memory: such sectors are
// few, and the code stays small.
namespace taylor {
// 1/k for k = 1..32 (k = 0 unused): series and jet recursions multiply by it
__device__ __constant__ double inv_k[33] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,
    1.0 / 9,    1.0 / 10,   1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17,
    1.0 / 18,   1.0 / 19,   1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26,
    1.0 / 27,   1.0 / 28,   1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32};

// Series: index i holds the order i - OFF. out = a b truncated above order hmax.
template <int NT, int OFF>
__device__ __forceinline__ void ser_mul(const double *a, const double *b, double *out, int hmax) {
#pragma unroll 1
    for (int i = 0; i < NT; ++i) {
        double v = 0.0;
        if (i - OFF <= hmax) {
#pragma unroll 1
            for (int k = 0; k < NT; ++k) {
                const int j = i + OFF - k;
                if (j >= 0 && j < NT) v = fma(a[k], b[j], v);
            }
        }
        out[i] = v;
    }
}

// c = a b over the box: index i has packed digits dig[i] (4 bits per jet
// dimension); a digit sum overflows its radix iff its nibble of
// dig[i] + dig[j] + off reaches 8 (off holds 8 - radix per nibble), and
// without overflow the flat index of the product term is i + j.
__device__ __forceinline__ void jet_mul(const double *a, const double *b, double *c, int J, const uint16_t *dig,
                                        uint32_t off) {
#pragma unroll 1
    for (int k = 0; k < J; ++k) c[k] = 0.0;
#pragma unroll 1
    for (int i = 0; i < J; ++i) {
        const double ai = a[i];
#pragma unroll 1
        for (int j = 0; i + j < J; ++j)
            if ((((uint32_t)dig[i] + dig[j] + off) & 0x8888u) == 0u) c[i + j] = fma(ai, b[j], c[i + j]);
    }
}
}  // namespace taylor

template <int DMAX, int SMAX, int LMAX, int JMAX>
__device__ __noinline__ void eval_real_taylor(const TileSmem<LMAX> &S, const double (&t)[DMAX], int lo, int hi,
                                              int nord, double (&res)[LMAX]) {
    constexpr int OFF = SMAX;            // series index i holds the order i - OFF
    constexpr int NT = SMAX + LMAX;
    constexpr int PMAX = QMC_PMAX;
    const QmcSectorDev &sec = S.sec;
    const int d = sec.d, ns = sec.ns;
    const uint64_t *tab = S.logtab;
    const int Hm = hi + ns;              // orders every factor must carry
    // regular factors C = prod t_j^{a_j} and Lc = sum b_j ln t_j; slot of each variable
    double Cc = 1.0, Lc = 0.0;
    int slot[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        slot[j] = -1;
        if (j < d && ((sec.regular_mask >> j) & 1)) {
            if (sec.a[j] > 0) Cc *= ipow_signed<double>(t[j], 1.0, sec.a[j]);
            if (sec.b[j] != 0.0) Lc = fma(sec.b[j], qlog(t[j], tab), Lc);
        }
    }
    // per singular slot: psi_q = t^{-p+b eps} (kept) and phi_q(k) (at t = 0)
    double psi[SMAX][NT];
    double phi[SMAX][PMAX][NT];
    int p[SMAX];
#pragma unroll 1
    for (int q = 0; q < ns; ++q) {
        const int j = sec.sing[q];
        slot[j] = q;
        p[q] = -sec.a[j];
        const double tq = t[j], tinv = qrcp(tq), bq = sec.b[j];
        const double bl = bq * qlog(tq, tab);
        const double rb = qrcp(bq);
        double E[NT];                    // e^{eps b ln t}: orders 0..Hm
#pragma unroll 1
        for (int i = 0; i < NT; ++i) E[i] = 0.0;
        double e = 1.0;
#pragma unroll 1
        for (int i = 0; i <= Hm; ++i) {
            E[OFF + i] = e;
            e = e * bl * taylor::inv_k[i + 1];
        }
        const double tp = ipow_signed<double>(tq, tinv, -p[q]);
#pragma unroll 1
        for (int i = 0; i < NT; ++i) psi[q][i] = tp * E[i];
#pragma unroll 1
        for (int k = 0; k < p[q]; ++k) {
            const double c = ipow_signed<double>(tq, tinv, k - p[q]);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) phi[q][k][i] = -c * E[i];
            const int m = k - p[q] + 1;  // 1/(m + b eps), m <= 0
            if (m == 0) {
                phi[q][k][OFF - 1] += rb;
            } else {
                double v = -taylor::inv_k[-m];
                const double r = -bq * v;
#pragma unroll 1
                for (int i = 0; i <= Hm; ++i) {
                    phi[q][k][OFF + i] += v;
                    v *= r;
                }
            }
        }
    }
    double tpw[DMAX][QMC_EMAX];
    powers<DMAX, double>(t, d, sec.pad0, tpw);
    double acc[NT];
#pragma unroll 1
    for (int i = 0; i < NT; ++i) acc[i] = 0.0;

    double ju[JMAX], jf[JMAX], ja[JMAX], jb[JMAX], jx[JMAX], jy[JMAX];
    double ei[LMAX][JMAX];
    uint16_t dig[JMAX];
#pragma unroll 1
    for (int V = 0; V < (1 << ns); ++V) {
        // jet dimensions: the slots in V with p >= 2
        int rad[SMAX], stride[SMAX];
        int J = 1, K = 0, nd = 0;
        uint32_t off = 0;
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            rad[q] = 1;
            stride[q] = 0;
            if (((V >> q) & 1) && p[q] > 1) {
                rad[q] = p[q];
                stride[q] = J;
                J *= p[q];
                K += p[q] - 1;
                off |= (uint32_t)(8 - p[q]) << (4 * nd);
                ++nd;
            }
        }
#pragma unroll 1
        for (int i = 0; i < J; ++i) {
            uint32_t w = 0;
            int n4 = 0;
#pragma unroll 1
            for (int q = 0; q < ns; ++q)
                if (rad[q] > 1) {
                    w |= (uint32_t)((i / stride[q]) % rad[q]) << (4 * n4);
                    ++n4;
                }
            dig[i] = (uint16_t)w;
            ju[i] = 0.0;
            jf[i] = 0.0;
        }
        // U and F over the box: monomials whose exponent in a zeroed variable
        // is beyond the box (or > 0 where p = 1) drop out
#pragma unroll 1
        for (int m = 0; m < sec.nU + sec.nF; ++m) {
            const uint32_t ex = S.exps[m];
            double v = S.cval[m];
            int idx = 0;
            bool keep = true;
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                const uint32_t ej = (ex >> (4 * j)) & 15u;
                if (j >= d || ej == 0u) continue;
                const int q = slot[j];
                if (q >= 0 && ((V >> q) & 1)) {
                    if ((int)ej >= rad[q]) keep = false;
                    else idx += (int)ej * stride[q];
                } else {
                    v *= pow_sel<double>(tpw[j], ej);
                }
            }
            if (!keep) continue;
            if (m < sec.nU) ju[idx] += v;
            else jf[idx] += v;
        }
        const double U0 = ju[0], F0 = jf[0];
        const double rU = qrcp(U0), rF = qrcp(F0);
        ju[0] = 0.0;
        jf[0] = 0.0;
#pragma unroll 1
        for (int i = 1; i < J; ++i) {
            ju[i] *= rU;
            jf[i] *= rF;
        }
        // L = ln(1 + x) = x h, h = sum_{k<K} (-1)^k x^k / (k + 1) by Horner
#pragma unroll 1
        for (int w = 0; w < 2; ++w) {
            double *x = w == 0 ? ju : jf;
#pragma unroll 1
            for (int i = 0; i < J; ++i) jy[i] = 0.0;
            jy[0] = ((K - 1) & 1 ? -1.0 : 1.0) * taylor::inv_k[K > 0 ? K : 1];
#pragma unroll 1
            for (int k = K - 2; k >= 0; --k) {
                taylor::jet_mul(x, jy, jx, J, dig, off);
#pragma unroll 1
                for (int i = 0; i < J; ++i) jy[i] = jx[i];
                jy[0] += (k & 1 ? -1.0 : 1.0) * taylor::inv_k[k + 1];
            }
            taylor::jet_mul(x, jy, jx, J, dig, off);
#pragma unroll 1
            for (int i = 0; i < J; ++i) x[i] = K > 0 ? jx[i] : 0.0;
        }
#pragma unroll 1
        for (int i = 0; i < J; ++i) {
            ja[i] = fma(sec.u0, ju[i], sec.f0 * jf[i]);
            jb[i] = fma(sec.u1, ju[i], sec.f1 * jf[i]);
        }
        // exp(A) = 1 + A (1 + A/2 (1 + A/3 (...))) by Horner
#pragma unroll 1
        for (int i = 0; i < J; ++i) jy[i] = 0.0;
        jy[0] = 1.0;
#pragma unroll 1
        for (int k = K; k >= 1; --k) {
            taylor::jet_mul(ja, jy, jx, J, dig, off);
            const double r = taylor::inv_k[k];
#pragma unroll 1
            for (int i = 0; i < J; ++i) jy[i] = jx[i] * r;
            jy[0] += 1.0;
        }
        // E_i = exp(A) B^i / i!, i <= min(K, Hm)
        const int Imax = K < Hm ? K : Hm;
#pragma unroll 1
        for (int i = 0; i < J; ++i) ei[0][i] = jy[i];
#pragma unroll 1
        for (int n = 1; n <= Imax; ++n) {
            taylor::jet_mul(ei[n - 1], jb, ei[n], J, dig, off);
            const double r = taylor::inv_k[n];
#pragma unroll 1
            for (int i = 0; i < J; ++i) ei[n][i] *= r;
        }
        // T = sum_kappa (sum_i eps^i E_i[kappa]) prod_{q in V} phi_q(kappa_q)
        double T[NT];
#pragma unroll 1
        for (int i = 0; i < NT; ++i) T[i] = 0.0;
#pragma unroll 1
        for (int kap = 0; kap < J; ++kap) {
            double P[NT], Q[NT];
            bool first = true;
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                if (!((V >> q) & 1)) continue;
                const int k = rad[q] > 1 ? (kap / stride[q]) % rad[q] : 0;
                if (first) {
#pragma unroll 1
                    for (int i = 0; i < NT; ++i) P[i] = phi[q][k][i];
                    first = false;
                } else {
                    taylor::ser_mul<NT, OFF>(P, phi[q][k], Q, Hm);
#pragma unroll 1
                    for (int i = 0; i < NT; ++i) P[i] = Q[i];
                }
            }
            if (first) {                 // V empty: the factor 1
#pragma unroll 1
                for (int i = 0; i < NT; ++i) P[i] = i == OFF ? 1.0 : 0.0;
            }
            double g[NT];
#pragma unroll 1
            for (int i = 0; i < NT; ++i) g[i] = (i >= OFF && i - OFF <= Imax) ? ei[i - OFF][kap] : 0.0;
            taylor::ser_mul<NT, OFF>(g, P, Q, Hm);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) T[i] += Q[i];
        }
        // base: C U0^{u0} F0^{f0} e^{eps Lam0} prod_{q not in V} psi_q
        double Bv = Cc;
        Bv *= sec.u0_int ? ipow_signed<double>(U0, rU, (int)sec.u0) : exp(sec.u0 * qlog(U0, tab));
        Bv *= sec.f0_int ? ipow_signed<double>(F0, rF, (int)sec.f0) : exp(sec.f0 * qlog(F0, tab));
        const double Lam = Lc + sec.u1 * qlog(U0, tab) + sec.f1 * qlog(F0, tab);
        double base[NT], Q[NT];
        double e = Bv;
#pragma unroll 1
        for (int i = 0; i < NT; ++i) base[i] = 0.0;
#pragma unroll 1
        for (int i = 0; i <= Hm; ++i) {
            base[OFF + i] = e;
            e = e * Lam * taylor::inv_k[i + 1];
        }
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            if ((V >> q) & 1) continue;
            taylor::ser_mul<NT, OFF>(base, psi[q], Q, Hm);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) base[i] = Q[i];
        }
        taylor::ser_mul<NT, OFF>(base, T, Q, Hm);
#pragma unroll 1
        for (int i = 0; i < NT; ++i) acc[i] += Q[i];
    }
#pragma unroll
    for (int o = 0; o < LMAX; ++o) {
        res[o] = 0.0;
#pragma unroll 1
        for (int i = 0; i < NT; ++i)
            if (o < nord && i == lo + o + OFF) res[o] = acc[i];
    }
}

// ---------------------------------------------------------------- deformed integrand
// z_j = t_j - i lambda_j t_j (1 - t_j) dF/dt_j at the (corner) point, with
// rho_j = z_j / t_j for singular variables and J = dz/dt; every quantity of
// G is recomputed at each corner t' = t with t_V = 0.
template <int DMAX, int SMAX, int LMAX, bool MIXED>
__device__ __forceinline__ void eval_deformed(const TileSmem<LMAX> &S, const double (&t)[DMAX],
                                              const double (&omt)[DMAX], int lo, int hi, int nord,
                                              dc (&res)[LMAX], int &signfail) {
    static_assert(DMAX <= 3, "deformed evaluator handles d <= 3");
    constexpr int NG = 1 << SMAX;
    const QmcSectorDev &sec = S.sec;
    const int d = sec.d, ns = sec.ns;
    const int full = (1 << ns) - 1;
    const int dbase = sec.nU + sec.nF;
    const uint64_t *tab = S.logtab;
    const double *atab = S.atantab;
    dc BV[NG], LV[NG];
    double it[SMAX], lt[SMAX], bq[SMAX];
#pragma unroll
    for (int q = 0; q < SMAX; ++q) {
        it[q] = 0.0;
        lt[q] = 0.0;
        bq[q] = 0.0;
        if (q < ns) {
            double tq = 1.0, bb = 0.0;
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
                if (j == sec.sing[q]) {
                    tq = t[j];
                    bb = sec.b[j];
                }
            it[q] = qrcp(tq);
            bq[q] = bb;
            if (hi + ns - 1 >= 1) lt[q] = qlog(tq, tab);
        }
    }
#pragma unroll
    for (int V = 0; V < NG; ++V) {
        BV[V] = zero<dc>();
        LV[V] = zero<dc>();
        if (V > full) continue;
        const bool lam_here = hi + __popc(V) >= 1;
        double tc[DMAX], oc[DMAX];
        bool issing[DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            tc[j] = t[j];
            oc[j] = omt[j];
            issing[j] = false;
        }
#pragma unroll
        for (int q = 0; q < SMAX; ++q) {
            if (q < ns) {
#pragma unroll
                for (int j = 0; j < DMAX; ++j)
                    if (j == sec.sing[q]) {
                        issing[j] = true;
                        if (V & (1 << q)) {
                            tc[j] = 0.0;
                            oc[j] = 1.0;
                        }
                    }
            }
        }
        // derivatives of F at the corner point (real); MIXED: FP32 monomial
        // products and sums, converted to FP64 for V and det J
        double dF[DMAX], H[DMAX][DMAX];
        if constexpr (MIXED) {
            float tcf[DMAX], tpf[DMAX][QMC_EMAX];
#pragma unroll
            for (int j = 0; j < DMAX; ++j) tcf[j] = __double2float_rn(tc[j]);
            powers<DMAX, float>(tcf, d, sec.pad0, tpf);
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                dF[j] = 0.0;
                if (j < d)
                    dF[j] = (double)poly_sum<DMAX, float>(S.exps, S.cvalf, dbase + sec.dFoff[j],
                                                          dbase + sec.dFoff[j] + sec.dFn[j], tpf);
            }
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
#pragma unroll
                for (int k = j; k < DMAX; ++k) {
                    H[j][k] = 0.0;
                    if (j < d && k < d) {
                        const int h = j * QMC_DMAX - j * (j - 1) / 2 + (k - j);  // host packing order
                        H[j][k] = (double)poly_sum<DMAX, float>(S.exps, S.cvalf, dbase + sec.Hoff[h],
                                                                dbase + sec.Hoff[h] + sec.Hn[h], tpf);
                    }
                    H[k][j] = H[j][k];
                }
        } else {
            double tp[DMAX][QMC_EMAX];
            powers<DMAX, double>(tc, d, sec.pad0, tp);
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                dF[j] = 0.0;
                if (j < d)
                    dF[j] = poly_sum<DMAX, double>(S.exps, S.cval, dbase + sec.dFoff[j],
                                                   dbase + sec.dFoff[j] + sec.dFn[j], tp);
            }
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
#pragma unroll
                for (int k = j; k < DMAX; ++k) {
                    H[j][k] = 0.0;
                    if (j < d && k < d) {
                        const int h = j * QMC_DMAX - j * (j - 1) / 2 + (k - j);  // host packing order
                        H[j][k] = poly_sum<DMAX, double>(S.exps, S.cval, dbase + sec.Hoff[h],
                                                         dbase + sec.Hoff[h] + sec.Hn[h], tp);
                    }
                    H[k][j] = H[j][k];
                }
        }
        // J = 1 - i V with V real: V_jk = lambda_j (t_j (1-t_j) H_jk + delta_jk (1 - 2 t_j) dF_j).
        // det(1 + X) = 1 + tr X + E2(X) + det X (E2: sum of principal 2 x 2
        // minors) with X = -i V gives det J = (1 - E2(V)) + i (det V - tr V) in
        // real arithmetic (d = 2: (1 - det V) - i tr V; d = 1: 1 - i V_00).
        dc z[DMAX];
        dc rho[DMAX];
        double Vm[DMAX][DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            const double lam = S.job.lambda[j];
            const double g = lam * oc[j] * dF[j];  // rho_j = 1 - i g
            z[j] = C(tc[j], -tc[j] * g);
            rho[j] = C(1.0, -g);
#pragma unroll
            for (int k = 0; k < DMAX; ++k)
                Vm[j][k] = lam * (tc[j] * oc[j] * H[j][k] + (j == k ? (oc[j] - tc[j]) * dF[j] : 0.0));
            if (j >= d) {
                z[j] = C(1.0);
                rho[j] = C(1.0);
            }
        }
        dc detJ;
        if (d == 1) {
            detJ = C(1.0, -Vm[0][0]);
        } else if (d == 2) {
            const double detV = fma(Vm[0][0], Vm[1][1], -Vm[0][1] * Vm[1][0]);
            detJ = C(1.0 - detV, -(Vm[0][0] + Vm[1][1]));
        } else {
            const double c00 = fma(Vm[1][1], Vm[2][2], -Vm[1][2] * Vm[2][1]);
            const double c01 = fma(Vm[1][0], Vm[2][2], -Vm[1][2] * Vm[2][0]);
            const double c02 = fma(Vm[1][0], Vm[2][1], -Vm[1][1] * Vm[2][0]);
            const double detV = fma(Vm[0][0], c00, fma(-Vm[0][1], c01, Vm[0][2] * c02));
            const double e2 = c00 + fma(Vm[0][0], Vm[1][1], -Vm[0][1] * Vm[1][0]) +
                              fma(Vm[0][0], Vm[2][2], -Vm[0][2] * Vm[2][0]);
            const double trV = Vm[0][0] + Vm[1][1] + Vm[2][2];
            detJ = C(1.0 - e2, detV - trV);
        }
        dc U, F;
        if constexpr (MIXED) {
            // U and F at z from FP32 complex monomial products; everything
            // after (powers and logs of U and F, det J, the assembly) is FP64
            fc zf[DMAX], zpf[DMAX][QMC_EMAX];
#pragma unroll
            for (int j = 0; j < DMAX; ++j) zf[j] = to_fc(z[j]);
            powers<DMAX, fc>(zf, d, sec.pad0, zpf);
            U = to_dc(poly_sum<DMAX, fc>(S.exps, S.cvalf, sec.gU[0], sec.nU, zpf));
            F = to_dc(poly_sum<DMAX, fc>(S.exps, S.cvalf, sec.nU, sec.nU + sec.nF, zpf));
        } else {
            dc zp[DMAX][QMC_EMAX];
            powers<DMAX, dc>(z, d, sec.pad0, zp);
            U = poly_sum<DMAX, dc>(S.exps, S.cval, sec.gU[0], sec.nU, zp);
            F = poly_sum<DMAX, dc>(S.exps, S.cval, sec.nU, sec.nU + sec.nF, zp);
        }
        if (F.im > 0.0) ++signfail;
        // all exponents integers: the corner's eps exponent is one complex log,
        // ln X with X = prod rho_j^b_j prod z_j^b_j U^u1 F^f1, whose imaginary
        // part is restored to the sum of the factors' principal arguments by the
        // multiple of 2 pi that an FP32 estimate of that sum selects
        const bool comb_all = (sec.pad1 & 3) == 3;
        dc num = detJ, den = one<dc>();
        dc lsum = zero<dc>();
        dc Xn = one<dc>(), Xd = one<dc>();
        float sarg = 0.0f;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j >= d) continue;
            if (issing[j]) {
                den = den * rho[j];
                if (lam_here && sec.b[j] != 0.0) {
                    if (comb_all) {
                        mul_ipow<dc>(rho[j], sec.bi[j], Xn, Xd);
                        sarg = fmaf((float)sec.bi[j], arg32(rho[j], false), sarg);
                    } else {
                        lsum = lsum + clog_m0(rho[j], tab, atab) * sec.b[j];
                    }
                }
            } else if ((sec.regular_mask >> j) & 1) {
                if (sec.a[j] != 0) mul_ipow<dc>(z[j], sec.a[j], num, den);
                if (lam_here && sec.b[j] != 0.0) {
                    if (comb_all) {
                        mul_ipow<dc>(z[j], sec.bi[j], Xn, Xd);
                        sarg = fmaf((float)sec.bi[j], arg32(z[j], false), sarg);
                    } else {
                        lsum = lsum + clog_m0(z[j], tab, atab) * sec.b[j];
                    }
                }
            }
        }
        const bool needU = (lam_here && sec.u1 != 0.0 && !comb_all) || !sec.u0_int;
        const bool needF = (lam_here && sec.f1 != 0.0 && !comb_all) || !sec.f0_int;
        dc lU = zero<dc>(), lF = zero<dc>();
        if (needU) lU = clog_m0(U, tab, atab);
        if (needF) lF = clog_m0(F, tab, atab);
        if (sec.u0_int) mul_ipow<dc>(U, (int)sec.u0, num, den);
        else num = num * cexp_(lU * sec.u0);
        if (sec.f0_int) mul_ipow<dc>(F, (int)sec.f0, num, den);
        else num = num * cexp_(lF * sec.f0);
        BV[V] = num * cinv(den);
        if (lam_here) {
            if (comb_all) {
                mul_ipow<dc>(U, sec.u1i, Xn, Xd);
                sarg = fmaf((float)sec.u1i, arg32(U, false), sarg);
                mul_ipow<dc>(F, sec.f1i, Xn, Xd);
                sarg = fmaf((float)sec.f1i, arg32(F, true), sarg);
                const dc X = Xn * conj_(Xd);                  // |Xd|^2 Xn / Xd
                const double phi = qatan2(X.im, X.re, atab);
                const float kf = rintf((sarg - __double2float_rn(phi)) * 0.15915494f);
                LV[V] = dc{0.5 * qlog(norm_(Xn) * qrcp(norm_(Xd)), tab),
                           fma((double)kf, 2.0 * CUDART_PI, phi)};
            } else {
                LV[V] = lsum + lU * sec.u1 + lF * sec.f1;
            }
        }
    }
    double ib[SMAX];
#pragma unroll
    for (int q = 0; q < SMAX; ++q) ib[q] = S.invb[q];
    double A_empty = 1.0;
#pragma unroll
    for (int q = 0; q < SMAX; ++q)
        if (q < ns) A_empty = q == 0 ? it[0] : A_empty * it[q];
    assemble<SMAX, LMAX, dc>(ns, lo, hi, nord, BV, LV, it, lt, bq, ib, A_empty, S.invb_full, res);
}

// ---------------------------------------------------------------- Taylor subtraction, deformed
// Deformed sectors (d <= 3, <= 2 singular variables) with some a_q <= -2.
// The subtraction is that of eval_real_taylor; the Taylor coefficients of
//   G = det J prod_{singular} rho_j^{a_j+b_j eps} prod_{regular} z_j^{a_j+b_j eps}
//       U(z)^{u0+u1 eps} F(z)^{f0+f1 eps}
// in the zeroed variables come from every quantity of the deformation formed
// on jets: dF/dt_j and d2F/dt_j dt_l from their monomial tables (t_V^e lands
// at entry e), g_j = lambda_j (1 - t_j) dF_j, rho_j = 1 - i g_j, z_j = t_j rho_j,
// det J = (1 - E2(V)) + i (det V - tr V) with V_jl = lambda_j (t_j (1 - t_j)
// d2F_jl + delta_jl (1 - 2 t_j) dF_j), U(z) and F(z) from complex jet powers of
// z. Each power factor P^{e0 + e1 eps} enters through L_P = ln P0 + ln(1 + x):
// with A = sum e0 L_P and B = sum e1 L_P, G = det J exp(A) exp(eps B), and
//   G(eps) = sum_i eps^i det J exp(A) B^i / i!.
// Complex jets in local memory, plain loops: such sectors are few.
namespace taylor {
// c = a b over the box for complex jets (see jet_mul)
__device__ __forceinline__ void cjet_mul(const dc *a, const dc *b, dc *c, int J, const uint16_t *dig, uint32_t off) {
#pragma unroll 1
    for (int k = 0; k < J; ++k) c[k] = dc{0.0, 0.0};
#pragma unroll 1
    for (int i = 0; i < J; ++i) {
        const dc ai = a[i];
#pragma unroll 1
        for (int j = 0; i + j < J; ++j)
            if ((((uint32_t)dig[i] + dig[j] + off) & 0x8888u) == 0u) {
                const dc bj = b[j];
                dc &r = c[i + j];
                r.re = fma(ai.re, bj.re, fma(-ai.im, bj.im, r.re));
                r.im = fma(ai.re, bj.im, fma(ai.im, bj.re, r.im));
            }
    }
}
// principal log; on the real axis the argument from below (m0: F - i0) or above
__device__ __forceinline__ dc clog_br(dc a, bool m0, const uint64_t *tab, const double *atab) {
    double arg = (a.im == 0.0) ? (a.re < 0.0 ? (m0 ? -CUDART_PI : CUDART_PI) : 0.0) : qatan2(a.im, a.re, atab);
    return dc{0.5 * qlog(fma(a.re, a.re, a.im * a.im), tab), arg};
}
}  // namespace taylor

template <int LMAX, int JMAX>
__device__ __noinline__ void eval_deformed_taylor(const TileSmem<LMAX> &S, const double (&t)[3], const double (&omt)[3],
                                                  int lo, int hi, int nord, dc (&res)[LMAX], int &signfail) {
    constexpr int SMAX = 2, DM = 3;
    constexpr int OFF = SMAX;
    constexpr int NT = SMAX + LMAX;
    constexpr int PMAX = QMC_PMAX;
    const QmcSectorDev &sec = S.sec;
    const int d = sec.d, ns = sec.ns;
    const int dbase = sec.nU + sec.nF;
    const uint64_t *tab = S.logtab;
    const double *atab = S.atantab;
    const int Hm = hi + ns;
    int slot[DM];
#pragma unroll
    for (int j = 0; j < DM; ++j) slot[j] = -1;
    // per singular slot: psi_q = t^{-p+b eps} (kept) and phi_q(k) (at t = 0)
    double psi[SMAX][NT];
    double phi[SMAX][PMAX][NT];
    int p[SMAX];
#pragma unroll 1
    for (int q = 0; q < ns; ++q) {
        const int j = sec.sing[q];
        slot[j] = q;
        p[q] = -sec.a[j];
        const double tq = t[j], tinv = qrcp(tq), bq = sec.b[j];
        const double bl = bq * qlog(tq, tab);
        const double rb = qrcp(bq);
        double E[NT];
#pragma unroll 1
        for (int i = 0; i < NT; ++i) E[i] = 0.0;
        double e = 1.0;
#pragma unroll 1
        for (int i = 0; i <= Hm; ++i) {
            E[OFF + i] = e;
            e = e * bl * taylor::inv_k[i + 1];
        }
        const double tp = ipow_signed<double>(tq, tinv, -p[q]);
#pragma unroll 1
        for (int i = 0; i < NT; ++i) psi[q][i] = tp * E[i];
#pragma unroll 1
        for (int k = 0; k < p[q]; ++k) {
            const double c = ipow_signed<double>(tq, tinv, k - p[q]);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) phi[q][k][i] = -c * E[i];
            const int m = k - p[q] + 1;
            if (m == 0) {
                phi[q][k][OFF - 1] += rb;
            } else {
                double v = -taylor::inv_k[-m];
                const double r = -bq * v;
#pragma unroll 1
                for (int i = 0; i <= Hm; ++i) {
                    phi[q][k][OFF + i] += v;
                    v *= r;
                }
            }
        }
    }
    double tpw[DM][QMC_EMAX];
    powers<DM, double>(t, d, sec.pad0, tpw);
    double acc_re[NT], acc_im[NT];
#pragma unroll 1
    for (int i = 0; i < NT; ++i) acc_re[i] = acc_im[i] = 0.0;

    double tj[DM][JMAX], oj[DM][JMAX], Fj[DM][JMAX], Hs[DM][DM][JMAX], gj[DM][JMAX], wk[JMAX], wk2[JMAX];
    dc zj[DM][JMAX], rj[DM][JMAX], zp[DM][QMC_EMAX][JMAX], cu[JMAX], cf[JMAX], cx[JMAX], cy[JMAX], cA[JMAX],
        cB[JMAX], dJ[JMAX];
    dc gi[LMAX][JMAX];
    uint16_t dig[JMAX];
#pragma unroll 1
    for (int V = 0; V < (1 << ns); ++V) {
        int rad[SMAX], stride[SMAX];
        int J = 1, K = 0, nd = 0;
        uint32_t off = 0;
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            rad[q] = 1;
            stride[q] = 0;
            if (((V >> q) & 1) && p[q] > 1) {
                rad[q] = p[q];
                stride[q] = J;
                J *= p[q];
                K += p[q] - 1;
                off |= (uint32_t)(8 - p[q]) << (4 * nd);
                ++nd;
            }
        }
#pragma unroll 1
        for (int i = 0; i < J; ++i) {
            uint32_t w = 0;
            int n4 = 0;
#pragma unroll 1
            for (int q = 0; q < ns; ++q)
                if (rad[q] > 1) {
                    w |= (uint32_t)((i / stride[q]) % rad[q]) << (4 * n4);
                    ++n4;
                }
            dig[i] = (uint16_t)w;
        }
        // t_j and 1 - t_j as jets
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
#pragma unroll 1
            for (int i = 0; i < J; ++i) tj[j][i] = oj[j][i] = 0.0;
            const int q = slot[j];
            if (q >= 0 && ((V >> q) & 1)) {
                oj[j][0] = 1.0;
                if (rad[q] > 1) {
                    tj[j][stride[q]] = 1.0;
                    oj[j][stride[q]] = -1.0;
                }
            } else {
                tj[j][0] = t[j];
                oj[j][0] = omt[j];
            }
        }
        // a polynomial's monomials [m0, m1) of the staged table as a jet
        auto poly_jet = [&](int m0, int m1, double *out) {
#pragma unroll 1
            for (int i = 0; i < J; ++i) out[i] = 0.0;
#pragma unroll 1
            for (int m = m0; m < m1; ++m) {
                const uint32_t ex = S.exps[m];
                double v = S.cval[m];
                int idx = 0;
                bool keep = true;
#pragma unroll
                for (int j = 0; j < DM; ++j) {
                    const uint32_t ej = (ex >> (4 * j)) & 15u;
                    if (j >= d || ej == 0u) continue;
                    const int q = slot[j];
                    if (q >= 0 && ((V >> q) & 1)) {
                        if ((int)ej >= rad[q]) keep = false;
                        else idx += (int)ej * stride[q];
                    } else {
                        v *= pow_sel<double>(tpw[j], ej);
                    }
                }
                if (keep) out[idx] += v;
            }
        };
#pragma unroll 1
        for (int j = 0; j < d; ++j) poly_jet(dbase + sec.dFoff[j], dbase + sec.dFoff[j] + sec.dFn[j], Fj[j]);
#pragma unroll 1
        for (int j = 0; j < d; ++j)
#pragma unroll 1
            for (int l = j; l < d; ++l) {
                const int h = j * QMC_DMAX - j * (j - 1) / 2 + (l - j);   // host packing order
                poly_jet(dbase + sec.Hoff[h], dbase + sec.Hoff[h] + sec.Hn[h], Hs[j][l]);
#pragma unroll 1
                for (int i = 0; i < J; ++i) Hs[l][j][i] = Hs[j][l][i];
            }
        // g_j, rho_j = 1 - i g_j, z_j = t_j rho_j, and V_jl into Hs
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
            const double lam = S.job.lambda[j];
            taylor::jet_mul(oj[j], Fj[j], gj[j], J, dig, off);
#pragma unroll 1
            for (int i = 0; i < J; ++i) {
                gj[j][i] *= lam;
                rj[j][i] = dc{i == 0 ? 1.0 : 0.0, -gj[j][i]};
            }
            taylor::jet_mul(tj[j], gj[j], wk, J, dig, off);
#pragma unroll 1
            for (int i = 0; i < J; ++i) zj[j][i] = dc{tj[j][i], -wk[i]};
        }
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
            const double lam = S.job.lambda[j];
            taylor::jet_mul(tj[j], oj[j], wk, J, dig, off);       // t_j (1 - t_j)
#pragma unroll 1
            for (int l = 0; l < d; ++l) {
                taylor::jet_mul(wk, Hs[j][l], wk2, J, dig, off);
                if (l == j) {
                    double u[JMAX];
#pragma unroll 1
                    for (int i = 0; i < J; ++i) u[i] = oj[j][i] - tj[j][i];
                    double u2[JMAX];
                    taylor::jet_mul(u, Fj[j], u2, J, dig, off);
#pragma unroll 1
                    for (int i = 0; i < J; ++i) wk2[i] += u2[i];
                }
#pragma unroll 1
                for (int i = 0; i < J; ++i) gi[0][i].re = lam * wk2[i];   // scratch row
#pragma unroll 1
                for (int i = 0; i < J; ++i) Hs[j][l][i] = gi[0][i].re;    // Hs now holds V_jl
            }
        }
        // det J = (1 - E2) + i (det V - tr V) (d = 3); (1 - det V) - i tr V (d = 2); 1 - i V00 (d = 1)
        {
            double e2[JMAX], dv[JMAX], tr[JMAX];
#pragma unroll 1
            for (int i = 0; i < J; ++i) e2[i] = dv[i] = tr[i] = 0.0;
#pragma unroll 1
            for (int j = 0; j < d; ++j)
#pragma unroll 1
                for (int i = 0; i < J; ++i) tr[i] += Hs[j][j][i];
            auto minor2 = [&](int a, int b, int c, int e, double *out) {   // V_ab V_ce - V_ae V_cb
                taylor::jet_mul(Hs[a][b], Hs[c][e], out, J, dig, off);
                taylor::jet_mul(Hs[a][e], Hs[c][b], wk, J, dig, off);
#pragma unroll 1
                for (int i = 0; i < J; ++i) out[i] -= wk[i];
            };
            if (d == 2) {
                minor2(0, 0, 1, 1, dv);
            } else if (d == 3) {
                double m[JMAX];
                minor2(0, 0, 1, 1, m);
#pragma unroll 1
                for (int i = 0; i < J; ++i) e2[i] += m[i];
                minor2(0, 0, 2, 2, m);
#pragma unroll 1
                for (int i = 0; i < J; ++i) e2[i] += m[i];
                minor2(1, 1, 2, 2, m);
#pragma unroll 1
                for (int i = 0; i < J; ++i) e2[i] += m[i];
                // det V by the first row: V00 c00 - V01 c01 + V02 c02
                minor2(1, 1, 2, 2, m);
                taylor::jet_mul(Hs[0][0], m, dv, J, dig, off);
                minor2(1, 0, 2, 2, m);
                taylor::jet_mul(Hs[0][1], m, wk2, J, dig, off);
#pragma unroll 1
                for (int i = 0; i < J; ++i) dv[i] -= wk2[i];
                minor2(1, 0, 2, 1, m);
                taylor::jet_mul(Hs[0][2], m, wk2, J, dig, off);
#pragma unroll 1
                for (int i = 0; i < J; ++i) dv[i] += wk2[i];
            }
#pragma unroll 1
            for (int i = 0; i < J; ++i) {
                const double one = i == 0 ? 1.0 : 0.0;
                if (d == 3) dJ[i] = dc{one - e2[i], dv[i] - tr[i]};
                else if (d == 2) dJ[i] = dc{one - dv[i], -tr[i]};
                else dJ[i] = dc{one, -tr[i]};
            }
        }
        // powers of z_j, then U(z) and F(z)
#pragma unroll 1
        for (int j = 0; j < d; ++j) {
#pragma unroll 1
            for (int i = 0; i < J; ++i) zp[j][0][i] = zj[j][i];
#pragma unroll 1
            for (int e = 1; e < sec.pad0 && e < QMC_EMAX; ++e) taylor::cjet_mul(zp[j][e - 1], zj[j], zp[j][e], J, dig, off);
        }
#pragma unroll 1
        for (int w = 0; w < 2; ++w) {
            dc *P = w == 0 ? cu : cf;
            const int m0 = w == 0 ? 0 : sec.nU, m1 = w == 0 ? sec.nU : sec.nU + sec.nF;
#pragma unroll 1
            for (int i = 0; i < J; ++i) P[i] = dc{0.0, 0.0};
#pragma unroll 1
            for (int m = m0; m < m1; ++m) {
                const uint32_t ex = S.exps[m];
#pragma unroll 1
                for (int i = 0; i < J; ++i) cx[i] = dc{i == 0 ? S.cval[m] : 0.0, 0.0};
#pragma unroll 1
                for (int j = 0; j < d; ++j) {
                    const uint32_t ej = (ex >> (4 * j)) & 15u;
                    if (ej == 0u) continue;
                    taylor::cjet_mul(cx, zp[j][ej - 1], cy, J, dig, off);
#pragma unroll 1
                    for (int i = 0; i < J; ++i) cx[i] = cy[i];
                }
#pragma unroll 1
                for (int i = 0; i < J; ++i) P[i] = P[i] + cx[i];
            }
        }
        if (cf[0].im > 0.0) ++signfail;   // F on the wrong side of the cut at this corner
        // A = sum e0 L_P, B = sum e1 L_P over the power factors
#pragma unroll 1
        for (int i = 0; i < J; ++i) cA[i] = cB[i] = dc{0.0, 0.0};
#pragma unroll 1
        for (int f = 0; f < d + 2; ++f) {
            const dc *P;
            double e0, e1;
            bool m0 = false;
            if (f < d) {
                if (slot[f] >= 0) P = rj[f];
                else if (sec.a[f] != 0 || sec.b[f] != 0.0) P = zj[f];
                else continue;
                e0 = sec.a[f];
                e1 = sec.b[f];
            } else if (f == d) {
                P = cu;
                e0 = sec.u0;
                e1 = sec.u1;
            } else {
                P = cf;
                e0 = sec.f0;
                e1 = sec.f1;
                m0 = true;
            }
            if (e0 == 0.0 && e1 == 0.0) continue;
            // L = ln P0 + ln(1 + x), x = (P - P0) / P0, ln(1 + x) = x h by Horner
            const dc r0 = cinv(P[0]);
#pragma unroll 1
            for (int i = 0; i < J; ++i) cx[i] = i == 0 ? dc{0.0, 0.0} : P[i] * r0;
#pragma unroll 1
            for (int i = 0; i < J; ++i) cy[i] = dc{0.0, 0.0};
            cy[0] = dc{((K - 1) & 1 ? -1.0 : 1.0) * taylor::inv_k[K > 0 ? K : 1], 0.0};
#pragma unroll 1
            for (int k = K - 2; k >= 0; --k) {
                taylor::cjet_mul(cx, cy, gi[0], J, dig, off);
#pragma unroll 1
                for (int i = 0; i < J; ++i) cy[i] = gi[0][i];
                cy[0].re += (k & 1 ? -1.0 : 1.0) * taylor::inv_k[k + 1];
            }
            taylor::cjet_mul(cx, cy, gi[0], J, dig, off);
            const dc l0 = taylor::clog_br(P[0], m0, tab, atab);
#pragma unroll 1
            for (int i = 0; i < J; ++i) {
                const dc L = i == 0 ? l0 : (K > 0 ? gi[0][i] : dc{0.0, 0.0});
                cA[i] = cA[i] + L * e0;
                cB[i] = cB[i] + L * e1;
            }
        }
        // exp(A) = exp(A0) (1 + A~ (1 + A~/2 (1 + ...))), A~ = A - A0
        const dc ea = cexp_(cA[0]);
        cA[0] = dc{0.0, 0.0};
#pragma unroll 1
        for (int i = 0; i < J; ++i) cy[i] = dc{i == 0 ? 1.0 : 0.0, 0.0};
#pragma unroll 1
        for (int k = K; k >= 1; --k) {
            taylor::cjet_mul(cA, cy, cx, J, dig, off);
            const double r = taylor::inv_k[k];
#pragma unroll 1
            for (int i = 0; i < J; ++i) cy[i] = cx[i] * r;
            cy[0].re += 1.0;
        }
#pragma unroll 1
        for (int i = 0; i < J; ++i) cx[i] = cy[i] * ea;
        taylor::cjet_mul(dJ, cx, gi[0], J, dig, off);    // det J exp(A)
        // G_i = det J exp(A) B^i / i!
#pragma unroll 1
        for (int n = 1; n <= Hm; ++n) {
            taylor::cjet_mul(gi[n - 1], cB, gi[n], J, dig, off);
            const double r = taylor::inv_k[n];
#pragma unroll 1
            for (int i = 0; i < J; ++i) gi[n][i] = gi[n][i] * r;
        }
        // T = sum_kappa (sum_i eps^i G_i[kappa]) prod_{q in V} phi_q(kappa_q)
        double Tr[NT], Ti[NT];
#pragma unroll 1
        for (int i = 0; i < NT; ++i) Tr[i] = Ti[i] = 0.0;
#pragma unroll 1
        for (int kap = 0; kap < J; ++kap) {
            double P[NT], Q[NT], gr[NT], gim[NT];
            bool first = true;
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                if (!((V >> q) & 1)) continue;
                const int k = rad[q] > 1 ? (kap / stride[q]) % rad[q] : 0;
                if (first) {
#pragma unroll 1
                    for (int i = 0; i < NT; ++i) P[i] = phi[q][k][i];
                    first = false;
                } else {
                    taylor::ser_mul<NT, OFF>(P, phi[q][k], Q, Hm);
#pragma unroll 1
                    for (int i = 0; i < NT; ++i) P[i] = Q[i];
                }
            }
            if (first) {
#pragma unroll 1
                for (int i = 0; i < NT; ++i) P[i] = i == OFF ? 1.0 : 0.0;
            }
#pragma unroll 1
            for (int i = 0; i < NT; ++i) {
                const bool in = i >= OFF && i - OFF <= Hm;
                gr[i] = in ? gi[i - OFF][kap].re : 0.0;
                gim[i] = in ? gi[i - OFF][kap].im : 0.0;
            }
            taylor::ser_mul<NT, OFF>(gr, P, Q, Hm);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) Tr[i] += Q[i];
            taylor::ser_mul<NT, OFF>(gim, P, Q, Hm);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) Ti[i] += Q[i];
        }
        // prod_{q not in V} psi_q
        double base[NT], Q[NT];
#pragma unroll 1
        for (int i = 0; i < NT; ++i) base[i] = i == OFF ? 1.0 : 0.0;
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            if ((V >> q) & 1) continue;
            taylor::ser_mul<NT, OFF>(base, psi[q], Q, Hm);
#pragma unroll 1
            for (int i = 0; i < NT; ++i) base[i] = Q[i];
        }
        taylor::ser_mul<NT, OFF>(base, Tr, Q, Hm);
#pragma unroll 1
        for (int i = 0; i < NT; ++i) acc_re[i] += Q[i];
        taylor::ser_mul<NT, OFF>(base, Ti, Q, Hm);
#pragma unroll 1
        for (int i = 0; i < NT; ++i) acc_im[i] += Q[i];
    }
#pragma unroll
    for (int o = 0; o < LMAX; ++o) {
        res[o] = dc{0.0, 0.0};
#pragma unroll 1
        for (int i = 0; i < NT; ++i)
            if (o < nord && i == lo + o + OFF) res[o] = dc{acc_re[i], acc_im[i]};
    }
}

// ---------------------------------------------------------------- tile staging
template <int LMAX>
__device__ void stage_tile(TileSmem<LMAX> &S, const QmcLaunch &Lc, int jidx) {
    // called by all threads; S.job already holds the job
    const int sidx = S.job.sector;
    const int pidx = S.job.point;
    if (sidx != S.cached_sector || pidx != S.cached_point) {
        const QmcSectorDev *src = Lc.sectors + sidx;
        // header copy (plain words)
        const int nw = sizeof(QmcSectorDev) / 4;
        for (int i = threadIdx.x; i < nw; i += blockDim.x)
            reinterpret_cast<int32_t *>(&S.sec)[i] = reinterpret_cast<const int32_t *>(src)[i];
        const int m0 = src->monoU;
        const int nm = src->nmono;
        const double *kin = Lc.kin + (size_t)pidx * Lc.ninv;
        for (int m = threadIdx.x; m < nm; m += blockDim.x) {
            const QmcMono &M = Lc.monos[m0 + m];
            double v = M.coef[0];
            for (int i = 0; i < Lc.ninv && i + 1 < QMC_NCOEF; ++i) v = fma(M.coef[i + 1], kin[i], v);
            S.cval[m] = v;
            S.cvalf[m] = (float)v;
            S.exps[m] = M.exps;
            uint64_t dsc = 0;
            int k = 0;
            for (int j = 0; j < QMC_DMAX; ++j) {
                const uint32_t ej = (M.exps >> (4 * j)) & 15u;
                if (ej) {
                    dsc |= (uint64_t)(Lc.prow * j + ej - 1) << (3 + 5 * k);
                    ++k;
                }
            }
            S.mdesc[m] = dsc | (uint64_t)k;
        }
        __syncthreads();
        if (threadIdx.x < QMC_SMAX) {
            int q = threadIdx.x;
            double inv = 0.0;
            if (q < S.sec.ns) {
                int j = S.sec.sing[q];
                inv = 1.0 / S.sec.b[j];
            }
            S.invb[q] = inv;
        }
        if (threadIdx.x == 0) {
            S.cached_sector = sidx;
            S.cached_point = pidx;
            double af = 1.0;
            for (int q = 0; q < S.sec.ns; ++q) af *= 1.0 / S.sec.b[S.sec.sing[q]];
            S.invb_full = af;
            double w = S.sec.weight;   // the sector's constant factor, times 140^d for korobov3
            if (Lc.transform == 0)
                for (int j = 0; j < S.sec.d; ++j) w *= 140.0;
            S.w140d = w;
        }
    }
}

// ---------------------------------------------------------------- the evaluator
#ifndef QMC_MINB
// Resident 128-thread blocks per SM (or half as many of 256 threads) the
// real d <= 3 evaluator's registers must allow. With the logarithm, lattice
// and transform on the integer pipe the kernel is latency-bound, and 16
// warps per SM (128 registers, some spilled to L1) beat 12 without spills.
#define QMC_MINB 4
#endif

// The same for the deformed and the d <= 6 classes, which need up to 255
// registers without a bound: 3 blocks (170 registers, spills to L1) beat 2
// blocks by 12 to 24 %; the mixed-precision deformed class, with fewer live
// FP64 values, goes best at 4 (128 registers)
#ifndef QMC_MINB_WIDE
#define QMC_MINB_WIDE 3
#endif
#ifndef QMC_MINB_WIDE_MIXED
#define QMC_MINB_WIDE_MIXED 4
#endif

template <int BLOCK, bool WIDE, bool CPLX_MIXED, bool HS>
constexpr int qmc_min_blocks() {
    return HS ? 1
              : WIDE ? ((CPLX_MIXED ? QMC_MINB_WIDE_MIXED : QMC_MINB_WIDE) * 128 + BLOCK - 1) / BLOCK
                     : QMC_MINB * 128 / BLOCK;
}

// The thread's points [k0, kend) of the current tile: lattice walk, shifted
// point and transform, integrand, and acc[o] += W f_o for the output orders
// eps^(lo+o), o < nord. NSC, HIC >= 0: the tile's number of singular
// variables and highest order fixed at compile time (real sectors), the
// series summed per order eps^-NSC .. eps^HIC and mapped to the output orders
// once at the end; NSC = HIC = -1: the run-time general path.
template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, bool HS, int NSC, int HIC, class T>
__device__ __forceinline__ void thread_points(const TileSmem<LMAX> &S, const QmcLaunch &Lc, uint64_t k0,
                                              uint64_t kend, int lo, int hi, int nord, T (&acc)[LMAX],
                                              int &signfail_tile, unsigned char *ptab) {
    constexpr bool FIXED = NSC >= 0 && HIC >= 0;
    constexpr int NO = FIXED ? NSC + HIC + 1 : 1;
    double accN[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) accN[i] = 0.0;
    const int d = S.sec.d;
    const uint64_t n = S.job.n;
    const double nd = (double)n, inv_n = S.job.inv_n;
    // per coordinate only the walk lives in registers; z, the expansion of
    // z/n and the shift are read from shared memory
    LatticeWalk wk[DMAX];
    const uint32_t n32 = (uint32_t)n;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) walk_init(wk[j], (j < d) ? (k0 * (uint64_t)S.zmod[j]) % n : 0, n);
#pragma unroll 1
    for (uint64_t k = k0; k < kend; ++k) {
        double t[DMAX], omt[DMAX];
        double Ws = 1.0;  // prod u(1-u); the korobov3 weight is 140^d Ws^3
        bool zero_t = false;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            t[j] = 1.0;
            omt[j] = 0.0;
            if (j < d) {
                double u;
                if constexpr (!CPLX && DMAX > 3 && FIXED && QMC_WALK_CALL)
                    u = walk_coord_call(wk[j].Q, wk[j].r, wk[j].R, n32, nd, inv_n, S.delta[j], S.dfix[j]);
                else
                    u = walk_coord(wk[j], n32, nd, inv_n, S.delta[j], S.dfix[j], true);
                if (Lc.transform == 0) {          // korobov3
                    // integer pipe (with 1 - t for the deformed classes)
                    if constexpr (!CPLX && DMAX > 3 && !QMC_KOROBOV_INT6) {
                        const double u2 = u * u;
                        t[j] = u2 * u2 * fma(u, fma(u, fma(u, -20.0, 70.0), -84.0), 35.0);
                        Ws *= fma(-u, u, u);
                    } else {
                        double ws = 0.0, om = 1.0;
                        t[j] = 0.0;
                        if constexpr (!CPLX && DMAX > 3 && FIXED && QMC_KOROBOV_CALL) {
                            if (!nonneg_is_zero(u)) {
                                const K3 k3 = korobov3_call(u);
                                t[j] = k3.t;
                                ws = k3.ws;
                            }
                        } else {
                            if (!nonneg_is_zero(u)) korobov3_int<CPLX>(u, t[j], om, ws);
                        }
                        if (CPLX) omt[j] = om;
                        Ws = j == 0 ? ws : Ws * ws;
                    }
                } else if (Lc.transform == 1) {   // baker: t = 1 - |2u - 1|, weight 1
                    t[j] = u < 0.5 ? 2.0 * u : 2.0 * (1.0 - u);
                    omt[j] = u < 0.5 ? 1.0 - 2.0 * u : 2.0 * u - 1.0;
                } else {                          // no transform
                    t[j] = u;
                    omt[j] = 1.0 - u;
                }
                zero_t |= nonneg_is_zero(t[j]);
                walk_step(wk[j], S.zmod[j], S.qz[j], S.rz[j], n32);
            }
        }
        const double W = Lc.transform == 0 ? Ws * Ws * Ws : 1.0;   // 140^d: per tile
        if (nonneg_is_zero(W) || zero_t) continue;
        if constexpr (FIXED) {
            double resN[NO];
            eval_real_fx<DMAX, NSC, HIC, MIXED, LMAX>(S, t, resN, reinterpret_cast<double *>(ptab) + threadIdx.x,
                                                      reinterpret_cast<float *>(ptab) + threadIdx.x, (int)blockDim.x,
                                                      Lc.prow);
#pragma unroll
            for (int i = 0; i < NO; ++i) accN[i] = fma(resN[i], W, accN[i]);
        } else {
            T res[LMAX];
            if constexpr (CPLX && HS) {
                eval_deformed_taylor<LMAX, QMC_JMAX3>(S, t, omt, lo, hi, nord, res, signfail_tile);
            } else if constexpr (CPLX) {
                eval_deformed<DMAX, SMAX, LMAX, MIXED>(S, t, omt, lo, hi, nord, res, signfail_tile);
            } else {
                if constexpr (HS) {
                    eval_real_taylor<DMAX, SMAX, LMAX, (DMAX <= 3 ? QMC_JMAX3 : QMC_JMAX6)>(S, t, lo, hi, nord, res);
                } else if constexpr (DMAX <= 3) {
                    // one instantiation per number of singular variables (uniform per tile)
                    if (S.sec.ns == 2) eval_real<DMAX, SMAX, LMAX, MIXED, 2>(S, t, lo, hi, nord, res);
                    else if (S.sec.ns == 1) eval_real<DMAX, SMAX, LMAX, MIXED, 1>(S, t, lo, hi, nord, res);
                    else eval_real<DMAX, SMAX, LMAX, MIXED, 0>(S, t, lo, hi, nord, res);
                } else {
                    eval_real<DMAX, SMAX, LMAX, MIXED>(S, t, lo, hi, nord, res);
                }
            }
#pragma unroll
            for (int o = 0; o < LMAX; ++o)
                if (o < nord) acc[o] = acc[o] + mulsc(res[o], W);
        }
    }
    if constexpr (FIXED) {
        // output order o is eps^(lo+o), i.e. index lo + o + NSC of accN; orders
        // below the sector's leading pole are 0 (selected without local memory)
#pragma unroll
        for (int o = 0; o < LMAX; ++o) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < NO; ++i)
                if (i == lo + o + NSC) v = accN[i];
            if (o < nord) acc[o] = from_real<T>(v);
        }
    }
}

// FIX: the real classes' kernel for sums up to eps^0 (highest order 0, every
// sum the integrator forms), with only the compile-time paths; the general
// kernel (FIX = false) serves every other order window. Two instantiations
// keep each kernel's code, and its instruction-cache footprint, small.
template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, int BLOCK, bool HS = false, bool FIX = false>
__global__ void __launch_bounds__(BLOCK, qmc_min_blocks<BLOCK, (CPLX || DMAX > 3), (CPLX && MIXED), HS>()) qmc_eval_kernel(QmcLaunch Lc, int ppt) {
    __shared__ TileSmem<LMAX> S;
    // the fixed-order kernels' per-thread power tables (4 DMAX rows of BLOCK
    // doubles, dynamic shared memory; empty for the other kernels)
    extern __shared__ __align__(16) unsigned char qmc_ptab[];
    using T = typename std::conditional<CPLX, dc, double>::type;
    const int lo = Lc.lo, nord = Lc.norders;
    if (threadIdx.x == 0) {
        S.cached_sector = -1;
        S.cached_point = -1;
    }
    for (int i = threadIdx.x; i < 3 * QMC_LOG_TABLE_ROWS; i += blockDim.x) S.logtab[i] = kLogTable[i];
    if (CPLX)
        for (int i = threadIdx.x; i < 2 * QMC_ATAN_TABLE_ROWS; i += blockDim.x) S.atantab[i] = kAtanTable[i];
    for (;;) {
        int signfail_tile = 0;
        __syncthreads();  // previous tile fully consumed
        if (threadIdx.x == 0) {
            unsigned long long tile = atomicAdd(Lc.queue, 1ULL);
            S.tile = tile;
            int jidx = -1;
            if (tile < Lc.ntiles) {
                // last job with tile_begin <= tile
                int lo_j = 0, hi_j = Lc.njobs - 1;
                while (lo_j < hi_j) {
                    int mid = (lo_j + hi_j + 1) >> 1;
                    if (Lc.jobs[mid].tile_begin <= tile) lo_j = mid;
                    else hi_j = mid - 1;
                }
                jidx = lo_j;
            }
            S.job_index = jidx;
        }
        __syncthreads();
        const unsigned long long tile = S.tile;
        if (tile >= Lc.ntiles) break;
        const int jidx = S.job_index;
        {
            const int nw = sizeof(QmcJobDev) / 4;
            for (int i = threadIdx.x; i < nw; i += blockDim.x)
                reinterpret_cast<int32_t *>(&S.job)[i] = reinterpret_cast<const int32_t *>(Lc.jobs + jidx)[i];
        }
        __syncthreads();
        stage_tile<LMAX>(S, Lc, jidx);
        const uint64_t local = tile - S.job.tile_begin;
        const int s = (int)(local / (uint64_t)S.job.tiles_per_shift);
        const uint64_t chunk = local % (uint64_t)S.job.tiles_per_shift;
        if (threadIdx.x < QMC_DMAX) {
            int j = threadIdx.x;
            S.delta[j] = (j < S.sec.d && !(S.job.flags & 1))
                             ? splitmix_uniform(S.job.seed_state, (uint64_t)s * S.sec.d + j) : 0.0;
            S.dfix[j] = (uint64_t)(S.delta[j] * 18446744073709551616.0);   // exact: delta is a multiple of 2^-53
            uint64_t qz = 0, rz = 0, zm = (uint64_t)S.job.z[j] % S.job.n;
            if (j < S.sec.d) fixdiv64(zm, S.job.n, qz, rz);
            S.qz[j] = qz;
            S.rz[j] = (uint32_t)rz;
            S.zmod[j] = (uint32_t)zm;
        }
        __syncthreads();

        const uint64_t n = S.job.n;
        const int hi = lo + nord - 1;
        T acc[LMAX];
#pragma unroll
        for (int o = 0; o < LMAX; ++o) acc[o] = zero<T>();

        const uint64_t kt0 = chunk * (uint64_t)Lc.tile_k;
        const uint64_t kt1 = min(n, kt0 + (uint64_t)Lc.tile_k);
        const uint64_t k0 = kt0 + (uint64_t)threadIdx.x * (uint64_t)ppt;
        if (k0 < kt1) {
            const uint64_t kend = min(kt1, k0 + (uint64_t)ppt);
            if constexpr (!CPLX && !HS && FIX) {
                // real sectors up to eps^0: the compile-time path for the tile's
                // number of singular variables (the host launches this kernel
                // only for hi = 0)
                const int ns = S.sec.ns;
                if (ns == 0) thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, 0, 0>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
                else if (ns == 1) thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, 1, 0>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
                else if (ns == 2 || SMAX < 3) thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, (SMAX >= 2 ? 2 : 1), 0>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
                else if constexpr (SMAX >= 3) {
                    if (ns == 3 || SMAX < 4) thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, 3, 0>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
                    else thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, (SMAX >= 4 ? 4 : 3), 0>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
                }
            } else {
                thread_points<DMAX, SMAX, LMAX, CPLX, MIXED, HS, -1, -1>(S, Lc, k0, kend, lo, hi, nord, acc, signfail_tile, qmc_ptab);
            }
        }
        // sign-check failures of this tile: per job (if counted) and in total
        if (CPLX && __ballot_sync(0xffffffffu, signfail_tile != 0)) {
            const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)signfail_tile);
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(Lc.status, (unsigned long long)v);
                if (Lc.job_fail) atomicAdd(Lc.job_fail + jidx, v);
            }
        }
        // block reduction: warp shuffles, then warps in index order
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 0; o < LMAX; ++o) {
            if (o >= nord) continue;
            double vr = re_of(acc[o]);
            double vi = im_of(acc[o]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                vr += __shfl_down_sync(0xffffffffu, vr, off);
                if (CPLX) vi += __shfl_down_sync(0xffffffffu, vi, off);
            }
            if (lane == 0) {
                S.red[warp][2 * o] = vr;
                S.red[warp][2 * o + 1] = vi;
            }
        }
        __syncthreads();
        if (threadIdx.x < 2 * nord) {
            double sum = 0.0;
            for (int w = 0; w < BLOCK / 32; ++w) sum += S.red[w][threadIdx.x];
            sum *= S.w140d;   // the sector's constant factor and the korobov3 weight's 140^d
            // streaming store (evict first): the partials are read once, by the
            // finishing kernel, and at large lattices their stream would
            // otherwise push the spilled thread stacks out of L2
            __stcs(&Lc.partials[tile * (uint64_t)(2 * nord) + threadIdx.x], sum);
            if (!isfinite(sum)) atomicAdd(Lc.status + 1, 1ULL);
        }
    }
}

#if QMC_PART == 0
// Sum each (job, shift, component) over its tiles in tile order (Neumaier),
// divide by n, write the per-shift estimate; then re-arm the tile queue.
__global__ void qmc_finish_kernel(QmcLaunch Lc) {
    const int j = blockIdx.x;
    if (j >= Lc.njobs) return;
    const QmcJobDev &J = Lc.jobs[j];
    const int per = 2 * Lc.norders;
    const int total = J.shifts * per;
    const double inv_n = 1.0 / (double)J.n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int s = idx / per, q = idx % per;
        const uint64_t t0 = J.tile_begin + (uint64_t)s * J.tiles_per_shift;
        double sum = 0.0, comp = 0.0;
        for (uint64_t c = 0; c < (uint64_t)J.tiles_per_shift; ++c) {
            const double x = __ldcs(&Lc.partials[(t0 + c) * per + q]);
            const double tt = sum + x;
            comp += (fabs(sum) >= fabs(x)) ? (sum - tt) + x : (x - tt) + sum;
            sum = tt;
        }
        Lc.out[J.out_off + idx] = (sum + comp) * inv_n;
    }
    if (j == 0 && threadIdx.x == 0) *Lc.queue = 0ULL;
}

// Each thread walks kQmcLatticeRun consecutive indices with the evaluator's
// integer walk (the first one set up by division, the rest by steps).
constexpr int kQmcLatticeRun = 8;
__global__ void qmc_lattice_kernel(uint64_t n, double inv_n, const uint32_t *z, int d,
                                   const double *delta, uint64_t k0, uint64_t count, double *x,
                                   uint64_t *rout) {
    const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kQmcLatticeRun;
    if (i0 >= count) return;
    const uint64_t i1 = min(count, i0 + (uint64_t)kQmcLatticeRun);
    for (int j = 0; j < d; ++j) {
        const uint64_t zj = (uint64_t)z[j] % n;
        uint64_t qz, rz, D;
        fixdiv64(zj, n, qz, rz);
        const uint32_t n32 = (uint32_t)n;
        const bool dok = delta_fix(delta[j], D);
        LatticeWalk w;
        // ((k0 + i0) mod n) z < 2^64 for n < 2^32
        walk_init(w, (((k0 + i0) % n) * zj) % n, n);
        for (uint64_t i = i0; i < i1; ++i) {
            x[i * d + j] = walk_coord(w, n32, (double)n, inv_n, delta[j], D, dok);
            if (rout) rout[i * d + j] = w.r;
            walk_step(w, (uint32_t)zj, qz, (uint32_t)rz, n32);
        }
    }
}

__global__ void qmc_log_kernel(const double *x, uint64_t n, double *out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = qlog(x[i], kLogTable);
}

__global__ void qmc_korobov_kernel(const double *x, uint64_t n, double *out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t = 0.0, omt = 1.0, ws = 0.0;
    if (!nonneg_is_zero(x[i])) korobov3_int<true>(x[i], t, omt, ws);
    out[3 * i] = t;
    out[3 * i + 1] = omt;
    out[3 * i + 2] = ws;
}

__global__ void qmc_rcp_kernel(const double *x, uint64_t n, double *out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = qrcp(x[i]);
}

__global__ void qmc_atan2_kernel(const double *yx, uint64_t n, double *out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = qatan2(yx[2 * i], yx[2 * i + 1], kAtanTable);
}

__global__ void qmc_shift_kernel(uint64_t state, int m, int d, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m * d) out[i] = splitmix_uniform(state, (uint64_t)i);
}

// FP64 throughput probe: 8 independent DFMA chains per thread.
__global__ void qmc_fp64_probe_kernel(double *out, int iters) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1.0 + 1e-9 * (threadIdx.x + c);
    const double m1 = 0.999999999, m2 = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m1, m2);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678) out[0] = s;  // never true; keeps the loop alive
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

// FP32 throughput probe: 8 independent FFMA chains per thread.
__global__ void qmc_fp32_probe_kernel(float *out, int iters) {
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1.0f + 1e-6f * (float)(threadIdx.x + c);
    const float m1 = 0.9999999f, m2 = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fmaf(a[c], m1, m2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678f) out[0] = s;  // never true; keeps the loop alive
    if (threadIdx.x == 0 && blockIdx.x == 0) out[1] = s;
}

#endif  // QMC_PART == 0

// Blocks of 256 threads exist for the d <= 3 classes only: the d <= 6 classes
// run near the register limit, where a second warp set per block buys nothing
// (and their instantiations dominate the build).
// Dynamic shared memory of an evaluator kernel: the power tables of the
// fixed-order real kernels, prow rows of x^1..x^prow per variable
template <int DMAX, bool CPLX, bool HS, bool FIX>
constexpr int eval_dyn_smem(int block, int prow) {
    return (!CPLX && !HS && FIX) ? prow * DMAX * block * (int)sizeof(double) : 0;
}

// The attribute allows the largest table (QMC_EMAX rows); each launch asks for its own
template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, int BLOCK, bool HS, bool FIX>
bool allow_dyn_smem() {
    constexpr int dmax = eval_dyn_smem<DMAX, CPLX, HS, FIX>(BLOCK, QMC_EMAX);
    static const bool ok =
        dmax == 0 || cudaFuncSetAttribute(qmc_eval_kernel<DMAX, SMAX, LMAX, CPLX, MIXED, BLOCK, HS, FIX>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, dmax) == cudaSuccess;
    return ok;
}

template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, int BLOCK, bool HS, bool FIX>
int launch_block(const QmcLaunch *L, int ppt, int grid, cudaStream_t st) {
    if (L->prow < 1 || L->prow > QMC_EMAX) return -1;
    if (!allow_dyn_smem<DMAX, SMAX, LMAX, CPLX, MIXED, BLOCK, HS, FIX>()) return -1;
    const int dyn = eval_dyn_smem<DMAX, CPLX, HS, FIX>(BLOCK, L->prow);
    qmc_eval_kernel<DMAX, SMAX, LMAX, CPLX, MIXED, BLOCK, HS, FIX><<<grid, BLOCK, dyn, st>>>(*L, ppt);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, bool HS, bool FIX>
int launch_shape(const QmcLaunch *L, int block, int ppt, int grid, cudaStream_t st) {
    if constexpr (DMAX <= 3) {
        if (block == 256) return launch_block<DMAX, SMAX, LMAX, CPLX, MIXED, 256, HS, FIX>(L, ppt, grid, st);
    }
    return launch_block<DMAX, SMAX, LMAX, CPLX, MIXED, 128, HS, FIX>(L, ppt, grid, st);
}

template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, bool HS = false>
int launch_cls(const QmcLaunch *L, int block, int ppt, int grid, cudaStream_t st) {
    if constexpr (!CPLX && !HS) {
        if (L->lo + L->norders - 1 == 0) return launch_shape<DMAX, SMAX, LMAX, CPLX, MIXED, HS, true>(L, block, ppt, grid, st);
    }
    return launch_shape<DMAX, SMAX, LMAX, CPLX, MIXED, HS, false>(L, block, ppt, grid, st);
}

template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, int BLOCK, bool HS, bool FIX>
int occupancy_block(int prow) {
    if (!allow_dyn_smem<DMAX, SMAX, LMAX, CPLX, MIXED, BLOCK, HS, FIX>()) return 0;
    const int dyn = eval_dyn_smem<DMAX, CPLX, HS, FIX>(BLOCK, prow);
    int v = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &v, qmc_eval_kernel<DMAX, SMAX, LMAX, CPLX, MIXED, BLOCK, HS, FIX>, BLOCK, dyn);
    return e == cudaSuccess ? v : 0;
}

template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, bool HS, bool FIX>
int occupancy_shape(int block, int prow) {
    if constexpr (DMAX <= 3) {
        if (block == 256) return occupancy_block<DMAX, SMAX, LMAX, CPLX, MIXED, 256, HS, FIX>(prow);
    }
    return occupancy_block<DMAX, SMAX, LMAX, CPLX, MIXED, 128, HS, FIX>(prow);
}

// Resident blocks per SM of the class's kernels (the larger of the fixed-order
// and the general kernel: a persistent grid sized for it only over-subscribes
// the other, whose surplus blocks find the tile queue empty)
template <int DMAX, int SMAX, int LMAX, bool CPLX, bool MIXED, bool HS = false>
int occupancy_cls(int block, int prow) {
    int v = occupancy_shape<DMAX, SMAX, LMAX, CPLX, MIXED, HS, false>(block, prow);
    if constexpr (!CPLX && !HS) v = std::max(v, occupancy_shape<DMAX, SMAX, LMAX, CPLX, MIXED, HS, true>(block, prow));
    return v;
}

}  // namespace

// Per translation unit: the launcher and occupancy query of the classes it
// instantiates (-2 / 0 for the others). The evaluator classes are compiled in
// four translation units in parallel: part 0 the real d <= 3 classes (and
// everything that is not an evaluator), part 1 the deformed classes, part 2
// the d <= 6 classes, part 3 the Taylor-subtraction classes.
#define QMC_PART_FN2(name, part) name##_part##part
#define QMC_PART_FN(name, part) QMC_PART_FN2(name, part)

extern "C" int QMC_PART_FN(qmc_k_launch_eval, QMC_PART)(int cls, const QmcLaunch *L, int block, int ppt, int grid,
                                                         void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (cls) {
#if QMC_PART == 0
        case QMC_CLASS_REAL3: return launch_cls<3, 2, 4, false, false>(L, block, ppt, grid, st);
        case QMC_CLASS_REAL3M: return launch_cls<3, 2, 4, false, true>(L, block, ppt, grid, st);
#elif QMC_PART == 1
        case QMC_CLASS_CPLX3: return launch_cls<3, 2, 4, true, false>(L, block, ppt, grid, st);
        case QMC_CLASS_CPLX3M: return launch_cls<3, 2, 4, true, true>(L, block, ppt, grid, st);
#elif QMC_PART == 2
        // one d <= 6 kernel for 0..4 singular variables (the former REAL6S and
        // REAL6T classes included)
        case QMC_CLASS_REAL6:
        case QMC_CLASS_REAL6S:
        case QMC_CLASS_REAL6T: return launch_cls<6, 4, 6, false, false>(L, block, ppt, grid, st);
        case QMC_CLASS_REAL6M:
        case QMC_CLASS_REAL6SM:
        case QMC_CLASS_REAL6TM: return launch_cls<6, 4, 6, false, true>(L, block, ppt, grid, st);
#elif QMC_PART == 3
        case QMC_CLASS_REAL3H: return launch_cls<3, 2, 4, false, false, true>(L, block, ppt, grid, st);
        case QMC_CLASS_REAL6H: return launch_cls<6, 4, 6, false, false, true>(L, block, ppt, grid, st);
        case QMC_CLASS_CPLX3H: return launch_cls<3, 2, 4, true, false, true>(L, block, ppt, grid, st);
#endif
        default: return -2;
    }
}

extern "C" int QMC_PART_FN(qmc_k_occupancy, QMC_PART)(int cls, int block, int prow) {
    switch (cls) {
#if QMC_PART == 0
        case QMC_CLASS_REAL3: return occupancy_cls<3, 2, 4, false, false>(block, prow);
        case QMC_CLASS_REAL3M: return occupancy_cls<3, 2, 4, false, true>(block, prow);
#elif QMC_PART == 1
        case QMC_CLASS_CPLX3: return occupancy_cls<3, 2, 4, true, false>(block, prow);
        case QMC_CLASS_CPLX3M: return occupancy_cls<3, 2, 4, true, true>(block, prow);
#elif QMC_PART == 2
        case QMC_CLASS_REAL6:
        case QMC_CLASS_REAL6S:
        case QMC_CLASS_REAL6T: return occupancy_cls<6, 4, 6, false, false>(block, prow);
        case QMC_CLASS_REAL6M:
        case QMC_CLASS_REAL6SM:
        case QMC_CLASS_REAL6TM: return occupancy_cls<6, 4, 6, false, true>(block, prow);
#elif QMC_PART == 3
        case QMC_CLASS_REAL3H: return occupancy_cls<3, 2, 4, false, false, true>(block, prow);
        case QMC_CLASS_REAL6H: return occupancy_cls<6, 4, 6, false, false, true>(block, prow);
        case QMC_CLASS_CPLX3H: return occupancy_cls<3, 2, 4, true, false, true>(block, prow);
#endif
        default: return 0;
    }
}

#if QMC_PART == 0
extern "C" int qmc_k_launch_eval_part1(int, const QmcLaunch *, int, int, int, void *);
extern "C" int qmc_k_launch_eval_part2(int, const QmcLaunch *, int, int, int, void *);
extern "C" int qmc_k_launch_eval_part3(int, const QmcLaunch *, int, int, int, void *);
extern "C" int qmc_k_occupancy_part1(int, int, int);
extern "C" int qmc_k_occupancy_part2(int, int, int);
extern "C" int qmc_k_occupancy_part3(int, int, int);

extern "C" int qmc_k_launch_eval(int cls, const QmcLaunch *L, int block, int ppt, int grid, void *stream) {
    int (*const parts[4])(int, const QmcLaunch *, int, int, int, void *) = {
        qmc_k_launch_eval_part0, qmc_k_launch_eval_part1, qmc_k_launch_eval_part2, qmc_k_launch_eval_part3};
    for (auto f : parts) {
        const int rc = f(cls, L, block, ppt, grid, stream);
        if (rc != -2) return rc;
    }
    return -2;
}

extern "C" int qmc_k_launch_finish(const QmcLaunch *L, void *stream) {
    if (L->njobs <= 0) return 0;
    qmc_finish_kernel<<<L->njobs, 128, 0, (cudaStream_t)stream>>>(*L);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_lattice_points(uint64_t n, const uint32_t *z_dev, int d, const double *delta_dev,
                                    uint64_t k0, uint64_t count, double *x_dev, uint64_t *r_dev,
                                    void *stream) {
    if (count == 0) return 0;
    const uint64_t threads = (count + kQmcLatticeRun - 1) / kQmcLatticeRun;
    const unsigned grid = (unsigned)((threads + 255) / 256);
    qmc_lattice_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, 1.0 / (double)n, z_dev, d, delta_dev, k0,
                                                               count, x_dev, r_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_shifts(uint64_t state, int m, int d, double *out_dev, void *stream) {
    const int total = m * d;
    if (total <= 0) return 0;
    qmc_shift_kernel<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(state, m, d, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_log(const double *x_dev, uint64_t n, double *out_dev, void *stream) {
    if (n == 0) return 0;
    qmc_log_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_atan2(const double *yx_dev, uint64_t n, double *out_dev, void *stream) {
    if (n == 0) return 0;
    qmc_atan2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(yx_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_korobov(const double *x_dev, uint64_t n, double *out_dev, void *stream) {
    if (n == 0) return 0;
    qmc_korobov_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_rcp(const double *x_dev, uint64_t n, double *out_dev, void *stream) {
    if (n == 0) return 0;
    qmc_rcp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, out_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_fp64_probe(double *out_dev, int iters, int grid, int block, void *stream) {
    qmc_fp64_probe_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(out_dev, iters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_fp32_probe(float *out_dev, int iters, int grid, int block, void *stream) {
    qmc_fp32_probe_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(out_dev, iters);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_sm_count(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v;
}

extern "C" int qmc_k_occupancy(int cls, int block, int prow) {
    int (*const parts[4])(int, int, int) = {qmc_k_occupancy_part0, qmc_k_occupancy_part1, qmc_k_occupancy_part2,
                                            qmc_k_occupancy_part3};
    for (auto f : parts) {
        const int v = f(cls, block, prow);
        if (v) return v;
    }
    return 0;
}

// ---------------------------------------------------------------- no-allocation variant
// Fixed scratch for qmc_eval_jobs_noalloc: [0, 256) queue counter and status
// words, then the job table, then the tile partial sums. Every GPU that loads
// the library holds it until the process exits; every call shares it.
namespace {
constexpr size_t kNoallocJobOff = 256;
constexpr size_t kNoallocPartOff = kNoallocJobOff + (size_t)QMC_NOALLOC_MAX_JOBS * sizeof(QmcJobDev);
static_assert(kNoallocPartOff % 256 == 0, "partials must stay 256-byte aligned");
static_assert(QMC_NOALLOC_BYTES > kNoallocPartOff, "scratch too small");
__device__ __align__(256) unsigned char qmc_noalloc_scratch[QMC_NOALLOC_BYTES];
void *g_noalloc_ptr[64];  // device address of the array, per device (host stand-in is not one)
}  // namespace

extern "C" size_t qmc_k_noalloc_partial_capacity(void) {
    return (QMC_NOALLOC_BYTES - kNoallocPartOff) / sizeof(double);
}

// Set-up once per device (the device must be current): look up the array's
// device address. Not thread-safe against a concurrent first call on the
// same device.
extern "C" int qmc_k_noalloc_setup(int device, void **ptr) {
    if (device < 0 || device >= 64) return -1;
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, qmc_noalloc_scratch) != cudaSuccess || !p) return -1;
        g_noalloc_ptr[device] = p;
    }
    *ptr = g_noalloc_ptr[device];
    return 0;
}

// Queue the evaluation of `njobs` host job records of one kernel class into
// the fixed scratch, then copy the status words to `status_host`. The caller
// synchronises the stream before reading `status_host`.
extern "C" int qmc_k_noalloc_eval(int device, int cls, const QmcJobDev *jobs_host, int njobs,
                                  const QmcLaunch *tmpl, int block, int ppt, int sm_count,
                                  unsigned long long *status_host, void *stream) {
    void *base = nullptr;
    if (qmc_k_noalloc_setup(device, &base)) return -1;
    if (njobs < 1 || njobs > QMC_NOALLOC_MAX_JOBS) return -2;
    if (tmpl->ntiles * (uint64_t)(2 * tmpl->norders) > qmc_k_noalloc_partial_capacity()) return -2;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *b = (unsigned char *)base;
    QmcLaunch L = *tmpl;
    L.queue = (unsigned long long *)b;
    L.status = (unsigned long long *)(b + 64);
    L.jobs = (const QmcJobDev *)(b + kNoallocJobOff);
    L.partials = (double *)(b + kNoallocPartOff);
    L.njobs = njobs;
    // what must start at zero: the tile counter and the status words
    if (cudaMemsetAsync(b, 0, 128, st) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(b + kNoallocJobOff, jobs_host, (size_t)njobs * sizeof(QmcJobDev),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return -1;
    int occ = qmc_k_occupancy(cls, block, L.prow);
    if (occ < 1) occ = 1;
    uint64_t g = (uint64_t)sm_count * occ;
    if (L.ntiles < g) g = L.ntiles;
    const int grid = g < 1 ? 1 : (int)g;
    if (L.ntiles > 0 && qmc_k_launch_eval(cls, &L, block, ppt, grid, stream)) return -1;
    if (qmc_k_launch_finish(&L, stream)) return -1;
    if (cudaMemcpyAsync(status_host, b + 64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return -1;
    return 0;
}
#endif  // QMC_PART == 0
