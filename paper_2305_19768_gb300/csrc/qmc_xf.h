// Extended-mantissa floating point on the integer pipe.
//
// On this GPU an FP64 warp instruction occupies the FP64 pipe for tens of
// cycles and an integer one about two, so the exact parts of the real
// evaluator's corner stage run here in integer arithmetic (the subset sums of
// U and F, the reciprocals and integer powers of U and F at the corners, the
// eps series of each corner and the superset Moebius transform of the
// plus-distribution subtraction). Every result carries at least 56
// significant bits, more than FP64's 53, and is rounded once to nearest-even
// FP64 where it leaves this arithmetic.
//
// qmc_xf: |value| = m 2^(e - 63) with m in [2^63, 2^64) (normalised; m = 0 is
// zero) and a sign flag. Products keep the high 64 bits of the 128-bit
// mantissa product, shifted left by one where its top bit is clear (relative
// error below 2^-62 per product, always towards zero); sums align the
// smaller operand to the larger one (an error below 2^-62 of the larger).
//
// Written for both the device and a host compiler (tested on the CPU with
// g++ against 128-bit rational arithmetic in Python).
#pragma once
#include "qmc_ilog.h"

struct qmc_xf {
    uint64_t m;
    int32_t e;
    int32_t neg;
};

#define QMC_XF_ZERO_E (-(1 << 20))   // exponent of a zero (below every nonzero value's)

QMC_HD uint64_t qmc_umulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((qmc_u128)a * b) >> 64);
#endif
}

QMC_HD qmc_xf qmc_xf_one() { return qmc_xf{1ULL << 63, 0, 0}; }

// x (finite double) as xf: exact
QMC_HD qmc_xf qmc_xf_of(double x) {
    const uint64_t bits = qmc_bits_of(x);
    const int neg = (int)(bits >> 63);
    const int be = (int)((bits >> 52) & 0x7FF);
    const uint64_t frac = bits & 0xFFFFFFFFFFFFFULL;
    if (be != 0) return qmc_xf{(frac << 11) | (1ULL << 63), be - 1023, neg};
    if (frac == 0) return qmc_xf{0, QMC_XF_ZERO_E, neg};
    const int p = qmc_clz64(frac);                    // subnormal: normalise
    return qmc_xf{frac << p, -1011 - p, neg};
}

QMC_HD qmc_xf qmc_xf_mul(qmc_xf a, qmc_xf b) {
    const uint64_t h = qmc_umulhi(a.m, b.m);
    const int top = (int)(h >> 63);
    qmc_xf r;
    r.m = top ? h : (h << 1);
    r.e = a.e + b.e + top;
    r.neg = a.neg ^ b.neg;
    if (r.m == 0) r.e = QMC_XF_ZERO_E;
    return r;
}

// a + b: the operand of smaller magnitude is aligned to the larger one's
// exponent and the mantissas added or subtracted, then normalised; the bits
// shifted out (of the smaller operand, and of a sum that carries) are
// dropped: an error below 2^-62 of the larger operand
QMC_HD qmc_xf qmc_xf_add(qmc_xf a, qmc_xf b) {
    if (b.e > a.e || (b.e == a.e && b.m > a.m)) {    // zeros carry QMC_XF_ZERO_E
        const qmc_xf t = a;
        a = b;
        b = t;
    }
    const int d = a.e - b.e;
    const uint64_t bm = d < 64 ? (b.m >> d) : 0ULL;
    qmc_xf r;
    r.neg = a.neg;
    if (a.neg == b.neg) {
        const uint64_t s = a.m + bm;
        const int c = s < a.m ? 1 : 0;                 // carry out of bit 63
        r.m = c ? ((s >> 1) | (1ULL << 63)) : s;
        r.e = a.e + c;
    } else {
        const uint64_t s = a.m - bm;                   // |a| >= |b|
        if (s == 0) return qmc_xf{0, QMC_XF_ZERO_E, 0};
        const int p = qmc_clz64(s);
        r.m = s << p;
        r.e = a.e - p;
    }
    return r;
}

QMC_HD qmc_xf qmc_xf_neg(qmc_xf a) {
    a.neg ^= 1;
    return a;
}

// 1/a (a nonzero): Newton-Raphson y <- y + y (1 - m y) on m = a.m 2^-64 in
// [1/2, 1), y in Q62, from an FP32 reciprocal of the top 24 bits (error
// about 2^-22), two steps (2^-44, then the Q62 resolution). Relative error
// below 2^-59.
QMC_HD qmc_xf qmc_xf_rcp(qmc_xf a) {
    qmc_xf r;
    r.neg = a.neg;
    if (a.m == (1ULL << 63)) {                         // a power of two: exact
        r.m = a.m;
        r.e = -a.e;
        return r;
    }
    uint32_t fb = (126u << 23) | (uint32_t)((a.m >> 40) & 0x7FFFFFu);   // m rounded down to float
    float f, y0;
#if defined(__CUDA_ARCH__)
    f = __int_as_float((int)fb);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(f));
    const uint32_t yb = (uint32_t)__float_as_int(y0);
#else
    memcpy(&f, &fb, 4);
    y0 = 1.0f / f;
    uint32_t yb;
    memcpy(&yb, &y0, 4);
#endif
    // y0 in (1, 2]: Q62 from its bits (2.0 clamps just below 2^63)
    int64_t Y = ((yb >> 23) & 0xFF) >= 128 ? (int64_t)0x7FFFFFFFFFFFFFFFLL
                                           : (int64_t)((1ULL << 62) | ((uint64_t)(yb & 0x7FFFFFu) << 39));
    for (int it = 0; it < 2; ++it) {
        const int64_t P = (int64_t)qmc_umulhi(a.m, (uint64_t)Y);    // m y 2^62
        const int64_t E = (int64_t)(1ULL << 62) - P;                 // (1 - m y) 2^62
        Y += qmc_smulhi(Y, E) << 2;
        if (Y < 0) Y = 0x7FFFFFFFFFFFFFFFLL;            // (never: y < 2)
    }
    // 1/|a| = y 2^(-a.e - 1) with y = Y 2^-62 in (1, 2)
    r.m = (uint64_t)Y << 1;
    r.e = -a.e - 1;
    return r;
}

// a 2^k (k >= 0 small): exponent only
QMC_HD qmc_xf qmc_xf_ldexp(qmc_xf a, int k) {
    a.e += k;
    return a;
}

// RN(a) as a double (overflow to +-inf, gradual underflow)
QMC_HD double qmc_xf_to_double(qmc_xf a) {
    const uint64_t sgn = (uint64_t)a.neg << 63;
    if (a.m == 0) return qmc_double_of(sgn);
    int be = a.e + 1023;
    if (be >= 2047) return qmc_double_of(sgn | 0x7FF0000000000000ULL);
    int sh = 11;
    if (be < 1) {
        sh += 1 - be;
        be = 0;
        if (sh > 64) return qmc_double_of(sgn);        // below half the smallest subnormal
        if (sh == 64) return qmc_double_of(sgn | (a.m > (1ULL << 63) ? 1ULL : 0ULL));   // tie -> 0
    }
    uint64_t mant = a.m >> sh;
    const uint64_t rb = (a.m >> (sh - 1)) & 1ULL;
    const uint64_t sticky = a.m & ((1ULL << (sh - 1)) - 1ULL);
    mant += (rb && (sticky || (mant & 1ULL))) ? 1ULL : 0ULL;
    // normal: (be - 1) 2^52 + mant (mant holds the implicit bit, a carry moves
    // into the exponent); subnormal: mant itself
    const uint64_t bits = be >= 1 ? (((uint64_t)(be - 1) << 52) + mant) : mant;
    return qmc_double_of(sgn | bits);
}

// x^k for an integer |k| <= 4 from x and 1/x (ri): repeated products
QMC_HD qmc_xf qmc_xf_ipow(qmc_xf x, qmc_xf ri, int k) {
    const qmc_xf b = k < 0 ? ri : x;
    const int a = k < 0 ? -k : k;
    qmc_xf p = qmc_xf_one();
    if (a >= 1) p = b;
    for (int i = 1; i < a; ++i) p = qmc_xf_mul(p, b);
    return p;
}

// 1/i for i = 1..6 as xf (RN of the 64-bit mantissa)
QMC_HD qmc_xf qmc_xf_inv_int(int i) {
    switch (i) {
        case 2: return qmc_xf{1ULL << 63, -1, 0};
        case 3: return qmc_xf{0xAAAAAAAAAAAAAAABULL, -2, 0};
        case 4: return qmc_xf{1ULL << 63, -2, 0};
        case 5: return qmc_xf{0xCCCCCCCCCCCCCCCDULL, -3, 0};
        case 6: return qmc_xf{0xAAAAAAAAAAAAAAABULL, -3, 0};
        default: return qmc_xf_one();
    }
}

#define QMC_LN2 0.6931471805599453   // RN(ln 2)

// ln x for x > 0 given as xf (the logarithm of qmc_ilog.h on the 63-bit
// fraction), rounded once; a negative or zero x gives NaN / -inf like the
// double version. Exponents beyond the double range (|e| > 1000, products of
// powers) take e RN(ln 2) + ln(mantissa), two roundings.
QMC_HD double qmc_ilog_xf(qmc_xf x, const uint64_t *tab) {
    if (x.m == 0) return qmc_double_of(0xFFF0000000000000ULL);
    if (x.neg) return qmc_double_of(0x7FF8000000000000ULL);
    const uint64_t f = x.m & 0x7FFFFFFFFFFFFFFFULL;
    if (x.e > 1000 || x.e < -1000) return (double)x.e * QMC_LN2 + qmc_ilog_core(0, f, tab);
    return qmc_ilog_core(x.e, f, tab);
}
