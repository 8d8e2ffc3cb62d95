// Natural logarithm of a double in integer fixed-point arithmetic.
//
// The evaluator's logarithms run here on the integer pipe instead of the
// FP64 pipe (on this GPU one FP64 warp instruction occupies the FP64 pipe for
// tens of cycles, an integer one for about two). The method is Tang's
// table-driven reduction (ACM TOMS 16, 1990) carried out exactly in fixed
// point:
//   x = 2^e m, m in [1, 2); F = 1 + j/1024 nearest to m (j = 0..1024);
//   f = (m - F)/F, |f| <= 2^-11, held as f 2^74 in an int64;
//   log1p(f) = f (1 - f c(f)),  c(f) = 1/2 - f/3 + f^2/4 - f^3/5 + f^4/6
//     (truncation below 2^-79 relative), c by Horner in Q63;
//   ln x = e ln2 + ln F + log1p(f), summed in a signed 128-bit Q116 number
//     (|ln x| < 745 < 2^9.6, and the smallest nonzero result, near x = 1,
//     still has 64 significant bits), and rounded once to nearest-even.
// The table row j holds RN(2^63/F) and RN(2^116 ln F) (low, high words); both
// are exact for F = 1 and F = 2, where e ln2 + ln F cancels. Measured
// against 50-digit logarithms: within 0.501 ulp (correctly rounded except
// next to a rounding tie). Subnormal inputs are normalised first; zero gives
// -inf, +inf gives +inf, negative numbers and NaN give NaN.
//
// Written for both the device (the evaluator) and a host compiler, with the
// 128-bit integer type of GCC and NVCC.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define QMC_HD __host__ __device__ __forceinline__
#else
#define QMC_HD static inline
#include <string.h>
#endif

#define QMC_ILOG_LN2_LO 0x9abc9e3b39803f2fULL   // RN(2^116 ln 2), low word
#define QMC_ILOG_LN2_HI 0xb17217f7d1cf7ULL      //                  high word
#define QMC_ILOG_C2 0x4000000000000000LL        // RN(2^63 / k), k = 2..6
#define QMC_ILOG_C3 0x2aaaaaaaaaaaaaabLL
#define QMC_ILOG_C4 0x2000000000000000LL
#define QMC_ILOG_C5 0x199999999999999aLL
#define QMC_ILOG_C6 0x1555555555555555LL

typedef unsigned __int128 qmc_u128;

QMC_HD uint64_t qmc_bits_of(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}
QMC_HD double qmc_double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}
QMC_HD int qmc_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}
// high 64 bits of the signed 128-bit product
QMC_HD int64_t qmc_smulhi(int64_t a, int64_t b) {
#if defined(__CUDA_ARCH__)
    return __mul64hi(a, b);
#else
    return (int64_t)(((__int128)a * b) >> 64);
#endif
}

// ln(2^e (1 + frac63 2^-63)), frac63 in [0, 2^63), |e| <= 1074: the
// reduction and the Q116 sum, rounded once. tab: 3 words per row
// j = 0..1024: RN(2^63/F_j), RN(2^116 ln F_j) low, high.
QMC_HD double qmc_ilog_core(int e, uint64_t frac63, const uint64_t *tab) {
    const int j = (int)((frac63 + (1ULL << 52)) >> 53);   // 0..1024
    const int64_t ri = (int64_t)frac63 - ((int64_t)j << 53);   // (m - F) 2^63, in [-2^52, 2^52)
    const bool fneg = ri < 0;
    const uint64_t ra = fneg ? (uint64_t)(-ri) : (uint64_t)ri;
    // |f| 2^74 = |m - F| 2^63 RN(2^63/F) 2^-52 (truncated; exact for F = 1, 2)
    const uint64_t fm = (uint64_t)(((qmc_u128)ra * tab[3 * j]) >> 52);
    const int64_t fq = fneg ? -(int64_t)fm : (int64_t)fm;
    // c(f) in Q63: each step c <- C_k - f c, with f c = (f 2^74)(c 2^63) 2^-74
    int64_t c = QMC_ILOG_C6;
    c = QMC_ILOG_C5 - (qmc_smulhi(fq, c) >> 10);
    c = QMC_ILOG_C4 - (qmc_smulhi(fq, c) >> 10);
    c = QMC_ILOG_C3 - (qmc_smulhi(fq, c) >> 10);
    c = QMC_ILOG_C2 - (qmc_smulhi(fq, c) >> 10);
    const uint64_t h = (1ULL << 63) - (uint64_t)(qmc_smulhi(fq, c) >> 10);   // (1 - f c) 2^63
    const qmc_u128 lp = ((qmc_u128)fm * h) >> 21;     // |log1p f| 2^116
    const uint64_t ea = (uint64_t)(e < 0 ? -e : e);
    const qmc_u128 el = (qmc_u128)ea * QMC_ILOG_LN2_LO + ((qmc_u128)(ea * QMC_ILOG_LN2_HI) << 64);
    const qmc_u128 lf = ((qmc_u128)tab[3 * j + 2] << 64) | tab[3 * j + 1];
    qmc_u128 S = lf + (fneg ? (qmc_u128)0 - lp : lp) + (e < 0 ? (qmc_u128)0 - el : el);   // mod 2^128
    const bool neg = (uint64_t)(S >> 127) != 0;
    if (neg) S = (qmc_u128)0 - S;
    const uint64_t hi = (uint64_t)(S >> 64), lo = (uint64_t)S;
    if ((hi | lo) == 0) return 0.0;                   // x = 1
    // round S 2^-116 to 53 bits: S < 2^126, so the leading bit is at 127 - lz, lz >= 2
    const int lz = hi ? qmc_clz64(hi) : 64 + qmc_clz64(lo);
    const qmc_u128 N = S << lz;
    const uint64_t nh = (uint64_t)(N >> 64), nl = (uint64_t)N;
    uint64_t mant = nh >> 11;
    const bool round_bit = ((nh >> 10) & 1) != 0;
    const bool sticky = (nh & 0x3FF) != 0 || nl != 0;
    mant += (round_bit && (sticky || (mant & 1))) ? 1 : 0;
    // value 2^(11 - lz) (mant 2^-52); a carry out of mant moves into the exponent
    const uint64_t out = ((uint64_t)(1023 + 11 - lz - 1) << 52) + mant;
    return qmc_double_of(out | ((uint64_t)neg << 63));
}

QMC_HD double qmc_ilog(double x, const uint64_t *tab) {
    const uint64_t bits = qmc_bits_of(x);
    if (bits - 1ULL >= 0x7FEFFFFFFFFFFFFFULL) {      // zero, inf, NaN or negative
        if ((bits << 1) == 0) return qmc_double_of(0xFFF0000000000000ULL);   // -inf
        if (bits == 0x7FF0000000000000ULL) return x;                          // +inf
        return qmc_double_of(0x7FF8000000000000ULL);                          // NaN
    }
    int e = (int)(bits >> 52) - 1023;
    uint64_t mb = bits & 0xFFFFFFFFFFFFFULL;
    if (e == -1023) {                                 // subnormal: normalise the mantissa
        const int p = 63 - qmc_clz64(bits);
        e = p - 1074;
        mb = (bits << (52 - p)) & 0xFFFFFFFFFFFFFULL;
    }
    return qmc_ilog_core(e, mb << 11, tab);
}
