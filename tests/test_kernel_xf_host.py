"""The evaluator's integer-pipe arithmetic of the corner stage
(csrc/qmc_xf.h: 64-bit-mantissa floating point products and sums, the
reciprocal, integer powers, RN to FP64 and the logarithm of a 64-bit
mantissa) is plain
integer C++ shared by the device and a host compiler. Built here with g++,
it is checked against exact rational arithmetic (Python integers and
fractions), so the bounds the kernel relies on are pinned on the CPU; the
GPU parity tests run the same code on the device."""
import ctypes
import shutil
import subprocess
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

from test_kernel_math_host import CSRC

HARNESS = r"""
#include "qmc_xf.h"
#include "qmc_log_table.h"
static const uint64_t kTab[3 * QMC_LOG_TABLE_ROWS] = QMC_LOG_TABLE_INIT;
static qmc_xf mk(const uint64_t *m, const int32_t *e, const int32_t *s, long i) { return qmc_xf{m[i], e[i], s[i]}; }
static void put(qmc_xf r, uint64_t *m, int32_t *e, int32_t *s, long i) { m[i] = r.m; e[i] = r.e; s[i] = r.neg; }
extern "C" {
void xf_of(const double *x, uint64_t *m, int32_t *e, int32_t *s, long n) {
    for (long i = 0; i < n; ++i) put(qmc_xf_of(x[i]), m, e, s, i);
}
void xf_to(const uint64_t *m, const int32_t *e, const int32_t *s, double *y, long n) {
    for (long i = 0; i < n; ++i) y[i] = qmc_xf_to_double(mk(m, e, s, i));
}
void xf_mul(const uint64_t *am, const int32_t *ae, const int32_t *as, const uint64_t *bm, const int32_t *be,
            const int32_t *bs, uint64_t *m, int32_t *e, int32_t *s, long n) {
    for (long i = 0; i < n; ++i) put(qmc_xf_mul(mk(am, ae, as, i), mk(bm, be, bs, i)), m, e, s, i);
}
void xf_add(const uint64_t *am, const int32_t *ae, const int32_t *as, const uint64_t *bm, const int32_t *be,
            const int32_t *bs, uint64_t *m, int32_t *e, int32_t *s, long n) {
    for (long i = 0; i < n; ++i) put(qmc_xf_add(mk(am, ae, as, i), mk(bm, be, bs, i)), m, e, s, i);
}
void xf_rcp(const uint64_t *am, const int32_t *ae, const int32_t *as, uint64_t *m, int32_t *e, int32_t *s, long n) {
    for (long i = 0; i < n; ++i) put(qmc_xf_rcp(mk(am, ae, as, i)), m, e, s, i);
}
void xf_ipow(const uint64_t *am, const int32_t *ae, const int32_t *as, const int32_t *k, uint64_t *m, int32_t *e,
             int32_t *s, long n) {
    for (long i = 0; i < n; ++i) {
        const qmc_xf x = mk(am, ae, as, i);
        put(qmc_xf_ipow(x, qmc_xf_rcp(x), k[i]), m, e, s, i);
    }
}
void xf_log(const uint64_t *am, const int32_t *ae, const int32_t *as, double *y, long n) {
    for (long i = 0; i < n; ++i) y[i] = qmc_ilog_xf(mk(am, ae, as, i), kTab);
}
// the d <= 6 kernel's corner sequence: U, F, Cc exact, reciprocals where a
// negative exponent needs them, B = Cc U^u0 F^f0 rounded once, ln(U^u1 F^f1)
void corner(const double *U, const double *F, const double *C, const int32_t *k, double *B, double *L, long n) {
    for (long i = 0; i < n; ++i) {
        const int u0 = k[4 * i], f0 = k[4 * i + 1], u1 = k[4 * i + 2], f1 = k[4 * i + 3];
        const qmc_xf u = qmc_xf_of(U[i]), f = qmc_xf_of(F[i]), c = qmc_xf_of(C[i]);
        const qmc_xf ru = (u0 < 0 || u1 < 0) ? qmc_xf_rcp(u) : u;
        const qmc_xf rf = (f0 < 0 || f1 < 0) ? qmc_xf_rcp(f) : f;
        B[i] = qmc_xf_to_double(qmc_xf_mul(c, qmc_xf_mul(qmc_xf_ipow(u, ru, u0), qmc_xf_ipow(f, rf, f0))));
        L[i] = qmc_ilog_xf(qmc_xf_mul(qmc_xf_ipow(u, ru, u1), qmc_xf_ipow(f, rf, f1)), kTab);
    }
}
}
"""

U64, I32 = np.uint64, np.int32


@pytest.fixture(scope="module")
def X(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("xf")
    src, lib = d / "h.cpp", d / "libxf.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(lib)],
                   check=True, capture_output=True)
    return ctypes.CDLL(str(lib))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _arrs(n):
    return np.zeros(n, U64), np.zeros(n, I32), np.zeros(n, I32)


def xf_of(X, x):
    x = np.ascontiguousarray(x, np.float64)
    m, e, s = _arrs(x.size)
    X.xf_of(_p(x), _p(m), _p(e), _p(s), ctypes.c_long(x.size))
    return m, e, s


def exact(m, e, s):
    """The xf values as exact fractions."""
    out = []
    for mi, ei, si in zip(m.tolist(), e.tolist(), s.tolist()):
        v = Fraction(int(mi)) * Fraction(2) ** (int(ei) - 63)
        out.append(-v if si else v)
    return out


def rand_xf(rng, n, emin=-300, emax=300):
    m = rng.integers(0, 2 ** 63, n, dtype=np.uint64) | np.uint64(1 << 63)
    e = rng.integers(emin, emax, n).astype(I32)
    s = rng.integers(0, 2, n).astype(I32)
    return m, e, s


def test_xf_of_double_is_exact_and_rounds_back(X):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(2000) * np.exp(rng.uniform(-700, 700, 2000)),
                        [5e-324, -1e-310, 2.2250738585072014e-308, 1.7976931348623157e308, 1.0, -0.5]])
    m, e, s = xf_of(X, x)
    for xi, v in zip(x.tolist(), exact(m, e, s)):
        assert v == Fraction(xi)
    assert np.all(m >> np.uint64(63) == 1)
    y = np.empty_like(x)
    X.xf_to(_p(m), _p(e), _p(s), _p(y), ctypes.c_long(x.size))
    assert np.array_equal(y, x)


def test_xf_to_double_rounds_to_nearest_even(X):
    rng = np.random.default_rng(2)
    m, e, s = rand_xf(rng, 4000, -1100, 1030)
    # ties and near-ties at the 53-bit rounding point
    m[:500] = (m[:500] & ~np.uint64((1 << 11) - 1)) | np.uint64(1 << 10)
    y = np.empty(m.size)
    X.xf_to(_p(m), _p(e), _p(s), _p(y), ctypes.c_long(m.size))
    for yi, v in zip(y.tolist(), exact(m, e, s)):
        try:
            ref = float(v)        # Fraction -> float is correctly rounded (ties to even)
        except OverflowError:
            ref = float("-inf") if v < 0 else float("inf")
        assert yi == ref or (yi == 0.0 and ref == 0.0), (yi, ref)


def test_xf_products_truncate_below_2_62(X):
    rng = np.random.default_rng(3)
    a, b = rand_xf(rng, 3000), rand_xf(rng, 3000)
    m, e, s = _arrs(3000)
    X.xf_mul(*map(_p, a), *map(_p, b), _p(m), _p(e), _p(s), ctypes.c_long(3000))
    assert np.all(m >> np.uint64(63) == 1)
    for va, vb, vr in zip(exact(*a), exact(*b), exact(m, e, s)):
        p = va * vb
        assert (vr >= 0) == (p >= 0)
        err = (abs(p) - abs(vr)) / abs(p)
        assert 0 <= err < Fraction(1, 2 ** 62)


def test_xf_sums_within_2_62_of_the_larger_operand(X):
    rng = np.random.default_rng(8)
    n = 4000
    a, b = rand_xf(rng, n, -20, 20), rand_xf(rng, n, -20, 20)
    # cancellation: equal exponents and nearby mantissas of opposite sign, exact
    # negatives, exponent gaps 0..70, and zeros on either side
    b[0][:500] = a[0][:500] ^ rng.integers(0, 2 ** 20, 500).astype(U64)
    b[1][:500] = a[1][:500]
    b[2][:500] = 1 - a[2][:500]
    b[0][500:600], b[1][500:600], b[2][500:600] = a[0][500:600], a[1][500:600], 1 - a[2][500:600]
    b[1][600:1300] = a[1][600:1300] - np.arange(700) // 10
    a[0][1300:1350] = 0
    a[1][1300:1350] = -(1 << 20)
    b[0][1350:1400] = 0
    b[1][1350:1400] = -(1 << 20)
    m, e, s = _arrs(n)
    X.xf_add(*map(_p, a), *map(_p, b), _p(m), _p(e), _p(s), ctypes.c_long(n))
    for va, vb, (mi, vr) in zip(exact(*a), exact(*b), zip(m.tolist(), exact(m, e, s))):
        ref = va + vb
        assert mi == 0 or mi >= 2 ** 63
        if ref == 0:
            assert vr == 0
            continue
        assert abs(vr - ref) < max(abs(va), abs(vb)) * Fraction(1, 2 ** 62)
        assert abs(vr - ref) < abs(ref) * Fraction(1, 2 ** 61) or abs(va + vb) < max(abs(va), abs(vb)) / 2


def test_xf_reciprocal_within_2_59(X):
    rng = np.random.default_rng(4)
    a = rand_xf(rng, 3000)
    # edges of the mantissa range: 1, just above 1, just below 2, FP32 seeds at 2.0
    a[0][:6] = np.array([1 << 63, (1 << 63) + 1, (1 << 64) - 1, (1 << 63) + (1 << 39), (1 << 63) + (1 << 40) - 1,
                         0xC000000000000000], dtype=np.uint64)
    m, e, s = _arrs(3000)
    X.xf_rcp(*map(_p, a), _p(m), _p(e), _p(s), ctypes.c_long(3000))
    assert np.all(m >> np.uint64(63) == 1)
    for va, vr in zip(exact(*a), exact(m, e, s)):
        ref = 1 / va
        assert (vr >= 0) == (ref >= 0)
        assert abs(vr - ref) / abs(ref) < Fraction(1, 2 ** 59)


def test_xf_integer_powers(X):
    rng = np.random.default_rng(5)
    a = rand_xf(rng, 900, -60, 60)
    k = np.tile(np.arange(-4, 5, dtype=I32), 100)
    m, e, s = _arrs(900)
    X.xf_ipow(*map(_p, a), _p(k), _p(m), _p(e), _p(s), ctypes.c_long(900))
    for va, ki, vr in zip(exact(*a), k.tolist(), exact(m, e, s)):
        ref = va ** int(ki)
        assert abs(vr - ref) / abs(ref) < Fraction(5, 2 ** 59)


def test_log_of_64_bit_mantissas_against_exact_values(X):
    rng = np.random.default_rng(7)
    n = 3000
    a = rand_xf(rng, n, -1000, 1000)
    a[2][:] = 0
    # next to 1 (both sides), at table points and at the extremes of the mantissa
    a[0][:400] = np.uint64(1 << 63) + rng.integers(0, 2 ** 20, 400).astype(U64)
    a[1][:400] = 0
    a[0][400:800] = np.uint64((1 << 64) - 1) - rng.integers(0, 2 ** 20, 400).astype(U64)
    a[1][400:800] = -1
    y = np.empty(n)
    X.xf_log(*map(_p, a), _p(y), ctypes.c_long(n))
    getcontext().prec = 60
    worst = 0.0
    for (mi, ei), yi in zip(zip(a[0].tolist(), a[1].tolist()), y.tolist()):
        x = Decimal(int(mi)) * Decimal(2) ** (int(ei) - 63)
        ref = x.ln()
        if ref == 0:
            assert yi == 0.0
            continue
        worst = max(worst, float(abs(Decimal(yi) - ref) / Decimal(float(np.spacing(abs(float(ref)))))))
    assert worst <= 0.51, worst
    # exponents beyond the double range (products of powers): e RN(ln 2) +
    # ln(mantissa), within 1.5 ulp
    b = rand_xf(rng, 200, 1001, 4000)
    b[1][100:] *= -1
    b[2][:] = 0
    yb = np.empty(200)
    X.xf_log(*map(_p, b), _p(yb), ctypes.c_long(200))
    for (mi, ei), yi in zip(zip(b[0].tolist(), b[1].tolist()), yb.tolist()):
        ref = (Decimal(int(mi)) * Decimal(2) ** (int(ei) - 63)).ln()
        assert abs(Decimal(yi) - ref) <= Decimal(1.5) * Decimal(float(np.spacing(abs(float(ref))))), (ei, yi)
    # zero and negative inputs
    z = (np.array([0, 1 << 63], U64), np.array([0, 3], I32), np.array([0, 1], I32))
    yz = np.empty(2)
    X.xf_log(*map(_p, z), _p(yz), ctypes.c_long(2))
    assert yz[0] == -np.inf and np.isnan(yz[1])


def test_corner_values_within_one_rounding_of_exact(X):
    """The corner sequence of the d <= 6 kernel (B_V = Cc U^u0 F^f0 and
    ln(U^u1 F^f1) from exact conversions, integer reciprocals and products)
    against exact rational powers: B within 0.5 ulp plus the 2^-56 the
    products may lose, the logarithm within 0.51 ulp of the exact logarithm
    of the exact power."""
    rng = np.random.default_rng(11)
    n = 600
    U = np.exp(rng.uniform(-5, 8, n))
    F = np.exp(rng.uniform(-6, 6, n))
    C = np.exp(rng.uniform(-40, 0, n))
    # the double box's (1, -3, 3, -2), the box's (0, -2, 2, -1), random others
    k = rng.integers(-4, 5, (n, 4)).astype(I32)
    k[:100] = (1, -3, 3, -2)
    k[100:200] = (0, -2, 2, -1)
    k = np.ascontiguousarray(k)
    B, L = np.empty(n), np.empty(n)
    X.corner(_p(U), _p(F), _p(C), _p(k), _p(B), _p(L), ctypes.c_long(n))
    getcontext().prec = 60
    worst_b = worst_l = 0.0
    for i in range(n):
        u0, f0, u1, f1 = (int(v) for v in k[i])
        fu, ff, fc = Fraction(float(U[i])), Fraction(float(F[i])), Fraction(float(C[i]))
        b = fc * fu ** u0 * ff ** f0
        worst_b = max(worst_b, float(abs(Fraction(float(B[i])) - b) / Fraction(float(np.spacing(float(b))))))
        x = fu ** u1 * ff ** f1
        ref = (Decimal(x.numerator) / Decimal(x.denominator)).ln()
        if ref != 0:
            worst_l = max(worst_l, float(abs(Decimal(float(L[i])) - ref) / Decimal(float(np.spacing(abs(float(ref)))))))
    assert worst_b <= 0.5 + 2.0 ** -3, worst_b
    assert worst_l <= 0.51, worst_l
