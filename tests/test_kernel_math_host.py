"""The evaluator's integer fixed-point logarithm (csrc/qmc_ilog.h) is plain
integer C++ shared by the device and a host compiler. Built here with g++,
it is checked on the CPU against the exact logarithm (50-digit decimal) and
against IEEE conventions, so the arithmetic the kernel runs is pinned even
without a GPU; the GPU test of the same function runs it on the device."""
import ctypes
import os
import shutil
import subprocess
from decimal import Decimal, getcontext

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2305_19768_gb300", "csrc")

HARNESS = r"""
#include "qmc_ilog.h"
#include "qmc_log_table.h"
static const uint64_t kTab[3 * QMC_LOG_TABLE_ROWS] = QMC_LOG_TABLE_INIT;
extern "C" void ilog_many(const double *x, double *y, long n) {
    for (long i = 0; i < n; ++i) y[i] = qmc_ilog(x[i], kTab);
}
"""


@pytest.fixture(scope="module")
def ilog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("ilog")
    src, lib = d / "h.cpp", d / "libilog.so"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(lib)],
                   check=True, capture_output=True)
    L = ctypes.CDLL(str(lib))

    def run(xs):
        xs = np.ascontiguousarray(xs, dtype=np.float64)
        ys = np.empty_like(xs)
        L.ilog_many(xs.ctypes.data_as(ctypes.c_void_p), ys.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(xs.size))
        return ys

    return run


def test_integer_log_against_exact_values(ilog):
    rng = np.random.default_rng(23)
    k = np.arange(1, 2001, dtype=np.float64)
    Fj = 1.0 + np.arange(1025) / 1024.0
    xs = np.concatenate([1.0 + k * 2.0 ** -52, 1.0 - k * 2.0 ** -53,
                         (Fj[:, None] * (1 + rng.uniform(-1e-6, 1e-6, (1025, 2)))).ravel(),
                         ((Fj[:-1] + 0.5 / 1024)[:, None] * (1 + rng.uniform(-1e-9, 1e-9, (1024, 2)))).ravel(),
                         np.exp(rng.uniform(-744, 709, 4000)), rng.uniform(0.5, 2.0, 4000),
                         np.array([5e-324, 1e-310, 2.2250738585072014e-308, 1.7976931348623157e308, 2.0, 0.5])])
    xs = xs[xs > 0]
    got = ilog(xs)
    getcontext().prec = 50
    worst = 0.0
    for x, g in zip(xs, got):
        exact = Decimal(float(x)).ln()
        if exact == 0:
            assert g == 0.0
            continue
        worst = max(worst, float(abs(Decimal(float(g)) - exact) / Decimal(float(np.spacing(abs(float(exact)))))))
    assert worst <= 0.51, worst


def test_integer_log_against_libm_and_special_values(ilog):
    rng = np.random.default_rng(29)
    xs = np.exp(rng.uniform(-700, 700, 200000))
    got, ref = ilog(xs), np.log(xs)
    assert (np.abs(got - ref) / np.spacing(np.abs(ref))).max() <= 1.0
    spec = ilog(np.array([1.0, 0.0, -0.0, np.inf, -1.0, np.nan, -np.inf]))
    assert spec[0] == 0.0 and not np.signbit(spec[0])
    assert spec[1] == -np.inf and spec[2] == -np.inf and spec[3] == np.inf
    assert np.isnan(spec[4:]).all()


def test_log_table_rows_are_exact_roundings():
    """Rows of qmc_log_table.h: RN(2^63 / F_j) checked with exact rationals,
    RN(2^116 ln F_j) with 60-digit decimal logarithms, on every 16th row and
    the ends (F = 1 and F = 2 must be exact: ln F cancels e ln 2 there)."""
    import re
    from fractions import Fraction

    text = open(os.path.join(CSRC, "qmc_log_table.h")).read()
    body = text[text.index("QMC_LOG_TABLE_INIT"):text.index("}", text.index("QMC_LOG_TABLE_INIT"))]
    words = [int(w, 16) for w in re.findall(r"0x[0-9a-f]+(?=ULL)", body)]
    assert len(words) == 3 * 1025
    getcontext().prec = 60
    for j in list(range(0, 1025, 16)) + [1, 1023, 1024]:
        F = Fraction(1024 + j, 1024)
        inv, lo, hi = words[3 * j:3 * j + 3]
        q = Fraction(2 ** 63) / F
        assert inv == round(q)                                   # round() on Fraction: nearest
        L = (Decimal(1024 + j) / Decimal(1024)).ln() * (Decimal(2) ** 116)
        assert (hi << 64) | lo == int(L.to_integral_value())     # ROUND_HALF_EVEN, no ties here
    assert words[0:3] == [2 ** 63, 0, 0]
    ln2 = int(((Decimal(2)).ln() * (Decimal(2) ** 116)).to_integral_value())
    assert (words[3 * 1024 + 2] << 64) | words[3 * 1024 + 1] == ln2 and words[3 * 1024] == 2 ** 62
