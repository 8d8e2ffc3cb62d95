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
