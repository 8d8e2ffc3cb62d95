"""Parity of the Taylor-subtraction evaluators (sectors with exponents
a_j <= -2; the d <= 3 and d <= 6 classes) against the oracle: per-shift sums
element by element, under korobov3 and under the baker transform, on toy
sectors of every subtraction degree (p = 2, 3, 4, one to three such
variables, d = 1 to 4) and on the one- and two-loop massless boxes in
D = 2 - 2 eps, including lattices whose tiles take 2048 points.

Under korobov3 the subtracted integrand cancels p orders of t near the border
(about 2^-53 |g| t^-p), so both sides' sums there are dominated by rounding;
the bound's corner-mass term (CTOL_TAYLOR times the summed magnitudes of the
terms before they cancel, Taylor-coefficient terms included) is what holds
them together. Under baker the sums are accurate to far better than that."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w
from paper_2305_19768_gb300.inputs.lattice import lattice_for

from parity import CTOL_TAYLOR, Gpu, assert_close
from subtraction_cases import CASES, DEFORMED_CASES
from test_oracle_pins import _toy_integral

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1], ids=["korobov3", "baker"])
def gpu_tr(request):
    g = Gpu(transform=request.param)
    yield g, request.param
    g.close()


def _toy(case):
    d, a, b, U, u0, u1, F, f0, f1, lo, no, _ = CASES[case]
    fr = lambda v: {e: Fraction(str(c)) for e, c in v.items()}
    return _toy_integral(d, a, [Fraction(x) for x in b], fr(U), u0=Fraction(str(u0)), u1=Fraction(str(u1)),
                         Fterms=fr(F), f0=Fraction(str(f0)), f1=Fraction(str(f1))), lo, no


def _compare(g, tr, I, inv, n, m, lo, no, sectors=None, seed=3, lam=None):
    iid = g.load(I)
    inv_arr = np.array([inv], dtype=np.float64) if inv else np.zeros((0, 0))
    qmc.qmc_set_kinematics(g.ctx, inv_arr)
    sectors = list(range(len(I.sectors))) if sectors is None else sectors
    specs = [dict(integral_id=iid, sector=s, point=0, shifts=m, n=n, seed=seed, stream=s,
                  **{"lambda": 0.0 if lam is None else lam}) for s in sectors]
    out, fails, rc = g.eval(iid, specs, lo, no)
    assert rc == 0, qmc.qmc_last_error(g.ctx)
    out = out.reshape(len(specs), m, no, 2)
    for i, sp in enumerate(specs):
        s = I.sectors[sp["sector"]]
        _, z = lattice_for(n, s.d)
        view = oracle.SectorView(I, sp["sector"], list(inv), lam, transform=tr)
        o, a, f, c = oracle.shift_sums(view, n, z, oracle.shifts(seed, sp["stream"], m, s.d), lo, no,
                                       with_cond=True)
        assert_close(out[i], o, a, c, lo=lo, ctol=CTOL_TAYLOR,
                     what=f"{I.name} tr={tr} n={n} sector {sp['sector']} a={list(s.a)}")


@pytest.mark.parametrize("case", range(len(CASES)))
def test_toy_sectors_every_degree(gpu_tr, case):
    g, tr = gpu_tr
    I, lo, no = _toy(case)
    _compare(g, tr, I, [], 4001, 4, lo, no)


def test_toy_sectors_large_tiles(gpu_tr):
    # n >= 16384: 2048-point tiles and the ragged last tile of each shift
    g, tr = gpu_tr
    for case in (1, 3, 6):
        I, lo, no = _toy(case)
        _compare(g, tr, I, [], 100003, 2, lo, no)


def test_massless_box_d2_all_sectors(gpu_tr):
    # D = 2 - 2 eps: 12 sectors with one or two a_j = -2 (the d <= 3 class)
    g, tr = gpu_tr
    I = w.box_massless_d2()
    _compare(g, tr, I, [-3.0, -2.0], 10007, 4, -2, 3)


def test_double_box_d2_sectors_of_every_box(gpu_tr):
    # D = 2 - 2 eps: one sector per (singular variables, Taylor box) pair, boxes
    # of 2 to 72 coefficients in up to four variables (the d <= 6 class)
    g, tr = gpu_tr
    I = w.double_box_massless_d2()
    seen, sel = set(), []
    for i, s in enumerate(I.sectors):
        key = (len(s.singular), int(np.prod([-a for a in s.a if a <= -1])))
        if key not in seen:
            seen.add(key)
            sel.append(i)
    _compare(g, tr, I, [-3.0, -1.0], 1009, 2, -4, 5, sectors=sel)


def _deformed_toy(case):
    d, a, b, U, u0, u1, F, f0, f1, lo, no, _, lam = DEFORMED_CASES[case]
    fr = lambda v: {e: Fraction(str(c)) for e, c in v.items()}
    I = _toy_integral(d, a, [Fraction(x) for x in b], fr(U), u0=Fraction(str(u0)), u1=Fraction(str(u1)),
                      Fterms=fr(F), f0=Fraction(str(f0)), f1=Fraction(str(f1)))
    I.sectors[0].deform = True
    return I, lo, no, float(Fraction(lam[0]))


@pytest.mark.parametrize("case", range(len(DEFORMED_CASES)))
def test_deformed_toy_sectors(gpu_tr, case):
    # contour-deformed sectors with a_j <= -2 (the deformed Taylor class); one
    # lambda for every variable of a job
    g, tr = gpu_tr
    I, lo, no, lam = _deformed_toy(case)
    _compare(g, tr, I, [], 4001, 4, lo, no, lam=lam)
    if case == 0:
        _compare(g, tr, I, [], 100003, 2, lo, no, lam=lam)


def test_deformed_massless_box_d2_physical(gpu_tr):
    # D = 2 - 2 eps at a physical point (s = 9, t = -2): all 12 sectors deformed
    g, tr = gpu_tr
    I = w.box_massless_d2(deform=True)
    _compare(g, tr, I, [9.0, -2.0], 4001, 4, -2, 3, lam=0.3)
