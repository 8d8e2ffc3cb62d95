"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Bit-exact: lattice indices r, shifted points x, random shifts. FP64 per-shift
sums: within RTOL = 1e-12 of the oracle (see tests/parity.py for the
derivation). Sizes span several tiles and a ragged tail (every n is prime,
so no tile size divides it); the full-size case is the bench workload.
"""
import numpy as np
import pytest

import oracle
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w
from paper_2305_19768_gb300.inputs.lattice import lattice_for, lattice_sizes

from parity import Gpu, assert_close, oracle_sums

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    g = Gpu()
    yield g
    g.close()


def _specs(iid, sectors, points, n, m, seed=1, lam=0.0, nsec_total=None):
    nsec_total = nsec_total or len(sectors)
    out = []
    for p in points:
        for s in sectors:
            out.append(dict(integral_id=iid, sector=s, point=p, shifts=m, n=n, seed=seed,
                            stream=p * nsec_total + s, **{"lambda": lam}))
    return out


# ---------------------------------------------------------------- bit-exact
# large primes with explicit generating vectors (every component < n is in U_n)
EXPLICIT_Z = {100000007: [1, 39435, 7612354, 23817, 99999, 12345678],
              4294967291: [4294967290, 3000000019]}


@pytest.mark.parametrize("n,d", [(1009, 3), (1000003, 3), (100000007, 6), (4294967291, 2)])
def test_lattice_points_bit_exact(gpu, n, d):
    if n in EXPLICIT_Z:
        z = np.array(EXPLICIT_Z[n][:d], dtype=np.uint32)
    else:
        z = np.array(lattice_for(n, d)[1], dtype=np.uint32)
    delta = oracle.shifts(5, 3, 1, d)[0]
    for k0 in (0, n // 3, n - 777):
        cnt = min(777, n - k0)
        xg, rg = qmc.qmc_lattice_points(gpu.ctx, n, z, delta, k0, cnt)
        xo, ro = oracle.lattice_points(n, z, delta, k0, cnt)
        assert np.array_equal(rg, ro)
        assert np.array_equal(xg.view(np.uint64), xo.view(np.uint64))


def test_lattice_points_bit_exact_whole_lattice(gpu):
    """Every point of shifted lattices, walked in runs the way the evaluator
    walks them: the integer path (rounding of r/n read off its 64-place
    binary expansion, exact sum with the shift, the fold above 1), the FP64
    path of the coordinates with r/n < 2^-12, and shifts that are not
    multiples of 2^-64 (FP64 path throughout)."""
    n = 1000003
    z = np.array(lattice_for(n, 3)[1], dtype=np.uint32)
    for s in range(2):
        delta = oracle.shifts(9, s, 1, 3)[0]
        xg, rg = qmc.qmc_lattice_points(gpu.ctx, n, z, delta, 0, n)
        xo, ro = oracle.lattice_points(n, z, delta, 0, n)
        assert np.array_equal(rg, ro)
        assert np.array_equal(xg.view(np.uint64), xo.view(np.uint64))
    rng = np.random.default_rng(12)
    for n in (4294967291, 2147483648, 99991):
        z = np.array([int(rng.integers(1, n)) | 1 for _ in range(3)], dtype=np.uint32)
        for delta in (oracle.shifts(3, 1, 1, 3)[0], np.array([0.5, 2.0 ** -60, 1.0 - 2.0 ** -53]),
                      np.array([3e-20, 0.7 + 2.0 ** -40, 1e-300])):
            k0 = int(rng.integers(0, max(1, n - 300000)))
            cnt = min(300000, n - k0)
            xg, rg = qmc.qmc_lattice_points(gpu.ctx, n, z, delta, k0, cnt)
            xo, ro = oracle.lattice_points(n, z, delta, k0, cnt)
            assert np.array_equal(rg, ro)
            assert np.array_equal(xg.view(np.uint64), xo.view(np.uint64)), (n, delta)


def test_lattice_division_exhaustive(gpu):
    # every r of one lattice, and random r near 2^32: the corrected division is RN(r/n)
    n = 1000003
    x, r = qmc.qmc_lattice_points(gpu.ctx, n, np.array([1], dtype=np.uint32), np.zeros(1), 0, n)
    expect = np.arange(n, dtype=np.float64) / float(n)
    assert np.array_equal(x[:, 0].view(np.uint64), expect.view(np.uint64))
    rng = np.random.default_rng(4)
    for n in (4294967291, 2147483647, 100000007, 65537, 3):
        z = np.array([int(rng.integers(1, n))], dtype=np.uint32)
        k0 = int(rng.integers(0, max(1, n - 100000)))
        cnt = min(100000, n - k0)
        xg, rg = qmc.qmc_lattice_points(gpu.ctx, n, z, np.zeros(1), k0, cnt)
        assert np.array_equal(xg[:, 0].view(np.uint64), (rg[:, 0].astype(np.float64) / float(n)).view(np.uint64))


def test_korobov3_against_exact_rationals(gpu):
    """The integer-pipe korobov3 (t = phi(u), 1 - t = phi(1 - u) and
    u (1 - u)) against the exact rational values at each double u: within
    0.55 ulp, on both halves of (0, 1), at the ends, at tiny u and at 1/2."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    us = np.concatenate([rng.uniform(0.0, 1.0, 20000), np.exp(rng.uniform(-55, 0, 5000)),
                         1.0 - np.exp(rng.uniform(-36, -1, 5000)),
                         np.array([0.5, np.nextafter(0.5, 0.0), np.nextafter(0.5, 1.0), 2.0 ** -60, 1e-25,
                                   np.nextafter(1.0, 0.0), 2.0 ** -11, 0.25, 0.75])])
    us = us[(us > 0) & (us < 1)]
    t, omt, ws = qmc.qmc_korobov3(gpu.ctx, us)

    def ulps(got, exact):
        return float(abs(Fraction(float(got)) - exact) / Fraction(float(np.spacing(float(exact)))))

    worst = [0.0, 0.0, 0.0]
    for u, gt, go, gw in zip(us, t, omt, ws):
        U = Fraction(float(u))
        V = 1 - U
        worst[0] = max(worst[0], ulps(gt, U ** 4 * (35 - 84 * U + 70 * U ** 2 - 20 * U ** 3)))
        worst[1] = max(worst[1], ulps(go, V ** 4 * (35 - 84 * V + 70 * V ** 2 - 20 * V ** 3)))
        worst[2] = max(worst[2], ulps(gw, U * V))
    assert max(worst) <= 0.55, worst
    t0, o0, w0 = qmc.qmc_korobov3(gpu.ctx, np.zeros(1))
    assert t0[0] == 0.0 and o0[0] == 1.0 and w0[0] == 0.0


def test_evaluator_reciprocal_within_one_ulp(gpu):
    rng = np.random.default_rng(6)
    xs = np.concatenate([rng.uniform(0.5, 2.0, 200000), np.exp(rng.uniform(-700, 700, 200000)),
                         np.exp(rng.uniform(-50, 50, 1000)),
                         np.array([1.0, 2.0, 3.0, 1e-300, 1e300, 0.1])])
    got = qmc.qmc_fp64_rcp(gpu.ctx, xs)
    ref = 1.0 / xs                      # IEEE division: correctly rounded
    err = np.abs(got - ref) / np.spacing(np.abs(ref))
    assert err.max() <= 1.0, (err.max(), xs[np.argmax(err)])


def test_evaluator_atan2_within_4_ulp(gpu):
    rng = np.random.default_rng(8)
    th = rng.uniform(-np.pi, np.pi, 100000)
    r = np.exp(rng.uniform(-20, 20, 100000))
    y = np.concatenate([r * np.sin(th), rng.uniform(-1, 1, 50000) * 10.0 ** rng.uniform(-30, 30, 50000),
                        np.array([0.0, -0.0, 1.0, -1.0, 1e-300, 0.0, -0.0])])
    x = np.concatenate([r * np.cos(th), rng.uniform(-1, 1, 50000) * 10.0 ** rng.uniform(-30, 30, 50000),
                        np.array([-1.0, -1.0, -0.0, 0.0, -1.0, 2.0, 3.0])])
    got = qmc.qmc_fp64_atan2(gpu.ctx, y, x)
    ref = np.arctan2(y, x)               # libm, within 1 ulp; signed-zero conventions of IEEE
    err = np.abs(got - ref) / np.maximum(np.spacing(np.abs(ref)), np.spacing(0.0))
    assert err.max() <= 4.0, (err.max(), y[np.argmax(err)], x[np.argmax(err)])
    assert np.array_equal(np.signbit(got), np.signbit(ref))


def test_evaluator_log_within_0_51_ulp(gpu):
    """The fixed-point logarithm: within 1 ulp of libm everywhere, within
    0.51 ulp of the exact logarithm (50-digit decimal) on inputs next to 1, at
    and between the table's points F_j = 1 + j/1024, over the exponent range
    and on subnormals; IEEE results for zero, infinity, negative and NaN."""
    from decimal import Decimal, getcontext
    rng = np.random.default_rng(5)
    k = np.arange(1, 5001, dtype=np.float64)
    Fj = 1.0 + np.arange(1025) / 1024.0
    xs = np.concatenate([rng.uniform(0.5, 2.0, 200000), np.exp(rng.uniform(-700, 700, 200000)),
                         1.0 + rng.uniform(-1e-3, 1e-3, 50000), 1.0 + k * 2.0 ** -52, 1.0 - k * 2.0 ** -53,
                         (Fj[:, None] * (1 + rng.uniform(-1e-6, 1e-6, (1025, 4)))).ravel(),
                         ((Fj[:-1] + 0.5 / 1024)[:, None] * (1 + rng.uniform(-1e-9, 1e-9, (1024, 4)))).ravel(),
                         np.array([1.0, 2.0, 0.5, 1e-300, 1e300, 5e-324, 1e-310, 2.2250738585072014e-308,
                                   1.7976931348623157e308])])
    got = qmc.qmc_fp64_log(gpu.ctx, xs)
    ref = np.log(xs)
    ulp = np.spacing(np.abs(ref))
    ulp[ref == 0] = np.spacing(0.0)
    assert (np.abs(got - ref) / ulp).max() <= 1.0
    getcontext().prec = 50
    sample = np.concatenate([np.arange(0, 450000, 450), np.arange(450000, len(xs))])
    worst = 0.0
    for i in sample:
        exact = Decimal(float(xs[i])).ln()
        err = abs(Decimal(float(got[i])) - exact) / Decimal(float(np.spacing(abs(float(exact)))))
        worst = max(worst, float(err))
    assert worst <= 0.51, worst
    spec = qmc.qmc_fp64_log(gpu.ctx, np.array([0.0, -0.0, np.inf, -1.0, np.nan, -np.inf]))
    assert spec[0] == -np.inf and spec[1] == -np.inf and spec[2] == np.inf and np.isnan(spec[3:]).all()


def test_shifts_bit_exact(gpu):
    for seed, stream, m, d in ((1, 0, 32, 3), (12345, 77, 7, 6), (2**63 + 5, 2**40, 3, 2)):
        g = qmc.qmc_shifts(gpu.ctx, seed, stream, m, d)
        o = oracle.shifts(seed, stream, m, d)
        assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


# ---------------------------------------------------------------- FP64 sums
def _compare_integral(gpu, I, inv_points, n, m, lo, norders, lam=None, sectors=None, seed=1):
    iid = gpu.load(I)
    inv_arr = np.array(inv_points, dtype=np.float64).reshape(len(inv_points), -1)
    qmc.qmc_set_kinematics(gpu.ctx, inv_arr if inv_arr.shape[1] else np.zeros((0, 0)))
    sectors = list(range(len(I.sectors))) if sectors is None else sectors
    pts = list(range(len(inv_points)))
    specs = _specs(iid, sectors, pts, n, m, seed=seed, lam=lam if lam is not None else 0.0,
                   nsec_total=len(I.sectors))
    out, fails, rc = gpu.eval(iid, specs, lo, norders)
    assert rc == 0, qmc.qmc_last_error(gpu.ctx)
    out = out.reshape(len(specs), m, norders, 2)
    worst = 0.0
    for i, sp in enumerate(specs):
        o, a, c = oracle_sums(I, sp["sector"], list(inv_points[sp["point"]]), n, m, seed,
                              sp["stream"], lo, norders, lam)
        worst = max(worst, assert_close(out[i], o, a, c, lo=lo,
                                        what=f"{I.name} n={n} sector {sp['sector']} point {sp['point']}"))
    return worst


def test_triangle_massive_sums(gpu):
    I = w.triangle_massive()
    _compare_integral(gpu, I, [[]], 10007, 8, 0, 1)


def test_massless_box_sums(gpu):
    I = w.box_massless()
    _compare_integral(gpu, I, [[-3.0, -2.0]], 20011, 4, -2, 3)


def test_massless_box_two_points_more_orders(gpu):
    I = w.box_massless()
    _compare_integral(gpu, I, [[-3.0, -2.0], [-5.0, -1.0]], 4001, 3, -2, 4, sectors=[0, 5, 11])


def test_deformed_massive_box_sums(gpu):
    I = w.box_massive()
    pts = [[12.0, -3.0], [7.5, -1.5], [19.0, -7.0]]
    _compare_integral(gpu, I, pts, 10007, 4, 0, 1, lam=0.3)


def test_deformed_bubbles_and_triangle(gpu):
    _compare_integral(gpu, w.bubble(1, "s"), [[10.0]], 4001, 4, 0, 2, lam=0.5)
    _compare_integral(gpu, w.bubble(0, "s"), [[10.0]], 4001, 4, 0, 2, lam=0.5)
    _compare_integral(gpu, w.triangle_one_offshell(0, "s"), [[10.0]], 4001, 4, -2, 3, lam=0.3)


def test_double_box_sectors_d6(gpu):
    # the d <= 6 evaluator: sectors with 1, 2, 3 and 4 singular variables, eps^-4..eps^0
    I = w.double_box_massless()
    by_ns = {}
    for i, s in enumerate(I.sectors):
        by_ns.setdefault(len(s.singular), i)
    sectors = [by_ns[k] for k in sorted(by_ns)]
    _compare_integral(gpu, I, [[-3.0, -1.0]], 1009, 2, -4, 5, sectors=sectors)


def test_baker_transform_sums():
    g = Gpu(transform=qmc.QMC_TRANSFORM_BAKER)
    try:
        I = w.box_massless()
        iid = g.load(I)
        qmc.qmc_set_kinematics(g.ctx, np.array([[-3.0, -2.0]]))
        specs = _specs(iid, [0, 4, 9], [0], 4001, 3, nsec_total=12)
        out, _, rc = g.eval(iid, specs, -2, 3)
        assert rc == 0
        out = out.reshape(3, 3, 3, 2)
        for i, sp in enumerate(specs):
            _, z = lattice_for(4001, 3)
            view = oracle.SectorView(I, sp["sector"], [-3.0, -2.0], transform=1)
            o, a, _, c = oracle.shift_sums(view, 4001, z, oracle.shifts(1, sp["stream"], 3, 3), -2, 3,
                                           with_cond=True)
            assert_close(out[i], o, a, c, what=f"baker sector {sp['sector']}")
    finally:
        g.close()


def test_median_rule_and_explicit_vectors(gpu):
    I = w.box_massless()
    iid = gpu.load(I)
    qmc.qmc_set_kinematics(gpu.ctx, np.array([[-3.0, -2.0]]))
    n, r, sector = 20011, 11, 5
    spec = dict(integral_id=iid, sector=sector, point=0, shifts=1, n=n, seed=1, stream=5)
    z, est = qmc.qmc_median_lattice(gpu.ctx, spec, -2, 3, r, 99)
    cands = qmc.qmc_median_candidates(n, 3, r, 99)
    view = oracle.SectorView(I, sector, [-3.0, -2.0])
    o_est = []
    for i in range(r):
        o, a, _, c = oracle.shift_sums(view, n, cands[i, :3], np.zeros((1, 3)), -2, 3, with_cond=True)
        assert_close(est[i][None], o, a, c, what=f"candidate {i}")
        o_est.append(o[0, 2, 0])
    assert list(z[:3]) == list(cands[int(np.argsort(o_est, kind="stable")[r // 2]), :3])
    # random shifts of the chosen lattice through an explicit generating vector
    spec2 = dict(spec, shifts=4, z=list(z))
    out, _, rc = gpu.eval(iid, [spec2], -2, 3)
    assert rc == 0
    o, a, _, c = oracle.shift_sums(view, n, z[:3], oracle.shifts(1, 5, 4, 3), -2, 3, with_cond=True)
    assert_close(out.reshape(4, 3, 2), o, a, c, what="median lattice with shifts")


def test_tiny_lattices_below_one_tile(gpu):
    # n smaller than one tile and than one thread's PPT span; custom lattices
    I = w.box_massless()
    iid = gpu.load(I)
    qmc.qmc_set_kinematics(gpu.ctx, np.array([[-3.0, -2.0]]))
    for n, z in ((2, [1, 1, 1]), (3, [1, 2, 1]), (7, [1, 3, 2]), (131, [1, 37, 55])):
        qmc.qmc_set_lattices(gpu.ctx, np.array([n], dtype=np.uint64),
                             np.array([z + [1, 1, 1]], dtype=np.uint32))
        specs = _specs(iid, [0, 4], [0], n, 2, nsec_total=12)
        out, _, rc = gpu.eval(iid, specs, -2, 3)
        assert rc == 0
        out = out.reshape(2, 2, 3, 2)
        for i, sp in enumerate(specs):
            view = oracle.SectorView(I, sp["sector"], [-3.0, -2.0])
            dl = oracle.shifts(1, sp["stream"], 2, 3)
            o, a, _, c = oracle.shift_sums(view, n, z, dl, -2, 3, with_cond=True)
            assert_close(out[i], o, a, c, what=f"n={n}")


def test_full_size_sampled_outputs():
    """Bench workload (massless box, n = 1000003, m = 32, all 12 sectors, same
    launch configuration as bench.py); the oracle recomputes sampled
    (sector, shift) outputs one by one at full n."""
    g = Gpu()
    try:
        I = w.box_massless()
        iid = g.load(I)
        qmc.qmc_set_kinematics(g.ctx, np.array([[-3.0, -2.0]]))
        n, m = 1000003, 32
        specs = _specs(iid, list(range(12)), [0], n, m)
        out, _, rc = g.eval(iid, specs, -2, 3)
        assert rc == 0
        out = out.reshape(12, m, 3, 2)
        for sector, shift in ((0, 0), (5, 17), (11, 31)):
            o, a, c = oracle_sums(I, sector, [-3.0, -2.0], n, m, 1, sector, -2, 3, shift_rows=[shift])
            assert_close(out[sector, shift][None], o, a, c, lo=-2,
                         what=f"box1L_massless n={n} full-size sector {sector} shift {shift}")
        # property at any size: the mean over shifts reproduces the closed form
        from golden_values import closed_form
        ex = closed_form("box1L_massless", "s=-3,t=-2")
        sec = out[..., 0] + 1j * out[..., 1]       # [12][m][3]
        tot = sec.sum(axis=0)                       # [m][3] sector sum per shift
        pref = np.array(I.prefactor)
        res = np.array([[sum(pref[p] * tot[s, o - p] for p in range(o + 1)) for o in range(3)]
                        for s in range(m)])
        mean = res.mean(0)
        err = res.real.std(0, ddof=1) / np.sqrt(m)
        for o, order in enumerate((-2, -1, 0)):
            assert abs(mean[o] - ex[order]) <= 4 * err[o] + 1e-12
    finally:
        g.close()


# ---------------------------------------------------------------- status / errors
def test_sign_check_reported(gpu):
    I = w.box_massive()
    iid = gpu.load(I)
    qmc.qmc_set_kinematics(gpu.ctx, np.array([[12.0, -3.0]]))
    specs = _specs(iid, [0], [0], 1009, 2, lam=-0.3, nsec_total=4)
    out, fails, rc = gpu.eval(iid, specs, 0, 1)
    assert rc == -6 and fails > 0
    specs = _specs(iid, [0], [0], 1009, 2, lam=0.3, nsec_total=4)
    out, fails, rc = gpu.eval(iid, specs, 0, 1)
    assert rc == 0 and fails == 0


def test_invalid_inputs_rejected(gpu):
    I = w.box_massless()
    iid = gpu.load(I)
    qmc.qmc_set_kinematics(gpu.ctx, np.array([[-3.0, -2.0]]))
    with pytest.raises(qmc.QmcError) as e:
        jobs, nj = qmc.make_jobs(_specs(iid, [0], [0], 1000, 2, nsec_total=12))  # 1000 not tabulated
        qmc.qmc_plan_create(gpu.ctx, jobs, nj, -2, 3)
    assert e.value.code == -1
    with pytest.raises(qmc.QmcError) as e:
        qmc.qmc_load_sectors_mem(gpu.ctx, "qmc-sectors 1 name broken")
    assert e.value.code == -2
    bad = I.to_text().replace("a -1 -1 0", "a -5 -1 0", 1)   # below a = -4: no Taylor subtraction
    with pytest.raises(qmc.QmcError) as e:
        qmc.qmc_load_sectors_mem(gpu.ctx, bad)
    assert e.value.code == -1
    with pytest.raises(qmc.QmcError) as e:
        qmc.qmc_set_lattices(gpu.ctx, np.array([10], dtype=np.uint64), np.array([[2, 1, 1, 1, 1, 1]]))
    assert e.value.code == -1


def test_degree1_subtraction_sectors(gpu):
    # sectors with one a_j = -2 variable (the d <= 3 Taylor-subtraction class)
    # against the oracle: the pinned 1-D and 2-D polynomial cases and a 3-D
    # sector with eps-dependent exponents of U and F and a second (a = -1)
    # singular variable
    from test_oracle_pins import _toy_integral

    I1 = _toy_integral(1, [-2], [1.25], {(0,): 1.0, (1,): 2.0, (2,): 3.0, (3,): -1.0})
    _compare_integral(gpu, I1, [[]], 4001, 4, -1, 4)
    I2 = _toy_integral(2, [-2, -1], [-1.5, 0.75],
                       {(0, 0): 1.0, (1, 0): -2.0, (0, 1): 0.5, (1, 1): 3.0, (2, 1): -2.0, (3, 0): 1.5})
    _compare_integral(gpu, I2, [[]], 4001, 4, -2, 4)
    I3 = _toy_integral(3, [-2, 0, -1], [1.0, 0.5, -2.0],
                       {(0, 0, 0): 1.0, (1, 0, 0): 1.0, (0, 1, 0): 2.0, (1, 1, 1): 0.5},
                       u0=-1, u1=2, Fterms={(0, 0, 0): 2.0, (1, 0, 1): 1.0, (0, 2, 0): 0.5}, f0=-2, f1=-1)
    _compare_integral(gpu, I3, [[]], 2003, 4, -2, 4)


def test_geometric_sectors_and_weights(gpu):
    # sectors from the geometric decomposition through the evaluator: the massless
    # box (all sectors), double-box sectors of every singular-variable count, and a
    # sector with a weight other than 1 (applied per tile on the device)
    I = w.box_massless(method="geometric")
    _compare_integral(gpu, I, [[-3.0, -2.0]], 10007, 4, -2, 3)
    D = w.double_box_massless(method="geometric")
    by_ns = {}
    for i, s in enumerate(D.sectors):
        by_ns.setdefault(len(s.singular), i)
    _compare_integral(gpu, D, [[-3.0, -1.0]], 2003, 2, -4, 5, sectors=sorted(by_ns.values()))
    T = w.triangle_massive(method="geometric")
    T.sectors[1].weight = 3
    _compare_integral(gpu, T, [[]], 4001, 4, 0, 1)
