"""FP64 and FP32 work per integrand evaluation (the roofline numerator).

One evaluation = one lattice point of one sector for one shift, all eps
orders, all subtraction corners. The count follows the evaluator's own
formulation of the method, operation by operation:

* FP64 flops: add, subtract and multiply count 1, a fused multiply-add 2.
  Steps that the evaluator computes on the integer pipe count 0 FP64 flops:
  the lattice coordinate (exact fixed-point walk), the korobov3 transform,
  every logarithm (fixed-point table reduction) and, in the d <= 6
  fixed-order kernel for sectors whose exponents are small integers, the
  corner stage (subset sums of U and F, their reciprocals and powers at the
  corners, in 64-bit-mantissa arithmetic).
  Multiplications by the constant 1 that the compiler folds away (first
  factors of products started at 1, the 1/1 of series recursions) are not
  counted.
* FP32 flops: the same rule for the monomial products of the
  mixed-precision classes.
* Transcendentals are counted separately, never as flops: logarithms
  (integer pipe), arctangents (table plus a series on the FP64 pipe; its
  FP64 operations are in the flop count), hardware reciprocal seeds
  (rcp.approx, followed by two Newton steps = 4 FMA counted as flops),
  exponentials and sine/cosine pairs (library); the integer-pipe
  reciprocals of the corner stage apart again (rcp_int).
* Only terms the requested orders need are counted: corner V carries its eps
  exponent only if hi + |V| >= 1, the ln t of a singular variable only if
  hi + ns - 1 >= 1, pole set P forms its series terms below hi + |P| + 1.

Workloads average the per-sector figures over their sectors (equal lattices).
"""
from __future__ import annotations

from dataclasses import dataclass, field

RCP_FLOPS = 8   # two Newton steps from the hardware seed: 4 FMA


@dataclass
class Work:
    fp64: float = 0.0
    fp32: float = 0.0
    log: float = 0.0
    atan2: float = 0.0
    rcp: float = 0.0
    exp: float = 0.0
    sincos: float = 0.0
    rcp_int: float = 0.0

    def add(self, other: "Work", scale: float = 1.0) -> "Work":
        for k in self.__dataclass_fields__:
            setattr(self, k, getattr(self, k) + scale * getattr(other, k))
        return self

    def as_dict(self):
        return {k: getattr(self, k) for k in self.__dataclass_fields__}

    def recip(self, count=1):
        self.fp64 += RCP_FLOPS * count
        self.rcp += count


def _popc(v: int) -> int:
    return bin(v).count("1")


def _sector_shape(sector):
    d = sector.d
    sing = [j for j in range(d) if sector.a[j] <= -1]
    ns = len(sing)
    emax = max(sector.U.max_var_exponent(), sector.F.max_var_exponent(), 1)
    for j in range(d):
        if sector.a[j] > 0:
            emax = max(emax, sector.a[j])
    return d, sing, ns, emax


def _is_small_int(x) -> bool:
    return float(x) == int(float(x)) and abs(float(x)) <= 4


def _grouped_poly(P, sing, ns):
    """Flops of the grouped monomial sums of one polynomial: per monomial its
    (nv - 1) power products and one FMA with the coefficient; the first
    monomial of each singular-mask group takes a multiply (or nothing, if
    constant) instead."""
    groups = {}
    for e in P.terms:
        mask = sum(1 << q for q, j in enumerate(sing) if e[j] > 0)
        groups.setdefault(mask, []).append(e)
    f = 0
    for mons in groups.values():
        for i, e in enumerate(mons):
            nv = sum(1 for x in e if x)
            if nv == 0:
                f += 0 if i == 0 else 1
            else:
                f += (nv - 1) + (1 if i == 0 else 2)
    return f


def _powers(d, emax):
    return d * ((emax >= 2) + (emax >= 3) + (emax >= 4))


def _assemble_fixed(ns, hi) -> float:
    """The real classes' assembly with the singular-variable count and the
    highest order fixed at compile time: corner series, superset Moebius
    transform, A_P and E_P by subset recursions, the pole sets' exponential
    series by Horner's rule (E/l, l >= 2, then one FMA per term), and every
    order from the leading pole eps^-ns up to eps^hi into the accumulator."""
    f = 0.0
    full = (1 << ns) - 1
    for V in range(full + 1):
        nV = hi + _popc(V) + 1
        for i in range(1, nV):
            f += 1 + (0 if i == 1 else 1)        # g_i = g_{i-1} Lambda (/ i)
    for q in range(ns):
        for P in range(full + 1):
            if not P & (1 << q):
                f += max(hi + _popc(P) + 1, 0)   # Moebius subtractions
    f += ns + max((1 << ns) - 2, 0)              # t_q / b_q, then A_P = A_{P-q} t_q / b_q
    f += ns                                      # b_q ln t_q
    for P in range(full):                        # E_P = E_{P+q} + b_q ln t_q
        q = (~P & -~P).bit_length() - 1
        if hi + _popc(P) + 1 > 1 and (P | (1 << q)) != full:
            f += 1
    for P in range(full + 1):
        np_ = _popc(P)
        nP = hi + np_ + 1
        if P != full:
            f += max(nP - 2, 0)                  # E / l, l >= 2
            f += sum(2 * k for k in range(nP))   # PE_k by Horner: k FMAs
        f += 2 * nP                              # res[k - |P|] += A_P PE_k
    f += 2 * (ns + hi + 1)                       # acc += res W, every order -ns .. hi
    return f


def _assemble(ns, lo, hi, nord, cplx: bool) -> float:
    """The general assembly (run-time orders; the deformed classes): corner
    series, superset Moebius transform, A_P, E_P and its exponential series,
    the convolution and res += A PE."""
    mul = 6 if cplx else 1          # value x value: complex product (2 FMA + 2 MUL) or one multiply
    fmul = 2 if cplx else 1         # value x real scalar
    f = 0.0
    full = (1 << ns) - 1
    for V in range(full + 1):
        nV = hi + _popc(V) + 1
        for i in range(1, nV):
            # g_i = g_{i-1} Lambda / i: complex x complex (cplx) or real x real, then x (1/i) unless i = 1
            f += mul + (0 if i == 1 else fmul)
    for q in range(ns):
        for P in range(full + 1):
            if P & (1 << q):
                continue
            nP = hi + _popc(P) + 1
            f += max(nP, 0) * (2 if cplx else 1)
    for P in range(full + 1):
        np_ = _popc(P)
        nP = hi + np_ + 1
        if nP < 1:
            continue
        if P not in (0, full):
            f += ns                          # A_P from its factors (runtime-selected start)
        if nP > 1 and P != full:
            f += 2 * (ns - np_)              # E_P = sum b_q ln t_q
            f += 2 * max(nP - 2, 0)          # e_l = e_{l-1} E / l, l >= 2
        for k in range(max(0, lo + np_), nP):
            if P != full:
                f += 2 * k * (2 if cplx else 1)   # PE_k += g_i e_{k-i}
        f += 2 * max(nord - max(0, -(lo + np_)), 0) * (2 if cplx else 1)   # res += A PE, every order in range
    return f


def _corners_fp64(w, ns, hi, u0, f0, u1, f1, u0i, f0i, comb, na_reg):
    """The corner stage in FP64: 1/F in pairs of corners, then per corner
    B = Cc U^u0 F^f0 and Lambda = Lc + ln(U^u1 F^f1)."""
    full = (1 << ns) - 1
    # 1/F at the corners that need it, in pairs
    needF = [V <= full and ((f0i and f0 < 0) or (hi + _popc(V) >= 1 and comb and f1 < 0))
             for V in range(1 << max(ns, 1))]
    for V in range(0, len(needF), 2):
        a, b = needF[V], (needF[V + 1] if V + 1 < len(needF) else False)
        if a and b:
            w.fp64 += 3
            w.recip()
        elif a or b:
            w.recip()
    for V in range(full + 1):
        lam_here = hi + _popc(V) >= 1
        if (u0i and u0 < 0) or (lam_here and comb and u1 < 0):
            w.recip()
        factors = 1 if na_reg else 0
        for e0, isint in ((u0, u0i), (f0, f0i)):
            if isint and e0 != 0:
                w.fp64 += abs(int(e0)) - 1
                factors += 1
            elif not isint:
                w.log += 1
                w.exp += 1
                w.fp64 += 1
                factors += 1
        w.fp64 += max(factors - 1, 0)    # B = Cc U^u0 F^f0
        if lam_here:
            if comb:
                # U^u1 F^f1 (each power 1 when its exponent is 0), then one log
                w.fp64 += max(abs(int(u1)) - 1, 0) + max(abs(int(f1)) - 1, 0) + 1
                w.log += 1
            else:
                w.log += 2
                w.fp64 += 3
            w.fp64 += 1                  # Lambda_V = Lc + log


def real_sector_work(sector, lo: int, norders: int, mixed: bool = False, fp64_corners: bool = False) -> Work:
    """Work of one evaluation in the real (undeformed) evaluator classes.
    fp64_corners: count the corner stage as FP64 work even where the kernel
    runs it on the integer pipe (the FP64-equivalent arithmetic of the
    formulation)."""
    d, sing, ns, emax = _sector_shape(sector)
    hi = lo + norders - 1
    w = Work()
    # transform on the integer pipe: only the product of the per-coordinate
    # weights u(1-u) is FP64
    w.fp64 += d - 1
    w.fp64 += 2                          # W = Ws^3
    # power tables and grouped monomial sums (FP32 in the mixed classes)
    pw = _powers(d, emax)
    polys = _grouped_poly(sector.U, sing, ns) + _grouped_poly(sector.F, sing, ns)
    if mixed:
        w.fp32 += pw + polys
        # the regular prefactor's powers t^a as FP64 products (the table is FP32)
        w.fp64 += sum(max(int(sector.a[j]) - 1, 0) for j in range(d) if sector.a[j] > 0)
    else:
        w.fp64 += pw + polys
    u0, f0, u1, f1 = (float(x) for x in (sector.u0, sector.f0, sector.u1, sector.f1))
    u0i, f0i = _is_small_int(u0), _is_small_int(f0)
    comb = _is_small_int(u1) and _is_small_int(f1)
    # the d <= 6 fixed-order kernel's integer-pipe corner stage (subset sums,
    # the reciprocals and powers of U and F at the corners); the d <= 3 kernel
    # keeps the FP64 corners
    xf = hi == 0 and u0i and f0i and comb and (d > 3 or ns > 2) and not fp64_corners
    if not xf:
        w.fp64 += 2 * ns * (1 << max(ns - 1, 0))   # subset sums of U and F
    need_lam = hi + ns >= 1
    nb_reg = sum(1 for j in range(d) if sector.a[j] > -1 and float(sector.b[j]) != 0.0)
    na_reg = sum(1 for j in range(d) if sector.a[j] > 0)
    if need_lam:
        w.log += nb_reg
        w.fp64 += 2 * nb_reg             # Lc += b_j ln t_j
    w.fp64 += max(na_reg - 1, 0)         # Cc = prod t^a
    if hi + ns - 1 >= 1:
        w.log += ns                      # ln t of the singular variables
    # A of the empty pole set, prod 1/t_q: one reciprocal per pair of singular
    # variables (of the pair's product) and one for an odd one left
    pairs, odd = ns // 2, ns % 2
    w.fp64 += pairs + max(pairs + odd - 1, 0)
    w.recip(pairs + odd)
    full = (1 << ns) - 1
    if xf:
        for V in range(full + 1):
            lam_here = hi + _popc(V) >= 1
            w.rcp_int += int(u0 < 0 or (lam_here and u1 < 0)) + int(f0 < 0 or (lam_here and f1 < 0))
            if lam_here:
                w.log += 1
                w.fp64 += 1 if nb_reg else 0     # Lambda_V = Lc + log
    else:
        _corners_fp64(w, ns, hi, u0, f0, u1, f1, u0i, f0i, comb, na_reg)
    if hi == 0:
        w.fp64 += _assemble_fixed(ns, hi)
    else:
        w.fp64 += _assemble(ns, lo, hi, norders, cplx=False)
        w.fp64 += 2 * norders            # acc += res W
    return w


def _derivative_flops(P, d: int):
    """Real flops of all first and second derivatives of P at a real point
    (the host's derivative tables: per derivative monomial its products and
    one FMA with the coefficient)."""
    f = 0
    for e in P.terms:
        vars_ = [j for j in range(d) if e[j]]
        nv = len(vars_)
        f += nv * (max(nv - 2, 0) + 2)
        f += (nv * (nv + 1) // 2) * (max(nv - 3, 0) + 2)
    return f


def _complex_poly_flops(P) -> int:
    # per monomial: (nv - 1) complex products (2 FMA + 2 MUL = 6) and the real
    # coefficient times the complex value added in (2 FMA = 4)
    f = 0
    for e in P.terms:
        nv = sum(1 for x in e if x)
        f += max(nv - 1, 0) * 6 + 4
    return f


def deformed_sector_work(sector, lo: int, norders: int, mixed: bool = False) -> Work:
    """Work of one evaluation in the deformed classes: korobov3 of u and 1 - u
    on the integer pipe; at each corner V the derivatives of F, the real
    matrix V_jk and det J in closed form, z and rho, U and F at z in complex
    arithmetic, the prefactor num/den with one complex reciprocal and, where
    the corner needs its eps exponent, one complex log of the product of its
    factors (a real log of the squared modulus and an atan2); then the
    assembly in complex arithmetic."""
    d, sing, ns, emax = _sector_shape(sector)
    hi = lo + norders - 1
    w = Work()
    w.fp64 += (d - 1) + 2                        # Ws products, W = Ws^3
    if ns:
        w.recip(ns)                              # 1/t of the singular variables
    if hi + ns - 1 >= 1:
        w.log += ns
    u0, f0, u1, f1 = (float(x) for x in (sector.u0, sector.f0, sector.u1, sector.f1))
    comb_all = (_is_small_int(u1) and _is_small_int(f1)
                and all(_is_small_int(b) for b in sector.b))
    nb = sum(1 for j in range(d) if float(sector.b[j]) != 0.0)
    na_reg = sum(1 for j in range(d) if sector.a[j] > 0)
    for V in range(1 << ns):
        per = Work()
        deriv = _derivative_flops(sector.F, d) + d * _powers(1, emax)
        if mixed:
            per.fp32 += deriv
        else:
            per.fp64 += deriv
        per.fp64 += 3 * d * d + 3 * d + 3 * d    # V_jk, rho = 1 - i g, z
        per.fp64 += {1: 0, 2: 5, 3: 26}.get(d, 26)   # det J in closed form
        cpoly = _complex_poly_flops(sector.U) + _complex_poly_flops(sector.F) + d * 6 * (emax - 1)
        if mixed:
            per.fp32 += cpoly
        else:
            per.fp64 += cpoly
        # num / den: complex products of the prefactor factors, 1/den, num x (1/den)
        nfac = ns + abs(int(u0)) + abs(int(f0)) + na_reg
        per.fp64 += 6 * nfac + 3 + 3 + 6
        per.recip()
        if hi + _popc(V) >= 1:
            if comb_all:
                per.fp64 += 6 * (nb + abs(int(u1)) + abs(int(f1))) + 6   # X = Xn conj(Xd)
                per.fp64 += 27                   # atan2: reduction, division, degree-7 series, octant
                per.atan2 += 1
                per.recip(2)                     # inside atan2 and 1/|Xd|^2
                per.fp64 += 3 + 3 + 1 + 1 + 2    # |Xn|^2, |Xd|^2, ratio, 0.5 x log, arg
                per.log += 1
            else:
                per.fp64 += 12 * (nb + 2)
                per.atan2 += nb + 2
                per.log += nb + 2
            per.fp64 += 12 * (hi + _popc(V))     # corner series B Lambda^i / i! (complex)
        w.add(per)
    w.fp64 += _assemble(ns, lo, hi, norders, cplx=True)
    w.fp64 += 4 * norders                        # acc += res W
    return w


def _ser_mul_pairs(NT: int, OFF: int, hmax: int) -> int:
    """FMAs of one truncated series product of the Taylor path (index i holds
    the order i - OFF; output orders above hmax skipped)."""
    return sum(1 for i in range(NT) if i - OFF <= hmax for k in range(NT) if 0 <= i + OFF - k < NT)


def taylor_sector_work(sector, lo: int, norders: int) -> Work:
    """Work of one evaluation of a sector with exponents a_j <= -2 (the
    Taylor-subtraction classes), counted along the kernel's loops: run-time
    series of NT = SMAX + LMAX orders, jets over the box prod_q p_q of each
    zeroed set V (products of two jets: prod_q p_q (p_q + 1) / 2 FMAs)."""
    d, sing, ns, _ = _sector_shape(sector)
    hi = lo + norders - 1
    p = [-int(sector.a[j]) for j in sing]
    box = 1
    for x in p:
        box *= x
    small = d <= 3 and ns <= 2 and box <= 16
    SMAX, LMAX = (2, 4) if small else (4, 6)
    NT, OFF = SMAX + LMAX, SMAX
    Hm = hi + ns
    smul = 2 * _ser_mul_pairs(NT, OFF, Hm)
    w = Work()
    w.fp64 += d - 1 + 2                        # korobov3 weight product, W = Ws^3
    for j in range(d):                         # regular factors
        if j in sing:
            continue
        a, b = int(sector.a[j]), float(sector.b[j])
        if a > 0:
            w.fp64 += a                        # t^a (a - 1) and Cc *= (1)
        if b != 0.0:
            w.log += 1
            w.fp64 += 2
    for pq in p:                               # per singular slot
        w.recip(2)                             # 1/t, 1/b
        w.log += 1
        w.fp64 += 1                            # b ln t
        w.fp64 += 2 * (Hm + 1)                 # e^{eps b ln t}
        w.fp64 += (pq - 1) + NT                # t^-p, psi
        for k in range(pq):
            w.fp64 += max(pq - k - 1, 0) + NT  # t^{k-p}, phi
            if k == pq - 1:
                w.fp64 += 1                    # pole 1/b
            else:
                w.fp64 += 1 + 2 * (Hm + 1)     # 1/(m + b eps)
    emax = max(sector.U.max_var_exponent(), sector.F.max_var_exponent(), 1)
    w.fp64 += _powers(d, emax)
    monos = list(sector.U.terms) + list(sector.F.terms)
    u0, f0 = float(sector.u0), float(sector.f0)
    for V in range(1 << ns):
        rad = [p[q] if (V >> q) & 1 and p[q] > 1 else 1 for q in range(ns)]
        J = 1
        pairs = 1
        for r in rad:
            J *= r
            pairs *= r * (r + 1) // 2
        K = sum(r - 1 for r in rad)
        jm = 2 * pairs                         # one jet product
        for e in monos:                        # U and F over the box
            keep = True
            for j in range(d):
                if e[j] == 0:
                    continue
                if j in sing and (V >> sing.index(j)) & 1:
                    q = sing.index(j)
                    if e[j] >= rad[q]:
                        keep = False
                else:
                    w.fp64 += 1
            if keep:
                w.fp64 += 1
        w.recip(2)                             # 1/U0, 1/F0
        w.fp64 += 2 * (J - 1)
        for _ in range(2):                     # ln(1 + x) by Horner
            w.fp64 += 1 + max(K - 1, 0) * (jm + 2) + jm
        w.fp64 += 6 * J                        # A, B
        w.fp64 += K * (jm + J + 1)             # exp(A) by Horner
        imax = min(K, Hm)
        w.fp64 += imax * (jm + J)              # E_i = E_{i-1} B / i
        inV = sum(1 for q in range(ns) if (V >> q) & 1)
        w.fp64 += J * (max(inV - 1, 0) * smul + smul + NT)   # sum_kappa g_kappa prod phi
        for e0 in (u0, f0):                    # base C U0^u0 F0^f0 e^{eps Lam0}
            if _is_small_int(e0):
                w.fp64 += max(abs(int(e0)) - 1, 0) + 1
            else:
                w.log += 1
                w.exp += 1
                w.fp64 += 2
        w.log += 2
        w.fp64 += 4                            # Lam0
        w.fp64 += 2 * (Hm + 1)
        w.fp64 += (ns - inV) * smul + smul + NT   # psi products, base x T, acc
    w.fp64 += 2 * norders                      # acc += res W
    return w


def _deriv_terms(terms, j):
    """Exponent tuples of dP/dt_j, merged by exponent (the host's table)."""
    out = []
    for e in terms:
        if e[j] == 0:
            continue
        f = list(e)
        f[j] -= 1
        f = tuple(f)
        if f not in out:
            out.append(f)
    return out


def deformed_taylor_sector_work(sector, lo: int, norders: int) -> Work:
    """Work of one evaluation of a deformed sector with exponents a_j <= -2
    (the deformed Taylor class), counted along the kernel's loops: real jet
    products of 2 flops per (i, j) pair, complex ones of 8, series products
    over NT = 6 orders."""
    d, sing, ns, _ = _sector_shape(sector)
    hi = lo + norders - 1
    p = [-int(sector.a[j]) for j in sing]
    SMAX, LMAX = 2, 4
    NT, OFF = SMAX + LMAX, SMAX
    Hm = hi + ns
    smul = 2 * _ser_mul_pairs(NT, OFF, Hm)
    emax = max(sector.U.max_var_exponent(), sector.F.max_var_exponent(), 1)
    for j in range(d):
        if sector.a[j] > 0:
            emax = max(emax, int(sector.a[j]))
    Fterms = list(sector.F.terms)
    dF = [_deriv_terms(Fterms, j) for j in range(d)]
    emax = max([emax] + [max(e) for tl in dF for e in tl if e])
    Hterms = {}
    for j in range(d):
        for l in range(j, d):
            Hterms[(j, l)] = _deriv_terms(dF[j], l)
    w = Work()
    w.fp64 += d - 1 + 2                        # korobov3 weight product, W = Ws^3
    for pq in p:                               # per singular slot (as the real class)
        w.recip(2)
        w.log += 1
        w.fp64 += 1 + 2 * (Hm + 1) + (pq - 1) + NT
        for k in range(pq):
            w.fp64 += max(pq - k - 1, 0) + NT
            w.fp64 += 1 if k == pq - 1 else 1 + 2 * (Hm + 1)
    w.fp64 += _powers(d, emax)
    u0, f0, u1, f1 = (float(x) for x in (sector.u0, sector.f0, sector.u1, sector.f1))
    nfac = sum(1 for j in range(d) if j in sing or int(sector.a[j]) != 0 or float(sector.b[j]) != 0.0)
    nfac += (u0 != 0 or u1 != 0) + (f0 != 0 or f1 != 0)
    for V in range(1 << ns):
        rad = [p[q] if (V >> q) & 1 and p[q] > 1 else 1 for q in range(ns)]
        J = 1
        pairs = 1
        for r in rad:
            J *= r
            pairs *= r * (r + 1) // 2
        K = sum(r - 1 for r in rad)
        jm, cjm = 2 * pairs, 8 * pairs
        zeroed = [sing[q] for q in range(ns) if (V >> q) & 1]

        def poly_jet(terms):
            f = 0
            for e in terms:
                keep = True
                for j in range(d):
                    if e[j] == 0:
                        continue
                    if j in zeroed:
                        q = sing.index(j)
                        if e[j] >= rad[q]:
                            keep = False
                    else:
                        f += 1
                f += 1 if keep else 0
            return f

        for j in range(d):
            w.fp64 += poly_jet(dF[j])
        for key in Hterms:
            w.fp64 += poly_jet(Hterms[key])
        w.fp64 += d * (2 * jm + J)             # g_j, z_j
        w.fp64 += d * jm + d * d * (jm + J) + d * (2 * J + jm)   # V_jl
        minor2 = 2 * jm + J
        w.fp64 += d * J                        # tr V
        if d == 3:
            w.fp64 += 6 * minor2 + 3 * jm + 5 * J + 2 * J
        elif d == 2:
            w.fp64 += minor2 + 2 * J
        else:
            w.fp64 += J
        w.fp64 += d * max(emax - 1, 0) * cjm   # powers of z
        for P in (sector.U.terms, sector.F.terms):
            for e in P:
                w.fp64 += sum(1 for j in range(d) if e[j] > 0) * cjm + 2 * J
        for _ in range(nfac):                  # ln P0 + ln(1 + x), into A and B
            w.recip()
            w.fp64 += 5 + 6 * (J - 1) + 1 + max(K - 1, 0) * (cjm + 2) + cjm + 3 + 8 * J
            w.log += 1
            w.atan2 += 1
        w.exp += 1
        w.sincos += 1
        w.fp64 += 2 + K * (cjm + 2 * J + 1) + 6 * J + cjm   # exp(A), det J exp(A)
        w.fp64 += max(Hm, 0) * (cjm + 2 * J)   # G_i
        inV = len(zeroed)
        w.fp64 += J * (max(inV - 1, 0) * smul + 2 * smul + 2 * NT)
        w.fp64 += (ns - inV) * smul + 2 * smul + 2 * NT
    w.fp64 += 4 * norders                      # acc += res W (complex)
    return w


def sector_work(sector, lo: int, norders: int, mixed: bool = False, fp64_corners: bool = False) -> Work:
    if getattr(sector, "deform", False):
        if any(int(a) <= -2 for a in sector.a):
            return deformed_taylor_sector_work(sector, lo, norders)
        return deformed_sector_work(sector, lo, norders, mixed)
    if any(int(a) <= -2 for a in sector.a):
        return taylor_sector_work(sector, lo, norders)
    return real_sector_work(sector, lo, norders, mixed, fp64_corners)


def workload_work(integral, lo: int, norders: int, mixed: bool = False, fp64_corners: bool = False) -> Work:
    """Mean work per evaluation over the integral's sectors (equal lattices)."""
    tot = Work()
    for s in integral.sectors:
        tot.add(sector_work(s, lo, norders, mixed, fp64_corners))
    n = max(1, len(integral.sectors))
    return Work(**{k: v / n for k, v in tot.as_dict().items()})


def workload_flops(integral, lo: int, norders: int, deform: bool = False) -> float:
    """Mean FP64 flops per evaluation (no credit for integer-pipe steps)."""
    return workload_work(integral, lo, norders).fp64
