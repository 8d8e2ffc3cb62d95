"""Geometric sector decomposition (the decomposition method the paper names
as its default: one Feynman parameter eliminated with the delta-constraint,
the sectors read off the Newton polytope).

With x_N = 1 the projective integrand over the simplex equals the integral
over (0, inf)^(N-1) (Cheng-Wu). Let P = U F in the remaining d = N - 1
variables and Delta its Newton polytope (the convex hull of the exponent
vectors of P, i.e. the Minkowski sum of those of U and F). The inward facet
normals of Delta span its normal fan, which covers R^d; every maximal cone
(the normal cone of a vertex v) is split into simplicial cones spanned by d
of its rays n_1 .. n_d (primitive integer vectors). On such a cone the
substitution x_j = prod_k t_k^{(n_k)_j}, t in (0, 1]^d, covers
log x in -cone(n_1..n_d); there every monomial x^e of U (of F) equals
prod_k t_k^{n_k . e}, the smallest exponent for every k belongs to one vertex,
so U = prod_k t_k^{min_e n_k . e} U~(t) with U~(0) != 0, and likewise F. The
Jacobian is |det N| prod_k t_k^{sum_j (n_k)_j - 1}. A sector is therefore

    |det N| prod_k t_k^{a_k + b_k eps} U~^{u0 + u1 eps} F~^{f0 + f1 eps},
    a_k + b_k eps = sum_j (n_k)_j - 1 + (u0 + u1 eps) min_U(n_k) + (f0 + f1 eps) min_F(n_k),

with the integer weight |det N|. The combinatorics (the hull, the
triangulation of each vertex cone) use floating point; every quantity that
enters a sector (normals, minima, exponents, determinants) is exact integer
arithmetic.
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .polynomial import LinPoly
from .secdec import DecompositionError, Sector

Vec = Tuple[int, ...]


def _primitive(v: Sequence[Fraction]) -> Vec:
    den = 1
    for x in v:
        den = den * Fraction(x).denominator // gcd(den, Fraction(x).denominator)
    ints = [int(Fraction(x) * den) for x in v]
    g = 0
    for x in ints:
        g = gcd(g, abs(x))
    return tuple(x // g for x in ints) if g else tuple(ints)


def _nullspace_vector(rows: List[List[int]], d: int) -> Vec:
    """A nonzero integer vector orthogonal to the d-1 independent integer rows
    (exact Gaussian elimination over the rationals)."""
    M = [[Fraction(x) for x in r] for r in rows]
    piv_cols, r = [], 0
    for c in range(d):
        p = next((i for i in range(r, len(M)) if M[i][c] != 0), None)
        if p is None:
            continue
        M[r], M[p] = M[p], M[r]
        pv = M[r][c]
        M[r] = [x / pv for x in M[r]]
        for i in range(len(M)):
            if i != r and M[i][c] != 0:
                f = M[i][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[r])]
        piv_cols.append(c)
        r += 1
    free = [c for c in range(d) if c not in piv_cols]
    if len(free) != 1:
        raise DecompositionError("degenerate facet")
    fc = free[0]
    v = [Fraction(0)] * d
    v[fc] = Fraction(1)
    for i, c in enumerate(piv_cols):
        v[c] = -M[i][fc]
    return _primitive(v)


def _det(rows: List[Vec]) -> int:
    M = [[Fraction(x) for x in r] for r in rows]
    n, det = len(M), Fraction(1)
    for c in range(n):
        p = next((i for i in range(c, n) if M[i][c] != 0), None)
        if p is None:
            return 0
        if p != c:
            M[c], M[p] = M[p], M[c]
            det = -det
        det *= M[c][c]
        for i in range(c + 1, n):
            f = M[i][c] / M[c][c]
            M[i] = [a - f * b for a, b in zip(M[i], M[c])]
    return int(det)


def _dot(a: Sequence[int], b: Sequence[int]) -> int:
    return sum(x * y for x, y in zip(a, b))


def newton_facets(points: List[Vec]):
    """(vertices, primitive inward integer facet normals) of conv(points) in Z^d."""
    from scipy.spatial import ConvexHull

    d = len(points[0])
    pts = sorted(set(points))
    if d == 1:
        return [min(pts), max(pts)], [(1,), (-1,)]
    X = np.array(pts, dtype=float)
    hull = ConvexHull(X)
    centroid = [sum(Fraction(p[j]) for p in pts) / len(pts) for j in range(d)]
    normals = set()
    scale = 1.0 + np.abs(X).max()
    for eq in hull.equations:
        # all points on this facet (qhull's simplices may be degenerate); the
        # exact normal is the integer kernel of their differences (rank d - 1)
        on = [pts[i] for i in np.nonzero(np.abs(X @ eq[:-1] + eq[-1]) < 1e-7 * scale)[0]]
        rows = [[q[j] - on[0][j] for j in range(d)] for q in on[1:]]
        n = _nullspace_vector(rows, d)
        if sum(Fraction(n[j]) * (centroid[j] - on[0][j]) for j in range(d)) < 0:
            n = tuple(-x for x in n)
        c = _dot(n, on[0])
        if any(_dot(n, q) < c for q in pts):
            raise DecompositionError("facet normal does not support the polytope")
        normals.add(n)
    normals = sorted(normals)
    # vertices: the points whose tight facets span R^d (checked exactly)
    verts = []
    for p in (pts[i] for i in sorted(hull.vertices)):
        tight = [n for n in normals if _dot(n, p) == min(_dot(n, q) for q in pts)]
        if len(tight) >= d and np.linalg.matrix_rank(np.array(tight, dtype=float)) == d:
            verts.append(p)
    return verts, normals


def _triangulate_cone(rays: List[Vec], h) -> List[List[Vec]]:
    """Simplicial cones covering cone(rays) exactly once, using only the given
    (extreme) rays: a regular triangulation of the cross-section polytope
    {x in cone : h.x = 1} (h.r > 0 for every ray), read off the lower hull of
    its vertices lifted to seeded random heights (generic heights make every
    lower facet a simplex)."""
    d = len(rays[0])
    if len(rays) == d:
        return [list(rays)]
    R = np.array(rays, dtype=float)
    h = np.asarray(h, dtype=float)
    if np.any(R @ h <= 0):
        raise DecompositionError("cross-section direction does not separate the cone")
    P = R / (R @ h)[:, None]                     # on the hyperplane h.x = 1
    Q, _ = np.linalg.qr(np.column_stack([h] + [np.eye(d)[:, i] for i in range(d)]))
    X = (P - P[0]) @ Q[:, 1:d]                   # (d-1)-dimensional cross-section
    if d - 1 == 1:
        order = np.argsort(X[:, 0])
        return [[rays[order[0]], rays[order[-1]]]]
    from scipy.spatial import ConvexHull

    rng = np.random.default_rng(20230531)
    lifted = np.column_stack([X, rng.uniform(0.0, 1.0, len(rays)) * (1.0 + np.abs(X).max())])
    hull = ConvexHull(lifted)
    out = []
    for simplex, eq in zip(hull.simplices, hull.equations):
        if eq[-2] < -1e-12:                      # lower facet (outward normal points down)
            out.append([rays[i] for i in simplex])
    return out


def decompose_geometric(U: LinPoly, F: LinPoly, u0, u1, f0, f1, *, deform: bool = False) -> List[Sector]:
    """Sectors of U^{u0+u1 eps} F^{f0+f1 eps} (projective, over the simplex) by
    the geometric method; each carries the integer weight |det N|."""
    N = U.nvars
    d = N - 1

    def restrict(P: LinPoly) -> Dict[Vec, tuple]:
        out: Dict[Vec, list] = {}
        for e, c in P.terms.items():
            k = tuple(e[:-1])
            if k in out:
                out[k] = [a + b for a, b in zip(out[k], c)]
            else:
                out[k] = list(c)
        return {k: tuple(v) for k, v in out.items() if any(x != 0 for x in v)}

    Ur, Fr = restrict(U), restrict(F)
    pts = [tuple(a + b for a, b in zip(eu, ef)) for eu in Ur for ef in Fr]
    verts, normals = newton_facets(pts)
    allp = sorted(set(pts))
    centroid = np.array(allp, dtype=float).mean(axis=0)
    sectors: List[Sector] = []
    for v in verts:
        tight = [n for n in normals if _dot(n, v) == min(_dot(n, p) for p in allp)]
        # every ray r of the normal cone of v has r.(p - v) >= 0 on the polytope,
        # strictly somewhere: centroid - v is a cross-section direction
        for cone in _triangulate_cone(tight, centroid - np.array(v, dtype=float)):
            det = _det(cone)
            if det == 0:
                continue
            a, b = [], []
            Ut: Dict[Vec, tuple] = {}
            Ft: Dict[Vec, tuple] = {}
            minU = [min(_dot(n, e) for e in Ur) for n in cone]
            minF = [min(_dot(n, e) for e in Fr) for n in cone]
            for k, n in enumerate(cone):
                ak = Fraction(sum(n) - 1) + Fraction(u0) * minU[k] + Fraction(f0) * minF[k]
                bk = Fraction(u1) * minU[k] + Fraction(f1) * minF[k]
                if ak.denominator != 1:
                    raise DecompositionError("non-integer monomial exponent")
                a.append(int(ak))
                b.append(bk)
            for src, dst, mins in ((Ur, Ut, minU), (Fr, Ft, minF)):
                for e, c in src.items():
                    key = tuple(_dot(n, e) - mins[k] for k, n in enumerate(cone))
                    if key in dst:
                        dst[key] = tuple(x + y for x, y in zip(dst[key], c))
                    else:
                        dst[key] = c
            Up = LinPoly(d, U.ncoef, {e: c for e, c in Ut.items() if any(x != 0 for x in c)})
            Fp = LinPoly(d, F.ncoef, {e: c for e, c in Ft.items() if any(x != 0 for x in c)})
            for j in range(d):
                if a[j] < -2 or (a[j] <= -1 and b[j] == 0):
                    raise DecompositionError(f"geometric sector: exponent a_{j}={a[j]}, b={b[j]}")
            sectors.append(Sector(d, a, b, Up, Fp, Fraction(u0), Fraction(u1), Fraction(f0), Fraction(f1),
                                  deform, origin=f"cone {cone}", weight=abs(det)))
    return sectors
