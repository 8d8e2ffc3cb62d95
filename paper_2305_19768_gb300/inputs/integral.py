"""Sector description of one integral and its text serialisation.

The text format is what the C-ABI loader (``qmc_load_sectors_mem``) parses;
it plays the role of the paper's per-integral library description (the
`.json` that describes an integral to its integrator). Layout::

    qmc-sectors 1
    name <identifier>
    loops <L> propagators <N> dim <D0>
    invariants <k> <name_1> ... <name_k>
    prefactor <lowest order> <count> <re_0> <im_0> <re_1> <im_1> ...
    nsectors <S>
    sector <index> d <d> deform <0|1> [weight <w>]
    a <a_1> ... <a_d>
    b <b_1> ... <b_d>
    U <u0> <u1> <nterms>
    <e_1> ... <e_d> <c_0> <c_1> ... <c_k>        (nterms rows)
    F <f0> <f1> <nterms>
    <e_1> ... <e_d> <c_0> <c_1> ... <c_k>        (nterms rows)
    ...                                            (S sectors)
    end

A monomial row means (c_0 + c_1 inv_1 + ... + c_k inv_k) * prod_j t_j^{e_j}.
The sector integrand is prod_j t_j^{a_j + b_j eps} U^{u0 + u1 eps}
F^{f0 + f1 eps} on [0,1]^d; the integral is prefactor(eps) times the sum of
the sector integrals. Numbers are written with Python's shortest round-trip
``repr`` so that both readers see identical doubles.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from typing import List, Sequence

import numpy as np

from .polynomial import LinPoly
from .secdec import Sector


def _num(x) -> str:
    return repr(float(x))


@dataclass
class Integral:
    name: str
    L: int
    N: int
    D0: int
    invariants: List[str]
    prefactor_lo: int
    prefactor: List[complex]
    sectors: List[Sector]

    @property
    def ninv(self) -> int:
        return len(self.invariants)

    @property
    def max_poles(self) -> int:
        return max((len(s.singular) for s in self.sectors), default=0)

    @property
    def dmax(self) -> int:
        return max(s.d for s in self.sectors)

    # -- serialisation -------------------------------------------------------
    def to_text(self) -> str:
        out = ["qmc-sectors 1", f"name {self.name}",
               f"loops {self.L} propagators {self.N} dim {self.D0}",
               " ".join(["invariants", str(self.ninv)] + list(self.invariants))]
        pf = ["prefactor", str(self.prefactor_lo), str(len(self.prefactor))]
        for c in self.prefactor:
            pf += [_num(complex(c).real), _num(complex(c).imag)]
        out.append(" ".join(pf))
        out.append(f"nsectors {len(self.sectors)}")
        for i, s in enumerate(self.sectors):
            head = f"sector {i} d {s.d} deform {1 if s.deform else 0}"
            if getattr(s, "weight", 1) != 1:
                head += f" weight {int(s.weight)}"
            out.append(head)
            out.append(" ".join(["a"] + [str(int(x)) for x in s.a]))
            out.append(" ".join(["b"] + [_num(x) for x in s.b]))
            for tag, P, e0, e1 in (("U", s.U, s.u0, s.u1), ("F", s.F, s.f0, s.f1)):
                out.append(f"{tag} {_num(e0)} {_num(e1)} {len(P)}")
                for e, c in P.sorted_terms():
                    out.append(" ".join([str(x) for x in e] + [_num(x) for x in c]))
        out.append("end")
        return "\n".join(out) + "\n"

    @classmethod
    def from_text(cls, text: str) -> "Integral":
        tok = text.split()
        pos = 0

        def nxt():
            nonlocal pos
            pos += 1
            return tok[pos - 1]

        assert nxt() == "qmc-sectors" and nxt() == "1"
        assert nxt() == "name"
        name = nxt()
        assert nxt() == "loops"
        L = int(nxt())
        assert nxt() == "propagators"
        N = int(nxt())
        assert nxt() == "dim"
        D0 = int(nxt())
        assert nxt() == "invariants"
        k = int(nxt())
        invs = [nxt() for _ in range(k)]
        assert nxt() == "prefactor"
        lo = int(nxt())
        cnt = int(nxt())
        pref = [complex(float(nxt()), float(nxt())) for _ in range(cnt)]
        assert nxt() == "nsectors"
        ns = int(nxt())
        secs = []
        for _ in range(ns):
            assert nxt() == "sector"
            nxt()
            assert nxt() == "d"
            d = int(nxt())
            assert nxt() == "deform"
            deform = bool(int(nxt()))
            weight = 1
            if tok[pos] == "weight":
                nxt()
                weight = int(nxt())
            assert nxt() == "a"
            a = [int(nxt()) for _ in range(d)]
            assert nxt() == "b"
            b = [Fraction(float(nxt())) for _ in range(d)]
            polys = []
            for tag in ("U", "F"):
                assert nxt() == tag
                e0 = Fraction(float(nxt()))
                e1 = Fraction(float(nxt()))
                nt = int(nxt())
                P = LinPoly(d, k + 1)
                for _ in range(nt):
                    e = tuple(int(nxt()) for _ in range(d))
                    c = tuple(Fraction(float(nxt())) for _ in range(k + 1))
                    P._acc(e, c)
                polys.append((P, e0, e1))
            (U, u0, u1), (F, f0, f1) = polys
            secs.append(Sector(d, a, b, U, F, u0, u1, f0, f1, deform, weight=weight))
        assert nxt() == "end"
        return cls(name, L, N, D0, invs, lo, pref, secs)

    # -- flat arrays (used by the oracle's ctypes wrapper and by tests) -------
    def coefficients_at(self, sector: int, which: str, inv: Sequence[float]):
        """(exponents int32[nterms][d], values float64[nterms]) of U or F of a
        sector at the kinematic point ``inv``."""
        s = self.sectors[sector]
        P = s.U if which == "U" else s.F
        terms = P.sorted_terms()
        ex = np.array([e for e, _ in terms], dtype=np.int32).reshape(len(terms), s.d)
        vals = np.array([float(c[0]) + sum(float(ci) * v for ci, v in zip(c[1:], inv))
                         for _, c in terms], dtype=np.float64)
        return ex, vals
