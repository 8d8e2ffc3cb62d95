"""CPU FP64 oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package. It is a plain, slow restatement of the
randomized lattice rule over eps-expanded sector integrands (see
``rqmc_oracle.c`` for what is computed and which passage each step follows)
plus plain host-side combination and allocation (``combine.py``). It shares
no code with the CUDA path; the only thing both sides read is the sector
description and kinematics produced by ``paper_2305_19768_gb300.inputs``.

Parity status: every function here is pinned by the CPU test suite against
closed forms, invariants or brute force (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rqmc_oracle.c")
_lock = threading.Lock()
_lib = None

DMAX = 8


class OrcSector(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("a", ctypes.c_int * DMAX), ("b", ctypes.c_double * DMAX),
                ("u0", ctypes.c_double), ("u1", ctypes.c_double), ("f0", ctypes.c_double),
                ("f1", ctypes.c_double), ("nU", ctypes.c_int), ("nF", ctypes.c_int),
                ("Ue", ctypes.POINTER(ctypes.c_int)), ("Uc", ctypes.POINTER(ctypes.c_double)),
                ("Fe", ctypes.POINTER(ctypes.c_int)), ("Fc", ctypes.POINTER(ctypes.c_double)),
                ("deform", ctypes.c_int), ("lam", ctypes.c_double * DMAX),
                ("transform", ctypes.c_int), ("weight", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            L.orc_shifts.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     P(ctypes.c_double)]
            L.orc_lattice_points.argtypes = [ctypes.c_uint64, P(ctypes.c_uint32), ctypes.c_int,
                                             P(ctypes.c_double), ctypes.c_uint64, ctypes.c_uint64,
                                             P(ctypes.c_double), P(ctypes.c_uint64)]
            L.orc_korobov3.argtypes = [ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double),
                                       P(ctypes.c_double)]
            L.orc_baker.argtypes = [ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double),
                                    P(ctypes.c_double)]
            L.orc_point_value.argtypes = [P(OrcSector), P(ctypes.c_double), ctypes.c_int,
                                          ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int)]
            L.orc_point_value.restype = ctypes.c_int
            L.orc_integrand_at.argtypes = [P(OrcSector), P(ctypes.c_double), ctypes.c_int,
                                           ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int)]
            L.orc_shift_sums.argtypes = [P(OrcSector), ctypes.c_uint64, P(ctypes.c_uint32),
                                         ctypes.c_int, P(ctypes.c_double), ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int]
            L.orc_shift_sums.restype = ctypes.c_long
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class SectorView:
    """An ``OrcSector`` plus the numpy arrays it points into."""

    def __init__(self, integral, sector: int, inv, lam=None, transform: int = 0):
        s = integral.sectors[sector]
        box = 1
        for x in s.a:
            if int(x) <= -1:
                box *= -int(x)
        if box > 128:
            raise ValueError("the subtraction's Taylor box prod_j (-a_j) exceeds 128 coefficients")
        self.d = s.d
        self.Ue, self.Uc = integral.coefficients_at(sector, "U", inv)
        self.Fe, self.Fc = integral.coefficients_at(sector, "F", inv)
        self.Ue = np.ascontiguousarray(self.Ue, dtype=np.int32)
        self.Fe = np.ascontiguousarray(self.Fe, dtype=np.int32)
        st = OrcSector()
        st.d = s.d
        for j in range(s.d):
            st.a[j] = int(s.a[j])
            st.b[j] = float(s.b[j])
        st.u0, st.u1, st.f0, st.f1 = float(s.u0), float(s.u1), float(s.f0), float(s.f1)
        st.nU, st.nF = len(self.Uc), len(self.Fc)
        st.Ue = self.Ue.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        st.Uc = _dptr(self.Uc)
        st.Fe = self.Fe.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        st.Fc = _dptr(self.Fc)
        st.deform = 1 if (s.deform and lam is not None) else 0
        if lam is not None:
            lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (s.d,))
            for j in range(s.d):
                st.lam[j] = float(lam[j])
        st.transform = transform
        st.weight = float(getattr(s, "weight", 1))
        self.st = st
        self.nsing = len(s.singular)


def shifts(seed: int, sector_id: int, m: int, d: int) -> np.ndarray:
    out = np.zeros((m, d), dtype=np.float64)
    lib().orc_shifts(seed, sector_id, m, d, _dptr(out))
    return out


def lattice_points(n: int, z, delta, k0: int, count: int):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    d = len(z)
    delta = np.ascontiguousarray(delta, dtype=np.float64).reshape(d)
    x = np.zeros((count, d), dtype=np.float64)
    r = np.zeros((count, d), dtype=np.uint64)
    lib().orc_lattice_points(n, z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), d, _dptr(delta),
                             k0, count, _dptr(x), r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return x, r


def korobov3(u: float):
    t, omt, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_korobov3(u, ctypes.byref(t), ctypes.byref(omt), ctypes.byref(w))
    return t.value, omt.value, w.value


def baker(u: float):
    t, omt, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_baker(u, ctypes.byref(t), ctypes.byref(omt), ctypes.byref(w))
    return t.value, omt.value, w.value


def point_value(view: SectorView, u, lo: int, norders: int):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(2 * norders)
    sf = ctypes.c_int(0)
    lib().orc_point_value(ctypes.byref(view.st), _dptr(u), lo, norders, _dptr(out), ctypes.byref(sf))
    return out.reshape(norders, 2), sf.value


def integrand_at(view: SectorView, t, lo: int, norders: int):
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.zeros(2 * norders)
    sf = ctypes.c_int(0)
    lib().orc_integrand_at(ctypes.byref(view.st), _dptr(t), lo, norders, _dptr(out), ctypes.byref(sf))
    return out.reshape(norders, 2)


def shift_sums(view: SectorView, n: int, z, delta, lo: int, norders: int, k0: int = 0,
               k1: int | None = None, nthreads: int = 0, with_cond: bool = False):
    """Per-shift estimates [m][norders][2], absolute mass (1/n) sum |f| [m][norders],
    sign failures; with ``with_cond`` also the corner-term mass [m][norders]
    (the size of what cancels inside the subtraction)."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    m = delta.shape[0]
    out = np.zeros((m, norders, 2))
    absout = np.zeros((2 * m, norders))
    if k1 is None:
        k1 = n
    fails = lib().orc_shift_sums(ctypes.byref(view.st), n, z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 m, _dptr(delta), k0, k1, lo, norders, _dptr(out), _dptr(absout),
                                 nthreads)
    if with_cond:
        return out, absout[:m], fails, absout[m:]
    return out, absout[:m], fails


def max_threads() -> int:
    return lib().orc_max_threads()
