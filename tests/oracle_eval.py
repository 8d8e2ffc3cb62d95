"""An evaluator for qmc_set_evaluator built on the CPU oracle (test
infrastructure): it lets the integration driver's host logic (allocation,
combination, median rules, rank partition) run in a host-only context on a
machine without a GPU, with every integrand evaluation done by the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2305_19768_gb300.inputs.lattice import lattice_for


def make_evaluator(integrals, kin, nthreads=0, transform=0):
    """integrals: {integral id: Integral}; kin: [npoints][ninv] kinematics;
    transform: the context's periodizing transform (0 korobov3, 1 baker)."""
    kin = np.asarray(kin, dtype=np.float64).reshape(len(kin), -1) if len(kin) else np.zeros((0, 0))

    def evaluate(jobs, lo, norders):
        out, fails = [], []
        for J in jobs:
            I = integrals[J["integral_id"]]
            sec = I.sectors[J["sector"]]
            inv = list(kin[J["point"]]) if I.ninv else []
            z = J["z"][:sec.d] if J["z"][0] != 0 else lattice_for(J["n"], sec.d)[1]
            m = J["shifts"]
            dl = np.zeros((m, sec.d)) if J["flags"] & 1 else oracle.shifts(J["seed"], J["stream"], m, sec.d)
            view = oracle.SectorView(I, J["sector"], inv, J["lambda"][0] if sec.deform else None,
                                     transform=transform)
            o, _, f = oracle.shift_sums(view, J["n"], z, dl, lo, norders, nthreads=nthreads)
            out.append(o)
            fails.append(int(f))
        return out, fails

    return evaluate
