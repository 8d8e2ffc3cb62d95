"""The roofline numerator (paper_2305_19768_gb300/flops.py) against counts
made by hand from the fixed-order assembly, so the reported FP64 fraction can
be reproduced: per pole-set formulation, FMA = 2 flops, add/multiply = 1."""
import pytest

from paper_2305_19768_gb300 import flops as F
from paper_2305_19768_gb300.inputs import workloads as w


def test_fixed_assembly_two_singular_variables_by_hand():
    # corner series 1 + 1 + (1 + 2) = 5; Moebius 3 + 3 = 6; t_q/b_q and A_P 2 + 2;
    # b_q ln t_q 2; E_P 0; pole sets: res 2 + 2*(2 + 4) + 6 = 20 with PE 2 + 2;
    # acc 2 * 3 = 6
    assert F._assemble_fixed(2, 0) == 5 + 6 + 4 + 2 + 0 + 20 + 6


def test_fixed_assembly_four_singular_variables_by_hand():
    # corner series: 4 x 1 + 6 x 3 + 4 x 5 + 1 x 7 = 49
    series = 4 * 1 + 6 * 3 + 4 * 5 + 1 * 7
    # Moebius: per slot q, sum over the 8 sets without q of 1 + |P| = 20
    moebius = 4 * 20
    ap = 4 + 14            # t_q / b_q, then A_P for the 14 sets between empty and full
    bl = 4                 # b_q ln t_q
    ep = 4 + 6             # E_P for |P| = 1, 2
    horner = 6 * 1 + 4 * 2           # E / l, l >= 2, per pole set with |P| = 2, 3
    pe = 4 * 2 + 6 * (2 + 4) + 4 * (2 + 4 + 6)
    res = 2 * (1 * 1 + 4 * 2 + 6 * 3 + 4 * 4 + 1 * 5)
    acc = 2 * 5
    assert F._assemble_fixed(4, 0) == series + moebius + ap + bl + ep + horner + pe + res + acc == 373


def test_integer_corner_stage_counts_nothing_on_the_fp64_pipe():
    I = w.double_box_massless()
    sec = next(s for s in I.sectors if sum(1 for a in s.a if a <= -1) == 4)
    xf = F.real_sector_work(sec, -4, 5)
    eq = F.real_sector_work(sec, -4, 5, fp64_corners=True)
    # the FP64 corner stage adds the subset sums (2 x 4 x 8), the paired 1/F,
    # the per-corner powers and products; the integer one counts its
    # reciprocals apart
    assert eq.fp64 - xf.fp64 >= 2 * 4 * 8
    assert xf.rcp_int > 0 and eq.rcp_int == 0
    assert xf.log == eq.log
    # the one-loop box stays on the FP64 corner stage (the d <= 3 kernel)
    box = w.box_massless()
    for s in box.sectors:
        assert F.real_sector_work(s, -2, 3).fp64 == F.real_sector_work(s, -2, 3, fp64_corners=True).fp64


@pytest.mark.parametrize("name,lo,nord,ref", [("double_box_massless", -4, 5, 279.9), ("box_massless", -2, 3, 88.3)])
def test_workload_means_reported_by_the_bench(name, lo, nord, ref):
    I = getattr(w, name)()
    assert abs(F.workload_work(I, lo, nord).fp64 - ref) < 0.05
