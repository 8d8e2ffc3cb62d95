"""The amplitude scan on a small grid: plain (per point), batched and learned
(MLP-sized, spot-checked, mixed precision) agree within their errors and meet
the requested accuracy; the learned form reports its surrogate acceptances."""
import numpy as np
import pytest

from paper_2305_19768_gb300 import scan

pytestmark = pytest.mark.gpu


def test_scan_modes_agree_on_a_small_grid():
    P = scan.Problem(npoints=144, grid=(12, 12))
    eps = 1e-4
    plain = scan.run_plain(P, eps, sel=np.arange(0, 144, 12))
    batched = scan.run_batched(P, eps)
    learned = scan.run_learned(P, eps, ntrain=64, steps=600)
    assert batched["rc"] == 0 and plain["failures"] == 0
    rel = scan.relative_errors(batched["values"], batched["errors"])
    assert rel.max() <= eps * 1.0000001
    # plain and batched estimate the same sums: differences within 5 combined sigma
    sel = np.arange(0, 144, 12)
    d = np.abs(plain["values"] - batched["values"][sel])
    comb = np.hypot(np.abs(plain["errors"]), np.abs(batched["errors"][sel]))
    assert np.all(d <= 5 * comb + 1e-12 * np.abs(plain["values"]).max(axis=1, keepdims=True))
    # learned: every point meets the request (surrogate or QMC) and agrees with batched
    # within 5 combined sigma plus the requested error (its mixed-precision QMC carries
    # a ~1e-7 relative FP32-product bias that only shows where sigma is far below it)
    rel_l = scan.relative_errors(learned["values"], learned["errors"])
    assert rel_l.max() <= eps * 1.0000001
    d = np.abs(learned["values"] - batched["values"])
    comb = np.hypot(np.abs(learned["errors"]), np.abs(batched["errors"]))
    assert np.all(d <= 5 * comb + eps * np.abs(batched["values"]).max(axis=1, keepdims=True))
    print("learned accepted", learned["accepted"], "of", 144 - 64, "times", learned["seconds"],
          batched["seconds"])


def test_network_gain_over_the_unsized_method():
    # on the points after the training set, the network's lattice sizes and
    # deformation parameters replace the pilot pass and the presampling: the
    # sized QMC must spend fewer lattice points (presampling included) and less
    # wall time than the same QMC started from the pilot pass, and far fewer
    # points than the 10^4-point pilot of the plain method, at the same
    # requested accuracy
    P = scan.Problem(npoints=144, grid=(12, 12))
    eps = 1e-4
    learned = scan.run_learned(P, eps, ntrain=64, steps=600)
    rest = np.arange(64, 144)
    scan.run_unsized(P, eps, sel=rest[:8])          # warm-up of the same launch shapes
    unsized = scan.run_unsized(P, eps, sel=rest)
    paper = scan.run_batched(P, eps, sel=rest)
    assert unsized["rc"] == 0 and paper["rc"] == 0
    cost_l = learned["sized_evaluations"] + learned["sized_presample_evaluations"]
    cost_u = unsized["evaluations"] + unsized["presample_evaluations"]
    cost_p = paper["evaluations"] + paper["presample_evaluations"]
    print("rest-point lattice points: network", cost_l, "pilot 1009", cost_u, "pilot 10^4", cost_p)
    print("rest-point seconds: network", learned["sized_seconds"], "pilot 1009", unsized["seconds"])
    assert learned["sized_presample_evaluations"] == 0
    assert cost_l < cost_u < cost_p
    assert learned["sized_seconds"] < unsized["seconds"]
    assert scan.relative_errors(learned["values"], learned["errors"]).max() <= eps * 1.0000001


@pytest.mark.parametrize("sizing", ["variance", "both"])
def test_variance_head_sizing_meets_the_request(sizing):
    # the per-sector log-variance head sizes the lattices through Eq.
    # (adaptive-solution); the adaptive QMC then meets the request everywhere
    P = scan.Problem(npoints=144, grid=(12, 12))
    eps = 1e-4
    learned = scan.run_learned(P, eps, ntrain=64, steps=600, sizing=sizing)
    assert learned["sized_presample_evaluations"] == 0
    assert np.isfinite(learned["logw_fit_median_abs"])
    assert scan.relative_errors(learned["values"], learned["errors"]).max() <= eps * 1.0000001
