"""Pins of the segment-side oracle: Fig. 2's projection cases (hand values
in tests/golden), closed-form radii, the cylinder lower bound against brute
force, and the counterexample showing why Algorithm 1's subtraction of the
squared error is replaced by the cylinder bound."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2112_10408_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig2_projection_cases.txt")
SIG = (1.0, 1.0, 10.0, 0.01)


def _cases():
    out = []
    with open(GOLD) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            v = [float(x) for x in tok[1:]]
            out.append((tok[0], v[0:3], v[3:6], v[6:9], v[9], v[10]))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_fig2_projection_cases(case):
    name, P, A, B, expected, _lam = case
    assert oracle.point_segment_sq(P, A, B) == pytest.approx(expected, rel=1e-15)


def test_segment_partition_counts():
    wl = synth.flights(7, 47, seed=2, n_routes=2)
    seg = oracle.segments(wl.xyzt, wl.traj_off, SIG, 10)
    # 47 samples in sets of 10 -> 5 segments, the last one with 7 points
    assert seg["first"].shape[0] == 7 * 5
    np.testing.assert_array_equal(seg["count"][:5], [10, 10, 10, 10, 7])
    assert seg["first"][5] == 47
    # A and B are the first and last members (scaled by sqrt(sigma))
    p0 = wl.xyzt[0].astype(np.float64)
    np.testing.assert_allclose(seg["A"][0], p0[:3] * np.sqrt(SIG[:3]))
    p9 = wl.xyzt[9].astype(np.float64)
    np.testing.assert_allclose(seg["B"][0], p9[:3] * np.sqrt(SIG[:3]))
    assert seg["tA"][0] == wl.xyzt[0, 3] and seg["tB"][0] == wl.xyzt[9, 3]


def test_radius_closed_forms():
    # collinear members -> radius 0
    t = np.arange(5, dtype=np.float64)
    line = np.column_stack([2 * t, 3 * t, np.zeros(5), t]).astype(np.float32)
    seg = oracle.segments(line, [0, 5], (1, 1, 1, 1), 5)
    assert seg["radius"][0] == pytest.approx(0.0, abs=1e-12)
    # a triangle: A=(0,0), apex (5,3), B=(10,0) -> radius 3
    tri = np.array([[0, 0, 0, 0], [5, 3, 0, 1], [10, 0, 0, 2]], np.float32)
    seg = oracle.segments(tri, [0, 3], (1, 1, 1, 1), 3)
    assert seg["radius"][0] == pytest.approx(3.0, rel=1e-15)
    # with sigma_y = 4 the metric doubles y distances -> radius 6
    seg = oracle.segments(tri, [0, 3], (1, 4, 1, 1), 3)
    assert seg["radius"][0] == pytest.approx(6.0, rel=1e-15)


def test_cylinder_bound_never_exceeds_true_minimum():
    wl = synth.flights(30, 60, seed=4, n_routes=4)
    K = 10
    seg = oracle.segments(wl.xyzt, wl.traj_off, SIG, K)
    rng = np.random.default_rng(0)
    qrows = rng.choice(wl.n, 40, replace=False)
    for lag in (0.0, 100.0):
        for q in qrows:
            qp = wl.xyzt[q]
            for s in range(seg["first"].shape[0]):
                f, c = int(seg["first"][s]), int(seg["count"][s])
                lb = oracle.cylinder_lb(qp, SIG, lag, seg["A"][s], seg["B"][s],
                                        seg["tA"][s], seg["tB"][s], seg["radius"][s])
                members = wl.xyzt[f:f + c]
                valid = members[:, 3].astype(np.float64) < float(qp[3]) - lag
                if not valid.any():
                    assert math.isinf(lb)
                    continue
                true_min = min(oracle.d2(qp, p, SIG) for p in members[valid])
                assert lb <= true_min * (1 + 1e-12) + 1e-12


def test_paper_alg1_is_not_a_lower_bound_but_the_cylinder_is():
    # A segment along x whose middle member sits rho = 1 off the axis, and a
    # query a = 10 away on the same side: Algorithm 1 returns a^2 - rho^2 = 99
    # for this segment, but the member is only (a - rho)^2 = 81 away, so with
    # a k-th candidate at 90 the printed rule would discard a true neighbour.
    sigma = (1.0, 1.0, 1.0, 0.0)
    members = np.array([[0, 0, 0, 0], [5, 1, 0, 1], [10, 0, 0, 2]], np.float32)
    seg = oracle.segments(members, [0, 3], sigma, 3)
    rho = seg["radius"][0]
    assert rho == pytest.approx(1.0)
    q = np.array([5, 10, 0, 10], np.float32)
    true_min = min(oracle.d2(q, p, sigma) for p in members)
    assert true_min == pytest.approx(81.0)
    paper = oracle.paper_alg1(q, sigma, 0.0, [0, 0, 0], [10, 0, 0], 0.0, 2.0, rho ** 2)
    assert paper == pytest.approx(99.0)
    assert paper > true_min
    lb = oracle.cylinder_lb(q, sigma, 0.0, seg["A"][0], seg["B"][0], 0.0, 2.0, rho)
    assert lb == pytest.approx(81.0) and lb <= true_min


def test_temporal_term_uses_time_since_segment_end():
    # Eq. masked temporal part: t_s^w = min(t, t_B); a segment that ended
    # 50 s before the query has a temporal bound st * 50^2 (Algorithm 1's
    # printed max(t_B - t, 0) would give 0 here).
    sigma = (1.0, 1.0, 1.0, 0.01)
    q = np.array([0, 0, 0, 100], np.float32)
    lb = oracle.cylinder_lb(q, sigma, 0.0, [0, 0, 0], [0, 0, 0], 10.0, 50.0, 0.0)
    assert lb == pytest.approx(0.01 * 50.0 ** 2)
    # and the lag raises it when the segment ended less than lag ago
    lb = oracle.cylinder_lb(q, sigma, 80.0, [0, 0, 0], [0, 0, 0], 10.0, 50.0, 0.0)
    assert lb == pytest.approx(0.01 * 80.0 ** 2)
    # a segment that starts at or after t_q - lag holds nothing valid
    assert math.isinf(oracle.cylinder_lb(q, sigma, 80.0, [0, 0, 0], [0, 0, 0], 20.0, 50.0, 0.0))
