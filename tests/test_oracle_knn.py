"""Pins of the k-NN oracle to things other than itself: a library k-d tree
(the unmasked and per-query-masked special cases reduce to a plain Euclidean
k-NN in sigma-scaled coordinates), closed forms on straight trajectories,
index tie-breaks and the exact mask semantics."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2112_10408_gb300 import synth

SIG = (1.0, 1.0, 10.0, 0.01)


def _scaled(p, sigma):
    return p.astype(np.float64) * np.sqrt(np.asarray(sigma, np.float64))[None, :]


@pytest.mark.parametrize("sigma", [SIG, (0.3, 2.0, 5.0, 0.1), (1.0, 1.0, 1.0, 0.0)])
def test_unmasked_matches_kdtree(sigma):
    # All data strictly before every query: the mask keeps everything, and the
    # scalable metric is the Euclidean norm of sqrt(sigma)-scaled coordinates.
    rng = np.random.default_rng(1)
    n, m, k = 3000, 200, 16
    pts = np.column_stack([rng.uniform(0, 100, n), rng.uniform(0, 100, n),
                           rng.uniform(0, 12, n), rng.uniform(0, 1000, n)]).astype(np.float32)
    qs = np.column_stack([rng.uniform(0, 100, m), rng.uniform(0, 100, m),
                          rng.uniform(0, 12, m), rng.uniform(2000, 3000, m)]).astype(np.float32)
    idx, d2 = oracle.knn(pts, k, sigma, lag=0.0, queries=qs)
    tree = cKDTree(_scaled(pts, sigma))
    dd, ii = tree.query(_scaled(qs, sigma), k=k)
    np.testing.assert_array_equal(idx, ii.astype(np.int32))
    np.testing.assert_allclose(d2.astype(np.float64), dd ** 2, rtol=1e-6, atol=1e-6)


def test_masked_self_query_matches_per_query_kdtree():
    wl = synth.flights(12, 40, seed=5, n_routes=3)
    pts = wl.xyzt
    k, lag = 6, 30.0
    idx, d2, d64 = oracle.knn(pts, k, SIG, lag=lag, want_d64=True)
    sc = _scaled(pts, SIG)
    t = pts[:, 3].astype(np.float64)
    for q in range(0, pts.shape[0], 7):
        valid = np.nonzero(t < t[q] - lag)[0]
        if valid.size == 0:
            assert (idx[q] == -1).all() and np.isinf(d2[q]).all()
            continue
        kk = min(k, valid.size)
        dd, ii = cKDTree(sc[valid]).query(sc[q], k=kk)
        ii = np.atleast_1d(valid[np.atleast_1d(ii)])
        np.testing.assert_array_equal(idx[q, :kk], ii)
        np.testing.assert_allclose(d64[q, :kk], np.atleast_1d(dd) ** 2, rtol=1e-9)
        assert (idx[q, kk:] == -1).all()


def test_straight_line_closed_form():
    # One aircraft on a straight line at constant velocity (0.75 km east and
    # 1 km north per 4 s sample -- steps exact in binary -- at constant
    # altitude), a second one 500 km away.  For lag 0 the k neighbours of
    # sample i are its k predecessors, and the n-th one is at
    # n^2 (sx 0.75^2 + sy 1^2) + st n^2 4^2.
    S, k = 60, 8
    t = 4.0 * np.arange(S)
    a = np.column_stack([0.75 * np.arange(S), 1.0 * np.arange(S), np.full(S, 10.0), t])
    b = np.column_stack([500 + 0.75 * np.arange(S), np.zeros(S), np.full(S, 10.0), t + 2.0])
    pts = np.concatenate([a, b]).astype(np.float32)
    idx, d2, d64 = oracle.knn(pts, k, SIG, want_d64=True)
    for i in range(k, S):
        n = np.arange(1, k + 1)
        np.testing.assert_array_equal(idx[i], i - n)
        exact = n ** 2 * (1.0 * 0.5625 + 1.0 * 1.0 + 0.01 * 16.0)
        np.testing.assert_allclose(d64[i], exact, rtol=1e-12)


def test_tie_break_by_index_and_duplicates():
    # Three identical points (same place and time) and a fourth at the same
    # distance from the query: ordering is by (distance, index).
    pts = np.array([[1, 0, 0, 0], [0, 0, 0, 5], [1, 0, 0, 0], [-1, 0, 0, 0],
                    [1, 0, 0, 0], [0, 0, 0, 10]], dtype=np.float32)
    sigma = (1.0, 1.0, 1.0, 0.0)
    idx, d2 = oracle.knn(pts, 5, sigma)
    # query 5 (t=10): valid are rows 0..4, distances 1,0,1,1,1
    np.testing.assert_array_equal(idx[5], [1, 0, 2, 3, 4])
    np.testing.assert_array_equal(d2[5], [0, 1, 1, 1, 1])


def test_mask_is_strict_and_lag_shifts_it():
    pts = np.array([[0, 0, 0, t] for t in (0, 1, 2, 3, 4)], dtype=np.float32)
    sigma = (1.0, 1.0, 1.0, 1.0)
    idx, _ = oracle.knn(pts, 5, sigma, lag=0.0)
    # row i sees exactly rows 0..i-1 (strict mask excludes itself)
    for i in range(5):
        assert sorted(idx[i][idx[i] >= 0].tolist()) == list(range(i))
    idx, _ = oracle.knn(pts, 5, sigma, lag=2.0)
    # t_j < t_i - 2: row 4 sees rows 0, 1; row 3 sees row 0; rows 0-2 none
    assert sorted(idx[4][idx[4] >= 0].tolist()) == [0, 1]
    assert sorted(idx[3][idx[3] >= 0].tolist()) == [0]
    assert (idx[2] == -1).all()


def test_scaling_all_weights_scales_distances():
    wl = synth.flights(8, 30, seed=9, n_routes=2)
    q = synth.query_sample(wl.n, 60, seed=3)
    i1, d1, e1 = oracle.knn(wl.xyzt, 5, SIG, qsel=q, want_d64=True)
    i4, d4, e4 = oracle.knn(wl.xyzt, 5, tuple(4.0 * s for s in SIG), qsel=q, want_d64=True)
    np.testing.assert_array_equal(i1, i4)
    fin = np.isfinite(e1)
    np.testing.assert_allclose(e4[fin], 4.0 * e1[fin], rtol=1e-14)


def test_qsel_rows_equal_full_run():
    wl = synth.flights(10, 30, seed=11, n_routes=3)
    full_i, full_d = oracle.knn(wl.xyzt, 4, SIG, lag=8.0)
    q = synth.query_sample(wl.n, 50, seed=4)
    i, d = oracle.knn(wl.xyzt, 4, SIG, lag=8.0, qsel=q, nthreads=3)
    np.testing.assert_array_equal(i, full_i[q])
    np.testing.assert_array_equal(d, full_d[q])


def test_d2_formula_single_pair():
    a = np.array([1.5, -2.0, 9.0, 100.0], np.float32)
    b = np.array([4.5, 2.0, 9.5, 130.0], np.float32)
    # 1*3^2 + 2*4^2 + 10*0.5^2 + 0.01*30^2 = 9 + 32 + 2.5 + 9 = 52.5
    assert math.isclose(oracle.d2(a, b, (1.0, 2.0, 10.0, 0.01)), 52.5, rel_tol=1e-15)
