"""The input recipe: the generators draw what their docstrings state (sizes,
4 s sampling, time order inside every trajectory, boxes, seeding), so that
the workloads the tests and the bench use are the ones described."""
import math

import numpy as np

from paper_2112_10408_gb300 import synth


def _check_layout(wl, lens):
    n = int(sum(lens))
    assert wl.xyzt.shape == (n, 4) and wl.xyzt.dtype == np.float32
    assert wl.wind.shape == (n, 2) and wl.wind.dtype == np.float32
    assert wl.traj_off.dtype == np.int64 and wl.traj_off[0] == 0 and wl.traj_off[-1] == n
    assert np.array_equal(np.diff(wl.traj_off), np.asarray(lens))
    assert np.array_equal(wl.flight, np.repeat(np.arange(len(lens)), lens).astype(np.int32))
    assert np.isfinite(wl.xyzt).all() and np.isfinite(wl.wind).all()
    for f in range(len(lens)):
        t = wl.xyzt[wl.traj_off[f]:wl.traj_off[f + 1], 3]
        assert (np.diff(t) >= 0).all()  # time-sorted inside every trajectory


def test_flights_recipe():
    wl = synth.flights(30, 50, seed=123, n_routes=4)
    _check_layout(wl, [50] * 30)
    x, y, z, t = wl.xyzt.T.astype(np.float64)
    # 4 s sampling (float32 times near 2e4 s are spaced 2^-9 s apart at most)
    dt = np.diff(t.reshape(30, 50), axis=1)
    assert np.abs(dt - synth.SAMPLE_DT_S).max() <= 2 ** -8
    # cruise levels 8.5-12 km plus N(0, 50 m) jitter; the whole flight inside the 6 h span
    assert z.min() > 8.5 - 0.5 and z.max() < synth.Z_MAX_KM + 0.5
    assert t.min() >= 0.0 and t.max() <= synth.T_SPAN_S + 1e-3
    # waypoints in the 2000 km box; lateral offsets N(0, 5 km) keep points near it
    assert x.min() > -100.0 and x.max() < synth.BOX_XY_KM + 100.0
    assert y.min() > -100.0 and y.max() < synth.BOX_XY_KM + 100.0
    # ground speed 0.20-0.26 km/s: per-sample steps of 0.8-1.04 km, plus jitter
    step = np.hypot(np.diff(x.reshape(30, 50), axis=1), np.diff(y.reshape(30, 50), axis=1))
    assert np.median(step) > 0.7 and np.median(step) < 1.2
    # seeded: the same seed draws the same arrays, another seed others
    again = synth.flights(30, 50, seed=123, n_routes=4)
    assert np.array_equal(wl.xyzt, again.xyzt) and np.array_equal(wl.wind, again.wind)
    other = synth.flights(30, 50, seed=124, n_routes=4)
    assert not np.array_equal(wl.xyzt, other.xyzt)


def test_named_workload_sizes():
    assert synth.tiny().n == 10_000
    wl = synth.medium()
    assert wl.n == 400_000 and wl.n_traj == 2_000
    assert np.array_equal(np.diff(wl.traj_off), np.full(2_000, 200))


def test_stress_layouts():
    srw = synth.smoothed_random_walks(7, 90, seed=3)
    _check_layout(srw, [90] * 7)
    step = np.hypot(*np.diff(srw.xyzt[:90, :2].astype(np.float64), axis=0).T)
    assert np.allclose(step, 0.23 * synth.SAMPLE_DT_S, rtol=1e-3)  # constant speed
    rp = synth.random_points(1003, 20, seed=4)
    _check_layout(rp, [20] * 50 + [3])  # a ragged last group
    lat = synth.lattice(5, 40, seed=6, side=6)
    _check_layout(lat, [40] * 5)
    assert np.array_equal(lat.xyzt[:, :3], np.round(lat.xyzt[:, :3]))  # integer lattice
    assert lat.xyzt[:, :3].min() >= 0 and lat.xyzt[:, :3].max() <= 5


def test_batched_windows_and_samples():
    wins = synth.batched_windows(12, lo=1e3, hi=2e4, seed=9)
    assert len(wins) == 12
    for wl, k in wins:
        assert k in (16, 32, 64)
        assert wl.n % 200 == 0 and 200 <= wl.n <= 2e4 + 200
    sizes = [wl.n for wl, _ in wins]
    assert len(set(sizes)) > 1  # log-uniform, not one size
    q = synth.query_sample(1000, 100, seed=1)
    assert q.dtype == np.int64 and len(q) == 100 and len(np.unique(q)) == 100
    assert (np.diff(q) > 0).all() and q.min() >= 0 and q.max() < 1000
    assert np.array_equal(q, synth.query_sample(1000, 100, seed=1))
    assert len(synth.query_sample(10, 50)) == 10


def test_flight_split_is_by_flight():
    wl = synth.flights(40, 20, seed=5, n_routes=3)
    train, test = synth.flight_split(wl, frac_test=0.25)
    assert not (train & test).any() and (train | test).all()
    held = np.unique(wl.flight[test])
    assert len(held) == 10 and not np.isin(held, wl.flight[train]).any()
    assert math.isclose(test.mean(), 0.25)
