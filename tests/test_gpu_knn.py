"""Parity of the CUDA search (TNN and the linear-search comparator) with the
FP64 oracle, through the C ABI: neighbour indices bit-exact (ties by index),
distances within 1e-5 relative; plus the index and bound invariants."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2112_10408_gb300 import synth
from paper_2112_10408_gb300 import tnn
from tests._helpers import assert_knn_equal

pytestmark = pytest.mark.gpu
SIG = synth.SIGMA_DEFAULT


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_10408_gb300 import build
    build.build()
    tnn.load_library()
    torch.cuda.init()


def _index(wl, K, sigma=SIG):
    return tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, sigma, K)


def _both(ix, k, lag, q=None, **kw):
    ti, td = tnn.tnn_knn(ix, k, lag, q=q, **kw)
    bi, bd = tnn.tnn_knn_bruteforce(ix, k, lag, q=q, **kw)
    torch.cuda.synchronize()
    return ti.cpu().numpy(), td.cpu().numpy(), bi.cpu().numpy(), bd.cpu().numpy()


def test_tiny_config_all_queries():
    # 200 flights x 50 samples, k = 8, 10-point segments, mask t_j < t_i.
    wl = synth.tiny()
    ix = _index(wl, 10)
    ti, td, bi, bd = _both(ix, 8, 0.0)
    oi, od = oracle.knn(wl.xyzt, 8, SIG)
    assert_knn_equal(ti, td, oi, od, what="tnn tiny")
    assert_knn_equal(bi, bd, oi, od, what="linear tiny")


@pytest.mark.parametrize("k,lag,K", [(1, 0.0, 10), (5, 37.0, 7), (32, 0.0, 20),
                                     (64, 120.0, 13), (17, 0.0, 2), (40, 0.0, 64)])
def test_small_configs(k, lag, K):
    # several warps of queries and a ragged tail (2,173 rows)
    wl = synth.flights(41, 53, seed=100 + k, n_routes=5)
    ix = _index(wl, K)
    ti, td, bi, bd = _both(ix, k, lag)
    oi, od = oracle.knn(wl.xyzt, k, SIG, lag=lag)
    assert_knn_equal(ti, td, oi, od, what=f"tnn k={k} lag={lag} K={K}")
    assert_knn_equal(bi, bd, oi, od, what=f"linear k={k} lag={lag} K={K}")


@pytest.mark.parametrize("tuning", [dict(seed_segments=1, seed_window=32, extra=2),
                                    dict(seed_segments=6, seed_window=0, extra=32),
                                    dict(seed_segments=3, seed_window=17, extra=5)])
def test_tuning_knobs_do_not_change_results(tuning):
    wl = synth.flights(60, 70, seed=7, n_routes=6)
    ix = _index(wl, 12)
    ti, td = tnn.tnn_knn(ix, 16, 30.0, **tuning)
    oi, od = oracle.knn(wl.xyzt, 16, SIG, lag=30.0)
    assert_knn_equal(ti.cpu().numpy(), td.cpu().numpy(), oi, od, what=str(tuning))


@pytest.mark.parametrize("k,lag", [(8, 0.0), (32, 90.0), (64, 0.0)])
def test_sweep_and_grid_orders_agree_with_oracle(k, lag):
    # The two segment orders (t_A sweep, time-bucketed grid) must give the
    # same exact answer; also on smoothed random walks and random points.
    for wl in (synth.flights(80, 60, seed=300 + k, n_routes=7),
               synth.smoothed_random_walks(30, 90, seed=k),
               synth.random_points(2500, 20, seed=k)):
        ix = _index(wl, 12)
        gi, gd = tnn.tnn_knn(ix, k, lag)
        si, sd = tnn.tnn_knn(ix, k, lag, sweep=True)
        oi, od = oracle.knn(wl.xyzt, k, SIG, lag=lag)
        assert_knn_equal(gi.cpu().numpy(), gd.cpu().numpy(), oi, od, what=f"grid {wl.name} k={k}")
        assert_knn_equal(si.cpu().numpy(), sd.cpu().numpy(), oi, od, what=f"sweep {wl.name} k={k}")


def test_exact_d2_flag_gives_fp64_rounded_distances():
    wl = synth.flights(30, 40, seed=3, n_routes=4)
    ix = _index(wl, 10)
    ti, td = tnn.tnn_knn(ix, 12, 0.0, exact_d2=True)
    bi, bd = tnn.tnn_knn_bruteforce(ix, 12, 0.0, exact_d2=True)
    oi, od = oracle.knn(wl.xyzt, 12, SIG)
    for i, d in ((ti, td), (bi, bd)):
        np.testing.assert_array_equal(i.cpu().numpy(), oi)
        np.testing.assert_array_equal(d.cpu().numpy(), od)  # bit-identical


def test_tie_heavy_lattice_uses_exact_settlement():
    # integer lattice, integer times: many equal distances and duplicates
    wl = synth.lattice(40, 30, seed=11, side=4)
    sigma = (1.0, 1.0, 1.0, 1.0)
    ix = _index(wl, 6, sigma)
    for k in (3, 8, 20):
        ti, td, st = tnn.tnn_knn(ix, k, 0.0, stats=True)
        bi, bd = tnn.tnn_knn_bruteforce(ix, k, 0.0)
        oi, od = oracle.knn(wl.xyzt, k, sigma)
        assert_knn_equal(ti.cpu().numpy(), td.cpu().numpy(), oi, od, what=f"tnn lattice k={k}")
        assert_knn_equal(bi.cpu().numpy(), bd.cpu().numpy(), oi, od, what=f"linear lattice k={k}")
        assert st["fp64_rechecks"] > 0


def test_external_queries_and_future_queries():
    wl = synth.flights(50, 60, seed=21, n_routes=5)
    ix = _index(wl, 15)
    rng = np.random.default_rng(0)
    q = wl.xyzt[rng.choice(wl.n, 333, replace=False)].copy()
    q[:, :3] += rng.normal(0, 3.0, size=(333, 3)).astype(np.float32)
    q[::3, 3] = 1e5  # after every point: the whole set is valid
    q[1::7, 3] = -1.0  # before every point: nothing valid
    qd = torch.from_numpy(q).cuda()
    ti, td, bi, bd = _both(ix, 9, 15.0, q=qd)
    oi, od = oracle.knn(wl.xyzt, 9, SIG, lag=15.0, queries=q)
    assert_knn_equal(ti, td, oi, od, what="tnn external")
    assert_knn_equal(bi, bd, oi, od, what="linear external")
    assert (ti[1::7] == -1).all() and np.isinf(td[1::7]).all()


@pytest.mark.parametrize("sigma", [(1.0, 1.0, 1.0, 0.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 0.0),
                                   (3.0, 0.5, 40.0, 2.0)])
def test_sigma_special_cases(sigma):
    # st = 0: no temporal pruning; spatial weights 0: pure time; all 0: every
    # valid point ties at 0 and the order is by index.
    wl = synth.flights(25, 33, seed=5, n_routes=3)
    ix = _index(wl, 8, sigma)
    ti, td, bi, bd = _both(ix, 6, 0.0)
    oi, od = oracle.knn(wl.xyzt, 6, sigma)
    assert_knn_equal(ti, td, oi, od, what=f"tnn sigma={sigma}")
    assert_knn_equal(bi, bd, oi, od, what=f"linear sigma={sigma}")


def test_degenerate_inputs():
    # one point; trajectories of length 1; a single trajectory; k > N
    one = np.array([[1.0, 2.0, 3.0, 4.0]], np.float32)
    ix = tnn.tnn_build_segments(torch.from_numpy(one).cuda(), [0, 1], SIG, 4)
    i, d = tnn.tnn_knn(ix, 3, 0.0)
    assert (i.cpu().numpy() == -1).all() and np.isinf(d.cpu().numpy()).all()
    rng = np.random.default_rng(1)
    pts = np.column_stack([rng.uniform(0, 10, 97), rng.uniform(0, 10, 97),
                           rng.uniform(0, 1, 97), np.sort(rng.uniform(0, 100, 97))]).astype(np.float32)
    for off in ([0, 97], list(range(98))):
        ix = tnn.tnn_build_segments(torch.from_numpy(pts).cuda(), off, SIG, 5)
        for k in (1, 64):
            ti, td, bi, bd = _both(ix, k, 0.0)
            oi, od = oracle.knn(pts, k, SIG)
            assert_knn_equal(ti, td, oi, od, what=f"tnn degenerate off={len(off)} k={k}")
            assert_knn_equal(bi, bd, oi, od, what=f"linear degenerate off={len(off)} k={k}")


def test_invalid_inputs_are_rejected():
    bad = np.array([[0, 0, 0, 0], [np.nan, 0, 0, 1]], np.float32)
    with pytest.raises(tnn.TNNError, match="non-finite"):
        tnn.tnn_build_segments(torch.from_numpy(bad).cuda(), [0, 2], SIG, 2)
    unsorted = np.array([[0, 0, 0, 5], [0, 0, 0, 1]], np.float32)
    with pytest.raises(tnn.TNNError, match="sorted"):
        tnn.tnn_build_segments(torch.from_numpy(unsorted).cuda(), [0, 2], SIG, 2)
    wl = synth.flights(3, 10, seed=1, n_routes=1)
    ix = _index(wl, 5)
    with pytest.raises(tnn.TNNError, match="k must"):
        tnn.tnn_knn(ix, 65, 0.0)
    with pytest.raises(tnn.TNNError, match="self-query"):
        idx = torch.empty((5, 4), dtype=torch.int32, device="cuda")
        d2 = torch.empty((5, 4), dtype=torch.float32, device="cuda")
        ctypes_p = tnn.make_knn_params(4)
        import ctypes
        tnn._check(tnn._L().tnn_knn(ix.handle, None, 5, ctypes.byref(ctypes_p), tnn._ptr(idx),
                                    tnn._ptr(d2), None, tnn._stream()))


def test_stress_layouts_random_points_and_srw():
    # Sec. 4.2: random points (pathological: the bound prunes almost nothing,
    # comparisons approach the linear search) and smoothed random walks.
    rnd = synth.random_points(6000, 20, seed=4)
    srw = synth.smoothed_random_walks(40, 150, seed=4)
    for wl, name in ((rnd, "rand"), (srw, "srw")):
        ix = _index(wl, 20)
        ti, td, st = tnn.tnn_knn(ix, 32, 0.0, stats=True)
        bi, bd, sb = tnn.tnn_knn_bruteforce(ix, 32, 0.0, stats=True)
        q = synth.query_sample(wl.n, 700, seed=9)
        oi, od = oracle.knn(wl.xyzt, 32, SIG, qsel=q)
        assert_knn_equal(ti.cpu().numpy()[q], td.cpu().numpy()[q], oi, od, what=f"tnn {name}")
        assert_knn_equal(bi.cpu().numpy()[q], bd.cpu().numpy()[q], oi, od, what=f"linear {name}")
        if name == "srw":
            assert st["pairs"] < 0.5 * sb["pairs"]


def test_index_segments_match_oracle():
    wl = synth.flights(20, 47, seed=2, n_routes=3)
    ix = _index(wl, 10)
    seg, pm = tnn.tnn_index_export(ix)
    seg = seg.cpu().numpy()
    pm = pm.cpu().numpy()
    ref = oracle.segments(wl.xyzt, wl.traj_off, SIG, 10)
    S = ref["first"].shape[0]
    assert ix.n_segments == S
    bid = seg[:, 15].view(np.int32)
    # ordered by t_A, stable by build order
    order = np.lexsort((np.arange(S), ref["tA"]))
    np.testing.assert_array_equal(bid, order)
    np.testing.assert_array_equal(seg[:, 12].view(np.int32), ref["first"][bid])
    np.testing.assert_array_equal(seg[:, 13].view(np.int32), ref["count"][bid])
    np.testing.assert_allclose(seg[:, 0:3], ref["A"][bid], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(seg[:, 0:3] + seg[:, 8:11], ref["B"][bid], rtol=1e-6, atol=1e-4)
    assert (seg[:, 11] >= ref["radius"][bid] - 1e-4).all()
    assert (seg[:, 11] <= ref["radius"][bid] + 1e-3).all()
    np.testing.assert_array_equal(pm, np.maximum.accumulate(seg[:, 7]))
    # the info call waits for the build and reports the largest radius
    assert ix.max_radius == float(seg[:, 11].max())
    assert ix.coord_max >= float(np.abs(wl.xyzt[:, :3] * np.sqrt(np.asarray(SIG[:3]))).max()) * (1 - 1e-6)
    # every member within r of the stored segment [A', A' + AB'] (FP64 check)
    sq = np.sqrt(np.asarray(SIG[:3]))
    for s in range(S):
        f, c = seg[s, 12:14].view(np.int32)
        A = seg[s, 0:3].astype(np.float64)
        B = A + seg[s, 8:11].astype(np.float64)
        for p in wl.xyzt[f:f + c]:
            d = math.sqrt(oracle.point_segment_sq(p[:3].astype(np.float64) * sq, A, B))
            assert d <= seg[s, 11]


def test_lower_bounds_never_exceed_point_distances():
    wl = synth.flights(30, 50, seed=8, n_routes=4)
    ix = _index(wl, 10)
    seg, _ = tnn.tnn_index_export(ix)
    seg = seg.cpu().numpy()
    rng = np.random.default_rng(2)
    rows = rng.choice(wl.n, 64, replace=False)
    for lag in (0.0, 60.0):
        q = torch.from_numpy(wl.xyzt[rows]).cuda()
        lb = tnn.tnn_segment_lower_bounds(ix, q=q, lag=lag).cpu().numpy()
        for a, r in enumerate(rows):
            qp = wl.xyzt[r]
            for s in range(seg.shape[0]):
                f, c = seg[s, 12:14].view(np.int32)
                mem = wl.xyzt[f:f + c]
                valid = mem[:, 3].astype(np.float64) < float(qp[3]) - lag
                if not valid.any():
                    assert math.isinf(lb[a, s])
                    continue
                dmin = min(oracle.d2(qp, p, SIG) for p in mem[valid])
                assert lb[a, s] <= dmin * (1 - 2.0 ** -21), (a, s, lb[a, s], dmin)


def test_medium_config_sampled_queries():
    # 2,000 flights x 200 samples = 400,000 points, k = 32, 20-point segments
    wl = synth.medium()
    ix = _index(wl, 20)
    ti, td, st = tnn.tnn_knn(ix, 32, 0.0, stats=True)
    q = synth.query_sample(wl.n, 4096)
    oi, od = oracle.knn(wl.xyzt, 32, SIG, qsel=q)
    assert_knn_equal(ti.cpu().numpy()[q], td.cpu().numpy()[q], oi, od, what="tnn medium")
    assert st["queries"] == wl.n
    qd = torch.from_numpy(wl.xyzt[q]).cuda()
    bi, bd = tnn.tnn_knn_bruteforce(ix, 32, 0.0, q=qd)
    assert_knn_equal(bi.cpu().numpy(), bd.cpu().numpy(), oi, od, what="linear medium")
    # invariants on every query: sorted by (d2, idx), unique, mask respected
    ti = ti.cpu().numpy()
    td = td.cpu().numpy()
    assert (td[:, 1:] >= td[:, :-1]).all()  # +inf padding compares equal
    t = wl.xyzt[:, 3]
    valid = ti >= 0
    assert (t[np.where(valid, ti, 0)][valid] < np.repeat(t[:, None], 32, axis=1)[valid]).all()
    srt = np.sort(ti, axis=1)
    assert ((np.diff(srt, axis=1) != 0) | (srt[:, 1:] < 0)).all()


def test_precision_config_sampled_queries():
    # 20,000 flights x 200 samples = 4,000,000 points, k = 32
    wl = synth.precision()
    ix = _index(wl, 20)
    ti, td, st = tnn.tnn_knn(ix, 32, 0.0, stats=True)
    q = synth.query_sample(wl.n, 4096)
    oi, od = oracle.knn(wl.xyzt, 32, SIG, qsel=q)
    assert_knn_equal(ti.cpu().numpy()[q], td.cpu().numpy()[q], oi, od, what="tnn precision")
    assert st["exact_queries"] <= wl.n * 1e-4
    qd = torch.from_numpy(wl.xyzt[q]).cuda()
    bi, bd = tnn.tnn_knn_bruteforce(ix, 32, 0.0, q=qd)
    assert_knn_equal(bi.cpu().numpy(), bd.cpu().numpy(), oi, od, what="linear precision")


def test_batched_windows_match_oracle():
    wins = synth.batched_windows(n_windows=9, lo=2e3, hi=3e4, seed=77)
    idxs = [_index(wl, 20) for wl, _ in wins]
    ks = [k for _, k in wins]
    b = tnn.Batch(idxs, ks)
    for _ in range(2):  # replaying the graph gives the same answer
        b.run()
    torch.cuda.synchronize()
    st = b.stats()
    assert st["queries"] == sum(wl.n for wl, _ in wins)
    for w, (wl, k) in enumerate(wins):
        q = synth.query_sample(wl.n, 300, seed=w)
        oi, od = oracle.knn(wl.xyzt, k, SIG, qsel=q)
        assert_knn_equal(b.idx[w].cpu().numpy()[q], b.d2[w].cpu().numpy()[q], oi, od,
                         what=f"window {w} k={k}")
    # one segment order per batch: mixing the sweep and the grid is refused
    with pytest.raises(tnn.TNNError):
        tnn.Batch(idxs[:2], ks[:2], tunings=[{"sweep": True}, {}])


def test_autotune_returns_valid_knobs():
    wl = synth.flights(200, 100, seed=12, n_routes=8)
    ix = _index(wl, 20)
    p = tnn.tnn_autotune(ix, 32, 0.0, m_sample=1024)
    assert 1 <= p["seed_segments"] <= 6 and p["seed_window"] >= 0 and 2 <= p["extra"] <= 32
    ti, td = tnn.tnn_knn(ix, 32, 0.0, **p)
    q = synth.query_sample(wl.n, 500)
    oi, od = oracle.knn(wl.xyzt, 32, SIG, qsel=q)
    assert_knn_equal(ti.cpu().numpy()[q], td.cpu().numpy()[q], oi, od, what="autotuned")


@pytest.mark.parametrize("k,extra", [(1, 2), (32, 4), (64, 32)])
def test_linear_search_tensor_core_and_cuda_core_paths(k, extra):
    # The tensor-core screen (128 x 128 distance tiles) and the direct FP32
    # distances must give the oracle's answer; 3,071 rows leave a ragged
    # 128-query tile and a ragged 128-point chunk.
    for wl in (synth.flights(37, 83, seed=500 + k, n_routes=4),
               synth.random_points(3071, 20, seed=k),
               synth.smoothed_random_walks(19, 97, seed=k)):
        ix = _index(wl, 16)
        oi, od = oracle.knn(wl.xyzt, k, SIG)
        for ffma in (False, True):
            bi, bd, st = tnn.tnn_knn_bruteforce(ix, k, 0.0, extra=extra, ffma=ffma, stats=True)
            assert_knn_equal(bi.cpu().numpy(), bd.cpu().numpy(), oi, od,
                             what=f"linear {wl.name} k={k} ffma={ffma}")
            assert st["queries"] == wl.n


def test_linear_tensor_core_far_and_large_coordinates():
    # Queries far outside the data (a large |q - centre| widens the screening
    # margin) and coordinates near 1e4 km, where FP32 spacing is coarse.
    wl = synth.flights(40, 64, seed=9, n_routes=5)
    xyzt = wl.xyzt.copy()
    xyzt[:, 0] += 9000.0
    xyzt[:, 1] -= 7000.0
    ix = tnn.tnn_build_segments(torch.from_numpy(xyzt).cuda(), wl.traj_off, SIG, 10)
    rng = np.random.default_rng(5)
    q = xyzt[rng.choice(len(xyzt), 400, replace=False)].copy()
    q[:100, :2] += rng.normal(0, 2000.0, size=(100, 2)).astype(np.float32)
    q[100:150, 3] = -5.0  # nothing causal for a whole run of queries
    q[150:200, 3] = 1e6
    qd = torch.from_numpy(q).cuda()
    oi, od = oracle.knn(xyzt, 10, SIG, lag=3.0, queries=q)
    for ffma in (False, True):
        bi, bd = tnn.tnn_knn_bruteforce(ix, 10, 3.0, q=qd, ffma=ffma)
        assert_knn_equal(bi.cpu().numpy(), bd.cpu().numpy(), oi, od, what=f"far ffma={ffma}")


def _ragged_flights(seed=71):
    # flights cut to random lengths of 0 to 70 samples (some empty, some 1)
    rng = np.random.default_rng(seed)
    wl = synth.flights(90, 70, seed=seed + 1, n_routes=6)
    lens = rng.integers(0, 71, size=wl.n_traj)
    lens[::17] = 0
    lens[1::13] = 1
    keep = np.concatenate([np.arange(wl.traj_off[f], wl.traj_off[f] + lens[f]) for f in range(wl.n_traj)])
    xyzt = np.ascontiguousarray(wl.xyzt[keep])
    off = np.zeros(wl.n_traj + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens)
    return xyzt, off


def test_trajectory_tiles_give_the_same_lists_as_query_order_tiles():
    """Self-queries are answered in tiles of one trajectory's consecutive
    samples, passed queries in tiles of 32 in array order: the lists must be
    bit-identical, also for ragged trajectories (1 to 70 samples, some empty),
    a run of rows starting inside a trajectory, and against the oracle."""
    xyzt, off = _ragged_flights()
    x = torch.from_numpy(xyzt).cuda()
    ix = tnn.tnn_build_segments(x, off, SIG, 10)
    si, sd = tnn.tnn_knn(ix, 12, 0.0)
    for kw in ({}, {"defer_cells": 0.3}, {"sweep": True}):
        ki, kd = tnn.tnn_knn(ix, 12, 0.0, **kw)
        qi, qd = tnn.tnn_knn(ix, 12, 0.0, q=x.clone(), **kw)
        torch.cuda.synchronize()
        assert torch.equal(ki, qi) and torch.equal(kd, qd), kw
        assert torch.equal(ki, si) and torch.equal(kd, sd), kw
    oi, od = oracle.knn(xyzt, 12, SIG, lag=0.0)
    assert_knn_equal(si.cpu().numpy(), sd.cpu().numpy(), oi, od, what="ragged trajectories")
    # a run of rows that starts and ends inside trajectories (tnn_knn_host's
    # slices): the host pipeline against the device path
    hi, hd = tnn.tnn_knn_host(xyzt, off, SIG, 10, 12, 0.0, chunks=5)
    assert torch.equal(hi, si.cpu()) and torch.equal(hd, sd.cpu())


@pytest.mark.parametrize("chunks,k,lag,kw", [(0, 12, 0.0, {}),
                                             (1, 12, 0.0, {"defer_cells": 0.3}),
                                             (3, 64, 0.0, {"exact_d2": True, "defer_cells": 0.3}),
                                             (7, 12, 60.0, {"sweep": True}),
                                             (64, 33, 0.0, {"defer_cells": 0.3})])
def test_mapped_host_outputs_match_the_device_path(chunks, k, lag, kw):
    """TNN_FLAG_MAPPED_OUT: the shared-tile kernel writes each finished
    tile's rows into the page-locked outputs itself, and the rows the
    per-query kernels finish afterwards are written by a kernel at the end.
    The lists must equal the device path's on ragged trajectories (tiles of
    1 to 32 rows), with many queries handed over, k above 32, and outputs
    that are a view into a larger page-locked block; `chunks` only matters
    to the copied path, which must agree too."""
    xyzt, off = _ragged_flights()
    n = xyzt.shape[0]
    ix = tnn.tnn_build_segments(torch.from_numpy(xyzt).cuda(), off, SIG, 10)
    di, dd, st = tnn.tnn_knn(ix, k, lag, stats=True, **kw)
    if "defer_cells" in kw:
        assert st["warp_queries"] > 100
    bi = torch.full((n + 9, k), -7, dtype=torch.int32).pin_memory()
    bd = torch.full((n + 9, k), -7.0, dtype=torch.float32).pin_memory()
    hi, hd = bi[4:4 + n], bd[4:4 + n]
    assert hi.is_pinned() and hi.is_contiguous()
    tnn.tnn_knn_host(xyzt, off, SIG, 10, k, lag, chunks=chunks, out=(hi, hd), **kw)
    assert torch.equal(hi, di.cpu()) and torch.equal(hd, dd.cpu())
    # rows outside the outputs are untouched
    assert (bi[:4] == -7).all() and (bi[4 + n:] == -7).all() and (bd[4 + n:] == -7.0).all()
    # the same call with the flag off copies every row after its slice ends
    pi, pd = tnn.tnn_knn_host(xyzt, off, SIG, 10, k, lag, chunks=chunks, mapped=False, **kw)
    assert torch.equal(pi, hi) and torch.equal(pd, hd)


def test_mapped_host_outputs_refuse_unmapped_memory():
    """TNN_FLAG_MAPPED_OUT with outputs that are not page-locked is an
    argument error, found before any device work."""
    xyzt, off = _ragged_flights()
    n = xyzt.shape[0]
    pinned = torch.empty((n, 8), dtype=torch.float32).pin_memory()
    for out in ((np.empty((n, 8), np.int32), np.empty((n, 8), np.float32)),
                (torch.empty((n, 8), dtype=torch.int32).pin_memory(), np.empty((n, 8), np.float32)),
                (np.empty((n, 8), np.int32), pinned)):
        with pytest.raises(tnn.TNNError, match="MAPPED_OUT"):
            tnn.tnn_knn_host(xyzt, off, SIG, 10, 8, 0.0, out=out, mapped=True)


def test_sweep_order_under_a_long_lag_matches_grid_order():
    """Under a long lag every bound carries the same large temporal part
    (sigma_t lag^2), so a query's k-th distance can exceed the F-th smallest
    segment bound at which the sweep's first pass stops.  The sweep may then
    skip the walk of the t_A table only if the temporal bound where that
    pass stopped also exceeds the key: with that check its lists equal the
    grid order's on all 200,000 rows (without it about one row in two
    thousand lost a neighbour), and a sample equals the oracle."""
    wl = synth.flights(1000, 200, 91)
    ix = _index(wl, 20)
    si, sd = tnn.tnn_knn(ix, 32, 1800.0, seed_segments=3, extra=4, sweep=True)
    gi, gd = tnn.tnn_knn(ix, 32, 1800.0, seed_segments=3, extra=4)
    torch.cuda.synchronize()
    assert torch.equal(si, gi) and torch.equal(sd, gd)
    q = synth.query_sample(wl.n, 512)
    oi, od = oracle.knn(wl.xyzt, 32, SIG, lag=1800.0, qsel=q)
    assert_knn_equal(si.cpu().numpy()[q], sd.cpu().numpy()[q], oi, od, what="sweep, lag 1800 s")


@pytest.mark.parametrize("offset", [(9000.0, -7000.0), (2e5, 1.5e5)])
def test_grid_search_far_from_the_origin(offset):
    # The grid's reach (cells within the k-th distance of a query) is taken in
    # FP32 with a slack that grows with the coordinates: data thousands of km
    # from the origin must give the oracle's lists, in both search orders.
    wl = synth.flights(80, 60, seed=17, n_routes=6)
    xyzt = wl.xyzt + np.array([offset[0], offset[1], 0.0, 0.0], np.float32)
    ix = tnn.tnn_build_segments(torch.from_numpy(xyzt).cuda(), wl.traj_off, SIG, 10)
    oi, od = oracle.knn(xyzt, 12, SIG, lag=0.0)
    for sweep in (False, True):
        ti, td = tnn.tnn_knn(ix, 12, 0.0, sweep=sweep)
        assert_knn_equal(ti.cpu().numpy(), td.cpu().numpy(), oi, od, what=f"offset {offset} sweep={sweep}")


def test_stop_certificate_every_skipped_segment_is_bounded_out():
    """Algorithm 2's stop rule and exclusion criterion, checked directly: the
    search records which segments it scanned for each query; every causal
    segment it skipped must have a cylinder bound above the query's final
    k-th distance (the bound it skipped against is the (k + extra)-th
    candidate, never below the k-th)."""
    far = synth.flights(60, 70, seed=43, n_routes=5)
    far = dataclasses.replace(far, xyzt=far.xyzt + np.array([3e4, -2e4, 0.0, 0.0], np.float32),
                              name="flights far from the origin")
    for wl, k, lag in ((synth.flights(60, 70, seed=41, n_routes=5), 16, 0.0),
                       (synth.flights(50, 80, seed=42, n_routes=4), 5, 90.0),
                       (synth.smoothed_random_walks(25, 90, seed=3), 32, 0.0),
                       (far, 16, 0.0)):
        ix = _index(wl, 12)
        idx, d2, path, seen = tnn.tnn_knn_trace(ix, k, lag, seen=True)
        lb = tnn.tnn_segment_lower_bounds(ix, lag=lag)
        seg, _ = tnn.tnn_index_export(ix)
        torch.cuda.synchronize()
        oi, od = oracle.knn(wl.xyzt, k, SIG, lag=lag)
        assert_knn_equal(idx.cpu().numpy(), d2.cpu().numpy(), oi, od, what=f"traced {wl.name}")
        seg = seg.cpu().numpy()
        first = seg[:, 12].view(np.int32)
        cnt = seg[:, 13].view(np.int32)
        bits = seen.cpu().numpy().view(np.uint32)
        pt_seen = ((bits[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(wl.n, -1)[:, :wl.n]
        # a segment counts as scanned for a query when its first member was
        # (members are recorded together)
        scanned = pt_seen[:, first].astype(bool)
        lbv = lb.cpu().numpy()
        dk = d2.cpu().numpy()[:, k - 1].astype(np.float64)
        p = path.cpu().numpy()
        rows = np.nonzero(p < 2)[0]
        assert rows.size > 0.9 * wl.n
        causal = np.isfinite(lbv)
        skipped = causal & ~scanned
        for q in rows:
            s = np.nonzero(skipped[q])[0]
            if s.size == 0:
                continue
            assert np.isfinite(dk[q]), (wl.name, q, "skipped a causal segment before k were found")
            worst = lbv[q, s].min()
            assert worst > dk[q] * (1.0 - 2.0 ** -18), (wl.name, q, worst, dk[q])
        # and the pruning did skip work
        assert skipped[rows].sum() > 0
        # every point of a segment scanned for a query was recorded with it
        scnt = pt_seen[rows].sum(axis=1)
        assert (scnt == (scanned[rows] * cnt[None, :]).sum(axis=1)).all()


def test_trace_paths_and_work_split_add_up():
    wl = synth.flights(300, 120, seed=61, n_routes=8)
    ix = _index(wl, 20)
    ti, td, st = tnn.tnn_knn(ix, 32, 0.0, stats=True)
    pi, pd, path = tnn.tnn_knn_trace(ix, 32, 0.0)
    torch.cuda.synchronize()
    assert torch.equal(pi, ti) and torch.equal(pd, td)
    p = path.cpu().numpy()
    assert set(np.unique(p).tolist()) <= {0, 1, 2}
    assert (p >= 1).sum() <= st["warp_queries"] and (p == 2).sum() == st["exact_queries"]
    total = tnn.tnn_knn_work(ix, 32, td)
    split = tnn.tnn_knn_work_split(ix, 32, td, path)
    for i in range(3):
        assert sum(split[c][i] for c in range(3)) == total[i]
    assert tnn.tnn_knn_work_split(ix, 32, td)[0] == list(total)


def test_expired_bounded_wait_is_reported_and_cleared():
    """A wait that nothing satisfies (the self-test kernel: an mbarrier no
    thread or copy arrives on, nothing in flight) gives up after its limit;
    the flag reaches the host as TNN_ERR_TIMEOUT at the next synchronising
    status call, once, and the context stays usable."""
    wl = synth.flights(30, 40, seed=5, n_routes=3)
    ix = _index(wl, 10)
    ref = tnn.tnn_knn(ix, 8, 0.0)
    tnn.tnn_sync_status()  # nothing pending
    tnn.tnn_selftest_bounded_wait(2000)
    with pytest.raises(tnn.TNNError) as ei:
        tnn.tnn_sync_status()
    assert ei.value.status == 4
    tnn.tnn_sync_status()  # reported once, then cleared
    again = tnn.tnn_knn(ix, 8, 0.0)
    torch.cuda.synchronize()
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1])
    # a search with statistics reports a pending flag too
    tnn.tnn_selftest_bounded_wait(1000)
    with pytest.raises(tnn.TNNError) as ei:
        tnn.tnn_knn(ix, 8, 0.0, stats=True)
    assert ei.value.status == 4
    tnn.tnn_sync_status()


def test_fp32_probe_measures_a_plausible_issue_rate():
    ops, ms = tnn.tnn_probe_fp32(1 << 14)
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM at no more than 2.2 GHz
    assert 0.3 * props.multi_processor_count * 128 * 1.0e9 < ops < props.multi_processor_count * 128 * 2.2e9
    assert ms > 0


def test_batched_full_config_sampled_against_oracle():
    """The batched configuration as timed: 64 windows of 10^4-5*10^5 points
    (log-uniform, whole 200-sample flights), k drawn from {16, 32, 64}, one
    persistent launch replayed from its CUDA graph; 512 sampled queries per
    window against the oracle."""
    wins = synth.batched_windows(n_windows=64)
    idxs = [_index(wl, 20) for wl, _ in wins]
    b = tnn.Batch(idxs, [k for _, k in wins])
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    st = b.stats()
    assert st["queries"] == sum(wl.n for wl, _ in wins)
    for w, (wl, k) in enumerate(wins):
        q = synth.query_sample(wl.n, 512, seed=0x5A00 + w)
        oi, od = oracle.knn(wl.xyzt, k, SIG, qsel=q)
        assert_knn_equal(b.idx[w].cpu().numpy()[q], b.d2[w].cpu().numpy()[q], oi, od,
                         what=f"window {w} ({wl.n} points) k={k}")
    b.destroy()
    for ix in idxs:
        ix.destroy()


def test_learned_config_contexts_sampled_against_oracle():
    """The learned form's contexts at full size: 5,000 flights x 200 samples
    = 1,000,000 points, k = 32, lag 1800 s, autotuned knobs; 4,096 sampled
    queries against the oracle."""
    wl = synth.learned()
    ix = _index(wl, 20)
    tune = tnn.tnn_autotune(ix, 32, 1800.0)
    ti, td, st = tnn.tnn_knn(ix, 32, 1800.0, stats=True, **tune)
    q = synth.query_sample(wl.n, 4096)
    oi, od = oracle.knn(wl.xyzt, 32, SIG, lag=1800.0, qsel=q)
    assert_knn_equal(ti.cpu().numpy()[q], td.cpu().numpy()[q], oi, od, what="learned 1M lag 1800")
    assert st["queries"] == wl.n


@pytest.mark.parametrize("k,lag,K", [(1, 0.0, 10), (8, 37.0, 7), (32, 0.0, 20), (64, 120.0, 13)])
def test_tensor_core_candidate_tiles_match_oracle(k, lag, K):
    """TNN with the candidate distances as tcgen05 tiles (TNN_FLAG_TC_TILES):
    the same exact answer as the FP32 member scan and the oracle, on flights,
    smoothed random walks and random points (several 128-query tiles and a
    ragged last one)."""
    for wl in (synth.flights(41, 53, seed=700 + k, n_routes=5),
               synth.smoothed_random_walks(23, 97, seed=k),
               synth.random_points(2771, 20, seed=k)):
        ix = _index(wl, K)
        ci, cd, st = tnn.tnn_knn(ix, k, lag, tc=True, stats=True)
        oi, od = oracle.knn(wl.xyzt, k, SIG, lag=lag)
        assert_knn_equal(ci.cpu().numpy(), cd.cpu().numpy(), oi, od, what=f"tc tiles {wl.name} k={k}")
        assert st["queries"] == wl.n
    # external queries, some before every point and some far outside the data
    wl = synth.flights(40, 64, seed=9, n_routes=5)
    ix = _index(wl, 10)
    rng = np.random.default_rng(5)
    q = wl.xyzt[rng.choice(len(wl.xyzt), 300, replace=False)].copy()
    q[:50, :2] += rng.normal(0, 500.0, size=(50, 2)).astype(np.float32)
    q[50:80, 3] = -5.0
    qd = torch.from_numpy(q).cuda()
    ci, cd = tnn.tnn_knn(ix, 10, 3.0, q=qd, tc=True)
    oi, od = oracle.knn(wl.xyzt, 10, SIG, lag=3.0, queries=q)
    assert_knn_equal(ci.cpu().numpy(), cd.cpu().numpy(), oi, od, what="tc tiles external queries")


def test_tensor_core_candidate_tiles_medium_and_precision_sampled():
    for wl in (synth.medium(), synth.precision()):
        ix = _index(wl, 20)
        ci, cd, st = tnn.tnn_knn(ix, 32, 0.0, tc=True, stats=True)
        q = synth.query_sample(wl.n, 4096)
        oi, od = oracle.knn(wl.xyzt, 32, SIG, qsel=q)
        assert_knn_equal(ci.cpu().numpy()[q], cd.cpu().numpy()[q], oi, od, what=f"tc tiles {wl.name}")
        assert st["queries"] == wl.n and st["segs_scanned"] > 0
        ti, td = tnn.tnn_knn(ix, 32, 0.0)
        assert torch.equal(ti, ci)
        ix.destroy()


def test_tensor_core_tiles_flag_is_for_single_searches():
    wl = synth.flights(20, 40, seed=3, n_routes=2)
    ix = _index(wl, 10)
    with pytest.raises(tnn.TNNError) as ei:
        tnn.Batch([ix, ix], [8, 8], tunings=[dict(tc=True), {}])
    assert ei.value.status == 1
    # the sweep order takes precedence over the tiles and is still exact
    si, sd = tnn.tnn_knn(ix, 8, 0.0, sweep=True, tc=True)
    oi, od = oracle.knn(wl.xyzt, 8, SIG)
    assert_knn_equal(si.cpu().numpy(), sd.cpu().numpy(), oi, od, what="sweep with tc flag")
