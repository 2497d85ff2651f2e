"""tnn_knn_noalloc: the search for callers that cannot allocate device
memory (a plugin whose host framework owns all device allocations, or a
real-time loop that must not call an allocator).  Its scratch is a static
device array of the library; these tests call it through the C ABI and
compare it with tnn_knn on the same inputs, twice in a row, since every call
reuses the array left by the previous one.  This file is collected last so
that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2112_10408_gb300 import synth
from paper_2112_10408_gb300 import tnn
from tests._helpers import D2_RTOL

pytestmark = pytest.mark.gpu
SIG = synth.SIGMA_DEFAULT


@pytest.fixture(scope="module")
def lib():
    from paper_2112_10408_gb300 import build
    build.build()
    return tnn.load_library()


def _noalloc(lib, ix, k, lag, q, m, **kw):
    p = tnn.make_knn_params(k, lag, **kw)
    idx = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
    d2 = torch.full((m, k), float("nan"), dtype=torch.float32, device="cuda")
    st = lib.tnn_knn_noalloc(ix.handle, tnn._ptr(q), m, ctypes.byref(p), tnn._ptr(idx),
                             tnn._ptr(d2), tnn._stream())
    assert st == 0, lib.tnn_last_error()
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


def _same(a, b):
    ai, ad = a
    bi, bd = b
    np.testing.assert_array_equal(ai, bi)
    fin = np.isfinite(bd)
    assert np.array_equal(np.isfinite(ad), fin)
    np.testing.assert_allclose(ad[fin], bd[fin], rtol=D2_RTOL, atol=0)


def test_noalloc_matches_tnn_knn_on_two_calls_in_a_row(lib):
    wl = synth.flights(150, 100, seed=2024, n_routes=8)  # 15,000 points
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 20)
    ref = tnn.tnn_knn(ix, 16, 0.0)
    ref = (ref[0].cpu().numpy(), ref[1].cpu().numpy())
    for _ in range(2):  # self-query, the whole index
        _same(_noalloc(lib, ix, 16, 0.0, None, wl.n), ref)
    # external queries with another k and lag, again twice
    q = torch.from_numpy(wl.xyzt[::3].copy()).cuda()
    ref2 = tnn.tnn_knn(ix, 8, 120.0, q=q)
    ref2 = (ref2[0].cpu().numpy(), ref2[1].cpu().numpy())
    for _ in range(2):
        _same(_noalloc(lib, ix, 8, 120.0, q, q.shape[0]), ref2)


def test_noalloc_rejects_more_queries_than_its_array_holds(lib):
    wl = synth.flights(400, 200, seed=7, n_routes=8)  # 80,000 points
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 20)
    p = tnn.make_knn_params(8)
    idx = torch.empty((wl.n, 8), dtype=torch.int32, device="cuda")
    d2 = torch.empty((wl.n, 8), dtype=torch.float32, device="cuda")
    st = lib.tnn_knn_noalloc(ix.handle, None, wl.n, ctypes.byref(p), tnn._ptr(idx),
                             tnn._ptr(d2), tnn._stream())
    assert st == 1 and b"at most 65536" in lib.tnn_last_error()
    # a slice within the limit still answers exactly
    q = torch.from_numpy(wl.xyzt[-60000:].copy()).cuda()
    ref = tnn.tnn_knn(ix, 8, 0.0, q=q)
    _same(_noalloc(lib, ix, 8, 0.0, q, q.shape[0]), (ref[0].cpu().numpy(), ref[1].cpu().numpy()))


def test_noalloc_at_exact_capacity_and_in_sweep_order(lib):
    """65,536 queries fill the static array to its end (both fallback lists
    and the handed-over keys); the sweep order runs another kernel over the
    same scratch.  Both against tnn_knn, twice in a row."""
    wl = synth.flights(400, 200, seed=11, n_routes=8)  # 80,000 points
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 20)
    q = torch.from_numpy(wl.xyzt[-65536:].copy()).cuda()
    ref = tnn.tnn_knn(ix, 32, 0.0, q=q)
    ref = (ref[0].cpu().numpy(), ref[1].cpu().numpy())
    for _ in range(2):
        _same(_noalloc(lib, ix, 32, 0.0, q, 65536), ref)
    q2 = torch.from_numpy(wl.xyzt[::7].copy()).cuda()
    ref2 = tnn.tnn_knn(ix, 16, 30.0, q=q2, sweep=True)
    ref2 = (ref2[0].cpu().numpy(), ref2[1].cpu().numpy())
    for _ in range(2):
        _same(_noalloc(lib, ix, 16, 30.0, q2, q2.shape[0], sweep=True), ref2)
    # nothing the kernels flagged is pending
    tnn.tnn_sync_status()


def test_noalloc_rejects_the_tensor_core_tiles_flag(lib):
    # the tiles read a key-ordered copy of the points that the index builds
    # on first use, i.e. an allocation: this entry point refuses the flag
    wl = synth.flights(20, 40, seed=4, n_routes=2)
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, SIG, 10)
    p = tnn.make_knn_params(8, tc=True)
    idx = torch.empty((wl.n, 8), dtype=torch.int32, device="cuda")
    d2 = torch.empty((wl.n, 8), dtype=torch.float32, device="cuda")
    st = lib.tnn_knn_noalloc(ix.handle, None, wl.n, ctypes.byref(p), tnn._ptr(idx), tnn._ptr(d2),
                             tnn._stream())
    assert st == 1 and b"TNN_FLAG_TC_TILES" in lib.tnn_last_error()
