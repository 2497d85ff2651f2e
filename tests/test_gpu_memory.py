"""Library memory pool: index arrays and scratch are taken in stream order
from a pool that keeps freed memory reserved; trimming hands it back."""
import numpy as np
import pytest
import torch

from paper_2112_10408_gb300 import synth, tnn

pytestmark = pytest.mark.gpu


def test_pool_reuse_and_trim():
    tnn.load_library()
    wl = synth.flights(200, 50, synth.SEED_TINY)
    x = torch.from_numpy(wl.xyzt).cuda()
    torch.cuda.synchronize()
    _, used0 = tnn.tnn_memory_reserved()  # indexes other tests still hold
    ref = None
    for _ in range(3):
        ix = tnn.tnn_build_segments(x, wl.traj_off, synth.SIGMA_DEFAULT, 10)
        idx, d2 = tnn.tnn_knn(ix, 8, 0.0)
        got = idx.cpu().numpy()
        if ref is None:
            ref = got
        assert np.array_equal(got, ref)
        ix.destroy()
    reserved, used = tnn.tnn_memory_reserved()
    assert reserved > used and used == used0  # freed arrays stay reserved
    tnn.tnn_memory_trim(0)
    reserved2, used = tnn.tnn_memory_reserved()
    assert reserved2 < reserved and used == used0
    ix = tnn.tnn_build_segments(x, wl.traj_off, synth.SIGMA_DEFAULT, 10)
    idx, _ = tnn.tnn_knn(ix, 8, 0.0)
    assert np.array_equal(idx.cpu().numpy(), ref)
    _, used = tnn.tnn_memory_reserved()
    assert used > used0
    ix.destroy()
    with pytest.raises(Exception):
        tnn.tnn_memory_trim(-1)


@pytest.mark.parametrize("chunks", [0, 1, 3, 8])
def test_host_pipeline_matches_device_path(chunks):
    """tnn_knn_host (host buffers in and out, sliced search with overlapped
    copies) gives exactly the device path's lists."""
    tnn.load_library()
    wl = synth.flights(200, 50, synth.SEED_TINY)
    x = torch.from_numpy(wl.xyzt).cuda()
    ix = tnn.tnn_build_segments(x, wl.traj_off, synth.SIGMA_DEFAULT, 10)
    idx_d, d2_d = tnn.tnn_knn(ix, 8, 0.0)
    ix.destroy()
    h_x = torch.from_numpy(wl.xyzt).pin_memory() if chunks == 3 else wl.xyzt
    idx_h, d2_h = tnn.tnn_knn_host(h_x, wl.traj_off, synth.SIGMA_DEFAULT, 10, 8, 0.0, chunks=chunks)
    assert not idx_h.is_cuda
    assert torch.equal(idx_h, idx_d.cpu())
    assert torch.equal(d2_h, d2_d.cpu())
