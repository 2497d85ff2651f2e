"""Shared helpers of the test-suite (comparison of k-NN results)."""
import numpy as np

# FP32 distances against the oracle's FP64 value rounded to float32.
D2_RTOL = 1e-5


def assert_knn_equal(gi, gd, oi, od, rtol=D2_RTOL, what=""):
    gi = np.asarray(gi)
    gd = np.asarray(gd)
    bad = np.nonzero((gi != oi).any(axis=1))[0]
    if bad.size:
        r = bad[0]
        raise AssertionError(f"{what}: {bad.size} query rows differ; first row {r}:\n"
                             f"  gpu idx {gi[r].tolist()}\n  ora idx {oi[r].tolist()}\n"
                             f"  gpu d2 {gd[r].tolist()}\n  ora d2 {od[r].tolist()}")
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin), f"{what}: padding differs"
    np.testing.assert_allclose(gd[fin], od[fin], rtol=rtol, atol=0, err_msg=what)
