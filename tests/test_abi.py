"""The C-ABI library loads and exports every entry point include/tnn.h
declares; argument checks answer before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2112_10408_gb300 import build as tnn_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tnn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = tnn_build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_binding_covers_header():
    from paper_2112_10408_gb300 import tnn
    assert set(declared_functions()) == set(tnn.exported_symbols())


def test_argument_errors_without_device(lib):
    from paper_2112_10408_gb300 import tnn
    L = tnn.load_library()
    h = ctypes.c_void_p()
    p = tnn.tnn_build_params()
    p.seg_len = 1  # K < 2
    off = (ctypes.c_int64 * 2)(0, 10)
    st = L.tnn_build_segments(ctypes.c_void_p(16), 10, off, 1, ctypes.byref(p), None, ctypes.byref(h))
    assert st == 1 and b"seg_len" in L.tnn_last_error()
    p.seg_len = 10
    p.sigma[3] = -1.0
    st = L.tnn_build_segments(ctypes.c_void_p(16), 10, off, 1, ctypes.byref(p), None, ctypes.byref(h))
    assert st == 1 and b"sigma" in L.tnn_last_error()
    kp = tnn.make_knn_params(0)
    st = L.tnn_knn(ctypes.c_void_p(8), None, 10, ctypes.byref(kp), None, None, None, None)
    assert st == 1 and b"k must" in L.tnn_last_error()
    kp = tnn.make_knn_params(8, lag=-1.0)
    st = L.tnn_knn(ctypes.c_void_p(8), None, 10, ctypes.byref(kp), None, None, None, None)
    assert st == 1 and b"lag" in L.tnn_last_error()
    st = L.tnn_mlp_create(100, 256, 0, ctypes.byref(h))
    assert st == 1 and b"d_in" in L.tnn_last_error()
    assert L.tnn_status_string(0) == b"ok"


def test_host_pipeline_and_memory_argument_errors(lib):
    from paper_2112_10408_gb300 import tnn
    L = tnn.load_library()
    bp = tnn.tnn_build_params()
    bp.seg_len = 10
    for i in range(4):
        bp.sigma[i] = 1.0
    kp = tnn.make_knn_params(8)
    off = (ctypes.c_int64 * 2)(0, 10)
    buf = (ctypes.c_float * 40)()
    oi = (ctypes.c_int32 * 80)()
    od = (ctypes.c_float * 80)()
    # NULL outputs
    st = L.tnn_knn_host(buf, 10, off, 1, ctypes.byref(bp), ctypes.byref(kp), 0, None, None, None)
    assert st == 1 and b"NULL" in L.tnn_last_error()
    # no points
    st = L.tnn_knn_host(buf, 0, off, 1, ctypes.byref(bp), ctypes.byref(kp), 0, oi, od, None)
    assert st == 1 and b"n must" in L.tnn_last_error()
    # k out of range
    kp0 = tnn.make_knn_params(65)
    st = L.tnn_knn_host(buf, 10, off, 1, ctypes.byref(bp), ctypes.byref(kp0), 0, oi, od, None)
    assert st == 1 and b"k must" in L.tnn_last_error()
    # too many slices
    st = L.tnn_knn_host(buf, 10, off, 1, ctypes.byref(bp), ctypes.byref(kp), 65, oi, od, None)
    assert st == 1 and b"chunks" in L.tnn_last_error()
    st = L.tnn_memory_trim(-1)
    assert st == 1 and b"keep_bytes" in L.tnn_last_error()
    st = L.tnn_memory_reserved(None, None)
    assert st == 1 and b"NULL" in L.tnn_last_error()


def test_measurement_and_baseline_entry_points_check_arguments(lib):
    from paper_2112_10408_gb300 import tnn
    L = tnn.load_library()
    ops, ms = ctypes.c_double(), ctypes.c_double()
    st = L.tnn_probe_fp32(0, ctypes.byref(ops), ctypes.byref(ms), None)
    assert st == 1 and b"iters" in L.tnn_last_error()
    st = L.tnn_probe_fp32(64, None, None, None)
    assert st == 1 and b"NULL" in L.tnn_last_error()
    st = L.tnn_selftest_bounded_wait(0, None)
    assert st == 1 and b"limit_us" in L.tnn_last_error()
    st = L.tnn_selftest_bounded_wait(2000000, None)
    assert st == 1 and b"limit_us" in L.tnn_last_error()
    buf = (ctypes.c_float * 8)()
    st = L.tnn_window_average(None, buf, None, 4, 5400.0, 1800.0, buf, None)
    assert st == 1 and b"NULL" in L.tnn_last_error()
    assert L.tnn_mlp_save(None, b"x.bin") == 1 and b"NULL" in L.tnn_last_error()
    assert L.tnn_mlp_load(None, b"x.bin") == 1 and b"NULL" in L.tnn_last_error()
    kp = tnn.make_knn_params(8)
    st = L.tnn_knn_trace(ctypes.c_void_p(8), None, 10, ctypes.byref(kp), buf, buf, None, None, None)
    assert st == 1 and b"d_path" in L.tnn_last_error()
    st = L.tnn_knn_work_split(ctypes.c_void_p(8), None, 10, 8, 0.0, buf, None, None, None)
    assert st == 1 and b"h_work" in L.tnn_last_error()
    # nothing recorded yet: zero time, zero launches
    k3 = (ctypes.c_double * 3)()
    n = ctypes.c_int64(-1)
    assert L.tnn_profile_read_kernels(k3, ctypes.byref(n), 1) == 0
    assert n.value == 0 and list(k3) == [0.0, 0.0, 0.0]
