"""TEST INFRASTRUCTURE ONLY -- the CPU oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path and is
never part of the product path.

* ``knn`` -- exact causal k-NN by brute force in IEEE double (plain C,
  ``tnn_oracle.c``; the scalable metric of Sec. 3.4, the strict causal mask,
  ties broken by index).
* ``segments`` / ``cylinder_lb`` / ``paper_alg1`` -- the segment table of
  Sec. 3.4 and the lower bounds used to check the index invariants.
* ``nowcast`` -- the context features, the inverse-distance-weighted
  average and the two-layer GELU MLP with its gradient and the AdamW
  update, in float64 numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnn_oracle.c")
_LIB = os.path.join(_HERE, "libtnn_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no FMA contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.tnn_oracle_d2.restype = f64
        lib.tnn_oracle_d2.argtypes = [P, P, P]
        lib.tnn_oracle_knn.restype = ctypes.c_int
        lib.tnn_oracle_knn.argtypes = [P, i64, P, P, i64, P, f64, i32, P, P, P, i32]
        lib.tnn_oracle_point_segment_sq.restype = f64
        lib.tnn_oracle_point_segment_sq.argtypes = [P, P, P]
        lib.tnn_oracle_segments.restype = i64
        lib.tnn_oracle_segments.argtypes = [P, P, i64, P, i32, i64, P, P, P, P, P, P, P]
        lib.tnn_oracle_cylinder_lb.restype = f64
        lib.tnn_oracle_cylinder_lb.argtypes = [P, P, f64, P, P, f64, f64, f64]
        lib.tnn_oracle_paper_alg1.restype = f64
        lib.tnn_oracle_paper_alg1.argtypes = [P, P, f64, P, P, f64, f64, f64]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32x4(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    assert a.ndim == 2 and a.shape[1] == 4
    return a


def d2(a, b, sigma) -> float:
    """Canonical FP64 scaled squared distance between two float (x,y,z,t)."""
    lib = _load()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(4))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float32).reshape(4))
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(4))
    return float(lib.tnn_oracle_d2(_ptr(a), _ptr(b), _ptr(s)))


def knn(pts, k: int, sigma, lag: float = 0.0, queries=None, qsel=None,
        nthreads: int | None = None, want_d64: bool = False):
    """Exact causal k-NN.  ``queries`` defaults to ``pts`` (self-query);
    ``qsel`` selects query rows.  Returns (idx int32 [m,k], d2 float32 [m,k])
    and, with ``want_d64``, the float64 distances too."""
    lib = _load()
    pts = _f32x4(pts)
    qp = pts if queries is None else _f32x4(queries)
    if qsel is not None:
        qsel = np.ascontiguousarray(np.asarray(qsel, dtype=np.int64))
        m = int(qsel.shape[0])
    else:
        m = int(qp.shape[0])
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(4))
    idx = np.empty((m, k), dtype=np.int32)
    dd = np.empty((m, k), dtype=np.float32)
    d64 = np.empty((m, k), dtype=np.float64) if want_d64 else None
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.tnn_oracle_knn(_ptr(pts), pts.shape[0], _ptr(qp),
                            _ptr(qsel) if qsel is not None else None, m,
                            _ptr(s), float(lag), int(k), _ptr(idx), _ptr(dd),
                            _ptr(d64) if d64 is not None else None, int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle knn failed")
    return (idx, dd, d64) if want_d64 else (idx, dd)


def point_segment_sq(p, a, b) -> float:
    lib = _load()
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(3))
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(3))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(3))
    return float(lib.tnn_oracle_point_segment_sq(_ptr(p), _ptr(a), _ptr(b)))


def segments(pts, traj_off, sigma, K: int) -> dict:
    """Segment table in build order (see ``tnn_oracle_segments``)."""
    lib = _load()
    pts = _f32x4(pts)
    off = np.ascontiguousarray(np.asarray(traj_off, dtype=np.int64))
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(4))
    cap = int(sum((int(off[i + 1] - off[i]) + K - 1) // K for i in range(len(off) - 1)))
    first = np.empty(cap, np.int64); count = np.empty(cap, np.int32)
    A = np.empty((cap, 3)); B = np.empty((cap, 3))
    tA = np.empty(cap); tB = np.empty(cap); r = np.empty(cap)
    got = lib.tnn_oracle_segments(_ptr(pts), _ptr(off), len(off) - 1, _ptr(s),
                                  int(K), cap, _ptr(first), _ptr(count), _ptr(A),
                                  _ptr(B), _ptr(tA), _ptr(tB), _ptr(r))
    if got != cap:
        raise RuntimeError("oracle segments failed")
    return dict(first=first, count=count, A=A, B=B, tA=tA, tB=tB, radius=r)


def cylinder_lb(q, sigma, lag, A, B, tA, tB, r) -> float:
    lib = _load()
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float32).reshape(4))
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(4))
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(3))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(3))
    return float(lib.tnn_oracle_cylinder_lb(_ptr(q), _ptr(s), float(lag), _ptr(A),
                                            _ptr(B), float(tA), float(tB), float(r)))


def paper_alg1(q, sigma, lag, A_raw, B_raw, tA, tB, E_sq) -> float:
    lib = _load()
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float32).reshape(4))
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64).reshape(4))
    A = np.ascontiguousarray(np.asarray(A_raw, dtype=np.float64).reshape(3))
    B = np.ascontiguousarray(np.asarray(B_raw, dtype=np.float64).reshape(3))
    return float(lib.tnn_oracle_paper_alg1(_ptr(q), _ptr(s), float(lag), _ptr(A),
                                           _ptr(B), float(tA), float(tB), float(E_sq)))
