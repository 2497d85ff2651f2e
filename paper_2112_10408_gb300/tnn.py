"""Python binding of libtnn (include/tnn.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Tensors are
torch CUDA tensors on the current device; work is enqueued on torch's current
stream.  There is no CPU path: if libtnn.so is missing or the device is not
supported, the call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

_lib = None

c_i32, c_i64, c_f32, c_f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
c_p = ctypes.c_void_p


class TNNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libtnn status {status}: {msg}")
        self.status = status


class tnn_build_params(ctypes.Structure):
    _fields_ = [("sigma", c_f64 * 4), ("seg_len", c_i32)]


class tnn_index_info(ctypes.Structure):
    _fields_ = [("n_points", c_i64), ("n_traj", c_i64), ("n_segments", c_i64),
                ("seg_len", c_i32), ("coord_max", c_f32), ("max_radius", c_f32)]


class tnn_knn_params(ctypes.Structure):
    _fields_ = [("k", c_i32), ("lag", c_f64), ("seed_segments", c_i32),
                ("seed_window", c_i32), ("extra", c_i32), ("flags", c_i32),
                ("defer_cells", c_f32)]


class tnn_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_uint64), ("lb_evals", ctypes.c_uint64),
                ("pairs", ctypes.c_uint64), ("segs_scanned", ctypes.c_uint64),
                ("fp64_rechecks", ctypes.c_uint64), ("warp_queries", ctypes.c_uint64),
                ("exact_queries", ctypes.c_uint64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class tnn_adamw_params(ctypes.Structure):
    _fields_ = [("lr", c_f32), ("beta1", c_f32), ("beta2", c_f32), ("eps", c_f32),
                ("weight_decay", c_f32)]


TNN_FLAG_EXACT_D2 = 1
TNN_FLAG_SWEEP = 2
TNN_FLAG_FFMA = 4
TNN_FLAG_TC_TILES = 8
TNN_FLAG_MAPPED_OUT = 16
N_FEAT = 6

# (name, restype, argtypes)
_SIGNATURES = [
    ("tnn_status_string", ctypes.c_char_p, [c_i32]),
    ("tnn_last_error", ctypes.c_char_p, []),
    ("tnn_build_segments", c_i32, [c_p, c_i64, c_p, c_i64, ctypes.POINTER(tnn_build_params), c_p,
                                   ctypes.POINTER(c_p)]),
    ("tnn_index_destroy", None, [c_p]),
    ("tnn_index_get_info", c_i32, [c_p, ctypes.POINTER(tnn_index_info)]),
    ("tnn_index_export", c_i32, [c_p, c_p, c_p, c_p]),
    ("tnn_knn", c_i32, [c_p, c_p, c_i64, ctypes.POINTER(tnn_knn_params), c_p, c_p,
                        ctypes.POINTER(tnn_stats), c_p]),
    ("tnn_knn_bruteforce", c_i32, [c_p, c_p, c_i64, ctypes.POINTER(tnn_knn_params), c_p, c_p,
                                   ctypes.POINTER(tnn_stats), c_p]),
    ("tnn_knn_noalloc", c_i32, [c_p, c_p, c_i64, ctypes.POINTER(tnn_knn_params), c_p, c_p, c_p]),
    ("tnn_segment_lower_bounds", c_i32, [c_p, c_p, c_i64, c_f64, c_p, c_p]),
    ("tnn_knn_work", c_i32, [c_p, c_p, c_i64, c_i32, c_f64, c_p, c_p, c_p]),
    ("tnn_knn_work_split", c_i32, [c_p, c_p, c_i64, c_i32, c_f64, c_p, c_p, c_p, c_p]),
    ("tnn_knn_trace", c_i32, [c_p, c_p, c_i64, ctypes.POINTER(tnn_knn_params), c_p, c_p, c_p, c_p,
                              c_p]),
    ("tnn_profile_enable", c_i32, [c_i32]),
    ("tnn_profile_read", c_i32, [ctypes.POINTER(c_f64), ctypes.POINTER(c_i64), c_i32]),
    ("tnn_profile_read_kernels", c_i32, [c_p, ctypes.POINTER(c_i64), c_i32]),
    ("tnn_probe_fp32", c_i32, [c_i32, ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_p]),
    ("tnn_sync_status", c_i32, [c_p]),
    ("tnn_selftest_bounded_wait", c_i32, [c_i32, c_p]),
    ("tnn_knn_host", c_i32, [c_p, c_i64, c_p, c_i64, ctypes.POINTER(tnn_build_params),
                             ctypes.POINTER(tnn_knn_params), c_i32, c_p, c_p, c_p]),
    ("tnn_memory_trim", c_i32, [c_i64]),
    ("tnn_memory_reserved", c_i32, [ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("tnn_batch_create", c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(c_p), ctypes.POINTER(c_i64),
                                 ctypes.POINTER(tnn_knn_params), c_i32, ctypes.POINTER(c_p),
                                 ctypes.POINTER(c_p), ctypes.POINTER(c_p)]),
    ("tnn_batch_run", c_i32, [c_p, c_p]),
    ("tnn_batch_stats", c_i32, [c_p, ctypes.POINTER(tnn_stats), c_p]),
    ("tnn_batch_destroy", None, [c_p]),
    ("tnn_autotune", c_i32, [c_p, ctypes.POINTER(tnn_knn_params), c_i64, c_p]),
    ("tnn_context_features", c_i32, [c_p, c_p, c_p, c_i64, c_p, c_p, c_i32, c_p, c_p, c_f32,
                                     c_p, c_p, c_p]),
    ("tnn_window_average", c_i32, [c_p, c_p, c_p, c_i64, c_f64, c_f64, c_p, c_p]),
    ("tnn_mlp_create", c_i32, [c_i32, c_i32, ctypes.c_uint64, ctypes.POINTER(c_p)]),
    ("tnn_mlp_save", c_i32, [c_p, ctypes.c_char_p]),
    ("tnn_mlp_load", c_i32, [c_p, ctypes.c_char_p]),
    ("tnn_mlp_destroy", None, [c_p]),
    ("tnn_mlp_num_params", c_i64, [c_p]),
    ("tnn_mlp_get_params", c_i32, [c_p, c_p, c_p, c_p, ctypes.POINTER(c_i64)]),
    ("tnn_mlp_set_params", c_i32, [c_p, c_p, c_p, c_p, c_i64]),
    ("tnn_mlp_forward", c_i32, [c_p, c_p, c_i64, c_p, c_p]),
    ("tnn_mlp_gradients", c_i32, [c_p, c_p, c_p, c_i64, c_p, c_p, c_p]),
    ("tnn_mlp_train_step", c_i32, [c_p, c_p, c_p, c_i64, ctypes.POINTER(tnn_adamw_params), c_p,
                                   c_p]),
    ("tnn_gka_create", c_i32, [c_p, ctypes.POINTER(c_p)]),
    ("tnn_gka_destroy", None, [c_p]),
    ("tnn_gka_get_params", c_i32, [c_p, c_p, ctypes.POINTER(c_i64)]),
    ("tnn_gka_set_params", c_i32, [c_p, c_p]),
    ("tnn_gka_forward", c_i32, [c_p, c_p, c_p, c_p, c_i64, c_p, c_i32, c_p, c_p]),
    ("tnn_gka_train_step", c_i32, [c_p, c_p, c_p, c_p, c_i64, c_p, c_i32,
                                   ctypes.POINTER(tnn_adamw_params), c_p, c_p, c_p]),
    ("tnn_gkamlp_create", c_i32, [c_p, c_i32, ctypes.c_uint64, ctypes.POINTER(c_p)]),
    ("tnn_gkamlp_destroy", None, [c_p]),
    ("tnn_gkamlp_num_params", c_i64, [c_p]),
    ("tnn_gkamlp_get_params", c_i32, [c_p, c_p, ctypes.POINTER(c_i64)]),
    ("tnn_gkamlp_set_params", c_i32, [c_p, c_p]),
    ("tnn_gkamlp_forward", c_i32, [c_p, c_p, c_p, c_p, c_i64, c_p, c_i32, c_p, c_p]),
    ("tnn_gkamlp_train_step", c_i32, [c_p, c_p, c_p, c_p, c_i64, c_p, c_i32,
                                      ctypes.POINTER(tnn_adamw_params), c_p, c_p, c_p]),
    ("tnn_nowcast", c_i32, [c_p, c_p, c_p, c_i64, ctypes.POINTER(tnn_knn_params), c_p, c_p, c_p,
                            c_f32, c_p, c_p]),
]


def exported_symbols():
    return [s[0] for s in _SIGNATURES]


def load_library(path: str | None = None):
    """Load libtnn.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2112_10408_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _L():
    return _lib if _lib is not None else load_library()


def _check(status: int):
    if status != 0:
        lib = _L()
        raise TNNError(status, lib.tnn_last_error().decode(errors="replace") or
                       lib.tnn_status_string(status).decode())


def _stream():
    return c_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype, shape_tail=None, name="tensor") -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [*, {', '.join(map(str, shape_tail))}]")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t):
    return c_p(t.data_ptr()) if t is not None else c_p(None)


# --------------------------------------------------------------------- index

class Index:
    """Owner of a tnn_index*; the points are copied into it."""

    def __init__(self, handle, sigma, seg_len, n_points, n_traj, n_segments):
        self._h = handle
        self.sigma = tuple(float(s) for s in sigma)
        self.n_points = int(n_points)
        self.n_traj = int(n_traj)
        self.n_segments = int(n_segments)
        self.seg_len = int(seg_len)
        self._info = None

    def _get_info(self):
        # waits for the build to finish (the segment fit's largest radius)
        if self._info is None:
            info = tnn_index_info()
            _check(_L().tnn_index_get_info(self.handle, ctypes.byref(info)))
            self._info = info
        return self._info

    @property
    def coord_max(self) -> float:
        return float(self._get_info().coord_max)

    @property
    def max_radius(self) -> float:
        return float(self._get_info().max_radius)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("index destroyed")
        return self._h

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.tnn_index_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tnn_build_segments(xyzt: torch.Tensor, traj_off, sigma, seg_len: int) -> Index:
    xyzt = _dev(xyzt, torch.float32, (4,), "xyzt")
    off = np.ascontiguousarray(np.asarray(traj_off, dtype=np.int64))
    p = tnn_build_params()
    for i in range(4):
        p.sigma[i] = float(sigma[i])
    p.seg_len = int(seg_len)
    h = c_p()
    _check(_L().tnn_build_segments(_ptr(xyzt), xyzt.shape[0], off.ctypes.data_as(c_p),
                                   off.shape[0] - 1, ctypes.byref(p), _stream(), ctypes.byref(h)))
    n_segments = int(((np.diff(off) + seg_len - 1) // seg_len).sum())
    return Index(h, sigma, seg_len, xyzt.shape[0], off.shape[0] - 1, n_segments)


def tnn_index_export(index: Index):
    """(segment records [S, 16] float32, running max of t_B [S])."""
    S = index.n_segments
    seg = torch.empty((S, 16), dtype=torch.float32, device="cuda")
    pm = torch.empty((S,), dtype=torch.float32, device="cuda")
    _check(_L().tnn_index_export(index.handle, _ptr(seg), _ptr(pm), _stream()))
    return seg, pm


def make_knn_params(k: int, lag: float = 0.0, seed_segments: int = 0, seed_window: int = 0,
                    extra: int = 0, exact_d2: bool = False, sweep: bool = False,
                    defer_cells: float = 0.0, ffma: bool = False, tc: bool = False) -> tnn_knn_params:
    p = tnn_knn_params()
    p.k = int(k)
    p.lag = float(lag)
    p.seed_segments = int(seed_segments)
    p.seed_window = int(seed_window)
    p.extra = int(extra)
    p.flags = ((TNN_FLAG_EXACT_D2 if exact_d2 else 0) | (TNN_FLAG_SWEEP if sweep else 0)
               | (TNN_FLAG_FFMA if ffma else 0) | (TNN_FLAG_TC_TILES if tc else 0))
    p.defer_cells = float(defer_cells)
    return p


def _knn_call(fn, index, k, lag, q, stats, out, **kw):
    p = make_knn_params(k, lag, **kw)
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    if out is None:
        idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    else:
        idx, d2 = out
        _dev(idx, torch.int32, (k,), "idx")
        _dev(d2, torch.float32, (k,), "d2")
    st = tnn_stats() if stats else None
    _check(fn(index.handle, _ptr(q), m, ctypes.byref(p), _ptr(idx), _ptr(d2),
              ctypes.byref(st) if st is not None else None, _stream()))
    if stats:
        return idx, d2, st.as_dict()
    return idx, d2


def tnn_knn(index: Index, k: int, lag: float = 0.0, q=None, stats: bool = False, out=None, **kw):
    """Exact causal k-NN by TNN.  Returns (idx int32 [m,k], d2 float32 [m,k])
    (+ counters dict when ``stats``)."""
    return _knn_call(_L().tnn_knn, index, k, lag, q, stats, out, **kw)


def tnn_knn_bruteforce(index: Index, k: int, lag: float = 0.0, q=None, stats: bool = False,
                       out=None, **kw):
    """The same k-NN by linear search (the comparator): the distance matrix
    on the tensor cores, or on the CUDA cores with ``ffma=True``."""
    return _knn_call(_L().tnn_knn_bruteforce, index, k, lag, q, stats, out, **kw)


def tnn_segment_lower_bounds(index: Index, q=None, lag: float = 0.0) -> torch.Tensor:
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    out = torch.empty((m, index.n_segments), dtype=torch.float32, device="cuda")
    _check(_L().tnn_segment_lower_bounds(index.handle, _ptr(q), m, float(lag), _ptr(out),
                                         _stream()))
    return out


def tnn_knn_work(index: Index, k: int, d2: torch.Tensor, lag: float = 0.0, q=None):
    """(segment bounds, member points, key bounds) any exact search over the
    index must evaluate, summed over the queries."""
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    _dev(d2, torch.float32, (k,), "d2")
    out = (ctypes.c_uint64 * 3)()
    _check(_L().tnn_knn_work(index.handle, _ptr(q), m, int(k), float(lag), _ptr(d2), out,
                             _stream()))
    return int(out[0]), int(out[1]), int(out[2])


def tnn_knn_trace(index: Index, k: int, lag: float = 0.0, q=None, out=None, seen: bool = False,
                  **kw):
    """tnn_knn that also returns, per query, the kernel that finished it
    (uint8 [m]: 0 tile kernel, 1 warp-per-query kernel, 2 FP64 definition)
    and, with ``seen``, the bitmap [m, ceil(n/32)] int32 of the points whose
    segment was scanned for each query (returned as a fourth value)."""
    p = make_knn_params(k, lag, **kw)
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    if out is None:
        idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    else:
        idx, d2 = out
        _dev(idx, torch.int32, (k,), "idx")
        _dev(d2, torch.float32, (k,), "d2")
    path = torch.empty((m,), dtype=torch.uint8, device="cuda")
    sn = (torch.empty((m, (index.n_points + 31) // 32), dtype=torch.int32, device="cuda")
          if seen else None)
    _check(_L().tnn_knn_trace(index.handle, _ptr(q), m, ctypes.byref(p), _ptr(idx), _ptr(d2),
                              _ptr(path), _ptr(sn), _stream()))
    return (idx, d2, path, sn) if seen else (idx, d2, path)


def tnn_knn_work_split(index: Index, k: int, d2: torch.Tensor, path=None, lag: float = 0.0, q=None):
    """[3][3] nested lists: per finishing kernel (row), the (segment bounds,
    member points, key bounds) any exact search must evaluate."""
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    _dev(d2, torch.float32, (k,), "d2")
    if path is not None:
        _dev(path, torch.uint8, (), "path")
    out = (ctypes.c_uint64 * 9)()
    _check(_L().tnn_knn_work_split(index.handle, _ptr(q), m, int(k), float(lag), _ptr(d2),
                                   _ptr(path), out, _stream()))
    return [[int(out[3 * c + i]) for i in range(3)] for c in range(3)]


def tnn_sync_status():
    """Synchronise the current stream and raise TNNError for a fault the
    search kernels flagged since the last report."""
    _check(_L().tnn_sync_status(_stream()))


def tnn_selftest_bounded_wait(limit_us: int):
    """Enqueue the bounded-wait self-test (tnn_sync_status then reports a
    timeout)."""
    _check(_L().tnn_selftest_bounded_wait(int(limit_us), _stream()))


def tnn_probe_fp32(iters: int = 1 << 16):
    """(measured FFMA lane-operations per second, launch ms)."""
    ops, ms = c_f64(), c_f64()
    _check(_L().tnn_probe_fp32(int(iters), ctypes.byref(ops), ctypes.byref(ms), _stream()))
    return float(ops.value), float(ms.value)


def _host(t, dtype, shape_tail, name):
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(t)
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host array")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape[1:]) != tuple(shape_tail) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous [*, {', '.join(map(str, shape_tail))}] array")
    return t


def tnn_knn_host(xyzt, traj_off, sigma, seg_len: int, k: int, lag: float = 0.0, chunks: int = 0,
                 out=None, mapped=None, **kw):
    """The whole pipeline on host buffers (C ABI tnn_knn_host): points in,
    index, every point's causal k-NN, neighbour lists out.  ``xyzt`` is a
    host float32 [n, 4] array (numpy or CPU tensor; page-locked tensors copy
    faster); returns host (idx int32 [n, k], d2 float32 [n, k]), written
    into ``out`` when given.  ``mapped`` sets TNN_FLAG_MAPPED_OUT; by
    default it is set when both outputs are page-locked tensors (each one
    block of mapped page-locked memory)."""
    x = _host(xyzt, torch.float32, (4,), "xyzt")
    n = x.shape[0]
    off = np.ascontiguousarray(np.asarray(traj_off, dtype=np.int64))
    bp = tnn_build_params()
    for i in range(4):
        bp.sigma[i] = float(sigma[i])
    bp.seg_len = int(seg_len)
    kp = make_knn_params(k, lag, **kw)
    if out is None:
        idx = torch.empty((n, k), dtype=torch.int32)
        d2 = torch.empty((n, k), dtype=torch.float32)
    else:
        idx = _host(out[0], torch.int32, (k,), "idx")
        d2 = _host(out[1], torch.float32, (k,), "d2")
        if idx.shape[0] != n or d2.shape[0] != n:
            raise ValueError("outputs must have n rows")
    if mapped is None:
        mapped = idx.is_pinned() and d2.is_pinned()
    if mapped:
        kp.flags |= TNN_FLAG_MAPPED_OUT
    _check(_L().tnn_knn_host(_ptr(x), n, off.ctypes.data_as(c_p), off.shape[0] - 1, ctypes.byref(bp),
                             ctypes.byref(kp), int(chunks), _ptr(idx), _ptr(d2), _stream()))
    return idx, d2


def tnn_memory_trim(keep_bytes: int = 0):
    """Release the library pool's reserved device memory down to keep_bytes."""
    _check(_L().tnn_memory_trim(int(keep_bytes)))


def tnn_memory_reserved():
    """(reserved, in use) bytes of the library's device memory pool."""
    r, u = c_i64(0), c_i64(0)
    _check(_L().tnn_memory_reserved(ctypes.byref(r), ctypes.byref(u)))
    return r.value, u.value


def tnn_profile_enable(on: bool = True):
    _check(_L().tnn_profile_enable(1 if on else 0))


def tnn_profile_read(reset: bool = True):
    """(summed device ms of the search-kernel launches, launch count)."""
    ms = c_f64()
    n = c_i64()
    _check(_L().tnn_profile_read(ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
    return float(ms.value), int(n.value)


def tnn_profile_read_kernels(reset: bool = True):
    """([main kernel ms, warp-per-query kernel ms, FP64 kernel ms], launches)."""
    ms = (c_f64 * 3)()
    n = c_i64()
    _check(_L().tnn_profile_read_kernels(ms, ctypes.byref(n), 1 if reset else 0))
    return [float(ms[i]) for i in range(3)], int(n.value)


def tnn_autotune(index: Index, k: int, lag: float = 0.0, m_sample: int = 4096, exact_d2=False):
    p = make_knn_params(k, lag, exact_d2=exact_d2)
    _check(_L().tnn_autotune(index.handle, ctypes.byref(p), int(m_sample), _stream()))
    return dict(seed_segments=p.seed_segments, seed_window=p.seed_window, extra=p.extra,
                sweep=bool(p.flags & TNN_FLAG_SWEEP), defer_cells=float(p.defer_cells))


# --------------------------------------------------------------------- batch

class Batch:
    """tnn_batch: many windows answered by one persistent launch (CUDA graph)."""

    def __init__(self, indexes, ks, lags=None, queries=None, tunings=None):
        n = len(indexes)
        lags = lags or [0.0] * n
        tunings = tunings or [{}] * n
        self.indexes = list(indexes)
        self.queries = list(queries) if queries is not None else [None] * n
        self.ms = [(q.shape[0] if q is not None else ix.n_points)
                   for ix, q in zip(self.indexes, self.queries)]
        self.ks = list(ks)
        self.idx = [torch.empty((m, k), dtype=torch.int32, device="cuda")
                    for m, k in zip(self.ms, self.ks)]
        self.d2 = [torch.empty((m, k), dtype=torch.float32, device="cuda")
                   for m, k in zip(self.ms, self.ks)]
        P = (tnn_knn_params * n)()
        for w in range(n):
            P[w] = make_knn_params(self.ks[w], lags[w], **tunings[w])
        ix_arr = (c_p * n)(*[ix.handle for ix in self.indexes])
        q_arr = (c_p * n)(*[(q.data_ptr() if q is not None else None) for q in self.queries])
        m_arr = (c_i64 * n)(*self.ms)
        i_arr = (c_p * n)(*[t.data_ptr() for t in self.idx])
        d_arr = (c_p * n)(*[t.data_ptr() for t in self.d2])
        h = c_p()
        torch.cuda.synchronize()
        _check(_L().tnn_batch_create(ix_arr, q_arr, m_arr, P, n, i_arr, d_arr, ctypes.byref(h)))
        self._h = h

    def run(self):
        _check(_L().tnn_batch_run(self._h, _stream()))

    def stats(self):
        st = tnn_stats()
        _check(_L().tnn_batch_stats(self._h, ctypes.byref(st), _stream()))
        return st.as_dict()

    def destroy(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.tnn_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------- nowcast

def tnn_context_features(index: Index, wind: torch.Tensor, idx: torch.Tensor, d2: torch.Tensor,
                         q=None, mean=None, std=None, idw_eps: float = 1e-6,
                         want_feat: bool = True, want_idw: bool = True):
    """(features bf16 [m, k*6] or None, idw float32 [m, 2] or None)."""
    wind = _dev(wind, torch.float32, (2,), "wind")
    m, k = idx.shape
    _dev(idx, torch.int32, (k,), "idx")
    _dev(d2, torch.float32, (k,), "d2")
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
    feat = torch.empty((m, k * N_FEAT), dtype=torch.bfloat16, device="cuda") if want_feat else None
    idw = torch.empty((m, 2), dtype=torch.float32, device="cuda") if want_idw else None
    hm = np.ascontiguousarray(np.asarray(mean, np.float32)) if mean is not None else None
    hs = np.ascontiguousarray(np.asarray(std, np.float32)) if std is not None else None
    _check(_L().tnn_context_features(
        index.handle, _ptr(wind), _ptr(q), m, _ptr(idx), _ptr(d2), k,
        hm.ctypes.data_as(c_p) if hm is not None else None,
        hs.ctypes.data_as(c_p) if hs is not None else None, float(idw_eps),
        _ptr(feat), _ptr(idw), _stream()))
    return feat, idw


def tnn_window_average(index: Index, wind: torch.Tensor, before_lo: float = 5400.0,
                       before_hi: float = 1800.0, q=None) -> torch.Tensor:
    """Mean wind [m, 2] of the indexed points measured in
    [t_q - before_lo, t_q - before_hi] (the hour average of Sec. 4.1 with the
    defaults; the day average with before_lo = inf, before_hi = -inf)."""
    wind = _dev(wind, torch.float32, (2,), "wind")
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    out = torch.empty((m, 2), dtype=torch.float32, device="cuda")
    _check(_L().tnn_window_average(index.handle, _ptr(wind), _ptr(q), m, float(before_lo),
                                   float(before_hi), _ptr(out), _stream()))
    return out


@dataclass
class AdamW:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weight_decay: float = 1e-2

    def c(self):
        return tnn_adamw_params(self.lr, self.beta1, self.beta2, self.eps, self.weight_decay)


class MLP:
    """tnn_mlp: d_in -> d_hidden (GELU) -> 2, trained by the library's kernels."""

    def __init__(self, d_in: int, d_hidden: int = 256, seed: int = 0):
        h = c_p()
        _check(_L().tnn_mlp_create(int(d_in), int(d_hidden), ctypes.c_uint64(seed), ctypes.byref(h)))
        self._h = h
        self.d_in, self.d_hidden = int(d_in), int(d_hidden)
        self.n_params = int(_L().tnn_mlp_num_params(h))

    @property
    def handle(self):
        return self._h

    def tnn_mlp_forward(self, x: torch.Tensor) -> torch.Tensor:
        x = _dev(x, torch.bfloat16, (self.d_in,), "x")
        y = torch.empty((x.shape[0], 2), dtype=torch.float32, device="cuda")
        _check(_L().tnn_mlp_forward(self._h, _ptr(x), x.shape[0], _ptr(y), _stream()))
        return y

    forward = tnn_mlp_forward

    def tnn_mlp_gradients(self, x: torch.Tensor, target: torch.Tensor):
        x = _dev(x, torch.bfloat16, (self.d_in,), "x")
        target = _dev(target, torch.float32, (2,), "target")
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        grad = torch.empty((self.n_params,), dtype=torch.float32, device="cuda")
        _check(_L().tnn_mlp_gradients(self._h, _ptr(x), _ptr(target), x.shape[0], _ptr(loss),
                                      _ptr(grad), _stream()))
        return loss, grad

    gradients = tnn_mlp_gradients

    def tnn_mlp_train_step(self, x: torch.Tensor, target: torch.Tensor, opt: AdamW,
                           loss: torch.Tensor | None = None):
        x = _dev(x, torch.bfloat16, (self.d_in,), "x")
        target = _dev(target, torch.float32, (2,), "target")
        o = opt.c()
        _check(_L().tnn_mlp_train_step(self._h, _ptr(x), _ptr(target), x.shape[0],
                                       ctypes.byref(o), _ptr(loss), _stream()))
        return loss

    train_step = tnn_mlp_train_step

    def tnn_mlp_get_params(self, with_moments: bool = False):
        P = self.n_params
        w = np.empty(P, np.float32)
        m = np.empty(P, np.float32) if with_moments else None
        v = np.empty(P, np.float32) if with_moments else None
        step = c_i64()
        _check(_L().tnn_mlp_get_params(self._h, w.ctypes.data_as(c_p),
                                       m.ctypes.data_as(c_p) if m is not None else None,
                                       v.ctypes.data_as(c_p) if v is not None else None,
                                       ctypes.byref(step)))
        return (w, m, v, int(step.value)) if with_moments else w

    get_params = tnn_mlp_get_params

    def tnn_mlp_set_params(self, w, m=None, v=None, step: int = 0):
        w = np.ascontiguousarray(np.asarray(w, np.float32))
        assert w.shape == (self.n_params,)
        m = np.ascontiguousarray(np.asarray(m, np.float32)) if m is not None else None
        v = np.ascontiguousarray(np.asarray(v, np.float32)) if v is not None else None
        _check(_L().tnn_mlp_set_params(self._h, w.ctypes.data_as(c_p),
                                       m.ctypes.data_as(c_p) if m is not None else None,
                                       v.ctypes.data_as(c_p) if v is not None else None,
                                       int(step)))

    set_params = tnn_mlp_set_params

    def unflatten(self, w):
        """Split a flat parameter vector into (W1, b1, W2, b2) views."""
        di, dh = self.d_in, self.d_hidden
        o = 0
        W1 = w[o:o + di * dh].reshape(di, dh); o += di * dh
        b1 = w[o:o + dh]; o += dh
        W2 = w[o:o + 2 * dh].reshape(dh, 2); o += 2 * dh
        b2 = w[o:o + 2]
        return W1, b1, W2, b2

    def tnn_mlp_save(self, path: str):
        """Checkpoint (C ABI tnn_mlp_save): parameters, AdamW moments, step."""
        _check(_L().tnn_mlp_save(self._h, os.fsencode(path)))

    save = tnn_mlp_save

    def tnn_mlp_load(self, path: str):
        """Restore a checkpoint of an MLP of the same shape (tnn_mlp_load)."""
        _check(_L().tnn_mlp_load(self._h, os.fsencode(path)))

    load = tnn_mlp_load

    def destroy(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.tnn_mlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class GKA:
    """tnn_gka: Gaussian kernel averaging over TNN contexts (Eq. GKA) with
    scales (s_xy, s_z, s_t) trained by Adam."""

    def __init__(self, sigma=(1.0, 10.0, 0.01)):
        h = c_p()
        sig = np.ascontiguousarray(np.asarray(sigma, np.float32))
        _check(_L().tnn_gka_create(sig.ctypes.data_as(c_p), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def tnn_gka_get_params(self):
        """(sigma [3] float32, Adam step)."""
        sig = np.empty(3, np.float32)
        step = c_i64()
        _check(_L().tnn_gka_get_params(self._h, sig.ctypes.data_as(c_p), ctypes.byref(step)))
        return sig, int(step.value)

    get_params = tnn_gka_get_params

    def tnn_gka_set_params(self, sigma):
        sig = np.ascontiguousarray(np.asarray(sigma, np.float32))
        _check(_L().tnn_gka_set_params(self._h, sig.ctypes.data_as(c_p)))

    set_params = tnn_gka_set_params

    def tnn_gka_forward(self, index: Index, wind: torch.Tensor, idx: torch.Tensor, q=None):
        wind = _dev(wind, torch.float32, (2,), "wind")
        m, k = idx.shape
        _dev(idx, torch.int32, (k,), "idx")
        if q is not None:
            q = _dev(q, torch.float32, (4,), "q")
        uv = torch.empty((m, 2), dtype=torch.float32, device="cuda")
        _check(_L().tnn_gka_forward(self._h, index.handle, _ptr(wind), _ptr(q), m, _ptr(idx), k,
                                    _ptr(uv), _stream()))
        return uv

    forward = tnn_gka_forward

    def tnn_gka_train_step(self, index: Index, wind: torch.Tensor, rows: torch.Tensor,
                           idx: torch.Tensor, opt: "AdamW | None" = None, loss=None, grad=None):
        wind = _dev(wind, torch.float32, (2,), "wind")
        rows = _dev(rows, torch.int32, None, "rows")
        _dev(idx, torch.int32, (idx.shape[1],), "idx")
        o = opt.c() if opt is not None else None
        _check(_L().tnn_gka_train_step(self._h, index.handle, _ptr(wind), _ptr(rows), rows.shape[0],
                                       _ptr(idx), idx.shape[1], ctypes.byref(o) if o is not None else None,
                                       _ptr(loss), _ptr(grad), _stream()))

    train_step = tnn_gka_train_step

    def gradients(self, index: Index, wind, rows, idx):
        """(loss, d loss / d log sigma [3]) on the batch; no update."""
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        grad = torch.empty((3,), dtype=torch.float32, device="cuda")
        self.tnn_gka_train_step(index, wind, rows, idx, None, loss, grad)
        return loss, grad

    def destroy(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.tnn_gka_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class GKAMLP:
    """tnn_gkamlp: GKA whose scales are an MLP of the normalised location."""

    def __init__(self, sigma=(1.0, 10.0, 0.01), hidden: int = 32, seed: int = 0):
        h = c_p()
        sig = np.ascontiguousarray(np.asarray(sigma, np.float32))
        _check(_L().tnn_gkamlp_create(sig.ctypes.data_as(c_p), int(hidden), ctypes.c_uint64(seed),
                                      ctypes.byref(h)))
        self._h = h
        self.hidden = int(hidden)
        self.n_params = int(_L().tnn_gkamlp_num_params(h))

    @property
    def handle(self):
        return self._h

    def tnn_gkamlp_get_params(self):
        """(flat parameters float32, Adam step)."""
        w = np.empty(self.n_params, np.float32)
        step = c_i64()
        _check(_L().tnn_gkamlp_get_params(self._h, w.ctypes.data_as(c_p), ctypes.byref(step)))
        return w, int(step.value)

    get_params = tnn_gkamlp_get_params

    def tnn_gkamlp_set_params(self, w):
        w = np.ascontiguousarray(np.asarray(w, np.float32))
        if w.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {w.size}")
        _check(_L().tnn_gkamlp_set_params(self._h, w.ctypes.data_as(c_p)))

    set_params = tnn_gkamlp_set_params

    def tnn_gkamlp_forward(self, index: Index, wind: torch.Tensor, idx: torch.Tensor, q=None):
        wind = _dev(wind, torch.float32, (2,), "wind")
        m, k = idx.shape
        _dev(idx, torch.int32, (k,), "idx")
        if q is not None:
            q = _dev(q, torch.float32, (4,), "q")
        uv = torch.empty((m, 2), dtype=torch.float32, device="cuda")
        _check(_L().tnn_gkamlp_forward(self._h, index.handle, _ptr(wind), _ptr(q), m, _ptr(idx), k,
                                       _ptr(uv), _stream()))
        return uv

    forward = tnn_gkamlp_forward

    def tnn_gkamlp_train_step(self, index: Index, wind: torch.Tensor, rows: torch.Tensor,
                              idx: torch.Tensor, opt: "AdamW | None" = None, loss=None, grad=None):
        wind = _dev(wind, torch.float32, (2,), "wind")
        rows = _dev(rows, torch.int32, None, "rows")
        _dev(idx, torch.int32, (idx.shape[1],), "idx")
        o = opt.c() if opt is not None else None
        _check(_L().tnn_gkamlp_train_step(self._h, index.handle, _ptr(wind), _ptr(rows), rows.shape[0],
                                          _ptr(idx), idx.shape[1], ctypes.byref(o) if o is not None else None,
                                          _ptr(loss), _ptr(grad), _stream()))

    train_step = tnn_gkamlp_train_step

    def gradients(self, index: Index, wind, rows, idx):
        """(loss, gradient in the flat layout) on the batch; no update."""
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        grad = torch.empty((self.n_params,), dtype=torch.float32, device="cuda")
        self.tnn_gkamlp_train_step(index, wind, rows, idx, None, loss, grad)
        return loss, grad

    def destroy(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.tnn_gkamlp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tnn_nowcast(index: Index, wind: torch.Tensor, k: int, lag: float = 0.0, q=None,
                mlp: MLP | None = None, mean=None, std=None, idw_eps: float = 1e-6, **kw):
    wind = _dev(wind, torch.float32, (2,), "wind")
    if q is not None:
        q = _dev(q, torch.float32, (4,), "q")
        m = q.shape[0]
    else:
        m = index.n_points
    p = make_knn_params(k, lag, **kw)
    uv = torch.empty((m, 2), dtype=torch.float32, device="cuda")
    hm = np.ascontiguousarray(np.asarray(mean, np.float32)) if mean is not None else None
    hs = np.ascontiguousarray(np.asarray(std, np.float32)) if std is not None else None
    _check(_L().tnn_nowcast(index.handle, _ptr(wind), _ptr(q), m, ctypes.byref(p),
                            mlp.handle if mlp is not None else None,
                            hm.ctypes.data_as(c_p) if hm is not None else None,
                            hs.ctypes.data_as(c_p) if hs is not None else None,
                            float(idw_eps), _ptr(uv), _stream()))
    return uv
