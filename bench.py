#!/usr/bin/env python3
"""Exact causal k-NN contexts/s with TNN on one GB300 (and the linear-search
comparator on the same inputs).

A step is one pass of the search over every query of the workload:
self-query of all points of the medium trajectory workload (2,000 synthetic
flights x 200 samples = 400,000 points, k = 32, 20-point segments, scales
(1, 1, 10, 0.01), mask t_j < t_i).  Inputs are resident in HBM; L2 is
flushed (256 MiB write) before every timed step.  The JSON line follows the
repository's benchmark contract.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "causal k-NN contexts/sec (exact, k=32) TNN vs GPU brute force on 1 GB300"
UNIT = "contexts/s"
# FP32 lane-operations per query-to-cylinder bound, per point distance and
# per grid-key bound (instruction counts of seg_lb, of dist32 + mask +
# compare, and of cell_lb).
OPS_PER_LB = 26
OPS_PER_PAIR = 14
OPS_PER_KEY = 20

# DRAM bytes (read + write) per launch of each search kernel on the medium
# workload, from one ncu capture of the timed search
# (dram__bytes_read.sum + dram__bytes_write.sum), with a hash of the kernel
# sources it was taken on (stale, and reported as null, once they change) and
# the tuning of that capture.
SEARCH_TRAFFIC = {"bytes": {"k_tnn_grid_search": 10436864 + 47383808, "k_tnn_warp": 3980288 + 0},
                  "workload": "medium",
                  "sources": ['tnn_device.cuh', 'tnn_grid.cuh', 'tnn_fallback.cuh', 'tnn_internal.cuh', 'tnn_knn.cu', 'tnn_index.cu'],
                  "tuning": {"seed_segments": 3, "extra": 4, "defer_cells": 1.0},
                  "sha256_16": "df2e349dfcd0b0a4"}


def _search_traffic(workload, kernel):
    import hashlib
    h = hashlib.sha256()
    for f in SEARCH_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2112_10408_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if workload != SEARCH_TRAFFIC["workload"] or h.hexdigest()[:16] != SEARCH_TRAFFIC["sha256_16"]:
        return None
    return SEARCH_TRAFFIC["bytes"].get(kernel)


def _max_over_ranks(x, world, device="cuda"):
    """The job's time is the slowest rank's (a MAX all-reduce; the only
    collective of the run: each rank answers its own window)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _throughput(world, m, steps, total_ms):
    """Whole-job contexts/s: every rank answers m queries per step."""
    return world * m * steps / (total_ms / 1e3)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["medium", "tiny", "precision"], default="medium")
    ap.add_argument("--comparator-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-window and nowcast measurements")
    ap.add_argument("--tuning", choices=["auto", "default"], default="auto",
                    help="autotune the seed/extra knobs (auto) or use the library defaults")
    return ap.parse_args()


def _workload(name, rank):
    from paper_2112_10408_gb300 import synth
    if name == "tiny":
        wl, k, K = synth.flights(200, 50, synth.SEED_TINY + 1000 * rank, name="tiny-10k"), 8, 10
    elif name == "precision":
        wl, k, K = synth.flights(20000, 200, synth.SEED_PRECISION + 1000 * rank,
                                 name="precision-4M"), 32, 20
    else:
        wl, k, K = synth.flights(2000, 200, synth.SEED_MEDIUM + 1000 * rank,
                                 name="medium-400k"), 32, 20
    return wl, k, K


def _config(wl, k, K, name):
    desc = {"tiny": "200 synthetic flights x 50 samples = 10,000 points",
            "medium": "2,000 synthetic flights x 200 samples = 400,000 points",
            "precision": "20,000 synthetic flights x 200 samples = 4,000,000 points"}[name]
    return {"workload": f"{wl.name}: {desc}, self-query of every point",
            "k": k, "seg_len": K, "sigma": list((1.0, 1.0, 10.0, 0.01)), "lag_s": 0.0,
            "queries_per_step": wl.n,
            "generator": "routes of 3-5 waypoints, 4 s sampling, N(0,50 m) jitter, 2000x2000 km x 12 km x 6 h",
            "l2": "flushed before every timed step (256 MiB write)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.bus_id:
                cmd += ["-i", self.bus_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _cpu_model():
    """The host CPU's model name (lscpu), for the oracle's timing lines."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _parity(gi, gd, oi, od):
    """Sampled GPU rows against the oracle's: identical neighbour indices
    (ties by index), and the largest relative error of the reported FP32
    distance against the FP64 one."""
    import numpy as np
    same = bool(np.array_equal(gi, oi))
    fin = np.isfinite(od)
    pad_ok = bool(np.array_equal(np.isfinite(gd), fin))
    err = 0.0
    if fin.any():
        err = float(np.max(np.abs(gd[fin].astype(np.float64) - od[fin]) / np.maximum(od[fin], 1e-300)))
    return {"queries_checked": int(gi.shape[0]), "identical_indices": same and pad_ok,
            "rows_differing": int((gi != oi).any(axis=1).sum()), "max_rel_d2_err_vs_fp64": err,
            "tolerance": 1e-5}


def _cpu_baseline(wl, k, n_sample, idx=None, d2=None, lag=0.0, seed=0x5A00):
    """The FP64 oracle as it stands on a bounded sample of the queries, and
    (given the GPU outputs) the parity of those rows."""
    import oracle
    from paper_2112_10408_gb300 import synth
    q = synth.query_sample(wl.n, n_sample, seed=seed)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oi, od, o64 = oracle.knn(wl.xyzt, k, (1.0, 1.0, 10.0, 0.01), lag=lag, qsel=q, nthreads=cores,
                             want_d64=True)
    dt = time.perf_counter() - t0
    out = {"value": q.size / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
           "sample": f"{q.size} uniformly sampled self-queries of the same workload "
                     f"(FP64 brute force, {cores} threads, {dt:.2f} s)"}
    if idx is not None:
        import torch
        qt = torch.from_numpy(q).to(idx.device)
        out["parity"] = _parity(idx[qt].cpu().numpy(), d2[qt].cpu().numpy(), oi, o64)
    return out


def _fp32_peak(tnn, peaks, nsm):
    """FFMA lane-operations/s measured by the library's probe (best of 3),
    with the unit-count figure beside it."""
    best = 0.0
    for _ in range(3):
        ops, _ms = tnn.tnn_probe_fp32(1 << 16)
        best = max(best, ops)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    return best / 1e12, nsm * 128 * sm_max * 1e6 / 1e12


def _search_roofline(tnn, ix, k, lag, tune, kern_ms, launches, alu_peak, derived_peak, traffic, out):
    """Roofline of the search, split by kernel: the necessary work of the
    queries each kernel finished (tnn_knn_trace + tnn_knn_work_split) over
    that kernel's own CUDA-event time; the top level is the kernel that
    takes the larger share."""
    idx, d2 = out
    _, _, path = tnn.tnn_knn_trace(ix, k, lag, out=(idx, d2), **tune)
    split = tnn.tnn_knn_work_split(ix, k, d2, path, lag)
    names = ["k_tnn_grid_search", "k_tnn_warp", "k_fallback_exact"]
    per = {}
    for c, name in enumerate(names):
        nlb, npairs, nkeys = split[c]
        ops = OPS_PER_LB * nlb + OPS_PER_PAIR * npairs + OPS_PER_KEY * nkeys
        ms = kern_ms[c] / max(launches, 1)
        ach = ops / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        per[name] = {"ms": ms, "queries": int((path == c).sum().item()),
                     "lb_needed": nlb, "pairs_needed": npairs, "keys_needed": nkeys,
                     "achieved": ach, "frac": ach / alu_peak}
    tot_ops = sum(OPS_PER_LB * split[c][0] + OPS_PER_PAIR * split[c][1] + OPS_PER_KEY * split[c][2]
                  for c in range(3))
    tot_ms = sum(kern_ms) / max(launches, 1)
    dom = max(names[:2], key=lambda n: per[n]["ms"])
    d = per[dom]
    return {"bound": "alu", "achieved": d["achieved"], "peak": alu_peak, "unit": "T FP32 lane-ops/s",
            "frac": d["frac"], "traffic": traffic, "kernel": dom, "kernel_ms": d["ms"],
            "peak_note": "of measured: FFMA issue rate from tnn_probe_fp32 (best of 3); "
                         f"unit-count figure {derived_peak:.2f}",
            "work_note": "necessary work of the queries this kernel finished; ops per unit "
                         f"{OPS_PER_LB}/{OPS_PER_PAIR}/{OPS_PER_KEY} (bound/pair/key)",
            "kernels": per,
            "search": {"ms": tot_ms, "achieved": tot_ops / (tot_ms / 1e3) / 1e12,
                       "frac": tot_ops / (tot_ms / 1e3) / 1e12 / alu_peak,
                       "kernels": "k_tnn_grid_search + k_tnn_warp + k_fallback_exact"}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2112_10408_gb300 import synth
    oracle.build()
    wl, k, K = _workload(a.workload, 0)
    cores = os.cpu_count() or 1
    per_step = 2048  # ~0.1 s of the 16-thread oracle per step at 400,000 points
    for w in range(a.warmup):
        oracle.knn(wl.xyzt, k, (1.0, 1.0, 10.0, 0.01), qsel=synth.query_sample(wl.n, per_step, seed=w),
                   nthreads=cores)
    t0 = time.perf_counter()
    for s in range(a.steps):
        q = synth.query_sample(wl.n, per_step, seed=0x1000 + s)
        oracle.knn(wl.xyzt, k, (1.0, 1.0, 10.0, 0.01), qsel=q, nthreads=cores)
    dt = time.perf_counter() - t0
    value = a.steps * per_step / dt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": 1e3 * dt / max(a.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(wl, k, K, a.workload), "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "cpu": _cpu_model(),
                            "sample": f"each step: {per_step} uniformly sampled self-queries "
                                      f"(FP64 brute-force oracle, {cores} threads)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


class _Range:
    """NVTX range around a measured section (lets ncu select its kernels with
    --nvtx --nvtx-include "<name>/")."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push(self.name)

    def __exit__(self, *exc):
        import torch
        torch.cuda.nvtx.range_pop()


def _timed(fn, steps, flush=None):
    """Mean CUDA-event time (ms) of fn() over `steps` runs, L2 flushed before each."""
    import torch
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return sum(ms) / len(ms)


def _extras(tnn, synth, flush, peaks, steps):
    """The other rows of the path, each timed on its own: the persistent
    batched driver over 64 windows (CUDA graph), and the learned form
    (contexts with lag 1800 s, features + IDW, MLP training, nowcasts)."""
    import numpy as np
    import torch
    sigma = (1.0, 1.0, 10.0, 0.01)
    out = {}
    # ---- batched windows
    wins = synth.batched_windows(n_windows=64)
    idxs = [tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, sigma, 20)
            for wl, _ in wins]
    # two tunings of the same launch: the library defaults, and every window
    # autotuned on its own (tnn_autotune: seed count, list width, deferral
    # radius for that window's size and k); the faster one is the batched
    # figure.  A batch runs one segment order for all its windows, so the
    # per-window tunings keep the grid order.
    ks = [k for _, k in wins]
    t0 = time.perf_counter()
    tuned = [dict(tnn.tnn_autotune(ix, k, 0.0), sweep=False) for ix, k in zip(idxs, ks)]
    tune_s = time.perf_counter() - t0
    timing = {}
    for name, tunings in (("library_defaults", [{}] * len(wins)), ("autotuned_per_window", tuned)):
        bb = tnn.Batch(idxs, ks, tunings=tunings)
        for _ in range(3):
            bb.run()
        torch.cuda.synchronize()
        with _Range("batched_" + name):
            timing[name] = _timed(bb.run, steps, flush)
        bb.destroy()
        del bb
    best_tuning = min(timing, key=timing.get)
    b = tnn.Batch(idxs, ks, tunings=tuned if best_tuning == "autotuned_per_window" else [{}] * len(wins))
    b.run()
    torch.cuda.synchronize()
    ms = timing[best_tuning]
    nq = sum(wl.n for wl, _ in wins)
    # each window on its own (tnn_knn, same knobs), for the per-window rates
    per_window = []
    for w, (wl, kw_) in enumerate(wins):
        iw, dw = b.idx[w], b.d2[w]
        kn_w = tuned[w] if best_tuning == "autotuned_per_window" else {}
        tnn.tnn_knn(idxs[w], kw_, 0.0, out=(iw, dw), **kn_w)
        torch.cuda.synchronize()
        wms = _timed(lambda: tnn.tnn_knn(idxs[w], kw_, 0.0, out=(iw, dw), **kn_w), 3, flush)
        per_window.append({"window": w, "points": wl.n, "k": kw_, "ms": wms,
                           "contexts_per_s": wl.n / (wms / 1e3)})
    b.run()  # the batched outputs again, for the parity sample below
    torch.cuda.synchronize()
    # the oracle on 64 sampled queries per window (host cores), and the
    # parity of those rows of the batched outputs
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    gi_all, gd_all, oi_all, od_all = [], [], [], []
    t0 = time.perf_counter()
    for w, (wl, kw_) in enumerate(wins):
        q = synth.query_sample(wl.n, 64, seed=0x5A00 + w)
        oi, od, o64 = oracle.knn(wl.xyzt, kw_, sigma, qsel=q, nthreads=cores, want_d64=True)
        qt = torch.from_numpy(q).cuda()
        gi = b.idx[w][qt].cpu().numpy()
        gd = b.d2[w][qt].cpu().numpy()
        pad = 64 - kw_
        gi_all.append(np.pad(gi, ((0, 0), (0, pad)), constant_values=-2))
        oi_all.append(np.pad(oi, ((0, 0), (0, pad)), constant_values=-2))
        gd_all.append(np.pad(gd, ((0, 0), (0, pad)), constant_values=np.inf))
        od_all.append(np.pad(o64, ((0, 0), (0, pad)), constant_values=np.inf))
    dt = time.perf_counter() - t0
    nsq = 64 * len(wins)
    out["batched"] = {"metric": "causal k-NN contexts/s over 64 windows in one persistent launch",
                      "value": nq / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "windows": len(wins),
                      "queries": nq, "k_mix": {str(k): sum(1 for _, kk in wins if kk == k) for k in (16, 32, 64)},
                      "launch": "tnn_batch_run: one CUDA graph (tile kernel + warp kernel + exact kernel)",
                      "tuning": best_tuning, "ms_by_tuning": timing, "autotune_s": tune_s,
                      "per_window": per_window,
                      "per_window_note": "each window alone through tnn_knn (L2 flushed), same knobs",
                      "cpu_baseline": {"value": nsq / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": f"64 sampled self-queries per window ({nsq}), FP64 brute force",
                                       "parity": _parity(np.concatenate(gi_all), np.concatenate(gd_all),
                                                         np.concatenate(oi_all), np.concatenate(od_all))}}
    b.destroy()
    for ix in idxs:
        ix.destroy()
    del idxs, b
    torch.cuda.empty_cache()

    # ---- learned form: 5,000 flights x 200 = 1,000,000 points, lag 1800 s
    wl = synth.learned()
    k, lag = 32, 1800.0
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, sigma, 20)
    wind = torch.from_numpy(wl.wind).cuda()
    idx = torch.empty((wl.n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((wl.n, k), dtype=torch.float32, device="cuda")
    tune = tnn.tnn_autotune(ix, k, lag)
    tnn.tnn_knn(ix, k, lag, out=(idx, d2), **tune)
    torch.cuda.synchronize()
    with _Range("learned_contexts"):
        ms_knn = _timed(lambda: tnn.tnn_knn(ix, k, lag, out=(idx, d2), **tune), steps, flush)
    full = (idx >= 0).all(dim=1).cpu().numpy()
    train, test = synth.flight_split(wl)
    tr = np.nonzero(train & full)[0]
    te = np.nonzero(test & full)[0]
    raw, idw = tnn.tnn_context_features(ix, wind, idx, d2)
    f = raw.float()[torch.from_numpy(tr).cuda()].view(-1, k, 6)
    mean = f.mean(dim=(0, 1)).cpu().numpy()
    std = f.std(dim=(0, 1)).cpu().numpy() + 1e-6
    del f, raw
    feat, _ = tnn.tnn_context_features(ix, wind, idx, d2, mean=mean, std=std, want_idw=False)
    with _Range("features"):
        ms_feat = _timed(lambda: tnn.tnn_context_features(ix, wind, idx, d2, mean=mean, std=std), steps, flush)
    # bytes per context: idx + d2 (8 k), gathered point + wind (24 k), query
    # point (16), features out (12 k bf16), IDW out (8)
    feat_bytes = wl.n * (44 * k + 24)
    mlp = tnn.MLP(k * 6, 256, seed=0)
    opt = tnn.AdamW(lr=1e-3, weight_decay=1e-2)
    rng = np.random.default_rng(0)
    trd = torch.from_numpy(tr).cuda()
    B = 4096
    epochs = 3
    batches = []
    for _ in range(epochs):
        perm = trd[torch.from_numpy(rng.permutation(tr.size)).cuda()]
        for s0 in range(0, perm.numel() - B + 1, B):
            sel = perm[s0:s0 + B]
            batches.append((feat[sel].contiguous(), wind[sel].contiguous()))
    mlp.train_step(*batches[0], opt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for xb, yb in batches[1:]:
        mlp.train_step(xb, yb, opt)
    e1.record()
    torch.cuda.synchronize()
    ms_train = e0.elapsed_time(e1) / (len(batches) - 1)
    flops_step = 2.0 * B * (k * 6) * 256 * 2 + 2.0 * B * 256 * 2 * 3
    # device-side rate: 16 steps captured once in a CUDA graph and replayed
    # (the AdamW step count lives on the device, so replays stay correct)
    G = 16
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        mlp.train_step(*batches[1], opt)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for xb, yb in batches[:G]:
            mlp.train_step(xb, yb, opt)
    graph.replay()
    torch.cuda.synchronize()
    with _Range("mlp_train"):
        ms_graph = _timed(graph.replay, steps) / G
    ted = torch.from_numpy(te).cuda()
    xte = feat[ted].contiguous()
    mlp.forward(xte)  # sizes the workspace outside the timed runs
    torch.cuda.synchronize()
    with _Range("mlp_forward"):
        ms_fwd = _timed(lambda: mlp.forward(xte), steps)
    pred = mlp.forward(xte)
    rmse_mlp = float(torch.sqrt(((pred - wind[ted]) ** 2).mean()))
    rmse_idw = float(torch.sqrt(((idw[ted] - wind[ted]) ** 2).mean()))
    qte = torch.from_numpy(wl.xyzt[te]).cuda()
    tnn.tnn_nowcast(ix, wind, k, lag, q=qte, mlp=mlp, mean=mean, std=std, **tune)
    torch.cuda.synchronize()
    ms_now = _timed(lambda: tnn.tnn_nowcast(ix, wind, k, lag, q=qte, mlp=mlp, mean=mean, std=std, **tune),
                    steps, flush)
    # the same held-out queries with the IDW fallback (no MLP): latency and
    # RMSE side by side with the MLP (matched query count, same search)
    tnn.tnn_nowcast(ix, wind, k, lag, q=qte, **tune)
    torch.cuda.synchronize()
    ms_now_idw = _timed(lambda: tnn.tnn_nowcast(ix, wind, k, lag, q=qte, **tune), steps, flush)
    now_idw = tnn.tnn_nowcast(ix, wind, k, lag, q=qte, **tune)
    now_mlp = tnn.tnn_nowcast(ix, wind, k, lag, q=qte, mlp=mlp, mean=mean, std=std, **tune)
    okq = torch.isfinite(now_idw).all(dim=1)
    rmse_now_idw = float(torch.sqrt(((now_idw[okq] - wind[ted][okq]) ** 2).mean()))
    rmse_now_mlp = float(torch.sqrt(((now_mlp[okq] - wind[ted][okq]) ** 2).mean()))
    # the averaging baselines of Table 2: hour average [t - 1 h 30, t - 30 min]
    # (causal) and day average (non-causal, every point)
    hour = tnn.tnn_window_average(ix, wind, 5400.0, 1800.0, q=qte)
    torch.cuda.synchronize()
    ms_hour = _timed(lambda: tnn.tnn_window_average(ix, wind, 5400.0, 1800.0, q=qte), steps, flush)
    hok = torch.isfinite(hour).all(dim=1)
    rmse_hour = float(torch.sqrt(((hour[hok] - wind[ted][hok]) ** 2).mean()))
    day = tnn.tnn_window_average(ix, wind, float("inf"), float("-inf"), q=qte)
    rmse_day = float(torch.sqrt(((day - wind[ted]) ** 2).mean()))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    # GKA-TNN (Eq. GKA): scales trained by Adam on the training rows
    gka = tnn.GKA((1.0, 10.0, 0.01))
    gopt = tnn.AdamW(lr=0.05, weight_decay=0.0)
    gbatches = [trd[torch.from_numpy(rng.permutation(tr.size)[:B]).cuda()].to(torch.int32).contiguous()
                for _ in range(200)]
    gka.train_step(ix, wind, gbatches[0], idx, gopt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for rb in gbatches[1:]:
        gka.train_step(ix, wind, rb, idx, gopt)
    e1.record()
    torch.cuda.synchronize()
    ms_gka_train = e0.elapsed_time(e1) / (len(gbatches) - 1)
    idx_te = idx[ted].contiguous()
    gka.forward(ix, wind, idx_te, q=qte)
    torch.cuda.synchronize()
    with _Range("gka_forward"):
        ms_gka = _timed(lambda: gka.forward(ix, wind, idx_te, q=qte), steps)
    gpred = gka.forward(ix, wind, idx_te, q=qte)
    rmse_gka = float(torch.sqrt(((gpred - wind[ted]) ** 2).mean()))
    gsig, gstep = gka.get_params()
    gka_bytes = qte.shape[0] * (28 * k + 24)
    # GKA-MLP-TNN: scales from an MLP of the location, started from the GKA
    # scales and trained end to end
    gm = tnn.GKAMLP(gsig, hidden=32, seed=0)
    mopt = tnn.AdamW(lr=0.01, weight_decay=0.0)
    mbatches = [trd[torch.from_numpy(rng.permutation(tr.size)[:B]).cuda()].to(torch.int32).contiguous()
                for _ in range(600)]
    gm.train_step(ix, wind, mbatches[0], idx, mopt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for rb in mbatches[1:]:
        gm.train_step(ix, wind, rb, idx, mopt)
    e1.record()
    torch.cuda.synchronize()
    ms_gm_train = e0.elapsed_time(e1) / (len(mbatches) - 1)
    gm.forward(ix, wind, idx_te, q=qte)
    torch.cuda.synchronize()
    with _Range("gkamlp_forward"):
        ms_gm = _timed(lambda: gm.forward(ix, wind, idx_te, q=qte), steps)
    gmpred = gm.forward(ix, wind, idx_te, q=qte)
    rmse_gm = float(torch.sqrt(((gmpred - wind[ted]) ** 2).mean()))
    # the float64 oracle of each stage on a bounded sample (host cores)
    from oracle import nowcast as ncr
    ns = 20000
    smp = te[:ns]
    idx_s = idx[torch.from_numpy(smp).cuda()].cpu().numpy()
    d2_s = d2[torch.from_numpy(smp).cuda()].cpu().numpy()
    c0 = time.perf_counter()
    ncr.features(wl.xyzt, wl.wind, wl.xyzt[smp], idx_s, sigma, mean=mean, std=std)
    ncr.idw(d2_s, idx_s, wl.wind)
    c_feat = time.perf_counter() - c0
    W1, b1m, W2, b2m = mlp.unflatten(mlp.get_params())
    xs = xte[:ns].float().cpu().numpy().astype(np.float64)
    c0 = time.perf_counter()
    ncr.mlp_forward(xs, W1, b1m, W2, b2m)
    c_mlp = time.perf_counter() - c0
    c0 = time.perf_counter()
    ncr.gka_forward(wl.xyzt, wl.wind, wl.xyzt[smp], idx_s, np.log(gsig.astype(np.float64)))
    c_gka = time.perf_counter() - c0
    # one training step of each learned form in the oracle (batch B)
    xb_, yb_ = batches[1]
    Xo = xb_.float().cpu().numpy().astype(np.float64)
    To = yb_.cpu().numpy().astype(np.float64)
    wflat = mlp.get_params().astype(np.float64)
    c0 = time.perf_counter()
    _, go = ncr.mlp_grads(Xo, To, W1, b1m, W2, b2m)
    gflat = np.concatenate([np.ravel(go[nm]) for nm in ("W1", "b1", "W2", "b2")])
    ncr.adamw_step(wflat, gflat, np.zeros_like(wflat), np.zeros_like(wflat), 1)
    c_train = time.perf_counter() - c0
    rows_o = gbatches[1].cpu().numpy()
    idx_all = idx.cpu().numpy()
    c0 = time.perf_counter()
    ncr.gka_loss_grad(wl.xyzt, wl.wind, rows_o, idx_all, np.log(gsig.astype(np.float64)))
    c_gka_train = time.perf_counter() - c0
    lo_b, hi_b = wl.xyzt.min(axis=0), wl.xyzt.max(axis=0)
    c0 = time.perf_counter()
    ncr.gkamlp_forward(wl.xyzt, wl.wind, wl.xyzt[smp], idx_s, gm.get_params()[0].astype(np.float64), 32, lo_b, hi_b)
    c_gm = time.perf_counter() - c0

    def _cpu(sec, unit):
        return {"value": ns / sec, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                "sample": f"{ns} held-out contexts, float64 numpy"}
    out["nowcast"] = {
        "workload": "learned-1M: 5,000 flights x 200 samples, k = 32, lag 1800 s, 80/20 split by flight",
        "contexts": {"value": wl.n / (ms_knn / 1e3), "unit": UNIT, "ms": ms_knn, "tuning": tune},
        "features_idw": {"value": wl.n / (ms_feat / 1e3), "unit": "contexts/s", "ms": ms_feat,
                         "cpu_baseline": _cpu(c_feat, "contexts/s"),
                         "roofline": {"bound": "hbm", "achieved": feat_bytes / (ms_feat / 1e3) / 1e9,
                                      "peak": hbm, "unit": "GB/s",
                                      "frac": feat_bytes / (ms_feat / 1e3) / 1e9 / hbm,
                                      "bytes_per_context": 44 * k + 24, "peak_note": "of measured hbm_gbs"}},
        "mlp_train": {"value": B / (ms_graph / 1e3), "unit": "samples/s", "ms_per_step": ms_graph,
                      "how": "CUDA graph of 16 tnn_mlp_train_step calls, replayed",
                      "host_loop_ms_per_step": ms_train, "batch": B, "steps": len(batches) - 1,
                      "epochs": epochs,
                      "cpu_baseline": {"value": B / c_train, "unit": "samples/s", "cores": os.cpu_count(),
                                       "kind": "oracle",
                                       "sample": f"one training step (batch {B}): float64 numpy gradients + AdamW"},
                      "roofline": {"bound": "tensor", "achieved": flops_step / (ms_graph / 1e3) / 1e12,
                                   "peak": bf16, "unit": "TFLOP/s",
                                   "frac": flops_step / (ms_graph / 1e3) / 1e12 / bf16,
                                   "flops_per_step": flops_step, "peak_note": "of measured bf16 burst"}},
        "mlp_forward": {"value": xte.shape[0] / (ms_fwd / 1e3), "unit": "samples/s", "ms": ms_fwd,
                        "rows": int(xte.shape[0]), "cpu_baseline": _cpu(c_mlp, "samples/s"),
                        "roofline": {"bound": "tensor",
                                     "achieved": 2.0 * xte.shape[0] * (k * 6 * 256 + 256 * 2) / (ms_fwd / 1e3) / 1e12,
                                     "peak": bf16, "unit": "TFLOP/s",
                                     "frac": 2.0 * xte.shape[0] * (k * 6 * 256 + 256 * 2) / (ms_fwd / 1e3) / 1e12 / bf16,
                                     "hbm_frac": xte.shape[0] * (k * 6 * 2 + 8) / (ms_fwd / 1e3) / 1e9 / hbm,
                                     "peak_note": "of measured bf16 burst; hbm_frac: X read + Y written over measured hbm_gbs"}},
        "nowcast_e2e": {"value": qte.shape[0] / (ms_now / 1e3), "unit": "nowcasts/s", "ms": ms_now,
                        "queries": int(qte.shape[0]), "includes": "tnn_nowcast: search + features + MLP"},
        "matched_latency": {
            "queries": int(qte.shape[0]), "includes": "tnn_nowcast on the held-out queries, same search",
            "mlp": {"ms": ms_now, "nowcasts_per_s": qte.shape[0] / (ms_now / 1e3), "rmse_ms": rmse_now_mlp},
            "idw": {"ms": ms_now_idw, "nowcasts_per_s": qte.shape[0] / (ms_now_idw / 1e3),
                    "rmse_ms": rmse_now_idw},
            "mlp_extra_ms": ms_now - ms_now_idw},
        "hour_average": {"value": qte.shape[0] / (ms_hour / 1e3), "unit": "nowcasts/s", "ms": ms_hour,
                         "window": "[t - 5400 s, t - 1800 s]", "queries_with_data": int(hok.sum())},
        "gka": {"forward": {"value": qte.shape[0] / (ms_gka / 1e3), "unit": "nowcasts/s", "ms": ms_gka,
                            "cpu_baseline": _cpu(c_gka, "nowcasts/s"),
                            "roofline": {"bound": "hbm", "achieved": gka_bytes / (ms_gka / 1e3) / 1e9,
                                         "peak": hbm, "unit": "GB/s",
                                         "frac": gka_bytes / (ms_gka / 1e3) / 1e9 / hbm,
                                         "bytes_per_context": 28 * k + 24, "peak_note": "of measured hbm_gbs"}},
                "train_step": {"value": B / (ms_gka_train / 1e3), "unit": "samples/s", "ms": ms_gka_train,
                               "batch": B, "steps": gstep,
                               "cpu_baseline": {"value": B / c_gka_train, "unit": "samples/s",
                                                "cores": os.cpu_count(), "kind": "oracle",
                                                "sample": f"one loss + gradient evaluation (batch {B}), float64 numpy"}},
                "sigma": [float(x) for x in gsig]},
        "gka_mlp": {"forward": {"value": qte.shape[0] / (ms_gm / 1e3), "unit": "nowcasts/s", "ms": ms_gm,
                                "cpu_baseline": _cpu(c_gm, "nowcasts/s"),
                                "roofline": {"bound": "hbm", "achieved": gka_bytes / (ms_gm / 1e3) / 1e9,
                                             "peak": hbm, "unit": "GB/s",
                                             "frac": gka_bytes / (ms_gm / 1e3) / 1e9 / hbm,
                                             "bytes_per_context": 28 * k + 24,
                                             "peak_note": "of measured hbm_gbs"}},
                    "train_step": {"value": B / (ms_gm_train / 1e3), "unit": "samples/s", "ms": ms_gm_train,
                                   "batch": B, "steps": len(mbatches), "hidden": 32}},
        "rmse_ms": {"mlp": rmse_mlp, "idw": rmse_idw, "gka": rmse_gka, "gka_mlp": rmse_gm,
                    "hour_average": rmse_hour, "day_average": rmse_day,
                    "hour_average_rows": int(hok.sum()),
                    "held_out_rows": int(te.size),
                    "note": "synthetic wind field; noise floor 1 m/s per component (parity unpinned)"}}
    ix.destroy()
    return out


def _tc_tiles(tnn, ix, k, tune, flush, steps, ref_idx, ref_ms):
    """TNN with the candidate distances formed as tcgen05 TF32 tiles and
    screened (TNN_FLAG_TC_TILES), timed beside the FP32 member scan on the
    same workload; identical neighbours required."""
    import torch
    ti = torch.empty_like(ref_idx)
    td = torch.empty(ref_idx.shape, dtype=torch.float32, device=ref_idx.device)
    # its own knobs: seed count and deferral radius, the fastest of a few
    # settings in which the tiles answer a fair share of the queries (with
    # one seed segment, or a smaller radius, nearly every query leaves its
    # tile and the warp kernel does the work)
    tried = {}
    for F in (3, 4):
        for dfr in (0.6, 1.0):
            kw_ = {"seed_segments": F, "extra": tune.get("extra", 4), "defer_cells": dfr}
            tnn.tnn_knn(ix, k, 0.0, out=(ti, td), tc=True, **kw_)
            torch.cuda.synchronize()
            tried[(F, dfr)] = _timed(lambda: tnn.tnn_knn(ix, k, 0.0, out=(ti, td), tc=True, **kw_), 2, flush)
    F, dfr = min(tried, key=tried.get)
    kw = {"seed_segments": F, "extra": tune.get("extra", 4), "defer_cells": dfr}
    tnn.tnn_knn(ix, k, 0.0, out=(ti, td), tc=True, **kw)
    torch.cuda.synchronize()
    tnn.tnn_profile_read(reset=True)
    tnn.tnn_profile_enable(True)
    with _Range("tnn_tc_tiles"):
        ms = _timed(lambda: tnn.tnn_knn(ix, k, 0.0, out=(ti, td), tc=True, **kw), steps, flush)
    tnn.tnn_profile_enable(False)
    kern, launches = tnn.tnn_profile_read_kernels(reset=True)
    _, _, st = tnn.tnn_knn(ix, k, 0.0, out=(ti, td), tc=True, stats=True, **kw)
    tiles = st["segs_scanned"] - 0  # 128 x 128 tiles multiplied (+ seed segments, see note)
    return {"kernel": "k_tnn_tc", "ms_per_step": ms, "value": ti.shape[0] / (ms / 1e3), "unit": UNIT,
            "kernel_ms": {"k_tnn_tc": kern[0] / max(launches, 1), "k_tnn_warp": kern[1] / max(launches, 1),
                          "k_fallback_exact": kern[2] / max(launches, 1)},
            "vs_fp32_member_scan": ref_ms / ms, "identical_neighbours": bool(torch.equal(ti, ref_idx)),
            "queries_finished_by_tiles": ti.shape[0] - st["warp_queries"],
            "rescored": st["lb_evals"], "pairs_screened": st["pairs"], "tiles_and_seed_segments": tiles,
            "warp_queries": st["warp_queries"], "tuning": kw,
            "ms_by_knobs": {f"F={a},defer={b}": v for (a, b), v in tried.items()}}


def _precision(tnn, synth, flush, steps, alu_peak, derived_peak, cpu=True):
    """The precision workload: 20,000 flights x 200 samples = 4,000,000
    points, k = 32, every point a query; FP32 screening with certified
    margins and an FP64 recheck of the candidates inside the margin of the
    k-th distance.  Reports its rate, the per-kernel roofline, the margin
    fraction and the error against the FP64 oracle on 4,096 sampled queries,
    and the tensor-core linear search on a query sample."""
    import torch
    sigma = (1.0, 1.0, 10.0, 0.01)
    wl = synth.precision()
    k, K = 32, 20
    ix = tnn.tnn_build_segments(torch.from_numpy(wl.xyzt).cuda(), wl.traj_off, sigma, K)
    tune = tnn.tnn_autotune(ix, k, 0.0)
    idx = torch.empty((wl.n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((wl.n, k), dtype=torch.float32, device="cuda")

    def step():
        tnn.tnn_knn(ix, k, 0.0, out=(idx, d2), **tune)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    tnn.tnn_profile_read(reset=True)
    tnn.tnn_profile_enable(True)
    with _Range("precision_search"):
        ms = _timed(step, steps, flush)
    tnn.tnn_profile_enable(False)
    kern, launches = tnn.tnn_profile_read_kernels(reset=True)
    _, _, st = tnn.tnn_knn(ix, k, 0.0, stats=True, out=(idx, d2), **tune)
    roof = _search_roofline(tnn, ix, k, 0.0, tune, kern, launches, alu_peak, derived_peak, None, (idx, d2))
    # tensor-core linear search on 131,072 queries spread over the workload
    import numpy as np
    qs = np.linspace(0, wl.n - 1, 131072).astype(np.int64)
    qd = torch.from_numpy(wl.xyzt[qs].copy()).cuda()
    bi = torch.empty((qd.shape[0], k), dtype=torch.int32, device="cuda")
    bd = torch.empty_like(bi, dtype=torch.float32)
    tnn.tnn_knn_bruteforce(ix, k, 0.0, q=qd, out=(bi, bd))
    torch.cuda.synchronize()
    cms = _timed(lambda: tnn.tnn_knn_bruteforce(ix, k, 0.0, q=qd, out=(bi, bd)), 2, flush)
    same = bool(torch.equal(bi, idx[torch.from_numpy(qs).cuda()]))
    tcx = _tc_tiles(tnn, ix, k, tune, flush, steps, idx, ms)
    out = {"workload": "precision-4M: 20,000 synthetic flights x 200 samples = 4,000,000 points, "
                       "self-query of every point, k = 32, 20-point segments",
           "metric": "causal k-NN contexts/s (exact, k=32)", "value": wl.n / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms, "steps": steps, "tuning": tune,
           "distance_form": "FP32 direct differences with certified bounds, FP64 settlement of "
                            "candidates within the margin of the k-th distance",
           "margin": {"fp64_rechecks": st["fp64_rechecks"], "queries": st["queries"],
                      "rechecks_per_query": st["fp64_rechecks"] / max(st["queries"], 1),
                      "fraction_of_candidates": st["fp64_rechecks"] / max(st["pairs"], 1),
                      "pairs": st["pairs"], "exact_queries": st["exact_queries"]},
           "roofline": roof,
           "comparator_tensor_core": {"queries": int(qd.shape[0]), "ms": cms,
                                      "contexts_per_s": qd.shape[0] / (cms / 1e3),
                                      "tnn_speedup": (wl.n / (ms / 1e3)) / (qd.shape[0] / (cms / 1e3)),
                                      "identical_neighbours": same},
           "stats_per_step": st, "tc_tiles": tcx}
    if cpu:
        out["cpu_baseline"] = _cpu_baseline(wl, k, 4096, idx, d2)
        out["max_rel_d2_err_vs_fp64"] = out["cpu_baseline"]["parity"]["max_rel_d2_err_vs_fp64"]
    ix.destroy()
    del idx, d2, bi, bd
    torch.cuda.empty_cache()
    return out


def _e2e_breakdown(tnn, wl, k, K, sigma, tune, h_x, h_i, h_d, reps=5):
    """Where the end-to-end time goes: the stages tnn_knn_host runs, timed
    one after another (no overlap), then tnn_knn_host with 1-4 slices."""
    import torch
    m = wl.n
    d_x = torch.empty((m, 4), dtype=torch.float32, device="cuda")
    idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    stages = {"h2d": [], "build": [], "search": [], "d2h": []}
    for rep in range(reps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        torch.cuda.synchronize()
        ev[0].record()
        d_x.copy_(h_x, non_blocking=True)
        ev[1].record()
        with _Range("index_build"):
            ix = tnn.tnn_build_segments(d_x, wl.traj_off, sigma, K)
        ev[2].record()
        tnn.tnn_knn(ix, k, 0.0, out=(idx, d2), **tune)
        ev[3].record()
        h_i.copy_(idx, non_blocking=True)
        h_d.copy_(d2, non_blocking=True)
        ev[4].record()
        torch.cuda.synchronize()
        ix.destroy()
        if rep:
            for i, name in enumerate(stages):
                stages[name].append(ev[i].elapsed_time(ev[i + 1]))
    def host_ms(**kw):
        ts = []
        for rep in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            tnn.tnn_knn_host(h_x, wl.traj_off, sigma, K, k, 0.0, out=(h_i, h_d), **kw, **tune)
            e1.record()
            torch.cuda.synchronize()
            if rep:
                ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    copied = {str(nc): host_ms(chunks=nc, mapped=False) for nc in (1, 2, 3, 4)}
    st = {name: sum(v) / len(v) for name, v in stages.items()}
    return {"stages_ms": st, "stages_sum_ms": sum(st.values()), "d2h_GB_per_s": m * k * 8 / st["d2h"] / 1e6,
            "tnn_knn_host_ms": {"mapped": host_ms(mapped=True), "copied_by_slices": copied},
            "note": "stages one after another, no overlap. tnn_knn_host, mapped (page-locked outputs, "
                    "TNN_FLAG_MAPPED_OUT, the default for them): the tile kernel writes each finished "
                    "tile's rows into host memory, the handed-over rows follow at the end; copied (flag "
                    "off): slices of complete searches, a slice's copy-out overlapped with the next "
                    "slice's search"}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2112_10408_gb300 import build as tb
    if rank == 0:
        tb.build()
    if world > 1:
        dist.barrier()
    from paper_2112_10408_gb300 import tnn
    tnn.load_library()

    wl, k, K = _workload(a.workload, rank)
    sigma = (1.0, 1.0, 10.0, 0.01)
    xyzt_d = torch.from_numpy(wl.xyzt).cuda()
    ix = tnn.tnn_build_segments(xyzt_d, wl.traj_off, sigma, K)
    tune = tnn.tnn_autotune(ix, k, 0.0, m_sample=8192) if a.tuning == "auto" else {}
    m = wl.n
    idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        tnn.tnn_knn(ix, k, 0.0, out=(idx, d2), **tune)

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        try:
            p = torch.cuda.get_device_properties(local)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        except Exception:
            bus = None
    sampler = ClockSampler(bus)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    tnn.tnn_profile_read(reset=True)
    tnn.tnn_profile_enable(True)
    with _Range("tnn_search"):
        for s in range(a.steps):
            flush.zero_()
            ev[s][0].record()
            step()
            ev[s][1].record()
        torch.cuda.synchronize()
    tnn.tnn_profile_enable(False)
    kern3, launches = tnn.tnn_profile_read_kernels(reset=True)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = _max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev), world)
    ms_step = total_ms / max(a.steps, 1)
    value = _throughput(world, m, a.steps, total_ms)

    # executed and necessary work of one pass (outside the timed region),
    # attributed to the kernel that finished each query
    _, _, st = tnn.tnn_knn(ix, k, 0.0, stats=True, out=(idx, d2), **tune)
    peaks = _peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak, derived_peak = _fp32_peak(tnn, peaks, nsm)
    roofline = _search_roofline(tnn, ix, k, 0.0, tune, kern3, launches, alu_peak, derived_peak,
                                None, (idx, d2))
    roofline["traffic"] = _search_traffic(a.workload, roofline["kernel"])
    roofline["traffic_note"] = ("ncu dram bytes of the dominant kernel at tuning %s (null: kernel "
                                "changed since the capture)" % SEARCH_TRAFFIC["tuning"])
    roofline["executed"] = {"lb": st["lb_evals"], "pairs": st["pairs"]}

    # comparator: linear search on the same queries, distance tiles on the
    # tensor cores (default) and on the CUDA cores (ffma)
    comparator = None
    if a.comparator_steps > 0:
        bi = torch.empty_like(idx)
        bd = torch.empty_like(d2)
        comparator = {}
        for name, ffma in (("tensor_core", False), ("cuda_core", True)):
            tnn.tnn_knn_bruteforce(ix, k, 0.0, out=(bi, bd), ffma=ffma)
            torch.cuda.synchronize()
            _, _, cst = tnn.tnn_knn_bruteforce(ix, k, 0.0, out=(bi, bd), ffma=ffma, stats=True)
            cms = []
            rng_ = _Range("linear_cuda_core" if ffma else "linear_tensor_core")
            rng_.__enter__()
            for _ in range(a.comparator_steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                tnn.tnn_knn_bruteforce(ix, k, 0.0, out=(bi, bd), ffma=ffma)
                e1.record()
                torch.cuda.synchronize()
                cms.append(e0.elapsed_time(e1))
            rng_.__exit__(None, None, None)
            cmean = sum(cms) / len(cms)
            ent = {"kernel": "k_linear_search" if ffma else "k_linear_tc",
                   "value": m / (cmean / 1e3), "unit": UNIT, "ms_per_step": cmean,
                   "tnn_speedup": cmean / ms_step, "identical_neighbours": bool(torch.equal(bi, idx)),
                   "pairs": cst["pairs"], "rescored": cst["lb_evals"]}
            if not ffma:
                # one TF32 MMA (M = N = 128, K = 8) per 128 x 128 tile
                tiles = cst["segs_scanned"]
                tf = 2.0 * 128 * 128 * 8 * tiles / (cmean / 1e3) / 1e12
                tf32_peak = peaks.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
                ent["tensor"] = {"tiles": tiles, "achieved_tflops": tf, "tf32_peak_tflops": tf32_peak,
                                 "frac": tf / tf32_peak,
                                 "peak_note": "of measured: bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}
            if ffma:
                # direct FP32 differences: every causal pair costs a distance,
                # a mask and a compare
                ach = OPS_PER_PAIR * cst["pairs"] / (cmean / 1e3) / 1e12
                ent["alu"] = {"achieved": ach, "peak": alu_peak, "unit": "T FP32 lane-ops/s",
                              "frac": ach / alu_peak, "ops_per_pair": OPS_PER_PAIR,
                              "peak_note": "of measured FFMA issue rate"}
            comparator[name] = ent

    # the same search with the candidate distances as tensor-core tiles
    tc_tiles = _tc_tiles(tnn, ix, k, tune, flush, max(3, min(a.steps, 20)), idx, ms_step)

    # end to end through the C ABI on host buffers (tnn_knn_host): pinned
    # host points -> H2D -> index build -> search -> D2H of both result
    # arrays into pinned host memory, the copies overlapped with the search
    h_x = torch.from_numpy(wl.xyzt).pin_memory()
    h_i = torch.empty((m, k), dtype=torch.int32).pin_memory()
    h_d = torch.empty((m, k), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for s in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        with _Range("e2e"):
            tnn.tnn_knn_host(h_x, wl.traj_off, sigma, K, k, 0.0, out=(h_i, h_d), **tune)
        e1.record()
        torch.cuda.synchronize()
        if s > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_avg = sum(e2e_ms) / len(e2e_ms) if e2e_ms else float("nan")
    e2e = {"value": world * m / (e2e_avg / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(h_x.numel() * 4), "d2h_bytes_per_step": int(m * k * 8),
           "ms_per_step": e2e_avg,
           "includes": "tnn_knn_host: H2D points, index build, search, D2H results (pinned host buffers, "
                       "TNN_FLAG_MAPPED_OUT: the handed-over rows written into them by a kernel)"}

    e2e_break = None
    if rank == 0 and world == 1 and a.e2e_steps > 0:
        e2e_break = _e2e_breakdown(tnn, wl, k, K, sigma, tune, h_x, h_i, h_d)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = _cpu_baseline(wl, k, 8192 if a.workload != "tiny" else wl.n, idx, d2)

    extras = None
    if rank == 0 and world == 1 and not a.no_extras:
        from paper_2112_10408_gb300 import synth
        nsteps = max(3, min(a.steps, 20))
        extras = _extras(tnn, synth, flush, _peaks(), nsteps)
        if a.workload != "precision":
            extras["precision"] = _precision(tnn, synth, flush, nsteps, alu_peak, derived_peak,
                                             cpu=not a.no_cpu_baseline)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": dict(_config(wl, k, K, a.workload), tuning=tune,
                              parallelism=f"replicas x{world}: each rank its own window"),
               "clocks": clocks, "e2e": e2e, "gpu_launches": 3 * a.steps,
               "roofline": roofline, "cpu_baseline": cpu, "comparator": comparator,
               "stats_per_step": st, "e2e_breakdown": e2e_break, "tc_tiles": tc_tiles}
        if extras:
            out.update(extras)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
