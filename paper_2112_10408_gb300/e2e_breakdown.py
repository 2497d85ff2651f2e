"""Where the end-to-end time of one host-to-host search goes (medium
workload: 2,000 flights x 200 samples, k = 32, 20-point segments).

    python -m paper_2112_10408_gb300.e2e_breakdown [--reps 5]

Times, with CUDA events on the current stream, the stages the
host-buffer pipeline (tnn_knn_host) runs: the copy of the points in, the
index build, the search and the copy of the neighbour lists out, each on its
own (no overlap); then tnn_knn_host itself for 1-4 slices; and the copy
rate of a 102 MB device-to-host transfer.  Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json

import torch

from paper_2112_10408_gb300 import build, synth, tnn


def _ev():
    return torch.cuda.Event(enable_timing=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    build.build()
    tnn.load_library()
    wl = synth.medium()
    m, k, K = wl.n, 32, 20
    sigma = synth.SIGMA_DEFAULT
    x = torch.from_numpy(wl.xyzt).cuda()
    ix = tnn.tnn_build_segments(x, wl.traj_off, sigma, K)
    tune = tnn.tnn_autotune(ix, k, 0.0)
    tune = {key: tune[key] for key in ("seed_segments", "extra", "defer_cells")}
    ix.destroy()
    h_x = torch.from_numpy(wl.xyzt).pin_memory()
    h_i = torch.empty((m, k), dtype=torch.int32).pin_memory()
    h_d = torch.empty((m, k), dtype=torch.float32).pin_memory()
    d_x = torch.empty_like(x)
    idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    stages = {"h2d": [], "build": [], "search": [], "d2h": []}
    for rep in range(a.reps + 1):
        ev = [_ev() for _ in range(5)]
        torch.cuda.synchronize()
        ev[0].record()
        d_x.copy_(h_x, non_blocking=True)
        ev[1].record()
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
    out = {"workload": f"medium: {m} points, k = {k}", "tuning": tune,
           "stages_ms": {name: sum(v) / len(v) for name, v in stages.items()}}
    slices = {}
    for nc in (1, 2, 3, 4):
        ts = []
        for rep in range(a.reps + 1):
            e0, e1 = _ev(), _ev()
            torch.cuda.synchronize()
            e0.record()
            tnn.tnn_knn_host(h_x, wl.traj_off, sigma, K, k, 0.0, chunks=nc, out=(h_i, h_d), **tune)
            e1.record()
            torch.cuda.synchronize()
            if rep:
                ts.append(e0.elapsed_time(e1))
        slices[str(nc)] = sum(ts) / len(ts)
    out["tnn_knn_host_ms_by_slices"] = slices
    src = torch.empty(m * k * 2, dtype=torch.float32, device="cuda")
    dst = torch.empty(m * k * 2, dtype=torch.float32).pin_memory()
    dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = _ev(), _ev()
    e0.record()
    for _ in range(a.reps):
        dst.copy_(src, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    out["d2h_copy"] = {"bytes": m * k * 8, "ms": ms, "GB_per_s": m * k * 8 / ms / 1e6}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
