"""Segment length K x seed count F sweep of the TNN search (the ablation of
Sec. 4.2 / Fig. 3: speed-up over the linear search and the share of point
comparisons TNN makes, as functions of K and F).

    python -m paper_2112_10408_gb300.sweep_kf [--flights 2000] [--samples 200]

Prints one JSON object: for every (K, F) the search time, the speed-up over
the tensor-core linear search and the comparisons (point distances) as a
fraction of the linear search's.  Runs on the current CUDA device.
"""
from __future__ import annotations

import argparse
import json

import torch

from paper_2112_10408_gb300 import build, synth, tnn


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--flights", type=int, default=2000)
    ap.add_argument("--samples", type=int, default=200)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--seg-lens", default="5,10,20,40,64")
    ap.add_argument("--seeds", default="1,2,4,6")
    a = ap.parse_args()
    build.build()
    tnn.load_library()
    wl = synth.flights(a.flights, a.samples, synth.SEED_MEDIUM)
    xyzt = torch.from_numpy(wl.xyzt).cuda()
    sig = synth.SIGMA_DEFAULT
    rows = []
    lin = None
    for K in (int(x) for x in a.seg_lens.split(",")):
        ix = tnn.tnn_build_segments(xyzt, wl.traj_off, sig, K)
        idx = torch.empty((wl.n, a.k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((wl.n, a.k), dtype=torch.float32, device="cuda")
        if lin is None:
            ms_lin = _time(lambda: tnn.tnn_knn_bruteforce(ix, a.k, 0.0, out=(idx, d2)), 1)
            _, _, st_lin = tnn.tnn_knn_bruteforce(ix, a.k, 0.0, out=(idx, d2), stats=True)
            lin = {"ms": ms_lin, "pairs": st_lin["pairs"]}
        for F in (int(x) for x in a.seeds.split(",")):
            kw = dict(seed_segments=F)
            ms = _time(lambda: tnn.tnn_knn(ix, a.k, 0.0, out=(idx, d2), **kw), a.reps)
            _, _, st = tnn.tnn_knn(ix, a.k, 0.0, out=(idx, d2), stats=True, **kw)
            rows.append({"K": K, "F": F, "ms": ms, "speedup": lin["ms"] / ms,
                         "comparisons_pct": 100.0 * st["pairs"] / lin["pairs"],
                         "pairs_per_query": st["pairs"] / wl.n, "bounds_per_query": st["lb_evals"] / wl.n})
        ix.destroy()
    print(json.dumps({"workload": f"{a.flights} flights x {a.samples} samples = {wl.n} points, k = {a.k}",
                      "linear_search": lin, "sweep": rows}))


if __name__ == "__main__":
    main()
