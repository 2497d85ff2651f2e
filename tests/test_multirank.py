"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank
answers its own synthetic window, the only collective is the MAX over the
ranks' times, and the job's throughput counts every rank's queries."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl, k, K = bench._workload("tiny", rank)
        fp = torch.tensor([float(np.abs(wl.xyzt).sum())], dtype=torch.float64)
        fps = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(fps, fp)
        t = bench._max_over_ranks(10.0 + 5.0 * rank, world, device="cpu")
        value = bench._throughput(world, wl.n, 3, t)
        out[rank] = (wl.n, k, K, [float(x) for x in fps], t, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_answer_their_own_windows_and_time_the_slowest():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0[:3] == r1[:3] == (10000, 8, 10)          # same shape of window
    assert r0[3] == r1[3] and r0[3][0] != r0[3][1]     # different data per rank
    assert r0[4] == r1[4] == 15.0                       # MAX over ranks
    assert r0[5] == pytest.approx(2 * 10000 * 3 / 0.015)
