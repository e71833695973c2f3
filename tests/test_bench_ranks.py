"""The multi-rank path of bench.py (replicas, one process per GPU) on CPU:
two gloo ranks check the max-over-ranks timing, the whole-job rate and that
every rank gets its own problem."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1502_05037_gb300 import synth
        local_ms = [120.0, 150.0][rank]
        total = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
        wl = bench.replica_workload(synth.WORKLOADS["sara64_fp64"], rank)
        x, u, v, offs, nz = wl.draw()
        out[rank] = (total, bench.job_rate(world, 20, total), wl.index, float(u[:16].sum()), float(x.sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    # both ranks see the slowest rank's time, and the job rate counts every rank
    assert r0[0] == r1[0] == 150.0
    assert r0[1] == r1[1] == pytest.approx(2 * 20 / 0.150)
    # independent problems: distinct seeds and coverages
    assert r0[2] != r1[2]
    assert r0[3] != r1[3]


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.job_rate(1, 10, 500.0) == pytest.approx(20.0)
