"""The block-sharded form of the SDMM iteration (the visibility blocks of
Eq. 2 split over ranks, the image and the wavelet state replicated), emulated
on CPU with two gloo ranks and the FP64 oracle: each rank degrids and projects
only its own blocks, and every application of Re Phi^H is the sum over ranks
of the adjoints of the local blocks (one all-reduce of an N-pixel image).
Two iterations of it equal two iterations of the unsharded oracle."""
import os
import socket
import sys

import numpy as np
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


def _problem():
    from oracle import nufft as nf
    from oracle import sdmm
    from paper_1502_05037_gb300 import synth
    n, M, R = 16, 600, 4
    x = synth.sky(n, n, 7, n_points=5, n_blobs=1)
    u, v = synth.uv_coverage(M, 8, sigma=1.0)
    p = nf.NufftPlan(n, n, u, v, 4)
    y0 = nf.phi(p, x)
    s = sdmm.noise_sigma(y0, 30.0)
    offs = synth.block_offsets(synth.block_sizes(M, R, 9))
    y = y0 + s * synth.unit_noise(M, 10)
    eps = sdmm.epsilon_chi2(s, np.diff(offs))
    return sdmm.Problem(p, 2, y, offs, eps, mask=0b111)


def _sharded_iterations(prob, rank, world, iters, cg_iters):
    from oracle import sdmm
    own = np.zeros(prob.plan.M, dtype=bool)
    for i in range(rank, prob.R, world):            # blocks rank, rank + world, ...
        own[prob.offsets[i]:prob.offsets[i + 1]] = True

    def phi_n_own(x):                                # local degridding: own blocks only
        return np.where(own, prob.phi_n(x), 0.0)

    def adj_re(s):                                   # sum over ranks of the local adjoints
        t = torch.from_numpy(prob.phi_n_adj_re(np.where(own, s, 0.0)))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    def apply_A(x):
        return 2.0 * x + adj_re(phi_n_own(x))

    x = np.zeros((prob.plan.ny, prob.plan.nx))
    z1 = np.zeros_like(prob.psi_adj(x))
    z2 = np.zeros(prob.plan.M, dtype=complex)
    z3 = np.zeros_like(x)
    yn = prob.y / prob.nu
    for _ in range(iters):
        v1 = prob.psi_adj(x)
        s1 = sdmm.soft_threshold(v1 + z1, prob.gamma * prob.w())
        z1 = z1 + v1 - s1
        v2 = phi_n_own(x)
        t2 = v2 + z2
        s2 = np.zeros_like(t2)
        for i in range(rank, prob.R, world):
            a, b = prob.offsets[i], prob.offsets[i + 1]
            s2[a:b] = sdmm.proj_l2_ball(t2[a:b], yn[a:b], prob.eps[i] / prob.nu)
        z2 = z2 + v2 - s2
        s3 = sdmm.proj_positive(x + z3)
        z3 = z3 + x - s3
        b = prob.psi(s1 - z1) + adj_re(s2 - z2) + (s3 - z3)
        x, _, _ = sdmm.cg(apply_A, b, x, cg_iters)
    return x, z2, own


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem()
        x, z2, own = _sharded_iterations(prob, rank, world, iters=2, cg_iters=6)
        out[rank] = (x, z2[own], np.flatnonzero(own))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_block_sharded_iterations_equal_the_unsharded_ones():
    from oracle import sdmm
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    prob = _problem()
    ref = sdmm.sdmm_solve(prob, np.zeros((prob.plan.ny, prob.plan.nx)), 2, 6)
    scale = np.linalg.norm(ref.x)
    for r in range(world):
        x, z2_own, idx = out[r]
        # the replicated image is the same on every rank and equals the oracle's
        assert np.linalg.norm(x - ref.x) <= 1e-10 * scale
        # each rank's multipliers are the oracle's on its own blocks
        assert np.allclose(z2_own, ref.z2[idx], rtol=0, atol=1e-12 * np.abs(ref.z2).max())
    # the two ranks' blocks partition the visibilities
    assert sorted(np.concatenate([out[0][2], out[1][2]]).tolist()) == list(range(prob.plan.M))


# ------------------------------------------- the library's shard driver
def _driver_rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1502_05037_gb300 import sharded
        from shard_oracle import OracleShard
        prob = _problem()
        shard = OracleShard(prob, sharded.shard_blocks(prob.R, world, rank))
        drv = sharded.ShardedSdmm([shard], sharded.all_reduce_images, cg_iters=6)
        drv.iterate(2)
        out[rank] = (shard.x, shard.z2[shard.own], np.flatnonzero(shard.own), drv.exchanges)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_shard_driver_on_two_gloo_ranks_equals_the_unsharded_solve():
    # the host orchestration of purify_shard_* (the exchange points, their
    # order and the round-robin block assignment), each rank's steps computed
    # by the oracle, against the unsharded oracle SDMM
    from oracle import sdmm
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    mp.spawn(_driver_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    prob = _problem()
    ref = sdmm.sdmm_solve(prob, np.zeros((prob.plan.ny, prob.plan.nx)), 2, 6)
    scale = np.linalg.norm(ref.x)
    for r in range(world):
        x, z2_own, idx, nex = out[r]
        assert np.linalg.norm(x - ref.x) <= 1e-9 * scale
        assert np.allclose(z2_own, ref.z2[idx], rtol=0, atol=1e-11 * np.abs(ref.z2).max())
        assert nex == 2 * (1 + 6)     # one adjoint and one normal-operator exchange per CG step
    assert sorted(np.concatenate([out[0][2], out[1][2]]).tolist()) == list(range(prob.plan.M))


def test_shard_driver_in_one_process_equals_the_unsharded_solve():
    # three shards driven by one process (sum_in_place as the all-reduce)
    from oracle import sdmm
    from paper_1502_05037_gb300 import sharded
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from shard_oracle import OracleShard
    prob = _problem()
    shards = [OracleShard(prob, sharded.shard_blocks(prob.R, 3, k)) for k in range(3)]
    sharded.ShardedSdmm(shards, sharded.sum_in_place, cg_iters=6).iterate(2)
    ref = sdmm.sdmm_solve(prob, np.zeros((prob.plan.ny, prob.plan.nx)), 2, 6)
    for sh in shards:
        assert np.linalg.norm(sh.x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    idx, offs = sharded.shard_visibilities(prob.offsets, [1, 3])
    assert offs[-1] == idx.size and np.array_equal(idx[:3], np.arange(prob.offsets[1], prob.offsets[1] + 3))
