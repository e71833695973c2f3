"""Block-sharded SDMM (Sec. 1: the data split into R blocks, Eqs. 2-3, and
SDMM's parallel structure): host-side orchestration of the C ABI's shard
steps (purify_shard_* in include/purify.h).

Each shard holds a plan over its own blocks; x, the wavelet state and the
positivity state are replicated and updated identically by every shard. Per
iteration the shards exchange two kinds of N-pixel image, both summed over
all shards by `allreduce`:
    r  = Re Phi_k^H (s2_k - z2_k - Phi_k x / nu) / nu   (once per iteration)
    u  = Re Phi_k^H Phi_k r / nu^2                      (once per CG step)
so the x-update sees the full data term sum_k Phi_k^H Phi_k while every
gridding and degridding touches only local visibilities. The block
assignment is round-robin (block i to shard i mod S).

`allreduce(images)` receives the images of the shards this process drives
and must leave each holding the sum over every shard of every process:
sum_in_place for shards driven by one process, all_reduce_images for one
shard per process over torch.distributed (NCCL on GPUs). The arithmetic of
every step runs in the library.
"""
from __future__ import annotations

import numpy as np


def shard_blocks(R: int, shards: int, k: int) -> list:
    """Blocks of shard k when R blocks are dealt round-robin to `shards`."""
    if not (1 <= shards and 0 <= k < shards):
        raise ValueError("need 0 <= k < shards")
    return list(range(k, R, shards))


def shard_visibilities(offsets, blocks) -> tuple:
    """Caller-order indices of the given blocks' visibilities (block by block)
    and the block offsets of that subset."""
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.concatenate([np.arange(offsets[i], offsets[i + 1]) for i in blocks]).astype(np.int64)
    sizes = [int(offsets[i + 1] - offsets[i]) for i in blocks]
    return idx, np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def sum_in_place(images) -> None:
    """All-reduce over shards driven by one process: the sum in list order,
    copied into every image."""
    total = images[0].clone()
    for t in images[1:]:
        total += t
    for t in images:
        t.copy_(total)


def all_reduce_images(images) -> None:
    """All-reduce over processes (one or more shards each) with
    torch.distributed: the local sum first, then one all-reduce."""
    import torch.distributed as dist
    sum_in_place(images)
    dist.all_reduce(images[0], op=dist.ReduceOp.SUM)
    for t in images[1:]:
        t.copy_(images[0])


class LibraryShard:
    """One shard on a library plan (its solve already started with
    purify_sdmm_solve(max_iter=0) on the shard's data)."""

    def __init__(self, plan, device, dtype):
        import torch
        self.plan = plan
        self.r = torch.empty((plan.info.N,), dtype=dtype, device=device)
        self.u = torch.empty_like(self.r)

    def iterate_local(self, r_out):
        from . import _lib
        _lib.check(_lib.load().purify_shard_iterate_local(self.plan.handle, r_out.data_ptr()))

    def cg_begin(self, r_sum):
        from . import _lib
        _lib.check(_lib.load().purify_shard_cg_begin(self.plan.handle, r_sum.data_ptr()))

    def cg_apply(self, k, u_out):
        from . import _lib
        _lib.check(_lib.load().purify_shard_cg_apply(self.plan.handle, int(k), u_out.data_ptr()))

    def cg_combine(self, k, u_sum):
        from . import _lib
        _lib.check(_lib.load().purify_shard_cg_combine(self.plan.handle, int(k), u_sum.data_ptr()))

    def iterate_end(self, cg_steps):
        from . import _lib
        _lib.check(_lib.load().purify_shard_iterate_end(self.plan.handle, int(cg_steps)))


class ShardedSdmm:
    """SDMM iterations over shards. `shards` are the shard objects this
    process drives (each with buffers r, u and the five step methods);
    `allreduce` sums a list of their images over all shards everywhere."""

    def __init__(self, shards, allreduce, cg_iters: int):
        if cg_iters < 1:
            raise ValueError("cg_iters must be >= 1")
        self.shards = list(shards)
        self.allreduce = allreduce
        self.cg_iters = int(cg_iters)
        self.exchanges = 0

    def iterate(self, n: int = 1) -> None:
        for _ in range(n):
            for sh in self.shards:
                sh.iterate_local(sh.r)
            self.allreduce([sh.r for sh in self.shards])
            self.exchanges += 1
            for sh in self.shards:
                sh.cg_begin(sh.r)
            for k in range(self.cg_iters):
                for sh in self.shards:
                    sh.cg_apply(k, sh.u)
                self.allreduce([sh.u for sh in self.shards])
                self.exchanges += 1
                for sh in self.shards:
                    sh.cg_combine(k, sh.u)
            for sh in self.shards:
                sh.iterate_end(self.cg_iters)
