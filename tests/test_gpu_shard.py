"""GPU parity of the block-sharded SDMM data path (Sec. 1: the block split of
Eqs. 2-3 and SDMM's parallel structure): shards holding a plan over their own
blocks, driven through purify_shard_* by sharded.ShardedSdmm, the N-pixel
exchanges summed in one process (the all-reduce of a multi-GPU run reduces
the same images). Against the FP64 oracle and against the unsharded solve."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, rel
from oracle import nufft as onf
from oracle import sdmm as osd
from paper_1502_05037_gb300 import sharded, synth

pytestmark = pytest.mark.gpu


def data(nx, M, J, R, seed):
    x_true = synth.sky(nx, nx, 1000 + seed, n_points=8, n_blobs=2)
    u, v = synth.uv_coverage(M, 2000 + seed, dtype=np.float32)
    offs = synth.block_offsets(synth.block_sizes(M, R, 4000 + seed))
    op = onf.NufftPlan(nx, nx, u.astype(np.float64), v.astype(np.float64), J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, 30.0)
    y = (y0 + sig * synth.unit_noise(M, 3000 + seed)).astype(np.complex64)
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    return x_true, u, v, offs, y, eps, op


def make_shards(nx, J, levels, u, v, offs, y, eps, S, cg, gamma, nu):
    st = torch.cuda.current_stream(DEV)
    shards = []
    for k in range(S):
        blocks = sharded.shard_blocks(len(offs) - 1, S, k)
        idx, loffs = sharded.shard_visibilities(offs, blocks)
        plan = pk.Plan(nx, nx, torch.from_numpy(u[idx]).to(DEV), torch.from_numpy(v[idx]).to(DEV), kb_width=J,
                       levels=levels, block_offsets=loffs, stream=st)
        x0 = torch.zeros((nx, nx), dtype=torch.float32, device=DEV)
        pk.purify_sdmm_solve(plan, torch.from_numpy(y[idx]).to(DEV), eps[blocks], x0, max_iter=0, cg_iters=cg,
                             gamma=gamma, nu=nu)
        shards.append(sharded.LibraryShard(plan, DEV, torch.float32))
    return shards


def shard_result(shards, nx, cg):
    out, stats = [], []
    for sh in shards:
        x = torch.empty((nx, nx), dtype=torch.float32, device=DEV)
        stats.append(pk.purify_sdmm_solve(sh.plan, None, None, x, max_iter=0, resume=True, cg_iters=cg))
        out.append(x.cpu().numpy().astype(np.float64))
    return out, stats


@pytest.mark.parametrize("S", [1, 2, 3])
def test_sharded_iterations_match_oracle_and_unsharded_solve(S):
    nx, M, J, R, levels, cg, iters = 32, 4096, 6, 4, 3, 8, 10
    x_true, u, v, offs, y, eps, op = data(nx, M, J, R, seed=51)
    prob = osd.Problem(op, levels, y.astype(np.complex128), offs, eps)
    ref = osd.sdmm_solve(prob, np.zeros((nx, nx)), iters, cg).x
    shards = make_shards(nx, J, levels, u, v, offs, y, eps, S, cg, prob.gamma, prob.nu)
    drv = sharded.ShardedSdmm(shards, sharded.sum_in_place, cg)
    drv.iterate(iters)
    xs, stats = shard_result(shards, nx, cg)
    for x in xs:
        assert rel(x, ref) <= 1e-3
        assert rel(x, xs[0]) <= 1e-6          # the replicated image agrees over shards
    # the unsharded solve of the same problem
    plan = pk.Plan(nx, nx, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=J, levels=levels,
                   block_offsets=offs)
    xu = torch.zeros((nx, nx), dtype=torch.float32, device=DEV)
    stu = pk.purify_sdmm_solve(plan, torch.from_numpy(y).to(DEV), eps, xu, max_iter=iters, cg_iters=cg,
                               gamma=prob.gamma, nu=prob.nu)
    assert rel(xs[0], xu.cpu().numpy()) <= 1e-5
    # statistics: the objective on any shard, the residual ratio as the max over shards
    assert abs(stats[0].objective - stu.objective) <= 1e-5 * stu.objective
    assert abs(max(s.max_resid_over_eps for s in stats) - stu.max_resid_over_eps) <= 1e-5 * stu.max_resid_over_eps
    assert drv.exchanges == iters * (1 + cg)


def test_sharded_iterations_at_benchmark_size():
    # 256 x 256, M = 655,360, R = 8 blocks over 2 shards against the unsharded solve
    wl = synth.WORKLOADS["sara256_r8"]
    x_true, u, v, offs, nz = wl.draw()
    y0 = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs)
    pk.purify_phi(plan, torch.from_numpy(x_true.astype(np.float32)).to(DEV), y0)
    y = (y0.cpu().numpy().astype(np.complex128) + 0.01 * nz).astype(np.complex64)
    eps = osd.epsilon_chi2(0.01, np.diff(offs))
    xu = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=DEV)
    stu = pk.purify_sdmm_solve(plan, torch.from_numpy(y).to(DEV), eps, xu, max_iter=3, cg_iters=8)
    shards = make_shards(wl.nx, wl.J, wl.levels, u, v, offs, y, eps, 2, 8, stu.gamma, stu.nu)
    sharded.ShardedSdmm(shards, sharded.sum_in_place, 8).iterate(3)
    xs, _ = shard_result(shards, wl.nx, 8)
    assert rel(xs[0], xu.cpu().numpy()) <= 1e-4


def test_shard_steps_are_checked():
    nx, M, J = 32, 1000, 6
    x_true, u, v, offs, y, eps, op = data(nx, M, J, 2, seed=52)
    plan = pk.Plan(nx, nx, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=J, levels=2,
                   block_offsets=offs)
    r = torch.empty(nx * nx, dtype=torch.float32, device=DEV)
    lib = pk._lib.load()
    assert lib.purify_shard_iterate_local(plan.handle, r.data_ptr()) == pk._lib.PURIFY_EINVAL   # no solve yet
    x0 = torch.zeros((nx, nx), dtype=torch.float32, device=DEV)
    pk.purify_sdmm_solve(plan, torch.from_numpy(y).to(DEV), eps, x0, max_iter=0, gamma=1e-4, nu=1.0)
    host = np.zeros(nx * nx, dtype=np.float32)
    assert lib.purify_shard_cg_begin(plan.handle, host.ctypes.data) == pk._lib.PURIFY_EINVAL     # host image
    assert lib.purify_shard_cg_apply(plan.handle, -1, r.data_ptr()) == pk._lib.PURIFY_EINVAL      # negative step
