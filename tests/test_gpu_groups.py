"""GPU parity of the stochastic block-subset SDMM iterations (the paper's
closing paragraph: one data block, or a subset of blocks, per iteration)
against the FP64 oracle's sdmm_iteration_groups, through the C ABI: the
blocks dealt round-robin into G groups, one group per iteration from a
seeded sequence, the group's data term scaled by G in the x-update."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, make_plan, np_cplx, rel, snr_db
from oracle import nufft as onf
from oracle import sdmm as osd
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu


def problem(nx, M, J, R, levels, seed, dtype=pk.PURIFY_F32, grid_mode=0):
    plan, u, v, offs = make_plan(nx, nx, M, J, levels=levels, R=R, dtype=dtype, seed=seed, grid_mode=grid_mode)
    x_true = synth.sky(nx, nx, 1000 + seed, n_points=8, n_blobs=2)
    op = onf.NufftPlan(nx, nx, u.astype(np.float64), v.astype(np.float64), J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, 30.0)
    y = (y0 + sig * synth.unit_noise(M, 3000 + seed)).astype(np_cplx(dtype)).astype(np.complex128)
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    return plan, osd.Problem(op, levels, y, offs, eps), x_true


def oracle_groups(prob, nx, seq, G, cg):
    st = osd.init_state(prob, np.zeros((nx, nx)))
    for g in seq:
        osd.sdmm_iteration_groups(prob, st, cg, int(g), G)
    return st


def gpu(plan, prob, nx, iters, cg, G, seq):
    x = torch.zeros((nx, nx), dtype=torch.float32, device=DEV)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=iters, cg_iters=cg, gamma=prob.gamma, nu=prob.nu,
                              block_groups=G, group_seq=seq)
    return x.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("G", [1, 3])
def test_group_trajectory_matches_oracle(G):
    plan, prob, x_true = problem(32, 4096, 6, 5, 3, seed=41)
    iters, cg = 12, 8
    seq = synth.group_sequence(iters, G, 7000 + G)
    ref = oracle_groups(prob, 32, seq, G, cg)
    xg, st = gpu(plan, prob, 32, iters, cg, G, seq)
    assert rel(xg, ref.x) <= 1e-3
    assert abs(snr_db(x_true, xg) - snr_db(x_true, ref.x)) <= 0.05
    assert st.iters == iters and st.cg_iters_total == iters * cg


def test_one_group_equals_plain_solve():
    # G = 1 runs the group code path (lane kernels on the group's own run
    # lists, group chunk lists) and gives the plain iterates
    plan, prob, _ = problem(32, 4096, 6, 4, 3, seed=42)
    xg, _ = gpu(plan, prob, 32, 10, 8, 1, None)
    ref = osd.sdmm_solve(prob, np.zeros((32, 32)), 10, 8).x
    assert rel(xg, ref) <= 1e-3
    x = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=10, cg_iters=8, gamma=prob.gamma, nu=prob.nu)
    assert rel(xg, x.cpu().numpy()) <= 1e-5


def test_group_iterations_resume_and_replay():
    # a solve of 6 group iterations continued by 6 graph replays equals one
    # solve of 12 with the same sequence
    plan, prob, _ = problem(32, 3000, 6, 4, 3, seed=43)
    G, seq = 2, synth.group_sequence(12, 2, 7100)
    x12, _ = gpu(plan, prob, 32, 12, 6, G, seq)
    x = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=6, cg_iters=6, gamma=prob.gamma, nu=prob.nu,
                         block_groups=G, group_seq=seq[:6])
    pk.purify_sdmm_iterate_groups(plan, 6, seq[6:])
    st = pk.purify_sdmm_solve(plan, None, None, x, max_iter=0, resume=True, cg_iters=6, block_groups=G)
    assert st.iters == 12
    assert rel(x.cpu().numpy(), x12) <= 1e-5


def test_group_arguments_are_checked():
    plan, prob, _ = problem(32, 2000, 6, 3, 3, seed=44)
    x = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    kw = dict(max_iter=2, cg_iters=2, gamma=prob.gamma, nu=prob.nu)
    for bad in (dict(block_groups=4), dict(block_groups=2, group_seq=[0, 2]), dict(block_groups=2, toeplitz=True)):
        with pytest.raises(pk.PurifyError) as e:
            pk.purify_sdmm_solve(plan, y, prob.eps, x, **kw, **bad)
        assert e.value.status == pk._lib.PURIFY_EINVAL
    plan64, prob64, _ = problem(32, 2000, 6, 3, 3, seed=45, dtype=pk.PURIFY_F64)
    x64 = torch.zeros((32, 32), dtype=torch.float64, device=DEV)
    with pytest.raises(pk.PurifyError) as e:
        pk.purify_sdmm_solve(plan64, torch.from_numpy(prob64.y).to(DEV), prob64.eps, x64, block_groups=2, **kw)
    assert e.value.status == pk._lib.PURIFY_EINVAL


def test_groups_at_benchmark_size():
    # 256 x 256, M = 655,360, R = 8 blocks in G = 4 groups: one group
    # iteration from zero with 8 CG steps against the oracle
    wl = synth.WORKLOADS["sara256_r8"]
    x_true, u, v, offs, nz = wl.draw()
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs)
    op = onf.NufftPlan(wl.nx, wl.ny, u.astype(np.float64), v.astype(np.float64), wl.J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, wl.snr_db)
    y = (y0 + sig * nz).astype(np.complex64)
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    nu = float(np.sqrt(onf.power_norm_sq(op, iters=3)))
    prob = osd.Problem(op, wl.levels, y.astype(np.complex128), offs, eps, nu=nu)
    G, seq = 4, np.array([2], dtype=np.int32)
    ref = oracle_groups(prob, wl.nx, seq, G, 8)
    xg, st = gpu(plan, prob, wl.nx, 1, 8, G, seq)
    assert rel(xg, ref.x) <= 1e-3
