"""Deterministic gridding (grid_mode 6): each run's J x J patch is stored and
every grid cell sums the patches covering it in a fixed order, so G^H, the
CG normal operator and a whole SDMM solve give the same bits on every run.
Checked here: repeated operator calls are bit-identical; a solve of n
iterations continued by m more through resume equals one solve of n + m bit
for bit (plain and block-group iterations, and at 256 x 256 / R = 8); the
deterministic trajectory matches the FP64 oracle like every other mode."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, make_plan, np_cplx, rel, snr_db
from oracle import nufft as onf
from oracle import sdmm as osd
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu


def problem(nx, M, J, R, levels, seed):
    plan, u, v, offs = make_plan(nx, nx, M, J, levels=levels, R=R, seed=seed, grid_mode=6,
                                 uniform_fraction=0.1)
    x_true = synth.sky(nx, nx, 1000 + seed, n_points=8, n_blobs=2)
    op = onf.NufftPlan(nx, nx, u.astype(np.float64), v.astype(np.float64), J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, 30.0)
    y = (y0 + sig * synth.unit_noise(M, 3000 + seed)).astype(np_cplx(pk.PURIFY_F32)).astype(np.complex128)
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    return plan, osd.Problem(op, levels, y, offs, eps), x_true


def solve(plan, prob, nx, iters, cg, **kw):
    x = torch.zeros((nx, nx), dtype=torch.float32, device=DEV)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=iters, cg_iters=cg, gamma=prob.gamma, nu=prob.nu,
                              **kw)
    return x, st


def resume(plan, nx, iters, cg, **kw):
    x = torch.empty((nx, nx), dtype=torch.float32, device=DEV)
    st = pk.purify_sdmm_solve(plan, None, None, x, max_iter=iters, cg_iters=cg, resume=True, **kw)
    return x, st


def test_operators_are_bit_reproducible():
    nx, M = 64, 30011
    plan, u, v, _ = make_plan(nx, nx, M, 6, R=3, seed=61, grid_mode=6)
    assert plan.info.grid_mode == 6 and plan.info.normal_mode == 6
    g = np.random.default_rng(62)
    y = torch.from_numpy((g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex64)).to(DEV)
    xr = torch.from_numpy(g.standard_normal((nx, nx)).astype(np.float32)).to(DEV)
    a = [torch.empty((nx, nx), dtype=torch.complex64, device=DEV) for _ in range(3)]
    n = [torch.empty((nx, nx), dtype=torch.float32, device=DEV) for _ in range(3)]
    for k in range(3):
        pk.purify_phi_adj(plan, y, a[k])
        pk.purify_phi_normal(plan, xr, n[k])
    for k in (1, 2):
        assert torch.equal(a[k], a[0])
        assert torch.equal(n[k], n[0])
    op = onf.NufftPlan(nx, nx, u.astype(np.float64), v.astype(np.float64), 6)
    assert rel(a[0].cpu().numpy(), onf.phi_adj(op, y.cpu().numpy().astype(np.complex128))) <= 1e-5
    xr64 = xr.cpu().numpy().astype(np.float64)
    assert rel(n[0].cpu().numpy(), np.real(onf.phi_adj(op, onf.phi(op, xr64)))) <= 1e-5


def test_trajectory_matches_oracle():
    plan, prob, x_true = problem(32, 4096, 6, 4, 3, seed=63)
    iters, cg = 12, 8
    ref = osd.sdmm_solve(prob, np.zeros((32, 32)), iters, cg).x
    x, st = solve(plan, prob, 32, iters, cg)
    xg = x.cpu().numpy().astype(np.float64)
    assert rel(xg, ref) <= 1e-3
    assert abs(snr_db(x_true, xg) - snr_db(x_true, ref)) <= 0.05
    assert st.iters == iters


def test_save_and_resume_is_bit_exact():
    # 100 iterations, then 100 more by resume, equal one solve of 200: the
    # iterate and every statistic, bit for bit
    plan, prob, _ = problem(64, 20000, 6, 4, 3, seed=64)
    cg = 8
    x200, st200 = solve(plan, prob, 64, 200, cg)
    x100, _ = solve(plan, prob, 64, 100, cg)
    xr, str_ = resume(plan, 64, 100, cg)
    assert str_.iters == 200
    assert torch.equal(xr, x200)
    assert str_.objective == st200.objective
    assert str_.max_resid_over_eps == st200.max_resid_over_eps
    assert str_.cg_iters_total == st200.cg_iters_total
    # and a second full solve repeats the first
    x200b, _ = solve(plan, prob, 64, 200, cg)
    assert torch.equal(x200b, x200)


def test_block_group_iterations_resume_bit_exact():
    plan, prob, _ = problem(32, 6000, 6, 6, 3, seed=65)
    G, seq = 3, synth.group_sequence(40, 3, 7200)
    x40, _ = solve(plan, prob, 32, 40, 6, block_groups=G, group_seq=seq)
    x20, _ = solve(plan, prob, 32, 20, 6, block_groups=G, group_seq=seq[:20])
    pk.purify_sdmm_iterate_groups(plan, 20, seq[20:])
    xr, st = resume(plan, 32, 0, 6, block_groups=G)
    assert st.iters == 40
    assert torch.equal(xr, x40)


def test_resume_bit_exact_at_benchmark_size():
    # 256 x 256, M = 655,360, R = 8: 20 + 20 iterations equal 40, and the
    # deterministic solve agrees with the autotuned (atomic) one to rounding
    wl = synth.WORKLOADS["sara256_r8"]
    x_true, u, v, offs, nz = wl.draw()
    ud, vd = torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV)
    det = pk.Plan(wl.nx, wl.ny, ud, vd, kb_width=wl.J, levels=wl.levels, block_offsets=offs, grid_mode=6)
    y0 = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(det, torch.from_numpy(x_true.astype(np.float32)).to(DEV), y0)
    y = torch.from_numpy((y0.cpu().numpy().astype(np.complex128) + 0.01 * nz).astype(np.complex64)).to(DEV)
    eps = osd.epsilon_chi2(0.01, np.diff(offs))

    def run(plan, iters, **kw):
        x = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=DEV)
        st = pk.purify_sdmm_solve(plan, y, eps, x, max_iter=iters, cg_iters=8, **kw)
        return x, st

    x40, st40 = run(det, 40)
    run(det, 20, gamma=st40.gamma, nu=st40.nu)
    xr, st = resume(det, wl.nx, 20, 8)
    assert st.iters == 40
    assert torch.equal(xr, x40)
    auto = pk.Plan(wl.nx, wl.ny, ud, vd, kb_width=wl.J, levels=wl.levels, block_offsets=offs)
    xa, _ = run(auto, 40, gamma=st40.gamma, nu=st40.nu)
    assert rel(x40.cpu().numpy(), xa.cpu().numpy()) <= 1e-4
