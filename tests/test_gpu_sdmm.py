"""GPU parity of the SDMM solve of problem (3) (Sec. 1, Eqs. 1-3) and of SARA
reweighting against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, make_plan, np_cplx, np_real, rel, snr_db, t_real
from oracle import nufft as onf
from oracle import primal_dual as opd
from oracle import sdmm as osd
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu


def problem(nx, M, J, R, levels, dtype, seed, snr=30.0):
    plan, u, v, offs = make_plan(nx, nx, M, J, levels=levels, R=R, dtype=dtype, seed=seed)
    x_true = synth.sky(nx, nx, 1000 + seed, n_points=8, n_blobs=2)
    op = onf.NufftPlan(nx, nx, u.astype(np.float64), v.astype(np.float64), J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, snr)
    y = (y0 + sig * synth.unit_noise(M, 3000 + seed)).astype(np_cplx(dtype)).astype(np.complex128)
    offs = offs if offs is not None else np.array([0, M])
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    prob = osd.Problem(op, levels, y, offs, eps)
    return plan, prob, x_true


def gpu_solve(plan, prob, dtype, iters, cg, x0=None, **kw):
    nx = prob.plan.nx
    x = torch.zeros((nx, nx), dtype=t_real(dtype), device=DEV) if x0 is None else x0
    y = torch.from_numpy(prob.y.astype(np_cplx(dtype))).to(DEV)
    w = None if prob.weights is None else torch.from_numpy(prob.weights.astype(np_real(dtype))).to(DEV)
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, w=w, max_iter=iters, cg_iters=cg, gamma=prob.gamma,
                              nu=prob.nu, **kw)
    return x, st


@pytest.mark.parametrize("dtype,tol", [(pk.PURIFY_F32, 1e-3), (pk.PURIFY_F64, 1e-9)])
def test_fixed_iteration_trajectory(dtype, tol):
    plan, prob, x_true = problem(32, 4096, 6, 3, 3, dtype, seed=1)
    iters, cg = 25, 8
    ref = osd.sdmm_solve(prob, np.zeros((32, 32)), iters, cg)
    x, st = gpu_solve(plan, prob, dtype, iters, cg)
    xg = x.cpu().numpy().astype(np.float64)
    assert rel(xg, ref.x) <= tol
    assert abs(snr_db(x_true, xg) - snr_db(x_true, ref.x)) <= 0.05
    assert st.iters == iters and st.cg_iters_total == iters * cg
    # stats at the returned x
    assert abs(st.objective - osd.objective(prob, ref.x)) <= 10 * tol * osd.objective(prob, ref.x)
    assert abs(st.max_resid_over_eps - osd.residual_ratios(prob, ref.x).max()) <= 10 * tol


def test_cg_tolerance_trajectory():
    # CG stopped by ||r|| <= tol ||r_0|| inside every x-update: same step
    # counts and the same iterates as the oracle (FP64, so no stop decision
    # sits within rounding of the threshold)
    dtype = pk.PURIFY_F64
    plan, prob, _ = problem(32, 4096, 6, 3, 3, dtype, seed=9)
    iters, cap, tol = 12, 40, 1e-3
    ref = osd.sdmm_solve(prob, np.zeros((32, 32)), iters, cap, tol)
    counts = [h["cg"] for h in ref.history]
    assert max(counts) < cap and min(counts) >= 1
    x, st = gpu_solve(plan, prob, dtype, iters, cap, cg_tol=tol)
    assert st.iters == iters and st.cg_iters_total == ref.cg_iters
    assert rel(x.cpu().numpy(), ref.x) <= 1e-9


@pytest.mark.parametrize("dtype,tol,weighted", [(pk.PURIFY_F64, 1e-9, False), (pk.PURIFY_F32, 1e-3, False),
                                                (pk.PURIFY_F32, 1e-3, True)])
def test_primal_dual_trajectory(dtype, tol, weighted):
    # Chambolle-Pock iterations for problem (3) against the FP64 oracle's
    # (the same steps, sigma z kept as the ball dual on the GPU)
    plan, prob, x_true = problem(32, 4096, 6, 3, 3, dtype, seed=11)
    if weighted:
        prob.weights = 0.5 + np.random.default_rng(12).random((plan.info.q, 32, 32))
    iters, tau, sigma = 40, 0.05, 9.8
    ref = opd.chambolle_pock(prob, iters, tau=tau, sigma=sigma, x0=np.zeros((32, 32)))
    x = torch.zeros((32, 32), dtype=t_real(dtype), device=DEV)
    y = torch.from_numpy(prob.y.astype(np_cplx(dtype))).to(DEV)
    w = None if prob.weights is None else torch.from_numpy(prob.weights.astype(np_real(dtype))).to(DEV)
    st = pk.purify_pd_solve(plan, y, prob.eps, x, w=w, iters=iters, tau=tau, sigma=sigma, nu=prob.nu)
    xg = x.cpu().numpy().astype(np.float64)
    assert rel(xg, ref) <= tol
    assert st.iters == iters and st.cg_iters_total == 0 and st.status == 0
    assert abs(st.objective - osd.objective(prob, ref)) <= 10 * tol * osd.objective(prob, ref)
    assert abs(st.max_resid_over_eps - osd.residual_ratios(prob, ref).max()) <= 10 * tol
    # a second call starts over from its x (here the result): the step from
    # the oracle's result agrees as well
    ref2 = opd.chambolle_pock(prob, 5, tau=tau, sigma=sigma, x0=ref)
    pk.purify_pd_solve(plan, y, prob.eps, x, w=w, iters=5, tau=tau, sigma=sigma, nu=prob.nu)
    assert rel(x.cpu().numpy().astype(np.float64), ref2) <= 2 * tol


def test_weighted_trajectory_and_reweight():
    dtype = pk.PURIFY_F32
    plan, prob, x_true = problem(32, 3000, 4, 2, 2, dtype, seed=2)
    base = osd.sdmm_solve(prob, np.zeros((32, 32)), 10, 6).x
    rho = float(np.std(prob.psi_adj(base)))
    w_ref = osd.reweight(prob, base, rho)
    xb = torch.from_numpy(base.astype(np.float32)).to(DEV)
    w = torch.empty((plan.info.q, 32, 32), dtype=torch.float32, device=DEV)
    pk.purify_reweight(plan, xb, rho, w)
    assert rel(w.cpu().numpy(), w_ref) <= 1e-5
    assert abs(pk.purify_coef_std(plan, xb) - rho) <= 1e-5 * rho
    prob.weights = w_ref
    ref = osd.sdmm_solve(prob, base, 10, 6)
    x, _ = gpu_solve(plan, prob, dtype, 10, 6, x0=xb.clone())
    assert rel(x.cpu().numpy(), ref.x) <= 1e-3


def test_operator_norm_and_gamma_defaults():
    dtype = pk.PURIFY_F64
    plan, prob, _ = problem(32, 2000, 6, 1, 3, dtype, seed=3)
    nu2 = pk.purify_op_norm_sq(plan, 300)
    assert abs(nu2 - onf.power_norm_sq(prob.plan, iters=300)) <= 1e-6 * nu2
    # default gamma with the oracle's nu
    x = torch.zeros((32, 32), dtype=torch.float64, device=DEV)
    y = torch.from_numpy(prob.y).to(DEV)
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=0, nu=prob.nu)
    assert abs(st.gamma - prob.gamma) <= 1e-10 * prob.gamma


def test_resume_continues_the_same_sequence():
    dtype = pk.PURIFY_F32
    plan, prob, _ = problem(32, 3000, 6, 2, 3, dtype, seed=4)
    x_all, _ = gpu_solve(plan, prob, dtype, 16, 6)
    x_half, _ = gpu_solve(plan, prob, dtype, 8, 6)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    x2 = torch.empty_like(x_half)
    st = pk.purify_sdmm_solve(plan, None, None, x2, max_iter=8, cg_iters=6, resume=True)
    assert st.iters == 16
    assert rel(x2.cpu().numpy(), x_all.cpu().numpy()) <= 1e-5


def test_host_buffers_give_the_device_result():
    dtype = pk.PURIFY_F32
    plan, prob, _ = problem(32, 2000, 6, 2, 3, dtype, seed=5)
    xd, _ = gpu_solve(plan, prob, dtype, 5, 5)
    xh = np.zeros((32, 32), dtype=np.float32)
    pk.purify_sdmm_solve(plan, prob.y.astype(np.complex64), prob.eps, xh, max_iter=5, cg_iters=5,
                         gamma=prob.gamma, nu=prob.nu)
    assert rel(xh, xd.cpu().numpy()) <= 1e-5


def test_tolerance_mode_and_errors():
    dtype = pk.PURIFY_F32
    plan, prob, _ = problem(32, 3000, 6, 2, 3, dtype, seed=6)
    y = torch.from_numpy(prob.y.astype(np.complex64)).to(DEV)
    x = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=3, cg_iters=5, gamma=prob.gamma, nu=prob.nu,
                              rel_obj_tol=1e-12, eps_tol=0.0, check_every=1, raise_on_error=False)
    assert st.status == pk._lib.PURIFY_ENOTCONV
    x.zero_()
    st = pk.purify_sdmm_solve(plan, y, prob.eps, x, max_iter=2000, cg_iters=10, cg_tol=1e-6, gamma=prob.gamma,
                              nu=prob.nu, rel_obj_tol=1e-4, eps_tol=1e-2, check_every=5)
    assert st.status == 0 and st.iters < 2000 and st.max_resid_over_eps <= 1.0 + 1e-2 + 1e-3
    with pytest.raises(pk.PurifyError) as e:
        pk.purify_sdmm_solve(plan, y, -prob.eps, x, max_iter=1, gamma=prob.gamma, nu=prob.nu)
    assert e.value.status == pk._lib.PURIFY_EINVAL
    ybad = y.clone()
    ybad[7] = float("nan")
    with pytest.raises(pk.PurifyError) as e:
        pk.purify_sdmm_solve(plan, ybad, prob.eps, x, max_iter=1, gamma=prob.gamma, nu=prob.nu)
    assert e.value.status == pk._lib.PURIFY_ENAN


def test_full_size_iteration_against_sampled_properties():
    # 256 x 256, M = 655360, R = 8: after a few iterations the multipliers
    # obey the projection identities at every visibility, checked on the host
    wl = synth.WORKLOADS["sara256_r8"]
    x_true, u, v, offs, nz = wl.draw()
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs)
    op = onf.NufftPlan(wl.nx, wl.ny, u.astype(np.float64), v.astype(np.float64), wl.J)
    y0n = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0n, wl.snr_db)
    y = y0n + sig * nz
    eps = osd.epsilon_chi2(sig, np.diff(offs))
    x = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=DEV)
    st = pk.purify_sdmm_solve(plan, torch.from_numpy(y.astype(np.complex64)).to(DEV), eps, x, max_iter=30,
                              cg_iters=8)
    xr = x.cpu().numpy()
    assert np.isfinite(xr).all()
    assert st.nu > 0 and st.gamma > 0
    # residual ratio reported equals one recomputed from Phi on the GPU
    yr = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, x, yr)
    r = y - yr.cpu().numpy().astype(np.complex128)
    ratios = [np.linalg.norm(r[offs[i]:offs[i + 1]]) / eps[i] for i in range(len(eps))]
    assert abs(max(ratios) - st.max_resid_over_eps) <= 1e-4 * max(ratios)
    assert snr_db(x_true, xr) > 3.0


def test_toeplitz_trajectory_against_exact_normal_operator():
    # the CG normal operator by circulant embedding equals the exact model's
    # A^H A up to the NUFFT error of its point-spread function
    dtype = pk.PURIFY_F32
    plan, prob, x_true = problem(32, 3000, 6, 2, 3, dtype, seed=7)
    prob.normal = "exact"
    iters, cg = 12, 8
    ref = osd.sdmm_solve(prob, np.zeros((32, 32)), iters, cg)
    x, st = gpu_solve(plan, prob, dtype, iters, cg, toeplitz=True)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-3
    # and stays close to the NUFFT-operator trajectory
    prob.normal = "nufft"
    ref2 = osd.sdmm_solve(prob, np.zeros((32, 32)), iters, cg)
    assert rel(x.cpu().numpy(), ref2.x) <= 1e-2
