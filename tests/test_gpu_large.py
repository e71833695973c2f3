"""The 1024 x 1024 workload (M = 10,485,760 visibilities with 10% uniform
coverage, J = 6, 5 wavelet levels, R = 64 uneven blocks): sampled outputs of
Phi against the oracle one by one, the adjoint identity at full size, and a
few SDMM iterations with per-block statistics checked against Phi."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, rel
from oracle import nufft as onf
from paper_1502_05037_gb300 import problem, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    wl = synth.WORKLOADS["sara1024_r64"]
    x, u, v, offs, nz = wl.draw()
    plan = pk.Plan(wl.nx, wl.ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=wl.J,
                   levels=wl.levels, block_offsets=offs)
    return wl, plan, x, u, v, offs, nz


def test_large_phi_sampled_and_adjoint(large):
    wl, plan, x, u, v, offs, nz = large
    xf = x.astype(np.float32)
    y = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, torch.from_numpy(xf).to(DEV), y)
    idx = np.random.default_rng(1).choice(wl.M, 2000, replace=False)
    op = onf.NufftPlan(wl.nx, wl.ny, u[idx].astype(np.float64), v[idx].astype(np.float64), wl.J)
    assert rel(y.cpu().numpy()[idx], onf.phi(op, xf.astype(np.float64))) <= 1e-5
    g = np.random.default_rng(2)
    yv = torch.from_numpy((g.standard_normal(wl.M) + 1j * g.standard_normal(wl.M)).astype(np.complex64)).to(DEV)
    xa = torch.empty((wl.ny, wl.nx), dtype=torch.complex64, device=DEV)
    pk.purify_phi_adj(plan, yv, xa)
    lhs = torch.vdot(yv.to(torch.complex128), y.to(torch.complex128)).real.item()
    rhs = torch.sum(torch.from_numpy(xf).to(DEV).double() * xa.real.double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_large_sdmm_iterations(large):
    wl, plan, x, u, v, offs, nz = large
    y0 = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, torch.from_numpy(x.astype(np.float32)).to(DEV), y0)
    sigma = problem.noise_sigma_from_norm(float(torch.linalg.vector_norm(y0.to(torch.complex128))), wl.M, wl.snr_db)
    y = y0 + torch.from_numpy((sigma * nz).astype(np.complex64)).to(DEV)
    eps = problem.chi2_epsilon(sigma, np.diff(offs))
    xs = torch.zeros((wl.ny, wl.nx), dtype=torch.float32, device=DEV)
    st = pk.purify_sdmm_solve(plan, y, eps, xs, max_iter=6, cg_iters=4)
    assert st.iters == 6 and np.isfinite(st.objective) and st.nu > 0
    yr = torch.empty(wl.M, dtype=torch.complex64, device=DEV)
    pk.purify_phi(plan, xs, yr)
    r = (y - yr).to(torch.complex128).cpu().numpy()
    ratios = [np.linalg.norm(r[offs[i]:offs[i + 1]]) / eps[i] for i in range(len(eps))]
    assert abs(max(ratios) - st.max_resid_over_eps) <= 1e-4 * max(ratios)
