"""Batched channels: several independent problems advanced by one captured
graph must follow the same iterates as each plan on its own, and the oracle."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, make_plan, rel
from oracle import nufft as onf
from oracle import sdmm as osd
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu


def channel(n, M, J, R, levels, seed):
    plan, u, v, offs = make_plan(n, n, M, J, levels=levels, R=R, seed=seed)
    x_true = synth.sky(n, n, 1000 + seed, n_points=6, n_blobs=2)
    op = onf.NufftPlan(n, n, u.astype(np.float64), v.astype(np.float64), J)
    y0 = onf.phi(op, x_true)
    sig = osd.noise_sigma(y0, 30.0)
    y = (y0 + sig * synth.unit_noise(M, 3000 + seed)).astype(np.complex64).astype(np.complex128)
    offs = offs if offs is not None else np.array([0, M])
    prob = osd.Problem(op, levels, y, offs, osd.epsilon_chi2(sig, np.diff(offs)))
    return plan, prob


def start(plan, prob, cg):
    n = prob.plan.nx
    x = torch.zeros((n, n), dtype=torch.float32, device=DEV)
    pk.purify_sdmm_solve(plan, torch.from_numpy(prob.y.astype(np.complex64)).to(DEV), prob.eps, x, max_iter=0,
                         cg_iters=cg, gamma=prob.gamma, nu=prob.nu)


def current_x(plan, n):
    x = torch.empty((n, n), dtype=torch.float32, device=DEV)
    pk.purify_sdmm_solve(plan, None, None, x, max_iter=0, resume=True)
    return x.cpu().numpy()


def test_batch_matches_single_plans_and_oracle():
    specs = [(32, 3000, 6, 2, 3, 1), (64, 9000, 4, 3, 3, 2), (32, 2500, 6, 1, 2, 3)]
    cg, iters = 6, 7
    chans = [channel(*s) for s in specs]
    batch_plans = []
    for plan, prob in chans:
        start(plan, prob, cg)
        batch_plans.append(plan)
    stream = torch.cuda.Stream()
    b = pk.Batch(batch_plans, stream)
    pk.purify_batch_iterate(b, 3)
    pk.purify_batch_iterate(b, iters - 3)
    stream.synchronize()
    xb = [current_x(p, pr.plan.nx) for p, pr in chans]
    # the same problems one at a time on fresh plans
    for (spec, (plan, prob), got) in zip(specs, chans, xb):
        single, prob2 = channel(*spec)
        start(single, prob2, cg)
        pk.purify_sdmm_iterate(single, iters)
        want = current_x(single, prob2.plan.nx)
        assert rel(got, want) <= 1e-5
        ref = osd.sdmm_solve(prob, np.zeros((prob.plan.nx, prob.plan.nx)), iters, cg)
        assert rel(got, ref.x) <= 1e-3
    b.close()
