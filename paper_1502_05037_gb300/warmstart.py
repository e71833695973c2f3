"""Learned warm start for SARA (not in the paper; problem (3) is convex, so a
starting point changes only the time to reach a tolerance, never the
solution).

SARA (Sec. 1) solves a sequence of weighted problems: W = I first, then
passes whose weights are w = rho / (rho + |Psi^dagger x|) from the previous
pass's solution, rho halved each pass. Pipeline, every numerical step on the
GPU through the C ABI:
  1. problems: seeded 256 x 256 skies, M = 2N Gaussian (u, v), J = 4, L = 3,
     R = 1, 30 dB noise (the small-problem recipe scaled to 256 x 256);
  2. targets: SARA solutions (the W = I pass and three reweighted passes at
     fixed iteration counts), several problems advanced together as one
     batched graph;
  3. network input: the normalised dirty image Re Phi^H y / M (Phi delta_0 is
     close to 1 at every visibility, so the point-spread peak is about M);
  4. training: Adam on the mean-squared error of the U-Net output;
  5. evaluation: wall time of the plain SARA solve (W = I from x = 0, then
     the reweighted passes, each run until the relative objective change over
     10 iterations is below 1e-4 with every ||y_i - Phi_i x|| / eps_i <=
     1 + 1e-3) against the learned solve: the network's prediction, weights
     from it, and the final reweighted pass alone, run until its result is as
     good as the plain one (SNR against the true sky within 0.05 dB of the
     plain result's, constraint ratios within 1 + 1e-3; inference and the
     checks included). Reported beside the times: the prediction's SNR, the
     fraction of problems that reach the plain quality within the iteration
     cap, and the learned result's objective under the plain solve's final
     weights.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (Batch, Plan, Unet, problem, purify_batch_iterate, purify_coef_std, purify_phi, purify_phi_adj,
               purify_reweight, purify_sdmm_iterate, purify_sdmm_solve, synth)

N_SIDE = 256
M_VIS = 2 * N_SIDE * N_SIDE
J, LEVELS, SNR_DB = 4, 3, 30.0
CG_ITERS = 8
TRAIN_SEED0, EVAL_SEED0 = 0, 100000
PASSES = 3                    # reweighted passes after the W = I pass
PASS_REL_TOL, PASS_EPS_TOL = 1e-4, 1e-3


def sample_arrays(s: int):
    """Seeded sky, (u, v) and unit noise of problem s."""
    x = synth.sky(N_SIDE, N_SIDE, 10_000_000 + s, n_points=20, n_blobs=3)
    u, v = synth.uv_coverage(M_VIS, 20_000_000 + s, dtype=np.float32)
    nz = synth.unit_noise(M_VIS, 30_000_000 + s)
    return x, u, v, nz


@dataclass
class Problem:
    seed: int
    plan: Plan
    y: torch.Tensor
    eps: np.ndarray
    x_true: np.ndarray
    dirty: torch.Tensor
    nu: float = 0.0
    gamma: float = 0.0


def make_problem(s: int, dev) -> Problem:
    x, u, v, nz = sample_arrays(s)
    plan = Plan(N_SIDE, N_SIDE, torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev), kb_width=J, levels=LEVELS)
    xt = torch.from_numpy(x.astype(np.float32)).to(dev)
    y0 = torch.empty(M_VIS, dtype=torch.complex64, device=dev)
    purify_phi(plan, xt, y0)
    sigma = problem.noise_sigma_from_norm(float(torch.linalg.vector_norm(y0.to(torch.complex128))), M_VIS, SNR_DB)
    y = y0 + torch.from_numpy((sigma * nz).astype(np.complex64)).to(dev)
    eps = problem.chi2_epsilon(sigma, [M_VIS])
    xa = torch.empty((N_SIDE, N_SIDE), dtype=torch.complex64, device=dev)
    purify_phi_adj(plan, y, xa)
    dirty = (xa.real / M_VIS).contiguous()
    return Problem(s, plan, y, eps, x, dirty)


def start(p: Problem, x0: torch.Tensor, w: torch.Tensor | None = None):
    """Set up the solver state from x0 and weights w (W = I when None); nu and
    gamma by power iteration and from the data on first use."""
    st = purify_sdmm_solve(p.plan, p.y, p.eps, x0, w=w, max_iter=0, cg_iters=CG_ITERS, nu=p.nu, gamma=p.gamma)
    p.nu, p.gamma = st.nu, st.gamma
    return st


def current(p: Problem, x_out: torch.Tensor):
    return purify_sdmm_solve(p.plan, None, None, x_out, max_iter=0, resume=True)


def weights_from(p: Problem, x: torch.Tensor, rho: float) -> torch.Tensor:
    """w = rho / (rho + |Psi^dagger x|) (SARA reweighting)."""
    w = torch.empty((p.plan.info.q, N_SIDE, N_SIDE), dtype=torch.float32, device=x.device)
    purify_reweight(p.plan, x, rho, w)
    return w


def sara_targets(probs, dev, first_iters: int, pass_iters: int, chunk: int = 16):
    """SARA solutions at fixed iteration counts (the W = I pass, then PASSES
    reweighted passes), several problems advanced together as one batched
    graph per pass."""
    out = []
    stream = torch.cuda.Stream(dev)
    for i in range(0, len(probs), chunk):
        group = probs[i:i + chunk]
        xs = [torch.zeros((N_SIDE, N_SIDE), dtype=torch.float32, device=dev) for _ in group]
        rho = [0.0] * len(group)
        for ps in range(PASSES + 1):
            for k, p in enumerate(group):
                if ps == 0:
                    start(p, xs[k])
                else:
                    if ps == 1:
                        rho[k] = purify_coef_std(p.plan, xs[k])
                    else:
                        rho[k] *= 0.5
                    start(p, xs[k], weights_from(p, xs[k], rho[k]))
            torch.cuda.synchronize(dev)
            b = Batch([p.plan for p in group], stream)
            purify_batch_iterate(b, first_iters if ps == 0 else pass_iters)
            stream.synchronize()
            b.close()
            for k, p in enumerate(group):
                current(p, xs[k])
        out.extend(xs)
    return out


def solve_pass(p: Problem, x: torch.Tensor, w: torch.Tensor | None, max_iter: int = 3000):
    """One SARA pass from x (updated in place) to the pass stopping rule."""
    return purify_sdmm_solve(p.plan, p.y, p.eps, x, w=w, max_iter=max_iter, cg_iters=CG_ITERS, nu=p.nu,
                             gamma=p.gamma, rel_obj_tol=PASS_REL_TOL, eps_tol=PASS_EPS_TOL, check_every=10,
                             raise_on_error=False)


def sara_plain(p: Problem, dev):
    """Plain SARA from x = 0: returns (seconds, iterations, x, final weights,
    final stats)."""
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    x = torch.zeros((N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
    st = solve_pass(p, x, None)
    iters = st.iters
    rho = purify_coef_std(p.plan, x)
    w = None
    for ps in range(PASSES):
        w = weights_from(p, x, rho)
        st = solve_pass(p, x, w)
        iters += st.iters
        rho *= 0.5
    torch.cuda.synchronize(dev)
    return time.perf_counter() - t0, iters, x, w, st


def sara_learned(p: Problem, net: Unet, dev, snr_target: float, check: int = 10, max_iter: int = 3000,
                 max_passes: int = 2):
    """Learned SARA: the network's prediction, weights from it (rho from its
    coefficient spread, halved as often as the plain solve halves it before
    its last pass), then reweighted passes from the prediction until the
    result is as good as the plain solve's (SNR against the true sky at least
    snr_target, every constraint ratio <= 1 + PASS_EPS_TOL), checked every
    `check` iterations. A pass that stagnates first (the plain passes'
    stopping rule) is followed by one more pass with weights from its result
    and rho halved, up to max_passes passes and max_iter iterations in all.
    Returns (seconds, iterations, x, stats, reached, prediction SNR, passes)."""
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pred = torch.empty((1, N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
    net.forward(p.dirty.view(1, N_SIDE, N_SIDE), pred)
    x = torch.clamp_min(pred.view(N_SIDE, N_SIDE), 0.0).contiguous()
    rho = purify_coef_std(p.plan, x) * 0.5 ** (PASSES - 1)
    truth = torch.from_numpy(p.x_true.astype(np.float32)).to(dev)
    tn = float(torch.linalg.vector_norm(truth))
    pred_snr = 20.0 * np.log10(tn / float(torch.linalg.vector_norm(truth - x)))
    it, reached, passes = 0, False, 0
    st = None
    while not reached and passes < max_passes and it < max_iter:
        start(p, x, weights_from(p, x, rho))
        passes += 1
        prev = None
        while it < max_iter:
            purify_sdmm_iterate(p.plan, check)
            it += check
            st = current(p, x)
            snr = 20.0 * np.log10(tn / float(torch.linalg.vector_norm(truth - x)))
            ok = st.max_resid_over_eps <= 1.0 + PASS_EPS_TOL
            if snr >= snr_target and ok:
                reached = True
                break
            if prev is not None and ok and abs(st.objective - prev) <= PASS_REL_TOL * st.objective:
                break
            prev = st.objective
        rho *= 0.5
    torch.cuda.synchronize(dev)
    return time.perf_counter() - t0, it, x, st, reached, pred_snr, passes


def objective_at(p: Problem, x: torch.Tensor, w: torch.Tensor):
    """||W Psi^dagger x||_1 and the worst constraint ratio at x."""
    xc = x.clone()
    st = purify_sdmm_solve(p.plan, p.y, p.eps, xc, w=w, max_iter=0, cg_iters=CG_ITERS, nu=p.nu, gamma=p.gamma)
    return st.objective, st.max_resid_over_eps


def train(net: Unet, inputs: torch.Tensor, targets: torch.Tensor, epochs: int, batch: int, lr: float, seed: int = 0):
    """Adam on shuffled mini-batches, the step size halved every ten epochs;
    returns the per-epoch mean loss."""
    g = np.random.default_rng(seed)
    n = inputs.shape[0]
    losses = []
    for ep in range(epochs):
        lr_ep = lr * 0.5 ** (ep / 10.0)   # halved every ten epochs
        order = g.permutation(n)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[i:i + batch]).to(inputs.device)
            xb = inputs.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            want = (i // batch) % 20 == 0
            l = net.train_step(xb, tb, lr_ep, want_loss=want)
            if want:
                tot += l
                cnt += 1
        losses.append(tot / max(cnt, 1))
    return losses
