"""Learned warm start for SDMM (not in the paper; problem (3) is convex, so a
starting point changes only the time to reach a tolerance, never the
solution).

Pipeline, every numerical step on the GPU through the C ABI:
  1. problems: seeded 256 x 256 skies, M = 2N Gaussian (u, v), J = 4, L = 3,
     R = 1, 30 dB noise (the small-problem recipe scaled to 256 x 256);
  2. targets: SDMM solutions of the W = I problem (the first SARA pass),
     several problems advanced together as one batched graph;
  3. network input: the normalised dirty image Re Phi^H y / M (Phi delta_0 is
     close to 1 at every visibility, so the point-spread peak is about M);
  4. training: Adam on the mean-squared error of the U-Net output;
  5. evaluation: wall time for SDMM from x = 0 and from the network's output
     to reach objective <= (1 + 1e-3) * a long-run reference objective with
     every ||y_i - Phi_i x|| / eps_i <= 1 + 1e-3 (inference time included).
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (Batch, Plan, Unet, problem, purify_batch_iterate, purify_phi, purify_phi_adj, purify_sdmm_iterate,
               purify_sdmm_solve, synth)

N_SIDE = 256
M_VIS = 2 * N_SIDE * N_SIDE
J, LEVELS, SNR_DB = 4, 3, 30.0
CG_ITERS = 8
TRAIN_SEED0, EVAL_SEED0 = 0, 100000


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


def start(p: Problem, x0: torch.Tensor):
    """Set up the solver state from x0 (nu by power iteration on first use)."""
    st = purify_sdmm_solve(p.plan, p.y, p.eps, x0, max_iter=0, cg_iters=CG_ITERS, nu=p.nu, gamma=p.gamma)
    p.nu, p.gamma = st.nu, st.gamma
    return st


def current(p: Problem, x_out: torch.Tensor):
    return purify_sdmm_solve(p.plan, None, None, x_out, max_iter=0, resume=True)


def solve_batch(probs, iters: int, dev, chunk: int = 16):
    """SDMM solutions after `iters` iterations, several problems at a time."""
    out = []
    stream = torch.cuda.Stream(dev)
    for i in range(0, len(probs), chunk):
        group = probs[i:i + chunk]
        for p in group:
            start(p, torch.zeros((N_SIDE, N_SIDE), dtype=torch.float32, device=dev))
        torch.cuda.synchronize(dev)
        b = Batch([p.plan for p in group], stream)
        purify_batch_iterate(b, iters)
        stream.synchronize()
        b.close()
        for p in group:
            x = torch.empty((N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
            current(p, x)
            out.append(x)
    return out


def train(net: Unet, inputs: torch.Tensor, targets: torch.Tensor, epochs: int, batch: int, lr: float, seed: int = 0):
    """Adam on shuffled mini-batches; returns the per-epoch mean loss."""
    g = np.random.default_rng(seed)
    n = inputs.shape[0]
    losses = []
    for ep in range(epochs):
        order = g.permutation(n)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[i:i + batch]).to(inputs.device)
            xb = inputs.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            want = (i // batch) % 20 == 0
            l = net.train_step(xb, tb, lr, want_loss=want)
            if want:
                tot += l
                cnt += 1
        losses.append(tot / max(cnt, 1))
    return losses


def time_to_tolerance(p: Problem, x0: torch.Tensor, obj_ref: float, check: int = 5, max_iter: int = 2000,
                      pre=None):
    """Wall seconds (GPU-synchronised) and iterations for SDMM from x0 to reach
    objective <= (1 + 1e-3) obj_ref and every ratio <= 1 + 1e-3. `pre` (a
    callable returning x0) is timed as part of the run."""
    dev = p.y.device
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    if pre is not None:
        x0 = pre()
    start(p, x0)
    it = 0
    xo = torch.empty((N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
    st = current(p, xo)
    while it < max_iter and not (st.objective <= (1 + 1e-3) * obj_ref and st.max_resid_over_eps <= 1 + 1e-3):
        purify_sdmm_iterate(p.plan, check)
        it += check
        st = current(p, xo)
    torch.cuda.synchronize(dev)
    return time.perf_counter() - t0, it, xo, st
