"""Learned warm start for SARA (not in the paper; problem (3) is convex, so a
starting point changes only the time to reach a tolerance, never the
solution).

SARA (Sec. 1) solves a sequence of weighted problems: W = I first, then
passes whose weights are w = rho / (rho + |Psi^dagger x|) from the previous
pass's solution, rho halved each pass. Pipeline, every numerical step on the
GPU through the C ABI:
  1. problems: seeded skies, M = 2N Gaussian (u, v), J = 4, L = 3, R = 1,
     30 dB noise (the small-problem recipe; 256 x 256 for the benchmark);
  2. targets: SARA solutions (the W = I pass and the reweighted passes at
     fixed iteration counts), several problems advanced as one batched graph;
  3. network input: the normalised dirty image Re Phi^H y / M (Phi delta_0 is
     close to 1 at every visibility, so the point-spread peak is about M);
  4. training: Adam on the mean-squared error of the U-Net output;
  5. evaluation, both arms stopped by the same rule and never by the true sky:
     plain = the W = I pass from x = 0 and PASSES reweighted passes; learned =
     the network's prediction (inference timed), then LEARNED_PASSES
     reweighted passes from it (weights from the current iterate, rho from
     the prediction's coefficient spread scaled like the plain schedule's
     last passes); every pass runs until the relative objective change over
     10 iterations is below PASS_REL_TOL with every ||y_i - Phi_i x|| / eps_i
     <= 1 + PASS_EPS_TOL. Afterwards a learned result counts as reaching the
     plain one when, under the plain solve's final weights, its objective is
     within 1e-3 of the plain result's, its constraint ratios are within
     1 + 1e-3, and its SNR against the true sky is at most 0.05 dB below the
     plain result's; a problem that misses counts its learned attempt plus
     the plain solve.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (Batch, Plan, Unet, problem, purify_batch_iterate, purify_coef_std, purify_phi, purify_phi_adj,
               purify_reweight, purify_sdmm_solve, synth)

J, LEVELS, SNR_DB = 4, 3, 30.0
CG_ITERS = 8
TRAIN_SEED0, EVAL_SEED0 = 0, 100000
PASSES = 3                    # reweighted passes after the W = I pass
LEARNED_PASSES = 2            # reweighted passes after the prediction
PASS_REL_TOL, PASS_EPS_TOL = 1e-4, 1e-3
OBJ_TOL, SNR_TOL = 1e-3, 0.05


@dataclass(frozen=True)
class Size:
    """Image side n (N = n^2) and visibility count M = 2N."""
    n: int = 256

    @property
    def M(self) -> int:
        return 2 * self.n * self.n


BENCH = Size(256)
N_SIDE = BENCH.n
M_VIS = BENCH.M


def sample_arrays(s: int, size: Size = BENCH):
    """Seeded sky, (u, v) and unit noise of problem s."""
    x = synth.sky(size.n, size.n, 10_000_000 + s, n_points=20, n_blobs=3)
    u, v = synth.uv_coverage(size.M, 20_000_000 + s, dtype=np.float32)
    nz = synth.unit_noise(size.M, 30_000_000 + s)
    return x, u, v, nz


@dataclass
class Problem:
    seed: int
    plan: Plan
    y: torch.Tensor
    eps: np.ndarray
    x_true: np.ndarray
    dirty: torch.Tensor
    size: Size = BENCH
    nu: float = 0.0
    gamma: float = 0.0


def make_problem(s: int, dev, size: Size = BENCH) -> Problem:
    x, u, v, nz = sample_arrays(s, size)
    n, M = size.n, size.M
    plan = Plan(n, n, torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev), kb_width=J, levels=LEVELS)
    xt = torch.from_numpy(x.astype(np.float32)).to(dev)
    y0 = torch.empty(M, dtype=torch.complex64, device=dev)
    purify_phi(plan, xt, y0)
    sigma = problem.noise_sigma_from_norm(float(torch.linalg.vector_norm(y0.to(torch.complex128))), M, SNR_DB)
    y = y0 + torch.from_numpy((sigma * nz).astype(np.complex64)).to(dev)
    eps = problem.chi2_epsilon(sigma, [M])
    xa = torch.empty((n, n), dtype=torch.complex64, device=dev)
    purify_phi_adj(plan, y, xa)
    dirty = (xa.real / M).contiguous()
    return Problem(s, plan, y, eps, x, dirty, size)


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
    n = p.size.n
    w = torch.empty((p.plan.info.q, n, n), dtype=torch.float32, device=x.device)
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
        n = group[0].size.n
        xs = [torch.zeros((n, n), dtype=torch.float32, device=dev) for _ in group]
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
    n = p.size.n
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    x = torch.zeros((n, n), dtype=torch.float32, device=dev)
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


def predict(p: Problem, net: Unet) -> torch.Tensor:
    """The network's estimate of the SARA solution, clamped to R_+^N."""
    n = p.size.n
    pred = torch.empty((1, n, n), dtype=torch.float32, device=p.dirty.device)
    net.forward(p.dirty.view(1, n, n), pred)
    return torch.clamp_min(pred.view(n, n), 0.0).contiguous()


def sara_learned(p: Problem, net: Unet, dev, passes: int = LEARNED_PASSES):
    """Learned SARA: the network's prediction, then `passes` reweighted passes
    from it, each with weights from the current iterate and stopped by the
    plain passes' rule (the true sky is never looked at). rho starts from the
    prediction's coefficient spread scaled like the last `passes` passes of
    the plain schedule, and is halved per pass. Returns (seconds,
    iterations, x, final weights, final stats, prediction)."""
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    x = predict(p, net)
    pred = x.clone()
    rho = purify_coef_std(p.plan, x) * 0.5 ** (PASSES - passes)
    iters, w, st = 0, None, None
    for _ in range(passes):
        w = weights_from(p, x, rho)
        st = solve_pass(p, x, w)
        iters += st.iters
        rho *= 0.5
    torch.cuda.synchronize(dev)
    return time.perf_counter() - t0, iters, x, w, st, pred


def objective_at(p: Problem, x: torch.Tensor, w: torch.Tensor):
    """||W Psi^dagger x||_1 and the worst constraint ratio at x."""
    xc = x.clone()
    st = purify_sdmm_solve(p.plan, p.y, p.eps, xc, w=w, max_iter=0, cg_iters=CG_ITERS, nu=p.nu, gamma=p.gamma)
    return st.objective, st.max_resid_over_eps


def snr_db(x_true: np.ndarray, x: torch.Tensor) -> float:
    return float(20 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x.cpu().numpy())))


def compare(p: Problem, plain, learned) -> dict:
    """The success test of a learned solve against the plain one (see the
    module docstring) and the figures it rests on."""
    t_p, it_p, x_p, w_p, _ = plain
    t_l, it_l, x_l, _, _, pred = learned
    obj_p, ratio_p = objective_at(p, x_p, w_p)
    obj_l, ratio_l = objective_at(p, x_l, w_p)
    snr_p, snr_l = snr_db(p.x_true, x_p), snr_db(p.x_true, x_l)
    ok = obj_l <= (1 + OBJ_TOL) * obj_p and ratio_l <= 1 + PASS_EPS_TOL and snr_l >= snr_p - SNR_TOL
    return {"t_plain": t_p, "it_plain": it_p, "t_learned": t_l, "it_learned": it_l,
            "obj_excess": obj_l / obj_p - 1.0, "ratio_plain": ratio_p, "ratio_learned": ratio_l,
            "snr_plain": snr_p, "snr_learned": snr_l, "snr_prediction": snr_db(p.x_true, pred),
            "reached": bool(ok)}


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


def build_training_set(dev, size: Size, n_samples: int, first_iters: int, pass_iters: int, seed0: int = TRAIN_SEED0):
    """Dirty images and SARA targets of seeds seed0 .. seed0 + n_samples - 1."""
    dirty, target = [], []
    for i in range(0, n_samples, 32):
        probs = [make_problem(seed0 + s, dev, size) for s in range(i, min(i + 32, n_samples))]
        sols = sara_targets(probs, dev, first_iters, pass_iters)
        for p, x in zip(probs, sols):
            dirty.append(p.dirty)
            target.append(x)
        for p in probs:
            p.plan.close()
    return torch.stack(dirty).contiguous(), torch.stack(target).contiguous()
