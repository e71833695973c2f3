"""Oracle: an independent primal-dual solver for problem (3). It pins the
SDMM oracle's converged objective value, and it is the reference of the GPU
primal-dual solver (purify_pd_solve), whose iterations follow these steps.
It is pinned by its first two iterations written out with the dense
measurement matrix and by its converged objective matching SDMM's.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Chambolle & Pock 2011 ("A first-order primal-dual algorithm for convex
problems with applications to imaging", Algorithm 1, theta = 1) applied to
    min_x  g(x) + f(K x),   K = [Psi^dagger; Phi_1/nu; ...; Phi_R/nu],
with g the indicator of R_+^N and f(v, s_1..s_R) = ||W v||_1 +
sum_i indicator(||s_i - y_i/nu|| <= eps_i/nu). Complex blocks are treated as
real vectors, so K^* (v, s) = Psi v + Re Phi^H s / nu and ||K||^2 <= 2.
Dual prox steps come from Moreau's identity:
    prox_{sigma f*}(p) = p - sigma prox_{f/sigma}(p / sigma),
which gives a clip to [-w, w] for the l1 part and
p - sigma proj_{B(c, eps)}(p / sigma) for each ball.
It shares no iteration with SDMM: no CG, no augmented Lagrangian.
"""
from __future__ import annotations

import numpy as np

from .sdmm import Problem, proj_l2_ball


def chambolle_pock(prob: Problem, iters: int, tau: float = 0.05, sigma: float = 9.8,
                   x0: np.ndarray | None = None) -> np.ndarray:
    """Run `iters` primal-dual iterations; tau * sigma * ||K||^2 < 1 with
    ||K||^2 <= 2 for the default steps."""
    ny, nx = prob.plan.ny, prob.plan.nx
    x = np.zeros((ny, nx)) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    xbar = x.copy()
    p1 = np.zeros_like(prob.psi_adj(x))
    p2 = np.zeros(prob.plan.M, dtype=np.complex128)
    w = prob.w()
    yn = prob.y / prob.nu
    for _ in range(iters):
        # dual ascent on the l1 term: clip to the weighted l-infinity ball
        p1 = np.clip(p1 + sigma * prob.psi_adj(xbar), -w, w)
        # dual ascent on the ball constraints
        q = p2 + sigma * prob.phi_n(xbar)
        for i in range(prob.R):
            a, b = prob.offsets[i], prob.offsets[i + 1]
            q[a:b] = q[a:b] - sigma * proj_l2_ball(q[a:b] / sigma, yn[a:b], prob.eps[i] / prob.nu)
        p2 = q
        # primal descent with positivity
        x_new = np.maximum(x - tau * (prob.psi(p1) + prob.phi_n_adj_re(p2)), 0.0)
        xbar = 2.0 * x_new - x
        x = x_new
    return x
