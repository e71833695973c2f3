"""Pins for the oracle's prox operators, projections, CG and SDMM (CPU only).

The closed forms are checked against their defining variational properties;
CG against a dense direct solve; SDMM's converged point against the
Karush-Kuhn-Tucker conditions and Fenchel duality of problem (3) (Sec. 1,
Eq. 3), and against an independent Chambolle-Pock solve.
"""
import numpy as np
import pytest
import scipy.stats

from oracle import nufft as nf
from oracle import primal_dual, sdmm, wavelets
from paper_1502_05037_gb300 import synth


# ------------------------------------------------------------ prox / proj
def test_soft_threshold_closed_form_and_tie():
    v = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.5])
    s = sdmm.soft_threshold(v, 1.0)
    assert np.array_equal(s, [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.5])


def test_soft_threshold_is_prox_of_weighted_l1():
    # s minimises 0.5 (s - v)^2 + t |s| elementwise: check against a fine scan
    g = np.random.default_rng(0)
    v = g.standard_normal(50) * 2
    t = np.abs(g.standard_normal(50))
    s = sdmm.soft_threshold(v, t)
    grid = np.linspace(-8, 8, 160001)
    for vi, ti, si in zip(v, t, s):
        obj = 0.5 * (grid - vi) ** 2 + ti * np.abs(grid)
        assert abs(grid[np.argmin(obj)] - si) <= 2e-4


def test_moreau_decomposition():
    # v = prox_{t|.|}(v) + t * proj_{[-1,1]}(v / t)
    g = np.random.default_rng(1)
    v = g.standard_normal(1000) * 3
    t = 0.7
    assert np.allclose(sdmm.soft_threshold(v, t) + t * np.clip(v / t, -1, 1), v, atol=1e-14)


def test_projection_properties():
    g = np.random.default_rng(2)
    c = g.standard_normal(40) + 1j * g.standard_normal(40)
    eps = 1.5
    inside = c + 0.1 * (g.standard_normal(40) + 1j * g.standard_normal(40)) / 10
    assert np.array_equal(sdmm.proj_l2_ball(inside, c, eps), inside)
    out = c + 5 * (g.standard_normal(40) + 1j * g.standard_normal(40))
    p = sdmm.proj_l2_ball(out, c, eps)
    assert abs(np.linalg.norm(p - c) - eps) < 1e-12
    assert np.allclose(sdmm.proj_l2_ball(p, c, eps), p, atol=1e-14)
    # variational inequality Re <out - p, s - p> <= 0 for points s in the ball
    for _ in range(50):
        d = g.standard_normal(40) + 1j * g.standard_normal(40)
        s = c + d / np.linalg.norm(d) * eps * g.uniform()
        assert np.real(np.vdot(out - p, s - p)) <= 1e-10
    assert np.array_equal(sdmm.proj_l2_ball(c, c, 0.0), c)


def test_positive_projection():
    v = np.array([-1.0, 0.0, 2.0])
    assert np.array_equal(sdmm.proj_positive(v), [0.0, 0.0, 2.0])


def test_epsilon_is_chi2_mean_plus_two_std():
    # (2/sigma^2) eps^2 = 2M + 4 sqrt(M): the chi^2_{2M} mean plus two std
    sigma = 0.3
    for M in (10, 1000, 100000):
        e = sdmm.epsilon_chi2(sigma, np.array([M]))[0]
        k = 2 * M
        assert abs(2 * e * e / sigma ** 2 - (scipy.stats.chi2.mean(k) + 2 * scipy.stats.chi2.std(k))) < 1e-6 * k


def test_epsilon_bounds_noise_norm_usually():
    sigma = 0.2
    sizes = np.array([500] * 200)
    eps = sdmm.epsilon_chi2(sigma, sizes)
    hits = 0
    for i in range(200):
        n = sigma * synth.unit_noise(500, 10 + i)
        hits += np.linalg.norm(n) <= eps[i]
    assert hits >= 180  # ~97.7% expected


# -------------------------------------------------------------------- CG
def _tiny_problem(n=8, M=80, R=2, J=4, levels=2, mask=0b111, seed=3):
    x = synth.sky(n, n, seed, n_points=4, n_blobs=1)
    u, v = synth.uv_coverage(M, seed + 1, sigma=1.2)
    p = nf.NufftPlan(n, n, u, v, J)
    y0 = nf.phi(p, x)
    s = sdmm.noise_sigma(y0, 30.0)
    offs = synth.block_offsets(synth.block_sizes(M, R, seed + 2))
    y = y0 + s * synth.unit_noise(M, seed + 3)
    eps = sdmm.epsilon_chi2(s, np.diff(offs))
    return sdmm.Problem(p, levels, y, offs, eps, mask=mask), x


def test_cg_matches_dense_solve():
    n = 16
    u, v = synth.uv_coverage(300, 11, sigma=1.0)
    p = nf.NufftPlan(n, n, u, v, 4)
    A = nf.phi_matrix(p)
    nu2 = nf.power_norm_sq(p, iters=200)
    Ad = 2 * np.eye(n * n) + np.real(A.conj().T @ A) / nu2
    b = np.random.default_rng(12).standard_normal(n * n)
    want = np.linalg.solve(Ad, b)
    apply = lambda x: (Ad @ x.ravel()).reshape(x.shape)
    got, done, res = sdmm.cg(apply, b.reshape(n, n), np.zeros((n, n)), 200, 1e-14)
    assert np.linalg.norm(got.ravel() - want) <= 1e-12 * np.linalg.norm(want)
    # the operator form the solver uses is the same matrix
    prob_A = lambda x: 2 * x + np.real(nf.phi_adj(p, nf.phi(p, x))) / nu2
    xr = np.random.default_rng(13).standard_normal((n, n))
    assert np.allclose(prob_A(xr).ravel(), Ad @ xr.ravel(), atol=1e-10)


def test_cg_fixed_iterations_and_zero_residual():
    apply = lambda x: 3.0 * x
    b = np.ones(5)
    x, done, res = sdmm.cg(apply, b, b / 3.0, 10)
    assert done == 0 and res == 0.0
    x, done, res = sdmm.cg(apply, b, np.zeros(5), 1)
    assert done == 1 and np.allclose(x, b / 3.0)


def test_cg_tolerance_is_relative_to_the_warm_start_residual():
    # Independent of the recurrences: the k-th CG iterate from x0 is the
    # Galerkin solution over x0 + K_k(A, r0), computed here from an
    # orthonormal Krylov basis; the stop is the first k with
    # ||r_k|| <= tol ||r0||, a different k than ||b|| would give.
    n = 12
    d = np.linspace(1.0, 9.0, n)
    A = np.diag(d)
    apply = lambda x: d * x
    rng = np.random.default_rng(21)
    b = rng.standard_normal(n)
    x0 = np.linalg.solve(A, b) + 1e-3 * rng.standard_normal(n)   # ||r0|| << ||b||
    r0 = b - A @ x0
    tol = 1e-2

    def galerkin(k):
        K = np.stack([np.linalg.matrix_power(A, j) @ r0 for j in range(k)], axis=1)
        V, _ = np.linalg.qr(K)
        c = np.linalg.solve(V.T @ A @ V, V.T @ r0)
        return x0 + V @ c

    want_k = next(k for k in range(1, n + 1)
                  if np.linalg.norm(b - A @ galerkin(k)) <= tol * np.linalg.norm(r0))
    assert np.linalg.norm(r0) <= tol * np.linalg.norm(b)   # a ||b|| rule would stop at 0
    x, done, res = sdmm.cg(apply, b, x0, 50, tol)
    assert done == want_k
    assert np.allclose(x, galerkin(want_k), rtol=0, atol=1e-12 * np.abs(x).max())
    assert res <= tol * np.linalg.norm(r0) and np.isclose(res, np.linalg.norm(b - A @ x), rtol=1e-8)


# ------------------------------------------------------------------ SDMM
def _dual_certificate(prob, st):
    """Fenchel dual value and feasibility residual from SDMM's multipliers
    u_j = z_j / gamma (problem (3) in its normalised form)."""
    g = prob.gamma
    u1, u2, u3 = st.z1 / g, st.z2 / g, st.z3 / g
    yn = prob.y / prob.nu
    dual = 0.0
    for i in range(prob.R):
        a, b = prob.offsets[i], prob.offsets[i + 1]
        dual -= np.real(np.vdot(u2[a:b], yn[a:b])) + prob.eps[i] / prob.nu * np.linalg.norm(u2[a:b])
    feas = prob.psi(u1) + prob.phi_n_adj_re(u2) + u3
    return dual, u1, u3, np.linalg.norm(feas) / np.linalg.norm(prob.psi(u1))


@pytest.fixture(scope="module")
def converged():
    prob, x_true = _tiny_problem()
    prob.gamma *= 10.0   # any gamma > 0 converges; this one converges fast here
    st = sdmm.sdmm_solve(prob, np.zeros((8, 8)), 700, 30, 1e-12)
    return prob, st, x_true


def test_sdmm_kkt_and_duality_gap(converged):
    prob, st, _ = converged
    primal = sdmm.objective(prob, st.x)
    dual, u1, u3, feas = _dual_certificate(prob, st)
    assert np.all(np.abs(u1) <= 1 + 1e-9)            # u1 in the subdifferential box
    assert np.all(u3 <= 1e-12)                         # normal cone of R_+
    assert np.all(np.abs(u3[st.x > 1e-8]) <= 1e-6 * np.abs(u3).max() + 1e-12)
    assert feas <= 1e-7                                # sum_j L_j^T u_j = 0
    assert abs(primal - dual) <= 1e-9 * primal         # strong duality
    ratios = sdmm.residual_ratios(prob, st.x)
    assert np.all(ratios <= 1 + 1e-8)                  # constraints of Eq. 3
    assert st.x.min() >= -1e-8                         # positive orthant


def test_sdmm_objective_matches_chambolle_pock(converged):
    prob, st, _ = converged
    xc = primal_dual.chambolle_pock(prob, 6000, tau=0.05, sigma=9.8)
    oc, os_ = sdmm.objective(prob, xc), sdmm.objective(prob, st.x)
    assert abs(oc - os_) <= 1e-5 * os_
    assert np.all(sdmm.residual_ratios(prob, xc) <= 1 + 1e-3)
    assert np.linalg.norm(xc - st.x) <= 1e-2 * np.linalg.norm(st.x)


def test_chambolle_pock_first_two_iterations_by_hand():
    # Algorithm 1 of Chambolle & Pock with theta = 1, written out with the
    # dense measurement matrix: iteration 1 from x = 0 and iteration 2 from the
    # extrapolated point 2 x_1 (this pins the extrapolation, the signs of the
    # Moreau steps and the clip)
    prob, _ = _tiny_problem(R=1)
    tau, sigma = 0.05, 9.8
    A = nf.phi_matrix(prob.plan) / prob.nu
    yn, en = prob.y / prob.nu, prob.eps[0] / prob.nu

    def ball(t):
        d = t - yn
        nd = np.linalg.norm(d)
        return t if nd <= en else yn + d * (en / nd)

    def adj_re(s):
        return np.real(A.conj().T @ s).reshape(prob.plan.ny, prob.plan.nx)

    p2 = -sigma * ball(np.zeros(prob.plan.M, dtype=complex))
    x1 = np.maximum(-tau * adj_re(p2), 0.0)
    xb = 2.0 * x1
    p1 = np.clip(sigma * prob.psi_adj(xb), -1.0, 1.0)
    q = p2 + sigma * (A @ xb.ravel())
    p2 = q - sigma * ball(q / sigma)
    x2 = np.maximum(x1 - tau * (prob.psi(p1) + adj_re(p2)), 0.0)
    got = primal_dual.chambolle_pock(prob, 2, tau=tau, sigma=sigma)
    assert np.abs(x1).max() > 0 and np.abs(x2 - x1).max() > 0
    assert np.allclose(got, x2, rtol=0, atol=1e-12 * np.abs(x2).max())


def test_sdmm_first_iteration_from_zero_by_hand():
    # from x = 0, z = 0: s1 = 0, s3 = 0 and s2 = projection of 0 onto each
    # ball, z2 = -s2, so the CG right-hand side is Re Phi^H (s2 - z2) / nu
    # = 2 Re Phi^H s2 / nu
    prob, _ = _tiny_problem(R=1)
    st = sdmm.init_state(prob, np.zeros((8, 8)))
    sdmm.sdmm_iteration(prob, st, 50, 1e-14)
    yn = prob.y / prob.nu
    en = prob.eps[0] / prob.nu
    s2 = yn - yn * (en / np.linalg.norm(yn))        # centre + r eps/||r||, r = -yn
    b = prob.phi_n_adj_re(2.0 * s2)
    want, _, _ = sdmm.cg(prob.apply_A, b, np.zeros((8, 8)), 200, 1e-14)
    assert np.allclose(st.x, want, atol=1e-10 * np.abs(want).max())
    assert np.allclose(st.z2, -s2, atol=1e-14)


def _log_sum(c, rho):
    """The log-sum sparsity penalty rho sum_d log(rho + c_d) of magnitudes
    c_d = |coefficient| (evaluated as given, also slightly below 0), whose
    majorise-minimise steps are reweighted l1 problems (Candes, Wakin & Boyd
    2008); the paper (Sec. 1) describes the weights as essentially the
    inverse of the previous solution's coefficients."""
    return rho * float(np.sum(np.log(rho + np.asarray(c))))


def test_reweight_is_the_log_sum_slope():
    # the weights are the derivative of the log-sum penalty in |c_d| at the
    # previous solution's coefficients: a central difference in each
    # coefficient magnitude (a dropped rho, a square or a missing |.| fails)
    prob, x = _tiny_problem()
    c = prob.psi_adj(x)
    for rho in (0.03, 0.1, 0.7):
        w = sdmm.reweight(prob, x, rho)
        assert w.shape == c.shape
        # the penalty's term rho log(rho + a) is analytic in a > -rho, so a
        # symmetric difference also holds at a = 0
        h = 1e-5 * rho
        a = np.abs(c).ravel()
        term = lambda t: rho * np.log(rho + t)
        slope = (term(a + h) - term(a - h)) / (2 * h)
        assert np.max(np.abs(w.ravel() - slope)) <= 1e-8
        # and the whole penalty's change for one coefficient moved by +-h
        for d in np.random.default_rng(5).choice(a.size, 20, replace=False):
            up, dn = a.copy(), a.copy()
            up[d] += h
            dn[d] -= h
            fd = (_log_sum(up, rho) - _log_sum(dn, rho)) / (2 * h)
            assert abs(w.ravel()[d] - fd) <= 1e-5
    # x = 0: every coefficient is zero and every weight one
    assert np.array_equal(sdmm.reweight(prob, np.zeros_like(x), 0.2), np.ones_like(c))


def test_reweight_majorises_the_log_sum_penalty():
    # concavity: for every c, penalty(c) <= penalty(c_t) + sum w_t (|c| - |c_t|)
    # with w_t the weights at c_t, so the weighted l1 problem majorises it
    prob, x = _tiny_problem(seed=4)
    ct = prob.psi_adj(x)
    rho = 0.05
    wt = sdmm.reweight(prob, x, rho)
    g = np.random.default_rng(6)
    for _ in range(50):
        c = ct + g.standard_normal(ct.shape) * g.choice([1e-3, 0.1, 1.0])
        bound = _log_sum(np.abs(ct), rho) + float(np.sum(wt * (np.abs(c) - np.abs(ct))))
        assert _log_sum(np.abs(c), rho) <= bound + 1e-12


def test_reweighted_pass_does_not_increase_the_log_sum_penalty():
    # majorise-minimise descent: solving the problem weighted at x_0 from x_0
    # lowers the log-sum penalty of the analysis coefficients (x_0 is
    # feasible, so the weighted l1 minimiser is at most its value)
    prob, _ = _tiny_problem(seed=21)
    x0 = sdmm.sdmm_solve(prob, np.zeros((8, 8)), 400, 20).x
    assert np.all(sdmm.residual_ratios(prob, x0) <= 1.0 + 1e-3)
    rho = float(np.std(prob.psi_adj(x0)))
    prob.weights = sdmm.reweight(prob, x0, rho)
    x1 = sdmm.sdmm_solve(prob, x0, 400, 20).x
    assert np.all(sdmm.residual_ratios(prob, x1) <= 1.0 + 1e-3)
    assert _log_sum(np.abs(prob.psi_adj(x1)), rho) < _log_sum(np.abs(prob.psi_adj(x0)), rho)


def test_sara_reweighting_keeps_feasibility():
    prob, x_true = _tiny_problem(seed=21)
    x, rhos = sdmm.sara(prob, np.zeros((8, 8)), 300, passes=2, cg_iters=20)
    assert len(rhos) == 2 and rhos[1] == rhos[0] / 2
    assert np.all(sdmm.residual_ratios(prob, x) <= 1.01)
    assert x.min() >= -1e-6


def test_block_offsets_partition():
    for M, R, seed in ((100, 7, 1), (655360, 8, 4001), (50, 50, 2)):
        s = synth.block_sizes(M, R, seed)
        assert s.sum() == M and s.min() >= 1 and s.size == R


# ---------------------------------------------- block-subset iterations
def test_one_group_is_plain_sdmm():
    # G = 1: one group holding every block, the data term unscaled: the same
    # iterates as plain SDMM, bit for bit
    prob, _ = _tiny_problem(R=3, seed=31)
    a = sdmm.init_state(prob, np.zeros((8, 8)))
    b = sdmm.init_state(prob, np.zeros((8, 8)))
    for _ in range(4):
        sdmm.sdmm_iteration(prob, a, 12)
        sdmm.sdmm_iteration_groups(prob, b, 12, 0, 1)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.z2, b.z2) and np.array_equal(a.z1, b.z1)


def test_group_iteration_against_dense_restricted_system():
    # the x-update of a group iteration solves (2 I + G Re Phi_g^H Phi_g / nu^2) x = b
    # with the group's rows of the dense measurement matrix; blocks outside the
    # group keep their multipliers
    prob, _ = _tiny_problem(R=4, M=120, seed=32)
    G, g = 2, 1
    st = sdmm.init_state(prob, np.zeros((8, 8)))
    sdmm.sdmm_iteration(prob, st, 30, 1e-14)            # a non-trivial state
    x0, z1, z2, z3 = st.x.copy(), st.z1.copy(), st.z2.copy(), st.z3.copy()
    sdmm.sdmm_iteration_groups(prob, st, 200, g, G, 1e-14)
    A = nf.phi_matrix(prob.plan) / prob.nu
    rows = np.zeros(prob.plan.M, dtype=bool)
    for i in sdmm.block_group(prob, g, G):
        rows[prob.offsets[i]:prob.offsets[i + 1]] = True
    Ag = A[rows]
    n = 64
    # s and z of the iteration, written out from the definitions
    v1 = prob.psi_adj(x0)
    s1 = sdmm.soft_threshold(v1 + z1, prob.gamma)
    z1n = z1 + v1 - s1
    v2 = A @ x0.ravel()
    yn = prob.y / prob.nu
    z2n = z2.copy()
    s2 = np.zeros_like(z2)
    for i in sdmm.block_group(prob, g, G):
        a, b_ = prob.offsets[i], prob.offsets[i + 1]
        s2[a:b_] = sdmm.proj_l2_ball(v2[a:b_] + z2[a:b_], yn[a:b_], prob.eps[i] / prob.nu)
        z2n[a:b_] = z2[a:b_] + v2[a:b_] - s2[a:b_]
    s3 = np.maximum(x0 + z3, 0.0)
    z3n = z3 + x0 - s3
    rhs = prob.psi(s1 - z1n).ravel() + G * np.real(Ag.conj().T @ (s2 - z2n)[rows]) + (s3 - z3n).ravel()
    Ad = 2 * np.eye(n) + G * np.real(Ag.conj().T @ Ag)
    want = np.linalg.solve(Ad, rhs).reshape(8, 8)
    assert np.allclose(st.x, want, atol=1e-9 * np.abs(want).max())
    out = ~rows
    assert np.array_equal(st.z2[out], z2[out])
    assert np.allclose(st.z2[rows], z2n[rows], atol=1e-13)


def test_group_data_term_is_unbiased():
    # averaged over the G groups, the scaled group data terms are the full
    # data term: sum_g G Phi_g^H Phi_g / G = Phi^H Phi
    prob, _ = _tiny_problem(R=5, M=150, seed=33)
    A = nf.phi_matrix(prob.plan)
    G = 3
    acc = np.zeros((64, 64))
    for g in range(G):
        rows = np.zeros(prob.plan.M, dtype=bool)
        for i in sdmm.block_group(prob, g, G):
            rows[prob.offsets[i]:prob.offsets[i + 1]] = True
        acc += G * np.real(A[rows].conj().T @ A[rows]) / G
    assert np.allclose(acc, np.real(A.conj().T @ A), atol=1e-10 * np.abs(acc).max())
    assert sorted(i for g in range(G) for i in sdmm.block_group(prob, g, G)) == list(range(5))
