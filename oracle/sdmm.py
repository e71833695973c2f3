"""Oracle: prox operators, projections, CG, the SDMM iteration and SARA
reweighting for problem (3) of the paper (FP64, NumPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Problem (3) (Sec. 1, Eq. 3; the R = 1 case is Eq. 1):
    min_{x in R_+^N} || W Psi^dagger x ||_1
    subject to || y_i - Phi_i x ||_2 <= eps_i,  i = 1..R,
with y and Phi split into R contiguous row blocks (Eq. 2).

Solver: SDMM (simultaneous-direction method of multipliers, Combettes &
Pesquet 2011, "Proximal splitting methods in signal processing"; the paper
cites its own SDMM framework for this problem). The
functions and linear maps are
    f_1 = ||W .||_1 with L_1 = Psi^dagger,
    f_2 = indicator of {s : ||s_i - y_i|| <= eps_i for all i} with L_2 = Phi,
    f_3 = indicator of R_+^N with L_3 = I.
With the tight frame Psi Psi^dagger = I and real images, sum_j L_j^T L_j =
2 I + Re Phi^H Phi; the x-update solves that system by conjugate gradients.

Readings the paper leaves open (each shared with the CUDA path as a plan or
solver parameter):
* Scaling: the data term uses Phi / nu, y / nu, eps / nu with nu = ||Phi||_2
  (power iteration). The constraint set is unchanged; the CG system becomes
  2 I + Re Phi^H Phi / nu^2 with spectrum in [2, 3].
* Order inside one iteration (from the current x, z_j start at 0):
    1. v1 = Psi^dagger x;  s1 = soft(v1 + z1, gamma w);  z1 += v1 - s1
    2. v2 = Phi x / nu;    s2_i = proj_{B(y_i/nu, eps_i/nu)}(v2_i + z2_i);
                           z2 += v2 - s2
    3. s3 = max(x + z3, 0); z3 += x - s3
    4. x = CG solution of (2 I + Re Phi^H Phi / nu^2) x =
           Psi (s1 - z1) + Re Phi^H (s2 - z2) / nu + (s3 - z3),
       warm-started from the current x.
  This is the Combettes-Pesquet SDMM loop started from y_j = L_j x0, z_j = 0,
  whose first x-update returns x0, so it is the same sequence.
* gamma = 1e-3 max |Psi^dagger Re Phi^H y| / nu^2, computed once per problem.
* Ties: soft-thresholding at |v| = threshold gives 0; projecting a point
  with ||r|| = 0 returns the centre.
* eps_i = (sigma / sqrt 2) sqrt(2 M_i + 4 sqrt(M_i)) (mean plus two standard
  deviations of (sigma^2/2) chi^2_{2 M_i}), sigma = ||Phi x|| / sqrt(M) *
  10^(-SNR/20) for complex noise with E|n_m|^2 = sigma^2.
* SARA reweighting (Sec. 1: weights essentially the inverse of the previous
  solution's coefficients): w = rho / (rho + |Psi^dagger x|), rho_1 =
  std(Psi^dagger x^(0)), rho_{t+1} = rho_t / 2, each pass warm-started.
* Stochastic block-subset iterations (the paper's closing paragraph names
  using one data block or a subset of blocks per iteration as a way to lower
  the cost of an iteration): sdmm_iteration_groups, the blocks dealt
  round-robin into G groups, one group per iteration, its data term scaled
  by G in the x-update (see there).
* CG stopping (the paper names no rule): a fixed number of steps, or, with a
  tolerance, the first step at which ||r|| <= tol ||r_0||, r_0 the residual
  of the warm start of that x-update.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import nufft, wavelets


# ------------------------------------------------------------ closed forms
def soft_threshold(v: np.ndarray, thr) -> np.ndarray:
    """prox of thr*|.|: sign(v) max(|v| - thr, 0); exactly 0 at |v| = thr."""
    mag = np.abs(v) - thr
    return np.where(mag > 0, np.sign(v) * mag, 0.0)


def proj_l2_ball(v: np.ndarray, centre: np.ndarray, eps: float) -> np.ndarray:
    """Euclidean projection of v onto {s : ||s - centre||_2 <= eps}."""
    r = v - centre
    nr = float(np.sqrt(np.sum(np.abs(r) ** 2)))
    if nr <= eps:
        return np.array(v, copy=True)
    if nr == 0.0:
        return np.array(centre, copy=True)
    return centre + r * (eps / nr)


def proj_positive(v: np.ndarray) -> np.ndarray:
    return np.maximum(v, 0.0)


def noise_sigma(y_clean: np.ndarray, snr_db: float) -> float:
    return float(np.linalg.norm(y_clean) / np.sqrt(y_clean.size) * 10.0 ** (-snr_db / 20.0))


def epsilon_chi2(sigma: float, sizes: np.ndarray) -> np.ndarray:
    sizes = np.asarray(sizes, dtype=np.float64)
    return sigma / np.sqrt(2.0) * np.sqrt(2.0 * sizes + 4.0 * np.sqrt(sizes))


# -------------------------------------------------------------------- CG
def cg(apply_A, b: np.ndarray, x0: np.ndarray, iters: int, tol: float = 0.0):
    """Conjugate gradients on a symmetric positive definite system, warm
    started at x0. Runs `iters` iterations, stopping early when the residual
    norm reaches tol * ||r_0|| (tol > 0), r_0 = b - A x0 the residual of the
    warm start, or becomes exactly zero. Returns (x, iterations done, final
    residual norm)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    p = r.copy()
    rs = float(np.sum(r * r))
    r0norm = float(np.sqrt(rs))
    done = 0
    for _ in range(iters):
        if rs == 0.0 or (tol > 0.0 and np.sqrt(rs) <= tol * r0norm):
            break
        Ap = apply_A(p)
        alpha = rs / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rs_new = float(np.sum(r * r))
        p = r + (rs_new / rs) * p
        rs = rs_new
        done += 1
    return x, done, float(np.sqrt(rs))


# --------------------------------------------------------------- problem
@dataclass
class Problem:
    """Problem (3): operator, data, blocks, bounds and solver constants."""
    plan: nufft.NufftPlan
    levels: int
    y: np.ndarray                 # complex [M], caller order
    offsets: np.ndarray           # int64 [R+1], contiguous blocks (Eq. 2)
    eps: np.ndarray               # float [R]
    mask: int = wavelets.DEFAULT_MASK
    nu: float | None = None       # ||Phi||_2
    gamma: float | None = None
    weights: np.ndarray | None = None   # [q][ny][nx] or None for W = I
    normal: str = "nufft"               # CG normal operator: "nufft" or "exact"

    def __post_init__(self):
        self.y = np.asarray(self.y, dtype=np.complex128)
        self.offsets = np.asarray(self.offsets, dtype=np.int64)
        self.eps = np.asarray(self.eps, dtype=np.float64)
        if self.nu is None:
            self.nu = float(np.sqrt(nufft.power_norm_sq(self.plan)))
        if self.gamma is None:
            dirty = np.real(nufft.phi_adj(self.plan, self.y))
            self.gamma = 1e-3 * float(np.abs(self.psi_adj(dirty)).max()) / self.nu ** 2

    @property
    def R(self) -> int:
        return self.offsets.size - 1

    def psi_adj(self, x):
        return wavelets.psi_adj(x, self.levels, self.mask)

    def psi(self, c):
        return wavelets.psi(c, self.levels, self.mask)

    def phi_n(self, x):
        """Phi x / nu."""
        return nufft.phi(self.plan, x) / self.nu

    def phi_n_adj_re(self, y):
        """Re Phi^H y / nu."""
        return np.real(nufft.phi_adj(self.plan, y)) / self.nu

    def apply_A(self, x):
        """(2 I + Re Phi^H Phi / nu^2) x; with normal == "exact" the normal
        operator of the exact model (brute-force DFT) replaces the NUFFT one."""
        if self.normal == "exact":
            p = self.plan
            return 2.0 * x + np.real(nufft.phi_exact_adj(nufft.phi_exact(x, p.u, p.v), p.u, p.v, p.nx, p.ny)) / self.nu ** 2
        return 2.0 * x + self.phi_n_adj_re(self.phi_n(x))

    def w(self):
        if self.weights is None:
            return 1.0
        return self.weights


@dataclass
class State:
    x: np.ndarray
    z1: np.ndarray
    z2: np.ndarray
    z3: np.ndarray
    cg_iters: int = 0
    history: list = field(default_factory=list)


def init_state(prob: Problem, x0: np.ndarray) -> State:
    x0 = np.array(x0, dtype=np.float64, copy=True)
    q = len(wavelets.bases(prob.mask))
    return State(x=x0, z1=np.zeros((q,) + x0.shape), z2=np.zeros(prob.plan.M, dtype=np.complex128),
                 z3=np.zeros_like(x0))


def sdmm_iteration(prob: Problem, st: State, cg_iters: int, cg_tol: float = 0.0) -> State:
    """One SDMM iteration in the order stated in the module docstring."""
    x = st.x
    # f_1: weighted l1 on the analysis coefficients
    v1 = prob.psi_adj(x)
    s1 = soft_threshold(v1 + st.z1, prob.gamma * prob.w())
    st.z1 = st.z1 + v1 - s1
    # f_2: one l2 ball per data block (Eq. 3)
    v2 = prob.phi_n(x)
    t2 = v2 + st.z2
    s2 = np.empty_like(t2)
    yn = prob.y / prob.nu
    for i in range(prob.R):
        a, b = prob.offsets[i], prob.offsets[i + 1]
        s2[a:b] = proj_l2_ball(t2[a:b], yn[a:b], prob.eps[i] / prob.nu)
    st.z2 = st.z2 + v2 - s2
    # f_3: positive orthant
    s3 = proj_positive(x + st.z3)
    st.z3 = st.z3 + x - s3
    # x-update
    b = prob.psi(s1 - st.z1) + prob.phi_n_adj_re(s2 - st.z2) + (s3 - st.z3)
    x_new, done, _ = cg(prob.apply_A, b, x, cg_iters, cg_tol)
    st.cg_iters += done
    rel = float(np.linalg.norm(x_new - x) / max(np.linalg.norm(x_new), 1e-300))
    st.history.append({"rel_change": rel, "cg": done})
    st.x = x_new
    return st


def block_group(prob: Problem, g: int, G: int) -> list:
    """Blocks of group g when the R blocks are dealt round-robin into G
    groups: block i belongs to group i mod G."""
    return [i for i in range(prob.R) if i % G == g]


def sdmm_iteration_groups(prob: Problem, st: State, cg_iters: int, g: int, G: int,
                          cg_tol: float = 0.0) -> State:
    """One stochastic block-subset SDMM iteration (the paper's closing
    paragraph: use one data block, or a subset of blocks, per iteration).
    Reading: only the blocks i of group g (i mod G == g) take part; their
    data term, scaled by G so that its expectation over a uniformly drawn
    group is the full data term, replaces the full one in the x-update, and
    only their multipliers move:
        s1, z1 and s3, z3 as in sdmm_iteration;
        for i in the group: v2_i = Phi_i x / nu, s2_i = proj(v2_i + z2_i), z2_i += v2_i - s2_i;
        x = CG solution of (2 I + G Re sum_{i in group} Phi_i^H Phi_i / nu^2) x
            = Psi (s1 - z1) + (s3 - z3) + G sum_{i in group} Re Phi_i^H (s2_i - z2_i) / nu.
    With G = 1 (one group holding every block) this is sdmm_iteration."""
    x = st.x
    blocks = block_group(prob, g, G)
    mask = np.zeros(prob.plan.M)
    for i in blocks:
        mask[prob.offsets[i]:prob.offsets[i + 1]] = 1.0
    # f_1
    v1 = prob.psi_adj(x)
    s1 = soft_threshold(v1 + st.z1, prob.gamma * prob.w())
    st.z1 = st.z1 + v1 - s1
    # f_2 on the group's blocks
    v2 = prob.phi_n(x)
    yn = prob.y / prob.nu
    s2 = np.array(st.z2, copy=True)   # placeholder values outside the group (not used)
    z2 = np.array(st.z2, copy=True)
    for i in blocks:
        a, b = prob.offsets[i], prob.offsets[i + 1]
        s2[a:b] = proj_l2_ball(v2[a:b] + st.z2[a:b], yn[a:b], prob.eps[i] / prob.nu)
        z2[a:b] = st.z2[a:b] + v2[a:b] - s2[a:b]
    st.z2 = z2
    # f_3
    s3 = proj_positive(x + st.z3)
    st.z3 = st.z3 + x - s3
    # x-update with the group's data term, scaled by G
    b = prob.psi(s1 - st.z1) + G * prob.phi_n_adj_re(mask * (s2 - st.z2)) + (s3 - st.z3)

    def apply_group(v):
        return 2.0 * v + G * prob.phi_n_adj_re(mask * prob.phi_n(v))

    x_new, done, _ = cg(apply_group, b, x, cg_iters, cg_tol)
    st.cg_iters += done
    rel = float(np.linalg.norm(x_new - x) / max(np.linalg.norm(x_new), 1e-300))
    st.history.append({"rel_change": rel, "cg": done, "group": g})
    st.x = x_new
    return st


def objective(prob: Problem, x: np.ndarray) -> float:
    """|| W Psi^dagger x ||_1."""
    return float(np.sum(np.abs(prob.w() * prob.psi_adj(x))))


def residual_ratios(prob: Problem, x: np.ndarray) -> np.ndarray:
    """||y_i - Phi_i x|| / eps_i for each block."""
    r = prob.y - nufft.phi(prob.plan, x)
    out = np.empty(prob.R)
    for i in range(prob.R):
        a, b = prob.offsets[i], prob.offsets[i + 1]
        out[i] = np.linalg.norm(r[a:b]) / prob.eps[i]
    return out


def sdmm_solve(prob: Problem, x0: np.ndarray, iters: int, cg_iters: int,
               cg_tol: float = 0.0) -> State:
    st = init_state(prob, x0)
    for _ in range(iters):
        sdmm_iteration(prob, st, cg_iters, cg_tol)
    return st


def reweight(prob: Problem, x: np.ndarray, rho: float) -> np.ndarray:
    """SARA weights w = rho / (rho + |Psi^dagger x|)."""
    return rho / (rho + np.abs(prob.psi_adj(x)))


def sara(prob: Problem, x0: np.ndarray, iters: int, passes: int, cg_iters: int,
         cg_tol: float = 0.0) -> tuple[np.ndarray, list]:
    """Pass 0 with W = I, then `passes` reweighted passes, each warm-started
    from the previous solution. Returns (x, [rho_1, ...])."""
    prob.weights = None
    x = sdmm_solve(prob, x0, iters, cg_iters, cg_tol).x
    rho = float(np.std(prob.psi_adj(x)))
    rhos = []
    for _ in range(passes):
        prob.weights = reweight(prob, x, rho)
        rhos.append(rho)
        x = sdmm_solve(prob, x, iters, cg_iters, cg_tol).x
        rho *= 0.5
    return x, rhos


def snr_db(x_true: np.ndarray, x: np.ndarray) -> float:
    return float(20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x)))
