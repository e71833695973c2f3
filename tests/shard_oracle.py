"""A shard for paper_1502_05037_gb300.sharded.ShardedSdmm computed by the
FP64 oracle on CPU (test helper): the five shard steps of the C ABI
(purify_shard_* in include/purify.h) written out with the oracle's
operators on one shard's blocks, the CG in the Chronopoulos-Gear arrangement
with the step scalars of the library (beta = gamma / gamma_prev,
alpha = gamma / (delta - beta gamma / alpha_prev))."""
import numpy as np
import torch

from oracle import sdmm


class OracleShard:
    def __init__(self, prob, blocks):
        self.prob = prob
        self.blocks = list(blocks)
        self.own = np.zeros(prob.plan.M, dtype=bool)
        for i in self.blocks:
            self.own[prob.offsets[i]:prob.offsets[i + 1]] = True
        n = prob.plan.nx * prob.plan.ny
        self.shape = (prob.plan.ny, prob.plan.nx)
        self.x = np.zeros(self.shape)
        self.z1 = np.zeros_like(prob.psi_adj(self.x))
        self.z2 = np.zeros(prob.plan.M, dtype=complex)
        self.z3 = np.zeros(self.shape)
        self.r = torch.zeros(n, dtype=torch.float64)
        self.u = torch.zeros(n, dtype=torch.float64)
        self.cg = {}

    # this shard's Re Phi_k^H (.) / nu of a visibility vector
    def _adj(self, v):
        return self.prob.phi_n_adj_re(np.where(self.own, v, 0.0))

    def _phi(self, x):
        return np.where(self.own, self.prob.phi_n(x), 0.0)

    def iterate_local(self, r_out):
        p, x = self.prob, self.x
        v1 = p.psi_adj(x)
        s1 = sdmm.soft_threshold(v1 + self.z1, p.gamma * p.w())
        self.z1 = self.z1 + v1 - s1
        v2 = self._phi(x)
        t2 = v2 + self.z2
        s2 = np.zeros_like(t2)
        yn = p.y / p.nu
        for i in self.blocks:
            a, b = p.offsets[i], p.offsets[i + 1]
            s2[a:b] = sdmm.proj_l2_ball(t2[a:b], yn[a:b], p.eps[i] / p.nu)
        self.z2 = self.z2 + v2 - s2
        s3 = sdmm.proj_positive(x + self.z3)
        self.z3 = self.z3 + x - s3
        self.addend = p.psi(s1 - self.z1) + (s3 - self.z3) - 2.0 * x
        r_out.copy_(torch.from_numpy(self._adj(s2 - self.z2 - v2).ravel()))

    def cg_begin(self, r_sum):
        self.rv = r_sum.numpy().reshape(self.shape) + self.addend
        self.pv = np.zeros(self.shape)
        self.sv = np.zeros(self.shape)
        self.uv = np.zeros(self.shape)
        self.stopped = False
        self.pending = None

    def _apply_pending(self):
        if self.pending is None or self.stopped:
            return
        al, be = self.pending
        self.pv = self.rv + be * self.pv
        self.sv = self.uv + be * self.sv
        self.x = self.x + al * self.pv
        self.rv = self.rv - al * self.sv
        self.pending = None

    def cg_apply(self, k, u_out):
        self._apply_pending()
        u_out.copy_(torch.from_numpy(self._adj(self._phi(self.rv)).ravel()))

    def cg_combine(self, k, u_sum):
        if self.stopped:
            return
        self.uv = 2.0 * self.rv + u_sum.numpy().reshape(self.shape)
        gam = float(np.sum(self.rv * self.rv))
        dlt = float(np.sum(self.rv * self.uv))
        if k == 0:
            be = 0.0
            al = gam / dlt if dlt > 0 else 0.0
        else:
            be = gam / self.cg["gam"] if self.cg["gam"] > 0 else 0.0
            den = dlt - (be * gam / self.cg["al"] if self.cg["al"] > 0 else 0.0)
            al = gam / den if den > 0 else 0.0
        self.cg = {"gam": gam, "al": al}
        if gam == 0.0:
            self.stopped = True
        else:
            self.pending = (al, be)

    def iterate_end(self, cg_steps):
        self._apply_pending()
