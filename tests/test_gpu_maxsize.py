"""GPU parity at the largest sizes a plan accepts, element by element against
the FP64 oracle: images of 4096 x 4096 (the upper limit of nx and ny), so
oversampled grids of 8192 x 8192 and 8192-point FFTs (the longest transform),
and eight wavelet levels (the most a plan takes).

* F and F^H (the FFT of Phi = G F Z S, Sec. 1): K = 4096 and 8192, FP32 and
  FP64, both directions;
* Phi and Phi^dagger (Sec. 1, Eq. 1) at 4096 x 4096, M = 2^20 visibilities
  (30% uniform coverage, J = 6, R = 4 uneven blocks), in every gridding
  decomposition (autotuned, tile subproblems, run sets, lane pairs, and the
  deterministic lane form) and in an FP64 plan;
* Psi^dagger and Psi (the SARA dictionary, Sec. 1) at 4096 x 4096 with eight
  levels and all nine bases, FP32 and FP64.

Inputs are FP32-representable, so one oracle result serves both precisions.
FP32 tolerance: 2e-5 relative (twice the 1e-5 of the smaller cases), since the
FP32 rounding of the FFT grows with the number of stages (26 for an 8192^2
transform against 22 at 2048^2) and the fractional tap offsets are taken from
coordinates up to 4096 grid cells from the centre.
"""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, TOL, np_cplx, np_real, rel, t_cplx, t_real
from oracle import nufft as onf
from oracle import wavelets as owv
from paper_1502_05037_gb300 import synth

pytestmark = pytest.mark.gpu

NMAX = 4096
TOL_MAX = {pk.PURIFY_F32: 2e-5, pk.PURIFY_F64: TOL[pk.PURIFY_F64]}


def plan_for(u, v, offs, dtype, grid_mode=0, levels=3, J=6):
    return pk.Plan(NMAX, NMAX, torch.from_numpy(u.astype(np_real(dtype))).to(DEV),
                   torch.from_numpy(v.astype(np_real(dtype))).to(DEV), kb_width=J, levels=levels,
                   block_offsets=offs, dtype=dtype, grid_mode=grid_mode)


@pytest.mark.parametrize("K", [4096, 8192])
def test_fft2_longest_transforms(K):
    g = np.random.default_rng(K + 7)
    X = (g.standard_normal((K, K)) + 1j * g.standard_normal((K, K))).astype(np.complex64)
    X64 = X.astype(np.complex128)
    want = {False: onf.fft2(X64), True: onf.ifft2_unnormalised(X64)}
    del X64
    u = np.zeros(1, dtype=np.float32)
    for dtype in (pk.PURIFY_F32, pk.PURIFY_F64):
        plan = pk.Plan(K // 2, K // 2, torch.from_numpy(u.astype(np_real(dtype))).to(DEV),
                       torch.from_numpy(u.astype(np_real(dtype))).to(DEV), kb_width=4, levels=1, dtype=dtype)
        for inv in (False, True):
            t = torch.from_numpy(X.astype(np_cplx(dtype))).to(DEV)
            pk.purify_fft2(plan, t, inv)
            assert rel(t.cpu().numpy(), want[inv]) <= 3 * TOL_MAX[dtype], (K, dtype, inv)
            del t
        plan.close()
        torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def nufft_max():
    M, R = 1 << 20, 4
    u, v = synth.uv_coverage(M, 2000 + 4096, sigma=np.pi / 4, uniform_fraction=0.3, dtype=np.float32)
    offs = synth.block_offsets(synth.block_sizes(M, R, 4000 + 4096))
    x = synth.sky(NMAX, NMAX, 1000 + 4096, n_points=200, n_blobs=20).astype(np.float32)
    g = np.random.default_rng(4096)
    y = (g.standard_normal(M) + 1j * g.standard_normal(M)).astype(np.complex64)
    op = onf.NufftPlan(NMAX, NMAX, u.astype(np.float64), v.astype(np.float64), 6)
    want_phi = onf.phi(op, x.astype(np.float64))
    want_adj = onf.phi_adj(op, y.astype(np.complex128))
    return u, v, offs, x, y, want_phi, want_adj


@pytest.mark.parametrize("dtype,grid_mode", [
    (pk.PURIFY_F32, 0), (pk.PURIFY_F32, 1), (pk.PURIFY_F32, 2), (pk.PURIFY_F32, 4), (pk.PURIFY_F32, 6),
    (pk.PURIFY_F64, 0),
])
def test_phi_and_adjoint_at_the_largest_image(nufft_max, dtype, grid_mode):
    u, v, offs, x, y, want_phi, want_adj = nufft_max
    plan = plan_for(u, v, offs, dtype, grid_mode)
    if grid_mode:
        assert plan.info.grid_mode == grid_mode
    M = y.size
    yg = torch.empty(M, dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi(plan, torch.from_numpy(x.astype(np_real(dtype))).to(DEV), yg)
    assert rel(yg.cpu().numpy(), want_phi) <= TOL_MAX[dtype]
    del yg
    xa = torch.empty((NMAX, NMAX), dtype=t_cplx(dtype), device=DEV)
    pk.purify_phi_adj(plan, torch.from_numpy(y.astype(np_cplx(dtype))).to(DEV), xa)
    assert rel(xa.cpu().numpy(), want_adj) <= TOL_MAX[dtype]
    del xa
    plan.close()
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def wavelet_max():
    levels = 8
    g = np.random.default_rng(8)
    x = g.standard_normal((NMAX, NMAX)).astype(np.float32)
    c = g.standard_normal((len(owv.bases(owv.DEFAULT_MASK)), NMAX, NMAX)).astype(np.float32)
    want_c = owv.psi_adj(x.astype(np.float64), levels)
    want_x = owv.psi(c.astype(np.float64), levels)
    return levels, x, c, want_c, want_x


@pytest.mark.parametrize("dtype", [pk.PURIFY_F32, pk.PURIFY_F64])
def test_psi_pair_at_the_largest_image_and_depth(wavelet_max, dtype):
    levels, x, c, want_c, want_x = wavelet_max
    u = np.zeros(1, dtype=np.float32)
    plan = plan_for(u, u, None, dtype, levels=levels, J=4)
    q = plan.info.q
    assert q == c.shape[0]
    cg = torch.empty((q, NMAX, NMAX), dtype=t_real(dtype), device=DEV)
    pk.purify_psi_adj(plan, torch.from_numpy(x.astype(np_real(dtype))).to(DEV), cg)
    assert rel(cg.cpu().numpy(), want_c) <= TOL[dtype]
    cg.copy_(torch.from_numpy(c.astype(np_real(dtype))))
    xg = torch.empty((NMAX, NMAX), dtype=t_real(dtype), device=DEV)
    pk.purify_psi(plan, cg, xg)
    assert rel(xg.cpu().numpy(), want_x) <= TOL[dtype]
    del cg, xg
    plan.close()
    torch.cuda.empty_cache()
