"""GPU parity of the SARA dictionary Psi and its adjoint (Sec. 1) against the
FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, TOL, make_plan, np_real, rel, t_real
from oracle import wavelets as owv

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, levels, mask, dtype
    (64, 64, 3, 0, pk.PURIFY_F64),
    (256, 256, 4, 0, pk.PURIFY_F32),
    (32, 64, 3, 0, pk.PURIFY_F32),
    (8, 8, 3, 0, pk.PURIFY_F64),          # db8 on 2-sample bands: heavy wrapping
    (16, 16, 1, 0b11, pk.PURIFY_F32),
    (64, 32, 2, 0b100000001, pk.PURIFY_F64),
    (32, 32, 2, 0b1, pk.PURIFY_F32),       # Dirac only
    (128, 64, 5, 0b111111110, pk.PURIFY_F32),  # wavelets only
]


@pytest.mark.parametrize("nx,ny,levels,mask,dtype", CASES)
def test_psi_adj_matches_oracle(nx, ny, levels, mask, dtype):
    plan, _, _, _ = make_plan(nx, ny, 64, 4, levels=levels, dtype=dtype, mask=mask, seed=nx)
    q = plan.info.q
    x = np.random.default_rng(nx + ny).standard_normal((ny, nx)).astype(np_real(dtype))
    c = torch.empty((q, ny, nx), dtype=t_real(dtype), device=DEV)
    pk.purify_psi_adj(plan, torch.from_numpy(x).to(DEV), c)
    m = mask or owv.DEFAULT_MASK
    want = owv.psi_adj(x.astype(np.float64), levels, m)
    assert rel(c.cpu().numpy(), want) <= TOL[dtype]


@pytest.mark.parametrize("nx,ny,levels,mask,dtype", CASES)
def test_psi_matches_oracle(nx, ny, levels, mask, dtype):
    plan, _, _, _ = make_plan(nx, ny, 64, 4, levels=levels, dtype=dtype, mask=mask, seed=nx + 1)
    q = plan.info.q
    c = np.random.default_rng(nx * 3 + ny).standard_normal((q, ny, nx)).astype(np_real(dtype))
    x = torch.empty((ny, nx), dtype=t_real(dtype), device=DEV)
    pk.purify_psi(plan, torch.from_numpy(c).to(DEV), x)
    m = mask or owv.DEFAULT_MASK
    want = owv.psi(c.astype(np.float64), levels, m)
    assert rel(x.cpu().numpy(), want) <= TOL[dtype]


def test_tight_frame_on_gpu():
    nx = ny = 128
    plan, _, _, _ = make_plan(nx, ny, 64, 4, levels=4, seed=3)
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((ny, nx)).astype(np.float32)).to(DEV)
    c = torch.empty((plan.info.q, ny, nx), dtype=torch.float32, device=DEV)
    xr = torch.empty_like(x)
    pk.purify_psi_adj(plan, x, c)
    pk.purify_psi(plan, c, xr)
    assert rel(xr.cpu().numpy(), x.cpu().numpy()) <= 1e-6
    assert abs(c.double().norm().item() - x.double().norm().item()) <= 1e-6 * x.double().norm().item()


def test_full_size_1024_levels_5():
    nx = ny = 1024
    plan, _, _, _ = make_plan(nx, ny, 64, 6, levels=5, seed=5)
    x = np.random.default_rng(2).standard_normal((ny, nx)).astype(np.float32)
    c = torch.empty((plan.info.q, ny, nx), dtype=torch.float32, device=DEV)
    pk.purify_psi_adj(plan, torch.from_numpy(x).to(DEV), c)
    # plane-by-plane check on two bases (db1 and db8) plus the Dirac plane
    cc = c.cpu().numpy()
    for plane, p in ((1, 1), (8, 8)):
        want = owv.dwt2(x.astype(np.float64), p, 5) / 3.0
        assert rel(cc[plane], want) <= 1e-5
    assert rel(cc[0], x / 3.0) <= 1e-7
