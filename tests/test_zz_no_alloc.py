"""The allocation-free Psi^dagger entry point against the plan-based one.

purify_psi_adj_static serves callers that cannot call cudaMalloc (a host
callback on a stream, a process whose device memory another allocator has
reserved, a loop that must not allocate after start-up): its wavelet scratch
is a file-scope device array instead of plan workspaces. This file is named
so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, TOL, make_plan, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [pk.PURIFY_F32, pk.PURIFY_F64])
def test_static_scratch_matches_plan_entry_point_twice(dtype):
    nx, ny, levels = 128, 64, 4
    tr = torch.float32 if dtype == pk.PURIFY_F32 else torch.float64
    plan, _, _, _ = make_plan(nx, ny, 64, 4, levels=levels, dtype=dtype, seed=3)
    q = plan.info.q
    g = np.random.default_rng(11)
    # two calls in a row with different inputs: the second must not see the
    # first call's scratch contents
    for k in range(2):
        x = torch.from_numpy(g.standard_normal((ny, nx))).to(tr).to(DEV)
        want = torch.empty((q, ny, nx), dtype=tr, device=DEV)
        pk.purify_psi_adj(plan, x, want)
        got = torch.full((q, ny, nx), float("nan"), dtype=tr, device=DEV)
        pk.purify_psi_adj_static(x, got, nx, ny, levels, 0, dtype)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert rel(got.cpu().numpy(), want.cpu().numpy()) <= TOL[dtype]


def test_static_scratch_limits_and_masks():
    # partial basis sets, and sizes beyond the static array are rejected
    nx = ny = 64
    plan, _, _, _ = make_plan(nx, ny, 64, 4, levels=3, mask=0b100000011, seed=4)
    x = torch.from_numpy(np.random.default_rng(5).standard_normal((ny, nx)).astype(np.float32)).to(DEV)
    want = torch.empty((plan.info.q, ny, nx), dtype=torch.float32, device=DEV)
    pk.purify_psi_adj(plan, x, want)
    got = torch.empty_like(want)
    pk.purify_psi_adj_static(x, got, nx, ny, 3, 0b100000011, pk.PURIFY_F32)
    assert rel(got.cpu().numpy(), want.cpu().numpy()) <= TOL[pk.PURIFY_F32]
    big = torch.empty((1024, 1024), dtype=torch.float32, device=DEV)
    bigc = torch.empty((9, 1024, 1024), dtype=torch.float32, device=DEV)
    with pytest.raises(pk.PurifyError) as e:
        pk.purify_psi_adj_static(big, bigc, 1024, 1024, 3, 0, pk.PURIFY_F32)
    assert e.value.status == pk._lib.PURIFY_EINVAL
    with pytest.raises(pk.PurifyError):
        pk.purify_psi_adj_static(x.cpu().numpy(), got, nx, ny, 3, 0b100000011, pk.PURIFY_F32)   # host x


@pytest.mark.parametrize("dtype,nx,ny,levels,mask", [
    (pk.PURIFY_F32, 128, 64, 4, 0),
    (pk.PURIFY_F64, 128, 64, 4, 0),
    (pk.PURIFY_F32, 8, 8, 3, 0b100000001),      # db8 at 8 x 8: the filter wraps the band several times
    (pk.PURIFY_F64, 8, 8, 3, 0b100000001),
    (pk.PURIFY_F32, 512, 512, 5, 0),            # the largest FP32 square with every wavelet
    (pk.PURIFY_F64, 512, 256, 5, 0),            # the largest FP64 size with every wavelet
])
def test_static_scratch_matches_oracle(dtype, nx, ny, levels, mask):
    from oracle import wavelets as owv
    tr = torch.float32 if dtype == pk.PURIFY_F32 else torch.float64
    x = np.random.default_rng(nx + ny + levels).standard_normal((ny, nx))
    xt = torch.from_numpy(x).to(tr).to(DEV)
    want = owv.psi_adj(xt.cpu().numpy().astype(np.float64), levels, mask if mask else 0x1FF)
    got = torch.empty((want.shape[0], ny, nx), dtype=tr, device=DEV)
    for _ in range(2):
        got.fill_(float("nan"))
        pk.purify_psi_adj_static(xt, got, nx, ny, levels, mask, dtype)
        assert rel(got.cpu().numpy(), want) <= TOL[dtype]


def test_static_scratch_limit_edges_and_buffer_checks():
    # one step past the stated limits is rejected before any launch; short or
    # mistyped buffers are caught by the binding (the C side cannot see sizes)
    for dtype, nx, ny in ((pk.PURIFY_F32, 1024, 512), (pk.PURIFY_F64, 512, 512)):
        tr = torch.float32 if dtype == pk.PURIFY_F32 else torch.float64
        x = torch.zeros((ny, nx), dtype=tr, device=DEV)
        c = torch.zeros((9, ny, nx), dtype=tr, device=DEV)
        with pytest.raises(pk.PurifyError) as e:
            pk.purify_psi_adj_static(x, c, nx, ny, 3, 0, dtype)
        assert e.value.status == pk._lib.PURIFY_EINVAL
    x = torch.zeros((32, 32), dtype=torch.float32, device=DEV)
    with pytest.raises(ValueError):
        pk.purify_psi_adj_static(x, torch.zeros((8, 32, 32), dtype=torch.float32, device=DEV), 32, 32, 2)
    with pytest.raises(ValueError):
        pk.purify_psi_adj_static(x, torch.zeros((9, 32, 32), dtype=torch.float64, device=DEV), 32, 32, 2)
