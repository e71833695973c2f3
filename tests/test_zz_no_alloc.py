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
    with pytest.raises(pk.PurifyError) as e:
        pk.purify_psi_adj_static(big, big, 1024, 1024, 3, 0, pk.PURIFY_F32)
    assert e.value.status == pk._lib.PURIFY_EINVAL
    with pytest.raises(pk.PurifyError):
        pk.purify_psi_adj_static(x.cpu().numpy(), got, nx, ny, 3, 0, pk.PURIFY_F32)
