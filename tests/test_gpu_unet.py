"""GPU parity of the warm-start network's tensor-core kernels against the
FP64 oracle (the network is not in the paper; it only changes SDMM's start).
Inputs are rounded to BF16 before the oracle sees them, so the comparison
measures the FP32 accumulation of exact BF16 products."""
import numpy as np
import pytest
import torch

import paper_1502_05037_gb300 as pk
from gpu_util import DEV, rel
from oracle import unet as un

pytestmark = pytest.mark.gpu


def bf16_round(a: np.ndarray) -> np.ndarray:
    return torch.from_numpy(a.astype(np.float32)).bfloat16().float().numpy().astype(np.float64)


@pytest.mark.parametrize("B,H,W,Cin,Cout,k,relu", [
    (2, 16, 16, 1, 32, 3, True),
    (1, 32, 32, 32, 64, 3, False),
    (1, 8, 8, 64, 128, 3, True),
    (1, 16, 16, 96, 48, 3, False),
    (1, 12, 20, 256, 256, 3, True),
    (2, 8, 16, 32, 1, 1, False),
])
def test_conv2d_matches_oracle(B, H, W, Cin, Cout, k, relu):
    g = np.random.default_rng(B * 1000 + Cin + Cout)
    x = g.standard_normal((B, H, W, Cin)).astype(np.float32)
    w = (g.standard_normal((Cout, k, k, Cin)) / np.sqrt(k * k * Cin)).astype(np.float32)
    b = g.standard_normal(Cout).astype(np.float32)
    out = torch.empty((B, H, W, Cout), dtype=torch.float32, device=DEV)
    pk.purify_conv2d(torch.from_numpy(x).to(DEV), torch.from_numpy(w).to(DEV), torch.from_numpy(b).to(DEV), out, k,
                     relu)
    want = un.conv2d(bf16_round(x), bf16_round(w), b.astype(np.float64))
    if relu:
        want = un.relu(want)
    assert rel(out.cpu().numpy(), want) <= 1e-5
