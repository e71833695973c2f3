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


def oracle_params_from_flat(flat, levels, base):
    """Split the library's flat parameter vector by the oracle's layer list."""
    params, off = {}, 0
    for name, cout, k, cin in un.layer_shapes(levels, base):
        nw = cout * k * k * cin
        params[name + ".w"] = flat[off:off + nw].reshape(cout, k, k, cin).astype(np.float64)
        off += nw
        params[name + ".b"] = flat[off:off + cout].astype(np.float64)
        off += cout
    assert off == flat.size
    return params


def flat_from_oracle(grads, levels, base):
    return np.concatenate([np.concatenate([grads[n + ".w"].ravel(), grads[n + ".b"].ravel()])
                           for n, *_ in un.layer_shapes(levels, base)])


@pytest.fixture(scope="module")
def small_net():
    levels, base, H, W, B = 3, 8, 32, 32, 2
    net = pk.Unet(H, W, levels, base, max_batch=B, seed=5)
    flat = np.empty(net.num_params, dtype=np.float32)
    net.get_params(flat)
    g = np.random.default_rng(6)
    # non-zero biases exercise the bias path
    params = oracle_params_from_flat(flat, levels, base)
    for k in params:
        if k.endswith(".b"):
            params[k] = g.standard_normal(params[k].shape) * 0.05
    flat = flat_from_oracle(params, levels, base).astype(np.float32)
    net.set_params(flat)
    params = oracle_params_from_flat(flat, levels, base)
    x = g.standard_normal((B, H, W)).astype(np.float32)
    t = g.standard_normal((B, H, W)).astype(np.float32)
    return net, params, x, t, levels, base


def test_unet_forward_matches_oracle(small_net):
    net, params, x, t, levels, base = small_net
    xd = torch.from_numpy(x).to(DEV)
    y = torch.empty_like(xd)
    net.forward(xd, y)
    pred, _ = un.forward(params, x[..., None].astype(np.float64), levels, base)
    # compare the network's correction (output minus the residual input)
    assert rel(y.cpu().numpy() - x, pred[..., 0] - x) <= 3e-2


def test_unet_forward_matches_bf16_rounded_oracle(small_net):
    # The oracle rounds to BF16 exactly where the CUDA path stores tensor-core
    # operands (the input, the weights, every ReLU output; pooling, upsampling
    # and concatenation move rounded values unchanged). What is left is FP32
    # against FP64 accumulation, and the few BF16 roundings and ReLU or
    # pooling choices that difference flips: each moves one activation by at
    # most one BF16 unit (2^-8 relative), far below this bound, while a wrong
    # tap, channel or skip connection changes the correction by O(1).
    net, params, x, t, levels, base = small_net
    xd = torch.from_numpy(x).to(DEV)
    y = torch.empty_like(xd)
    net.forward(xd, y)
    pred, _ = un.forward(params, x[..., None].astype(np.float64), levels, base, q=bf16_round)
    assert rel(y.cpu().numpy() - x, pred[..., 0] - x) <= 5e-3


@pytest.mark.parametrize("rounding,tol_layer,tol_all", [("bf16", 3e-2, 1.5e-2), ("fp64", 2e-1, 5e-2)])
def test_unet_gradients_match_oracle(small_net, rounding, tol_layer, tol_all):
    # "bf16": the oracle rounds where the CUDA path stores BF16 tensor-core
    # operands (weights, input, ReLU outputs, gradients entering a backward
    # convolution), so only accumulation order, and the BF16 roundings, ReLU
    # masks and pooling choices it flips, differ; "fp64": the plain oracle.
    # Tolerances: on this 3-level network at initialisation the oracle's own
    # weight gradients move by 2-7 % per layer when its activations are
    # perturbed at the BF16 rounding level, so a per-layer deviation of a few
    # percent is rounding, while a wrong index or a missing term gives O(1).
    net, params, x, t, levels, base = small_net
    q = bf16_round if rounding == "bf16" else None
    xd, td = torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV)
    grads = torch.empty(net.num_params, dtype=torch.float32, device=DEV)
    loss = net.gradients(xd, td, grads)
    pred, cache = un.forward(params, x[..., None].astype(np.float64), levels, base, q=q)
    want_loss, gpred = un.mse(pred, t[..., None].astype(np.float64))
    assert abs(loss - want_loss) <= 1e-3 * want_loss
    want = un.backward(params, x[..., None].astype(np.float64), cache, gpred, levels, base)
    got = oracle_params_from_flat(grads.cpu().numpy(), levels, base)
    errs = {k: rel(got[k], want[k]) for k in want if np.linalg.norm(want[k]) > 0}
    bad = {k: round(e, 4) for k, e in errs.items() if e > tol_layer}
    assert not bad, bad
    assert rel(flat_from_oracle(got, levels, base), flat_from_oracle(want, levels, base)) <= tol_all


def test_unet_training_reduces_loss():
    H = W = 32
    net = pk.Unet(H, W, 3, 8, max_batch=4, seed=9)
    g = np.random.default_rng(10)
    x = torch.from_numpy(g.standard_normal((4, H, W)).astype(np.float32)).to(DEV)
    t = 0.5 * x   # the network must learn to halve its input
    first = net.train_step(x, t, 1e-3, want_loss=True)
    for _ in range(60):
        net.train_step(x, t, 1e-3)
    last = net.train_step(x, t, 1e-3, want_loss=True)
    assert last < 0.5 * first
