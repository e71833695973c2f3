"""Oracle: the learned warm start's network in FP64 NumPy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; the warm start is a U-Net that maps a
normalised dirty image to the SARA solution and only changes SDMM's starting
point (problem (3) is convex). Layout NHWC; 3x3 convolutions with zero
padding 1 (cross-correlation, as deep-learning libraries define "conv"),
1x1 convolutions, ReLU, 2x2 max pooling, nearest-neighbour x2 upsampling,
channel concatenation, mean-squared-error loss, Adam.

Architecture with L levels and base width c (channels c, 2c, 4c, ... ):
  encoder level l: conv3x3 -> ReLU -> conv3x3 -> ReLU (skip saved), maxpool
  bottom:          conv3x3 -> ReLU -> conv3x3 -> ReLU
  decoder level l: upsample x2 -> conv3x3 -> ReLU, concat(skip, .),
                   conv3x3 -> ReLU -> conv3x3 -> ReLU
  head:            conv1x1 (c -> 1), output = input + head (residual)
Weights are [Cout][kh][kw][Cin]; biases [Cout].

`forward` and `backward` take an optional `q` (a rounding function, identity
by default). Given one, the network is evaluated with q applied exactly where
a reduced-precision implementation stores its tensor-core operands: the input,
every weight, every ReLU output, and every gradient entering a convolution's
backward. The default is plain FP64.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------- primitives
def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """x [B][H][W][Cin], w [Cout][k][k][Cin] (k = 1 or 3, 'same' zero
    padding) -> [B][H][W][Cout]."""
    B, H, W, Cin = x.shape
    Cout, k, _, _ = w.shape
    r = k // 2
    xp = np.pad(x, ((0, 0), (r, r), (r, r), (0, 0)))
    out = np.zeros((B, H, W, Cout))
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + W, :]                 # [B][H][W][Cin]
            out += np.einsum("bhwc,oc->bhwo", patch, w[:, dy, dx, :])
    if b is not None:
        out += b
    return out


def conv2d_backward(x, w, gout):
    """Gradients of conv2d with respect to x, w and b."""
    B, H, W, Cin = x.shape
    Cout, k, _, _ = w.shape
    r = k // 2
    xp = np.pad(x, ((0, 0), (r, r), (r, r), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + W, :]
            gw[:, dy, dx, :] = np.einsum("bhwo,bhwc->oc", gout, patch)
            gxp[:, dy:dy + H, dx:dx + W, :] += np.einsum("bhwo,oc->bhwc", gout, w[:, dy, dx, :])
    gx = gxp[:, r:r + H, r:r + W, :]
    gb = gout.sum(axis=(0, 1, 2))
    return gx, gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def maxpool2(x):
    B, H, W, C = x.shape
    v = x.reshape(B, H // 2, 2, W // 2, 2, C)
    return v.max(axis=(2, 4))


def maxpool2_backward(x, gout):
    """Gradient goes to the first maximum of each 2x2 window (row-major)."""
    B, H, W, C = x.shape
    v = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 5, 2, 4).reshape(B, H // 2, W // 2, C, 4)
    idx = np.argmax(v, axis=-1)
    g = np.zeros_like(v)
    np.put_along_axis(g, idx[..., None], gout[..., None], axis=-1)
    g = g.reshape(B, H // 2, W // 2, C, 2, 2).transpose(0, 1, 4, 2, 5, 3).reshape(B, H, W, C)
    return g


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample2_backward(gout):
    B, H, W, C = gout.shape
    return gout.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(pred, target):
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size


# ------------------------------------------------------------------ network
def layer_shapes(levels: int = 4, base: int = 32):
    """Ordered list of (name, Cout, k, Cin) for every convolution."""
    shapes = []
    cin = 1
    for l in range(levels - 1):
        c = base << l
        shapes += [(f"e{l}a", c, 3, cin), (f"e{l}b", c, 3, c)]
        cin = c
    c = base << (levels - 1)
    shapes += [("ba", c, 3, cin), ("bb", c, 3, c)]
    for l in reversed(range(levels - 1)):
        c = base << l
        shapes += [(f"d{l}u", c, 3, 2 * c), (f"d{l}a", c, 3, 2 * c), (f"d{l}b", c, 3, c)]
    shapes.append(("head", 1, 1, base))
    return shapes


def init_params(levels=4, base=32, seed=0):
    """He-normal weights, zero biases (seeded)."""
    g = np.random.default_rng(seed)
    params = {}
    for name, cout, k, cin in layer_shapes(levels, base):
        std = np.sqrt(2.0 / (k * k * cin))
        params[name + ".w"] = g.standard_normal((cout, k, k, cin)) * std
        params[name + ".b"] = np.zeros(cout)
    return params


def _ident(a):
    return a


def forward(params, x, levels=4, base=32, q=None):
    """x [B][H][W][1] -> prediction [B][H][W][1]; returns (pred, cache)."""
    q = q or _ident
    params = {k: (q(v) if k.endswith(".w") else v) for k, v in params.items()}
    cache = {"params": params, "q": q}
    h = q(x)
    skips = []
    for l in range(levels - 1):
        for s in ("a", "b"):
            name = f"e{l}{s}"
            cache[name + ".in"] = h
            z = conv2d(h, params[name + ".w"], params[name + ".b"])
            h = q(relu(z))
            cache[name + ".out"] = h
        skips.append(h)
        cache[f"p{l}.in"] = h
        h = maxpool2(h)
    for s in ("a", "b"):
        name = "b" + s
        cache[name + ".in"] = h
        h = q(relu(conv2d(h, params[name + ".w"], params[name + ".b"])))
        cache[name + ".out"] = h
    for l in reversed(range(levels - 1)):
        name = f"d{l}u"
        hu = upsample2(h)
        cache[name + ".in"] = hu
        h = q(relu(conv2d(hu, params[name + ".w"], params[name + ".b"])))
        cache[name + ".out"] = h
        h = np.concatenate([skips[l], h], axis=-1)
        for s in ("a", "b"):
            name = f"d{l}{s}"
            cache[name + ".in"] = h
            h = q(relu(conv2d(h, params[name + ".w"], params[name + ".b"])))
            cache[name + ".out"] = h
    cache["head.in"] = h
    pred = x + conv2d(h, params["head.w"], params["head.b"])
    return pred, cache


def backward(params, x, cache, gpred, levels=4, base=32):
    """Gradients of the loss with respect to every parameter, given
    dLoss/dpred (uses the weights and rounding recorded by `forward`)."""
    params = cache["params"]
    q = cache["q"]
    grads = {}
    gh, gw, gb = conv2d_backward(cache["head.in"], params["head.w"], q(gpred))
    grads["head.w"], grads["head.b"] = gw, gb
    gskips = {}
    for l in range(levels - 1):
        c = base << l
        for s in ("b", "a"):
            name = f"d{l}{s}"
            gz = q(gh * (cache[name + ".out"] > 0))
            gh, grads[name + ".w"], grads[name + ".b"] = conv2d_backward(cache[name + ".in"], params[name + ".w"], gz)
        gskips[l] = gh[..., :c]
        gh = gh[..., c:]
        name = f"d{l}u"
        gz = q(gh * (cache[name + ".out"] > 0))
        ghu, grads[name + ".w"], grads[name + ".b"] = conv2d_backward(cache[name + ".in"], params[name + ".w"], gz)
        gh = upsample2_backward(ghu)
    for s in ("b", "a"):
        name = "b" + s
        gz = q(gh * (cache[name + ".out"] > 0))
        gh, grads[name + ".w"], grads[name + ".b"] = conv2d_backward(cache[name + ".in"], params[name + ".w"], gz)
    for l in reversed(range(levels - 1)):
        gh = maxpool2_backward(cache[f"p{l}.in"], gh) + gskips[l]
        for s in ("b", "a"):
            name = f"e{l}{s}"
            gz = q(gh * (cache[name + ".out"] > 0))
            gh, grads[name + ".w"], grads[name + ".b"] = conv2d_backward(cache[name + ".in"], params[name + ".w"], gz)
    return grads


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
