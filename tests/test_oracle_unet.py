"""Pins for the oracle's warm-start network (CPU only): convolution against a
direct loop, every backward against central finite differences, pooling and
upsampling by hand, Adam's first step in closed form."""
import numpy as np
import pytest

from oracle import unet as un


def test_conv2d_matches_direct_loops():
    g = np.random.default_rng(0)
    x = g.standard_normal((2, 5, 6, 3))
    w = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    out = un.conv2d(x, w, b)
    B, H, W, C = x.shape
    for bi in range(B):
        for i in range(H):
            for j in range(W):
                for o in range(4):
                    s = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            ii, jj = i + dy - 1, j + dx - 1
                            if 0 <= ii < H and 0 <= jj < W:
                                s += np.dot(w[o, dy, dx], x[bi, ii, jj])
                    assert abs(out[bi, i, j, o] - s) < 1e-12


@pytest.mark.parametrize("k", [1, 3])
def test_conv2d_backward_finite_differences(k):
    g = np.random.default_rng(k)
    x = g.standard_normal((1, 4, 5, 2))
    w = g.standard_normal((3, k, k, 2))
    b = g.standard_normal(3)
    go = g.standard_normal((1, 4, 5, 3))
    loss = lambda x_, w_, b_: np.sum(un.conv2d(x_, w_, b_) * go)
    gx, gw, gb = un.conv2d_backward(x, w, go)
    h = 1e-6
    for arr, grad in ((x, gx), (w, gw), (b, gb)):
        flat = arr.reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[i]
            flat[i] = old + h
            lp = loss(x, w, b)
            flat[i] = old - h
            lm = loss(x, w, b)
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - grad.reshape(-1)[i]) < 1e-6


def test_pool_and_upsample_by_hand():
    x = np.array([[1.0, 5.0, 2.0, 2.0], [3.0, 4.0, 0.0, 7.0]]).reshape(1, 2, 4, 1)
    assert np.array_equal(un.maxpool2(x).ravel(), [5.0, 7.0])
    g = un.maxpool2_backward(x, np.array([10.0, 20.0]).reshape(1, 1, 2, 1))
    assert np.array_equal(g.ravel(), [0, 10, 0, 0, 0, 0, 0, 20])
    # ties go to the first maximum in row-major order
    t = np.ones((1, 2, 2, 1))
    assert np.array_equal(un.maxpool2_backward(t, np.ones((1, 1, 1, 1))).ravel(), [1, 0, 0, 0])
    u = un.upsample2(np.array([1.0, 2.0]).reshape(1, 1, 2, 1))
    assert np.array_equal(u.ravel(), [1, 1, 2, 2, 1, 1, 2, 2])
    assert np.array_equal(un.upsample2_backward(np.arange(8.0).reshape(1, 2, 4, 1)).ravel(), [0 + 1 + 4 + 5, 2 + 3 + 6 + 7])


def test_network_backward_finite_differences():
    levels, base = 3, 2
    g = np.random.default_rng(3)
    params = un.init_params(levels, base, seed=4)
    for k in params:
        if k.endswith(".b"):
            params[k] = g.standard_normal(params[k].shape) * 0.1
    x = g.standard_normal((2, 8, 8, 1))
    target = g.standard_normal((2, 8, 8, 1))

    def loss_of(p):
        pred, _ = un.forward(p, x, levels, base)
        return un.mse(pred, target)[0]

    pred, cache = un.forward(params, x, levels, base)
    _, gpred = un.mse(pred, target)
    grads = un.backward(params, x, cache, gpred, levels, base)
    assert set(grads) == set(params)
    h = 1e-6
    for name in ("e0a.w", "e1b.w", "ba.b", "d1u.w", "d0a.w", "d0b.b", "head.w", "head.b"):
        flat = params[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 4)):
            old = flat[i]
            flat[i] = old + h
            lp = loss_of(params)
            flat[i] = old - h
            lm = loss_of(params)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[name].reshape(-1)[i]) < 1e-6 * max(1.0, abs(fd)), name


def test_adam_first_step_closed_form():
    p, g = np.array([1.0, -2.0]), np.array([0.5, -4.0])
    p1, m, v = un.adam_step(p, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    # bias-corrected first step moves each weight by lr * sign(g) (up to eps)
    assert np.allclose(p1, p - 0.1 * np.sign(g), atol=1e-7)


def test_layer_shapes_four_levels_base_32():
    s = un.layer_shapes(4, 32)
    chans = {n: c for n, c, _, _ in s}
    assert chans["e0a"] == 32 and chans["e2b"] == 128 and chans["bb"] == 256 and chans["head"] == 1
    assert [n for n, *_ in s][:2] == ["e0a", "e0b"] and s[-1][0] == "head"
