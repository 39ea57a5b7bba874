"""Pins of the FP64 reference network (oracle/unet.py), CPU only.

The reference is pinned to definitions it does not share code with: a
brute-force periodic convolution written with explicit modulo indices, the
central-difference derivative of its own loss, the adjointness of average
pooling and nearest upsampling, the translation equivariance a periodic
U-Net must have, and Adam's first step in closed form.
"""
import itertools

import numpy as np
import pytest

from oracle import unet


def _brute_conv(x, W, b):
    ndim = x.ndim - 1
    S = x.shape[1:]
    co, ci = W.shape[:2]
    k = W.shape[-1]
    out = np.zeros((co,) + S)
    for o in range(co):
        for p in itertools.product(*[range(n) for n in S]):
            acc = b[o]
            for c in range(ci):
                for t in itertools.product(*[range(k)] * ndim):
                    q = tuple((p[d] + t[d] - (k // 2)) % S[d] for d in range(ndim))
                    acc += W[(o, c) + t] * x[(c,) + q]
            out[(o,) + p] = acc
    return out


@pytest.mark.parametrize("shape,k", [((5, 4), 3), ((3, 4, 5), 3), ((4, 6), 1)])
def test_conv_matches_brute_force(shape, k):
    rng = np.random.default_rng(0)
    ndim = len(shape)
    x = rng.standard_normal((2,) + shape)
    W = rng.standard_normal((3, 2) + (k,) * ndim)
    b = rng.standard_normal(3)
    assert np.allclose(unet.conv(x, W, b), _brute_conv(x, W, b), rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["mse", "grad"])
@pytest.mark.parametrize("ndim,shape,channels", [(2, (8, 8), [3, 4]), (2, (8, 12), [2, 3, 4]), (3, (4, 4, 4), [2, 3])])
def test_gradient_matches_central_differences(ndim, shape, channels, kind):
    rng = np.random.default_rng(1)
    cin = 3
    theta = unet.init_params(ndim, cin, channels, seed=2)
    theta += 0.05 * rng.standard_normal(theta.size)     # non-zero biases too
    x = rng.standard_normal((cin,) + shape)
    x[1] = rng.uniform(0.0, 1.0, shape)          # the weight channel is a gas weight
    tgt = rng.standard_normal((ndim,) + shape)
    f = lambda th: unet.loss_and_grad(th, x, tgt, ndim, channels, kind=kind)
    loss, g = f(theta)
    assert g.shape == theta.shape
    h = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (f(tp)[0] - f(tm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_input_gradient_of_conv_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 5))
    W = rng.standard_normal((3, 2, 3, 3))
    gout = rng.standard_normal((3, 6, 5))
    gx, gW, gb = unet.conv_backward(x, W, gout)
    # <conv(x) - b, gout> is linear in x and in W
    lin = np.sum((unet.conv(x, W, np.zeros(3))) * gout)
    assert np.isclose(np.sum(gx * x), lin, rtol=1e-12)
    assert np.isclose(np.sum(gW * W), lin, rtol=1e-12)
    assert np.allclose(gb, gout.sum(axis=(1, 2)))


@pytest.mark.parametrize("shape", [(6, 4), (4, 2, 6)])
def test_pool_and_upsample_are_adjoint(shape):
    rng = np.random.default_rng(4)
    ndim = len(shape)
    x = rng.standard_normal((2,) + shape)
    y = rng.standard_normal((2,) + tuple(s // 2 for s in shape))
    assert np.isclose(np.sum(unet.avgpool2(x) * y), np.sum(x * unet.up2(y)) / 2 ** ndim, rtol=1e-12)
    c = np.full((1,) + shape, 3.5)
    assert np.allclose(unet.up2(unet.avgpool2(c)), c)


def test_network_is_periodic_translation_equivariant():
    rng = np.random.default_rng(5)
    channels = [3, 4, 5]
    theta = unet.init_params(2, 2, channels, seed=6)
    x = rng.standard_normal((2, 16, 8))
    y = unet.forward(theta, x, 2, channels)
    s = 2 ** (len(channels) - 1)             # shifts that commute with the pooling
    xs = np.roll(x, shift=(s, 2 * s), axis=(1, 2))
    ys = unet.forward(theta, xs, 2, channels)
    assert np.allclose(ys, np.roll(y, shift=(s, 2 * s), axis=(1, 2)), atol=1e-12)


def test_parameter_count_and_layout():
    shapes = unet.conv_shapes(2, 3, [16, 32, 64, 64])
    assert len(shapes) == 2 * 4 + 2 * 3 + 1
    assert shapes[0] == (3, 16, 9) and shapes[8] == (64 + 64, 64, 9) and shapes[-1] == (16, 2, 1)
    n = unet.n_params(2, 3, [16, 32, 64, 64])
    theta = np.arange(n, dtype=np.float64)
    assert np.array_equal(unet.pack(unet.unpack(theta, 2, 3, [16, 32, 64, 64])), theta)


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t1, m, v = unet.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first moment g, second g^2: step lr * g / (|g| + eps)
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_gradient_loss_ignores_translation_and_weights_stiff_cells():
    rng = np.random.default_rng(8)
    y = rng.standard_normal((2, 6, 8))
    w = rng.uniform(0.0, 1.0, (6, 8))
    # a rigid translation of the output costs nothing
    l0, _ = unet.output_loss(y, y + np.array([0.3, -1.2])[:, None, None], "grad", w)
    assert abs(l0) < 1e-25
    # a single-cell error e at q costs w_q-weighted squares of its differences:
    # sum_d [w_{q-1} e^2 + w_q e^2] / n
    t = y.copy()
    t[0, 2, 3] += 1.0
    l1, _ = unet.output_loss(y, t, "grad", w)
    want = (w[2, 2] + w[2, 3] + w[1, 3] + w[2, 3]) / y.size
    assert np.isclose(l1, want, rtol=1e-12)
