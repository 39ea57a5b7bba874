"""GPU parity of the warm-start network against the FP64 numpy reference
(oracle/unet.py): forward output, parameter gradient and the Adam step, in
2D and 3D.

Tolerances: activations and weights are BF16 (8-bit significand, unit
roundoff 2^-9 = 2e-3) with FP32 accumulation; a few layers of rounding put
the output within ~1% of the FP64 reference, so the output is held to 2e-2
relative L2 and the parameter gradient (which goes through every layer
twice) to 5e-2, with a cosine similarity above 0.998.  The Adam step is
FP32 arithmetic on the same gradient: 1e-6.
"""
import numpy as np
import pytest

from oracle import unet as ref

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _net(ndim, channels, seed):
    from paper_2111_11538_gb300.warmstart import WarmStartNet
    net = WarmStartNet(ndim=ndim, channels=channels, cin=3)
    theta = ref.init_params(ndim, 3, list(channels), seed=seed)
    # small random biases so that every bias path is exercised
    theta = theta + 0.02 * np.random.default_rng(seed + 1).standard_normal(theta.size)
    theta = theta.astype(np.float32).astype(np.float64)
    net.set_params(theta)
    return net, theta


def _data(shape, ndim, nb, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (nb,) + shape + (3,))
    t = 0.3 * rng.standard_normal((nb,) + shape + (ndim,))
    return x.astype(np.float32), t.astype(np.float32)


def _to_ref(a):
    # (nb, *S, C) -> list of (C, *S)
    return [np.moveaxis(a[b].astype(np.float64), -1, 0) for b in range(a.shape[0])]


CASES = [
    (2, (32, 64), (16, 32)),              # levels 2: nx % 32, ny % 16
    (2, (128, 128), (16, 32, 64, 64)),    # the default network
    (3, (8, 8, 32), (16, 32)),            # 3D: nz % 4, ny % 8, nx % 32
]


@pytest.mark.parametrize("ndim,shape,channels", CASES)
def test_forward_matches_reference(ndim, shape, channels):
    import torch
    net, theta = _net(ndim, channels, seed=11)
    x, _ = _data(shape, ndim, 2, seed=12)
    y = net.forward(torch.as_tensor(x, device="cuda")).cpu().numpy()
    for b, xb in enumerate(_to_ref(x)):
        yr = np.moveaxis(ref.forward(theta, xb, ndim, list(channels)), 0, -1)
        assert rel(y[b], yr) < 2e-2, (b, rel(y[b], yr))
    net.close()


@pytest.mark.parametrize("kind", ["mse", "grad"])
@pytest.mark.parametrize("ndim,shape,channels", [CASES[0], CASES[2]])
def test_gradient_matches_reference(ndim, shape, channels, kind):
    import torch
    net, theta = _net(ndim, channels, seed=21)
    net.set_loss(kind, weight_channel=1, floor=0.05)
    x, t = _data(shape, ndim, 2, seed=22)
    loss, g = net.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), want_grad=True)
    # the batch loss is the mean over samples of the per-sample means
    lr_, gr = 0.0, np.zeros_like(theta)
    for xb, tb in zip(_to_ref(x), _to_ref(t)):
        l, gb = ref.loss_and_grad(theta, xb, tb, ndim, list(channels), kind=kind, weight_channel=1, floor=0.05)
        lr_ += l / x.shape[0]
        gr += gb / x.shape[0]
    assert abs(loss - lr_) < 2e-2 * lr_
    cos = float(np.dot(g, gr) / (np.linalg.norm(g) * np.linalg.norm(gr)))
    assert cos > 0.998, cos
    assert rel(g.astype(np.float64), gr) < 5e-2, rel(g, gr)
    # every convolution's weight block and bias receives its own gradient
    o = 0
    for ci, co, taps in ref.conv_shapes(ndim, 3, list(channels)):
        nw = ci * co * taps
        for blk in (slice(o, o + nw), slice(o + nw, o + nw + co)):
            if np.linalg.norm(gr[blk]) > 1e-6 * np.linalg.norm(gr):
                assert rel(g[blk].astype(np.float64), gr[blk]) < 1e-1, (o, rel(g[blk], gr[blk]))
        o += nw + co
    net.close()


def test_adam_step_matches_reference():
    import torch
    ndim, shape, channels = CASES[0]
    net, theta = _net(ndim, channels, seed=31)
    x, t = _data(shape, ndim, 1, seed=32)
    _, g = net.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), want_grad=True)
    net.adam_step(1e-3)
    got = net.get_params().astype(np.float64)
    want, _, _ = ref.adam(theta, g.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1, lr=1e-3)
    assert np.max(np.abs(got - want)) < 1e-6
    net.close()


def test_training_lowers_the_loss():
    import torch
    ndim, shape, channels = CASES[0]
    net, _ = _net(ndim, channels, seed=41)
    x, _ = _data(shape, ndim, 4, seed=42)
    # a smooth target the network can represent: a local function of the input
    t = np.stack([x[..., 0] - 0.5 * x[..., 1], x[..., 2] * x[..., 0]], axis=-1).astype(np.float32)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    first = net.loss_grad(xd, td)
    for _ in range(300):
        net.loss_grad(xd, td)
        net.adam_step(3e-3)
    last = net.loss_grad(xd, td)
    assert last < 0.2 * first, (first, last)
    net.close()


def test_rejects_grid_not_divisible():
    import torch
    from paper_2111_11538_gb300.warmstart import UNetError
    net, _ = _net(2, (16, 32), seed=51)
    x = torch.zeros((1, 24, 64, 3), device="cuda")
    with pytest.raises(UNetError):
        net.forward(x)
    net.close()
