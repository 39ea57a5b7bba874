"""Plain FP64 reference of the warm-start network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline import this
package; the CUDA library never does.

The network supplies the initial guess of the displacement solve (the
mechanical equilibrium of Sec. 2.4, div sigma = 0): from per-cell inputs
(ferrite weight W_f, gas weight W_g and the prescribed mean stress, the
quantities that set the eigenstrain and the stiffness of Sec. 2.2) it
predicts the periodic displacement fluctuation, scaled by 1/|eig0|.

Architecture (every convolution is periodic, 3^D taps, with a bias):

  level l = 0..L-1 with channels c_l; input x_{-1} = the C_in input channels
  encoder   a_l = relu(conv(relu(conv(p_l))))          p_0 = input,
                                                        p_l = avgpool2(a_{l-1})
  decoder   d_{L-1} = a_{L-1}
            d_l = relu(conv(relu(conv(concat(a_l, up2(d_{l+1}))))))   l = L-2..0
  output    y = conv1x1(d_0)                           (C_out = D channels)

avgpool2 averages 2^D children, up2 copies a parent to its 2^D children
(nearest), concat stacks channels (skip channels first).

Parameter order (the flat FP32 vector both sides agree on): for each
convolution in the order enc_0a, enc_0b, enc_1a, enc_1b, ..., enc_{L-1}b,
dec_{L-2}a, dec_{L-2}b, ..., dec_0a, dec_0b, out: the weights W[c_out][c_in]
[taps] (taps row-major over (dz,) dy, dx, each in 0..2, tap offset = index-1)
followed by the bias b[c_out].

Loss, either of
  "mse":  mean over cells and output channels of (y - target)^2;
  "grad": (1/(cells * C_out)) sum over cells p, axes d and channels c of
          w_p (e_c(p + e_d) - e_c(p))^2, e = y - target, periodic forward
          differences, w_p = floor + (1 - floor)(1 - x_k(p)) with x_k an input
          channel (the gas weight: a stiffness weight, so that the loss
          follows the strain error where the material is stiff).

Everything here is written from the definitions above with numpy; a
convolution is a sum over taps of np.roll-shifted inputs contracted with the
tap's weight matrix.
"""
import numpy as np


def conv_shapes(ndim, cin, channels, cout=None):
    """(c_in, c_out, taps) of every convolution, in parameter order."""
    cout = ndim if cout is None else cout
    taps = 3 ** ndim
    L = len(channels)
    out = []
    prev = cin
    for l in range(L):
        out.append((prev, channels[l], taps))
        out.append((channels[l], channels[l], taps))
        prev = channels[l]
    for l in range(L - 2, -1, -1):
        # the decoder input of level l: skip a_l plus up2 of d_{l+1}
        cat = channels[l] + channels[l + 1]
        out.append((cat, channels[l], taps))
        out.append((channels[l], channels[l], taps))
    out.append((channels[0], cout, 1))
    return out


def n_params(ndim, cin, channels, cout=None):
    return sum(ci * co * t + co for ci, co, t in conv_shapes(ndim, cin, channels, cout))


def unpack(theta, ndim, cin, channels, cout=None):
    """Flat parameter vector -> list of (W (co, ci, *taps), b)."""
    res = []
    o = 0
    for ci, co, t in conv_shapes(ndim, cin, channels, cout):
        k = 3 if t > 1 else 1
        W = np.asarray(theta[o:o + ci * co * t], dtype=np.float64).reshape((co, ci) + (k,) * ndim)
        o += ci * co * t
        b = np.asarray(theta[o:o + co], dtype=np.float64)
        o += co
        res.append((W, b))
    assert o == len(theta)
    return res


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def init_params(ndim, cin, channels, seed, cout=None):
    """He-uniform weights, zero biases (an initialisation, not part of the
    method; both sides receive the same vector)."""
    rng = np.random.default_rng(seed)
    out = []
    for ci, co, t in conv_shapes(ndim, cin, channels, cout):
        bound = np.sqrt(6.0 / (ci * t))
        out.append(rng.uniform(-bound, bound, ci * co * t))
        out.append(np.zeros(co))
    return np.concatenate(out)


def _offsets(ndim, k):
    if k == 1:
        return [((0,) * ndim, (0,) * ndim)]
    res = []
    for idx in np.ndindex(*(3,) * ndim):
        res.append((idx, tuple(i - 1 for i in idx)))
    return res


def conv(x, W, b):
    """Periodic cross-correlation: out[o, p] = b[o] + sum_{c, t} W[o, c, t] x[c, p + t - 1]."""
    ndim = x.ndim - 1
    k = W.shape[-1]
    out = np.zeros((W.shape[0],) + x.shape[1:])
    axes = tuple(range(1, ndim + 1))
    for idx, off in _offsets(ndim, k):
        # xs[c, p] = x[c, p + off]
        xs = np.roll(x, shift=tuple(-o for o in off), axis=axes)
        out += np.tensordot(W[(slice(None), slice(None)) + idx], xs, axes=([1], [0]))
    out += b.reshape((-1,) + (1,) * ndim)
    return out


def conv_backward(x, W, gout):
    """Gradients of conv with respect to x, W and b."""
    ndim = x.ndim - 1
    k = W.shape[-1]
    axes = tuple(range(1, ndim + 1))
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for idx, off in _offsets(ndim, k):
        xs = np.roll(x, shift=tuple(-o for o in off), axis=axes)
        Wt = W[(slice(None), slice(None)) + idx]                   # (co, ci)
        gW[(slice(None), slice(None)) + idx] = np.tensordot(gout, xs, axes=(axes, axes))
        # d out[o, p] / d x[c, p + off] = W[o, c]  ->  gx[c, q] += sum_o W[o, c] gout[o, q - off]
        g = np.tensordot(Wt, gout, axes=([0], [0]))
        gx += np.roll(g, shift=off, axis=axes)
    gb = gout.sum(axis=axes)
    return gx, gW, gb


def avgpool2(x):
    ndim = x.ndim - 1
    s = x.shape
    shp = [s[0]]
    for n in s[1:]:
        assert n % 2 == 0
        shp += [n // 2, 2]
    y = x.reshape(shp)
    return y.mean(axis=tuple(range(2, 2 + 2 * ndim, 2)))


def up2(x):
    y = x
    for ax in range(1, x.ndim):
        y = np.repeat(y, 2, axis=ax)
    return y


def relu(x):
    return np.maximum(x, 0.0)


def forward(theta, x, ndim, channels, cout=None, keep=False):
    """y = net(x) for x of shape (C_in, *S); with keep=True also the tape."""
    cin = x.shape[0]
    P = unpack(theta, ndim, cin, channels, cout)
    L = len(channels)
    tape = []
    k = 0
    a = []
    h = x
    for l in range(L):
        if l > 0:
            h = avgpool2(a[-1])
        z1 = conv(h, *P[k]); r1 = relu(z1)
        z2 = conv(r1, *P[k + 1]); r2 = relu(z2)
        tape.append(("enc", l, h, r1, r2))
        k += 2
        a.append(r2)
    d = a[L - 1]
    for l in range(L - 2, -1, -1):
        cat = np.concatenate([a[l], up2(d)], axis=0)
        z1 = conv(cat, *P[k]); r1 = relu(z1)
        z2 = conv(r1, *P[k + 1]); r2 = relu(z2)
        tape.append(("dec", l, cat, r1, r2))
        k += 2
        d = r2
    y = conv(d, *P[k])
    if keep:
        return y, (P, tape, d)
    return y


def output_loss(y, target, kind="mse", weights=None):
    """Loss and its gradient with respect to the network output y (C, *S)."""
    n = y.size
    e = y - target
    if kind == "mse":
        return float(np.sum(e * e) / n), 2.0 * e / n
    ndim = y.ndim - 1
    loss = 0.0
    g = np.zeros_like(y)
    for ax in range(1, ndim + 1):
        de = np.roll(e, -1, axis=ax) - e                  # e(p + e_d) - e(p)
        wde = weights[None] * de
        loss += float(np.sum(wde * de))
        # d/d e(q) of w_p de(p)^2: +2 w_{q-1} de(q-1) - 2 w_q de(q)
        g += 2.0 * (np.roll(wde, 1, axis=ax) - wde)
    return loss / n, g / n


def loss_and_grad(theta, x, target, ndim, channels, cout=None, kind="mse", weight_channel=1, floor=0.01):
    """Loss of net(x) against target (see the module docstring) and its
    gradient with respect to the parameters (flat)."""
    y, (P, tape, d0) = forward(theta, x, ndim, channels, cout, keep=True)
    L = len(channels)
    wts = floor + (1.0 - floor) * (1.0 - x[weight_channel]) if kind == "grad" else None
    loss, gy = output_loss(y, target, kind, wts)
    grads = [None] * len(P)
    k = len(P) - 1
    gd, gW, gb = conv_backward(d0, P[k][0], gy)
    grads[k] = (gW, gb)
    # decoder, in reverse (level 0 first)
    dec = [t for t in tape if t[0] == "dec"]
    enc = [t for t in tape if t[0] == "enc"]
    ga = [np.zeros_like(t[4]) for t in enc]   # gradients reaching a_l
    g_next = gd
    kk = k - 1
    for _, l, cat, r1, r2 in reversed(dec):
        # r2 = relu(conv(r1)); r1 = relu(conv(cat))
        gz2 = g_next * (r2 > 0)
        g1, gW2, gb2 = conv_backward(r1, P[kk][0], gz2)
        gz1 = g1 * (r1 > 0)
        gcat, gW1, gb1 = conv_backward(cat, P[kk - 1][0], gz1)
        grads[kk] = (gW2, gb2)
        grads[kk - 1] = (gW1, gb1)
        kk -= 2
        cs = enc[l][4].shape[0]
        ga[l] += gcat[:cs]
        gup = gcat[cs:]
        # up2 backward: sum over the 2^D children
        g = gup
        ndim_ = g.ndim - 1
        shp = [g.shape[0]]
        for s in g.shape[1:]:
            shp += [s // 2, 2]
        g = g.reshape(shp).sum(axis=tuple(range(2, 2 + 2 * ndim_, 2)))
        g_next = g
    # the bottom of the decoder is a_{L-1}
    ga[L - 1] += g_next
    for _, l, h, r1, r2 in reversed(enc):
        gz2 = ga[l] * (r2 > 0)
        g1, gW2, gb2 = conv_backward(r1, P[kk][0], gz2)
        gz1 = g1 * (r1 > 0)
        gh, gW1, gb1 = conv_backward(h, P[kk - 1][0], gz1)
        grads[kk] = (gW2, gb2)
        grads[kk - 1] = (gW1, gb1)
        kk -= 2
        if l > 0:
            # avgpool2 backward: each child receives its parent's gradient / 2^D
            nd = gh.ndim - 1
            ga[l - 1] += up2(gh) / (2 ** nd)
    assert kk == -1
    return loss, pack(grads)


def adam(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1); t counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
