"""Learned warm start of the displacement solve: the network object (thin
binding of include/pf_unet.h) and its training on pairs from the library's
own converged solves.

The network predicts the rate of the displacement solution as the
ferrite/wuestite interface moves.  Inputs per cell (channels, in this
order): the ferrite weight W_f, the gas weight W_g, the prescribed mean
stress p / |eig0| (the same value in every cell) and the ferrite-weight rate
dW_f/dt over the last step; target: du/dt / |eig0| of the periodic
displacement fluctuation.  The solve of step n then starts from
u_{n-1} + |eig0| dt y.  The absolute displacement is not the target: with a
prestress on porous bodies whose gas channels span the box it is a
domain-scale field that a network with a finite receptive field cannot
predict, while its change under a small interface motion is mostly local.
"""
import ctypes

import numpy as np

from . import native
from .native import PF_OK

INPUT_CHANNELS = 4
DEFAULT_CHANNELS = (16, 32, 64, 64)


class UNetError(RuntimeError):
    pass


def _ptr(t):
    return int(t.data_ptr())


class WarmStartNet:
    """The periodic U-Net on the GPU.  Arrays are torch CUDA float32 tensors
    shaped (nb, [nz,] ny, nx, C) (channels last)."""

    def __init__(self, ndim=2, channels=DEFAULT_CHANNELS, cin=INPUT_CHANNELS):
        native.build_library()
        self.ndim = ndim
        self.channels = tuple(channels)
        self.cin = cin
        cfg = native.pf_unet_config()
        cfg.ndim, cfg.cin, cfg.levels = ndim, cin, len(channels)
        for i, c in enumerate(channels):
            cfg.channels[i] = c
        rc, h = native.pf_unet_create(cfg)
        if rc != PF_OK:
            raise UNetError(native.pf_unet_last_error(None))
        self.h = h
        self.nparam = native.pf_unet_param_count(h)

    def _check(self, rc):
        if rc != PF_OK:
            raise UNetError("status %d: %s" % (rc, native.pf_unet_last_error(self.h)))

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.nparam
        self._check(native.pf_unet_set_params(self.h, a))

    def get_params(self):
        a = np.zeros(self.nparam, dtype=np.float32)
        self._check(native.pf_unet_get_params(self.h, a))
        return a

    @staticmethod
    def _grid(x, ndim):
        s = x.shape[1:1 + ndim]
        if ndim == 2:
            return s[1], s[0], 1
        return s[2], s[1], s[0]

    def forward(self, x):
        import torch
        x = x.contiguous()
        nb = x.shape[0]
        nx, ny, nz = self._grid(x, self.ndim)
        out = torch.empty(x.shape[:-1] + (self.ndim,), dtype=torch.float32, device=x.device)
        stream = torch.cuda.current_stream().cuda_stream
        self._check(native.pf_unet_forward(self.h, _ptr(x), _ptr(out), nb, nx, ny, nz, stream))
        return out

    def loss_grad(self, x, target, want_grad=False):
        import torch
        x = x.contiguous()
        target = target.contiguous()
        nb = x.shape[0]
        nx, ny, nz = self._grid(x, self.ndim)
        g = np.zeros(self.nparam, dtype=np.float32) if want_grad else None
        stream = torch.cuda.current_stream().cuda_stream
        rc, loss = native.pf_unet_loss_grad(self.h, _ptr(x), _ptr(target), nb, nx, ny, nz, g, stream)
        self._check(rc)
        return (loss, g) if want_grad else loss

    def set_loss(self, kind="mse", weight_channel=1, floor=0.01):
        """Training loss: "mse" on the output, or "grad" -- the stiffness-
        weighted error of the output's forward differences (include/pf_unet.h)."""
        k = {"mse": native.PF_UNET_LOSS_MSE, "grad": native.PF_UNET_LOSS_GRAD}[kind]
        self._check(native.pf_unet_set_loss(self.h, k, weight_channel, floor))

    def adam_step(self, lr):
        import torch
        self._check(native.pf_unet_adam_step(self.h, lr, torch.cuda.current_stream().cuda_stream))

    def close(self):
        if getattr(self, "h", None):
            native.pf_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Training pairs from the library's own converged solves
# ---------------------------------------------------------------------------
def _h(x):
    return x * x * x * (x * (6.0 * x - 15.0) + 10.0)


def weights(phi_f, phi_w):
    """(W_f, W_g) of the model's phase interpolation, with
    theta = phi_f / (phi_f + phi_w) and phi_g = 1 - phi_f - phi_w."""
    s = phi_f + phi_w
    theta = np.where(s > 0.0, phi_f / np.where(s > 0.0, s, 1.0), 0.0)
    wg = _h(1.0 - s)
    return (1.0 - wg) * _h(theta), wg


def cell_inputs(phi_f, phi_w, prestress, eig0, wf_rate):
    """Network inputs of one grid (channels last, float32)."""
    wf, wg = weights(phi_f, phi_w)
    p = np.full_like(wf, prestress / abs(eig0))
    return np.stack([wf, wg, p, wf_rate], axis=-1).astype(np.float32)


def random_instance(shape, rng):
    """A seeded microstructure of the kinds the workloads use: a porous
    oxide with a ferrite rim around the pores, or a core-shell particle."""
    from . import inputs
    n = shape[-1]
    if rng.uniform() < 0.5:
        frac = rng.uniform(0.05, 0.3)
        grains = max(4, int(n * n / 4096))
        f = inputs.porous(shape, grains, frac, rng.uniform(0.02, 0.06) * n, 0.5, int(rng.integers(1 << 30)),
                          rim=rng.uniform(1.0, 6.0))
    else:
        r = rng.uniform(0.15, 0.4) * n
        f = inputs.core_shell(shape, r, rng.uniform(0.05, 0.25) * r)
    return f


def generate_pairs(count, shape, seed, record_steps=(1, 10, 40), cg_rtol=1e-11):
    """(inputs, targets) from converged FP64 solves.  For each of `count`
    seeded instances (random prestress in [0, 0.02]) the library advances
    the fields; at each step k in `record_steps` the solves of states k-1
    and k give the displacement rate (u_k - u_{k-1}) / dt, paired with the
    inputs of state k and its ferrite-weight rate.  The solves run to a
    tight residual so that the difference is not solver noise, and a rigid
    translation (which the periodic problem does not fix) is removed."""
    from . import Simulation, workloads
    rng = np.random.default_rng(seed)
    X, T = [], []
    for i in range(count):
        f = random_instance(shape, rng)
        p = float(rng.uniform(0.0, 0.02))
        prm = workloads.params(plasticity=0, prestress=p, cg_rtol=cg_rtol, cg_maxit=200000)
        ae = abs(prm["eig0"])
        sim = Simulation(shape, prm, precision="fp64")
        sim.set_fields(f)
        dt = sim.dt
        done = 0
        for k in record_steps:
            if k - 1 > done:
                sim.step(k - 1 - done)
            g0 = sim.get_fields(keys=("phi_f", "phi_w"))
            sim.step(1)
            ua = sim.get_fields(keys=("u",))["u"]
            g1 = sim.get_fields(keys=("phi_f", "phi_w"))
            sim.step(1)
            ub = sim.get_fields(keys=("u",))["u"]
            done = k + 1
            rate = (weights(g1["phi_f"], g1["phi_w"])[0] - weights(g0["phi_f"], g0["phi_w"])[0]) / dt
            du = (ub - ua) / (ae * dt)
            du -= du.reshape(-1, du.shape[-1]).mean(axis=0)
            X.append(cell_inputs(g1["phi_f"], g1["phi_w"], p, prm["eig0"], rate))
            T.append(du.astype(np.float32))
        sim.close()
    return np.stack(X), np.stack(T)


def augment(x, t, rng):
    """A random symmetry of the periodic square-grid problem applied to a
    2D batch (torch tensors, channels last): periodic shift, mirror in x
    and/or y, transpose.  Scalar inputs move with the cells; the displacement
    rate is a vector, so a mirror flips its component and a transpose swaps
    its components."""
    import torch
    sy, sx = int(rng.integers(x.shape[1])), int(rng.integers(x.shape[2]))
    x = torch.roll(x, shifts=(sy, sx), dims=(1, 2))
    t = torch.roll(t, shifts=(sy, sx), dims=(1, 2))
    sign = torch.ones(2, device=t.device)
    if rng.uniform() < 0.5:
        x, t = torch.flip(x, dims=(2,)), torch.flip(t, dims=(2,))
        sign[0] = -sign[0]
    if rng.uniform() < 0.5:
        x, t = torch.flip(x, dims=(1,)), torch.flip(t, dims=(1,))
        sign[1] = -sign[1]
    t = t * sign
    if x.shape[1] == x.shape[2] and rng.uniform() < 0.5:
        x = x.transpose(1, 2)
        t = t.transpose(1, 2)[..., [1, 0]]
    return x.contiguous(), t.contiguous()


def train(net, X, T, steps, batch=8, lr=1e-3, seed=0, log_every=0, symmetries=True):
    """Adam on mini-batches drawn from (X, T) (numpy, channels last; or lists
    of such arrays, one per grid size, visited in turn), each batch under a
    random symmetry of the problem (2D); the learning rate decays with a
    cosine to lr/20.  Returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    if not isinstance(X, (list, tuple)):
        X, T = [X], [T]
    Xd = [torch.as_tensor(x, device="cuda") for x in X]
    Td = [torch.as_tensor(t, device="cuda") for t in T]
    hist = []
    for it in range(steps):
        k = it % len(Xd)
        n = len(Xd[k])
        idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device="cuda")
        xb, tb = Xd[k][idx], Td[k][idx]
        if symmetries and net.ndim == 2:
            xb, tb = augment(xb, tb, rng)
        loss = net.loss_grad(xb, tb)
        a = lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * it / max(steps, 1))))
        net.adam_step(a)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print("train step %d loss %.4e lr %.2e" % (it, loss, a), flush=True)
    return hist


def save(net, path):
    np.savez_compressed(path, params=net.get_params(), ndim=net.ndim, channels=np.array(net.channels))


def load(path):
    d = np.load(path)
    net = WarmStartNet(ndim=int(d["ndim"]), channels=tuple(int(c) for c in d["channels"]))
    net.set_params(d["params"])
    return net


def init(ndim=2, channels=DEFAULT_CHANNELS, seed=0):
    """A network with He-uniform weights and zero biases."""
    net = WarmStartNet(ndim=ndim, channels=channels)
    rng = np.random.default_rng(seed)
    taps = 3 ** ndim
    parts = []
    prev = INPUT_CHANNELS
    shapes = []
    L = len(channels)
    for l in range(L):
        shapes += [(prev, channels[l], taps), (channels[l], channels[l], taps)]
        prev = channels[l]
    for l in range(L - 2, -1, -1):
        shapes += [(channels[l] + channels[l + 1], channels[l], taps), (channels[l], channels[l], taps)]
    shapes.append((channels[0], ndim, 1))
    for ci, co, t in shapes:
        b = np.sqrt(6.0 / (ci * t))
        parts += [rng.uniform(-b, b, ci * co * t), np.zeros(co)]
    theta = np.concatenate(parts).astype(np.float32)
    # the output layer starts small: the first guesses stay near zero
    theta[-(channels[0] * ndim + ndim):] *= 0.1
    net.set_params(theta)
    return net


def rate_error(net, X, T):
    """Relative L2 error of the predicted displacement rate on (X, T), and
    that of the previous-step guess (rate 0) -- 1 by definition."""
    import torch
    y = net.forward(torch.as_tensor(X, device="cuda")).cpu().numpy()
    return float(np.linalg.norm(y - T) / np.linalg.norm(T))


def main(argv=None):
    """Generate pairs on the GPU, train the 2D network with the library's own
    kernels and save it:  python -m paper_2111_11538_gb300.warmstart OUT.npz"""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("out")
    ap.add_argument("--instances", type=int, default=96)
    ap.add_argument("--instances-256", type=int, default=16)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--loss", default="grad", choices=["mse", "grad"])
    a = ap.parse_args(argv)
    t0 = time.time()
    X, T = generate_pairs(a.instances, (128, 128), seed=a.seed)
    X2, T2 = generate_pairs(a.instances_256, (256, 256), seed=a.seed + 1)
    Xh, Th = generate_pairs(8, (128, 128), seed=a.seed + 100)
    t1 = time.time()
    net = init(2, DEFAULT_CHANNELS, seed=a.seed)
    net.set_loss(a.loss)
    hist = train(net, [X, X2], [T, T2], a.steps, batch=8, lr=2e-3, seed=a.seed)
    t2 = time.time()
    save(net, a.out)
    info = {"loss": a.loss, "pairs": int(len(X) + len(X2)), "pair_seconds": t1 - t0, "train_steps": a.steps,
            "train_seconds": t2 - t1, "loss_first": hist[0], "loss_last50": float(np.mean(hist[-50:])),
            "heldout_rate_error": rate_error(net, Xh, Th), "heldout_pairs": int(len(Xh))}
    print(json.dumps(info))
    with open(a.out + ".json", "w") as fh:
        json.dump(info, fh)


if __name__ == "__main__":
    main()
