"""Learned warm start of the displacement solve: the network object (thin
binding of include/pf_unet.h) and its training on pairs from the library's
own converged solves.

Inputs per cell (channels, in this order): the ferrite weight W_f, the gas
weight W_g and the prescribed mean stress p / |eig0| (the same value in every
cell); target: the periodic displacement fluctuation divided by |eig0|.
"""
import ctypes

import numpy as np

from . import native
from .native import PF_OK

INPUT_CHANNELS = 3
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
