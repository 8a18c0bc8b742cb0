"""Learned warm start for the MH3D reconstruction.

The solve of Sec. 4.3 starts from zero.  Here a small 3D U-Net (the kernels
of include/mh3d_unet.h) maps the back-projection A^T d to an initial
iterate,

    x0 = (r / ||A||_2^2) * net(A^T d / r),    r = RMS(A^T d),

and CG starts from x0 with the device-side fallback to the zero start when
x0 is no better than zero (mh3d_solve_opts.x0_fallback).  The scaling makes
the network independent of the data's magnitude; 1 / ||A||_2^2 is the gain
of the operator's top singular direction.  Training minimises the mean
squared error between the scaled network output and the scaled CG solution
x* of the same problem (the iterate CG must reach), with Adam.

Every step runs in libmh3d.so's kernels: A^T d (mh3d_adjoint), the RMS,
the network, the loss and its gradient, Adam, and the solve.  This module
only sequences the calls.
"""
from __future__ import annotations

from typing import Iterable, Optional, Sequence, Tuple

from .mh3d import Plan, make_opts, mh3d_adjoint, mh3d_operator_norm2, mh3d_solve
from .unet import UNet

def layer_io(levels: int):
    """(input level, output level) of every convolution in parameter order
    (None: the one-channel input or output): the encoder's two per level,
    the decoder's two per level from the bottom up, the output
    convolution."""
    io = []
    for l in range(levels):
        io += [(None if l == 0 else l - 1, l), (l, l)]
    for l in range(levels - 2, -1, -1):
        io += [(l + 1, l), (l, l)]
    io.append((0, None))
    return tuple(io)


class WarmStart:
    """A warm-start network for one plan's grid."""

    def __init__(self, plan: Plan, channels: Sequence[int] = (16, 32, 64)):
        import torch

        self.plan = plan
        self.channels = tuple(int(c) for c in channels)
        self.net = UNet(plan.n, *self.channels)
        self.gain = 1.0 / mh3d_operator_norm2(plan)
        self.rhs = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
        self.x0 = torch.empty(plan.shape, dtype=torch.float32, device="cuda")

    # -- parameters -------------------------------------------------------
    def init_params(self, seed: int):
        """He-normal weights (std sqrt(2 / (27 cin))), zero biases, from a
        seeded generator."""
        import torch

        g = torch.Generator().manual_seed(int(seed))
        parts = []
        for ci, co in layer_io(len(self.channels)):
            cin = 1 if ci is None else self.channels[ci]
            cout = 1 if co is None else self.channels[co]
            parts.append(torch.randn(cout * 27 * cin, generator=g) * (2.0 / (27 * cin)) ** 0.5)
            parts.append(torch.zeros(cout))
        theta = torch.cat(parts).float().cuda()
        assert theta.numel() == self.net.nparam
        self.net.set_params(theta)

    def set_params(self, theta):
        self.net.set_params(theta)

    def get_params(self):
        return self.net.get_params()

    def save(self, path: str):
        """Writes the parameters (FP32), the channels and the grid to an .npz
        file.  The Adam state is not kept: a reloaded network resumes
        training with fresh moments."""
        import numpy as np

        np.savez(path, theta=self.get_params().cpu().numpy(), channels=np.array(self.channels),
                 n=np.array(self.plan.n))

    def load(self, path: str):
        import numpy as np
        import torch

        z = np.load(path)
        if tuple(int(c) for c in z["channels"]) != self.channels or tuple(int(v) for v in z["n"]) != tuple(self.plan.n):
            raise ValueError(f"{path}: saved for channels {tuple(z['channels'])} and grid {tuple(z['n'])}")
        self.set_params(torch.as_tensor(z["theta"], dtype=torch.float32).cuda())

    # -- training -----------------------------------------------------------
    def back_projection(self, d, out=None):
        out = self.rhs if out is None else out
        mh3d_adjoint(self.plan, d, out)
        return out

    def train_step(self, rhs, target, lr: float, want_loss: bool = False) -> Optional[float]:
        """One Adam step on one (A^T d, x*) pair; returns the scaled loss
        when asked (that synchronises)."""
        loss = self.net.loss_grad_scaled(rhs, target, self.gain, want_loss=want_loss)
        self.net.adam_step(lr)
        return loss

    def fit(self, rhs_list, target_list, epochs: int, lr_max: float = 1e-3, lr_min: float = 1e-5, seed: int = 0,
            log=None):
        """Adam over the pairs for `epochs` passes, in a seeded random order
        per epoch, the learning rate following a cosine from lr_max to
        lr_min over all steps.  Returns the mean scaled loss of each epoch
        (one synchronisation per step to read it)."""
        import math

        import torch

        n = len(rhs_list)
        total = max(epochs * n, 1)
        g = torch.Generator().manual_seed(int(seed))
        history = []
        step = 0
        for ep in range(epochs):
            order = torch.randperm(n, generator=g).tolist()
            acc = 0.0
            for i in order:
                lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * step / total))
                acc += self.train_step(rhs_list[i], target_list[i], lr, want_loss=True)
                step += 1
            history.append(acc / max(n, 1))
            if log:
                log(ep, history[-1])
        return history

    def loss(self, rhs, target) -> float:
        """Scaled loss of one pair without a parameter update."""
        return self.net.loss_grad_scaled(rhs, target, self.gain, want_loss=True)

    # -- use ------------------------------------------------------------------
    def predict(self, d, out=None):
        """x0 for portraits d (A^T d, then the network)."""
        out = self.x0 if out is None else out
        mh3d_adjoint(self.plan, d, self.rhs)
        self.net.forward_scaled(self.rhs, self.gain, out)
        return out

    def solve(self, d, rho, fallback: bool = True, **opts):
        """CG from the learned x0 (make_opts keywords); returns the info
        dict of mh3d_solve, with x0_rejected when the fallback fired."""
        self.predict(d)
        o = make_opts(x0=self.x0, x0_fallback=fallback, **opts)
        return mh3d_solve(self.plan, d, o, rho)
