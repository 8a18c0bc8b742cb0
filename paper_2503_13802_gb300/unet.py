"""Thin ctypes binding of the learned warm-start network (include/mh3d_unet.h).

Argument marshalling only: the network's convolutions, pooling, loss and
optimiser run in libmh3d.so's kernels.  Tensors are checked for device,
dtype, size and contiguity before their pointers are passed.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_void_p, c_char_p
from typing import Sequence

from .mh3d import MH3DError, _dev_ptr, _stream_ptr, load as _load_base

EXPORTS = ["mh3d_unet_param_count", "mh3d_unet_param_count_levels", "mh3d_unet_create",
           "mh3d_unet_create_levels", "mh3d_unet_destroy", "mh3d_unet_set_params",
           "mh3d_unet_get_params", "mh3d_unet_forward", "mh3d_unet_loss_grad", "mh3d_unet_forward_scaled",
           "mh3d_unet_loss_grad_scaled", "mh3d_unet_adam_step",
           "mh3d_unet_conv_forward", "mh3d_unet_conv_input_grad", "mh3d_unet_conv_weight_grad",
           "mh3d_unet_last_error"]


class mh3d_unet_conv_desc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("cin", c_int), ("cout", c_int),
                ("src_bf16", c_void_p), ("skip_bf16", c_void_p), ("src_f32", c_void_p), ("up", c_int)]


_ready = False


def load():
    global _ready
    lib = _load_base()
    if _ready:
        return lib
    P = c_void_p
    lib.mh3d_unet_param_count.argtypes = [c_int, c_int, c_int]
    lib.mh3d_unet_param_count.restype = c_longlong
    lib.mh3d_unet_param_count_levels.argtypes = [c_int, POINTER(c_int)]
    lib.mh3d_unet_param_count_levels.restype = c_longlong
    lib.mh3d_unet_create.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, POINTER(c_void_p)]
    lib.mh3d_unet_create_levels.argtypes = [c_int, c_int, c_int, c_int, POINTER(c_int), POINTER(c_void_p)]
    lib.mh3d_unet_destroy.argtypes = [P]
    lib.mh3d_unet_set_params.argtypes = [P, P, P]
    lib.mh3d_unet_get_params.argtypes = [P, P, P]
    lib.mh3d_unet_forward.argtypes = [P, P, P, P]
    lib.mh3d_unet_loss_grad.argtypes = [P, P, P, P, POINTER(c_double), P]
    lib.mh3d_unet_forward_scaled.argtypes = [P, P, c_float, P, P]
    lib.mh3d_unet_loss_grad_scaled.argtypes = [P, P, P, c_float, P, POINTER(c_double), P]
    lib.mh3d_unet_adam_step.argtypes = [P, c_float, P]
    lib.mh3d_unet_conv_forward.argtypes = [POINTER(mh3d_unet_conv_desc), P, P, c_int, P, P]
    lib.mh3d_unet_conv_input_grad.argtypes = [POINTER(mh3d_unet_conv_desc), P, P, P, P]
    lib.mh3d_unet_conv_weight_grad.argtypes = [POINTER(mh3d_unet_conv_desc), P, P, P, P]
    lib.mh3d_unet_last_error.argtypes = [P]
    lib.mh3d_unet_last_error.restype = c_char_p
    for name in EXPORTS:
        if name not in ("mh3d_unet_param_count", "mh3d_unet_param_count_levels", "mh3d_unet_last_error"):
            getattr(lib, name).restype = c_int
    _ready = True
    return lib


def mh3d_unet_param_count(*channels: int) -> int:
    """Parameters of the network with these channels per level (2..5
    levels)."""
    ch = (c_int * len(channels))(*channels)
    n = int(load().mh3d_unet_param_count_levels(len(channels), ch))
    if n < 0:
        raise ValueError(f"bad channel list {channels}")
    return n


class UNet:
    """The warm-start network for volumes of n = (nx, ny, nz) voxels."""

    def __init__(self, n: Sequence[int], *channels: int):
        """channels per level, full resolution first (2..5 levels; default
        (16, 32, 64))."""
        lib = load()
        self.n = tuple(int(v) for v in n)
        self.channels = tuple(int(c) for c in channels) if channels else (16, 32, 64)
        nx, ny, nz = self.n
        self.shape = (nz, ny, nx)
        self.V = nx * ny * nz
        self.nparam = mh3d_unet_param_count(*self.channels)
        self.handle = c_void_p()
        ch = (c_int * len(self.channels))(*self.channels)
        st = lib.mh3d_unet_create_levels(nx, ny, nz, len(self.channels), ch, ctypes.byref(self.handle))
        if st != 0:
            raise MH3DError(st, "mh3d_unet_create_levels")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                load().mh3d_unet_destroy(h)
            except Exception:
                pass
            self.handle = c_void_p()

    def _check(self, st: int, what: str):
        if st != 0:
            raise MH3DError(st, f"{what}: {load().mh3d_unet_last_error(self.handle).decode()}")

    def set_params(self, theta, stream=None):
        import torch

        p = _dev_ptr(theta, torch.float32, self.nparam, "theta")
        self._check(load().mh3d_unet_set_params(self.handle, c_void_p(p), c_void_p(_stream_ptr(stream))),
                    "set_params")

    def get_params(self, stream=None):
        import torch

        out = torch.empty(self.nparam, dtype=torch.float32, device="cuda")
        self._check(load().mh3d_unet_get_params(self.handle, c_void_p(out.data_ptr()),
                                                c_void_p(_stream_ptr(stream))), "get_params")
        return out

    def forward(self, inp, out, stream=None):
        import torch

        pi = _dev_ptr(inp, torch.float32, self.V, "in")
        po = _dev_ptr(out, torch.float32, self.V, "out")
        self._check(load().mh3d_unet_forward(self.handle, c_void_p(pi), c_void_p(po), c_void_p(_stream_ptr(stream))),
                    "forward")

    def loss_grad(self, inp, target, grad=None, want_loss: bool = True, stream=None):
        import torch

        pi = _dev_ptr(inp, torch.float32, self.V, "in")
        pt = _dev_ptr(target, torch.float32, self.V, "target")
        pg = _dev_ptr(grad, torch.float32, self.nparam, "grad") if grad is not None else None
        loss = c_double(0.0)
        self._check(load().mh3d_unet_loss_grad(self.handle, c_void_p(pi), c_void_p(pt), c_void_p(pg),
                                               ctypes.byref(loss) if want_loss else None,
                                               c_void_p(_stream_ptr(stream))), "loss_grad")
        return loss.value if want_loss else None

    def forward_scaled(self, inp, gain: float, out, stream=None):
        """out = (r gain) network(inp / r), r = RMS(inp) on the device."""
        import torch

        pi = _dev_ptr(inp, torch.float32, self.V, "in")
        po = _dev_ptr(out, torch.float32, self.V, "out")
        self._check(load().mh3d_unet_forward_scaled(self.handle, c_void_p(pi), c_float(gain), c_void_p(po),
                                                    c_void_p(_stream_ptr(stream))), "forward_scaled")

    def loss_grad_scaled(self, inp, target, gain: float, grad=None, want_loss: bool = True, stream=None):
        import torch

        pi = _dev_ptr(inp, torch.float32, self.V, "in")
        pt = _dev_ptr(target, torch.float32, self.V, "target")
        pg = _dev_ptr(grad, torch.float32, self.nparam, "grad") if grad is not None else None
        loss = c_double(0.0)
        self._check(load().mh3d_unet_loss_grad_scaled(self.handle, c_void_p(pi), c_void_p(pt), c_float(gain),
                                                      c_void_p(pg), ctypes.byref(loss) if want_loss else None,
                                                      c_void_p(_stream_ptr(stream))), "loss_grad_scaled")
        return loss.value if want_loss else None

    def adam_step(self, lr: float, stream=None):
        self._check(load().mh3d_unet_adam_step(self.handle, c_float(lr), c_void_p(_stream_ptr(stream))),
                    "adam_step")


def _desc(n, cin, cout, src=None, skip=None, src_f32=None, up=0):
    nx, ny, nz = n
    d = mh3d_unet_conv_desc()
    d.nx, d.ny, d.nz, d.cin, d.cout, d.up = nx, ny, nz, cin, cout, int(up)
    d.src_bf16 = src.data_ptr() if src is not None else None
    d.skip_bf16 = skip.data_ptr() if skip is not None else None
    d.src_f32 = src_f32.data_ptr() if src_f32 is not None else None
    return d


def _need(t, dtype, numel, what):
    import torch

    if t is None:
        return
    _dev_ptr(t, dtype, numel, what)


def mh3d_unet_conv_forward(n, cin, cout, W, b, out, src=None, skip=None, src_f32=None, up=0, relu=False,
                           stream=None):
    """out [V][cout] FP32 = conv(source) (+ReLU); sources as in the header."""
    import torch

    nx, ny, nz = n
    V = nx * ny * nz
    Vs = V // 8 if up else V
    _need(src, torch.bfloat16, Vs * cin, "src")
    _need(skip, torch.bfloat16, Vs * cin, "skip")
    _need(src_f32, torch.float32, V, "src_f32")
    _dev_ptr(W, torch.float32, cout * 27 * cin, "W")
    if b is not None:
        _dev_ptr(b, torch.float32, cout, "b")
    _dev_ptr(out, torch.float32, V * cout, "out")
    d = _desc(n, cin, cout, src, skip, src_f32, up)
    st = load().mh3d_unet_conv_forward(ctypes.byref(d), c_void_p(W.data_ptr()),
                                       c_void_p(b.data_ptr() if b is not None else None), int(relu),
                                       c_void_p(out.data_ptr()), c_void_p(_stream_ptr(stream)))
    if st != 0:
        raise MH3DError(st, "mh3d_unet_conv_forward")


def mh3d_unet_conv_input_grad(n, cin, cout, g, W, gin, stream=None):
    import torch

    nx, ny, nz = n
    V = nx * ny * nz
    _dev_ptr(g, torch.bfloat16, V * cout, "g")
    _dev_ptr(W, torch.float32, cout * 27 * cin, "W")
    _dev_ptr(gin, torch.float32, V * cin, "gin")
    d = _desc(n, cin, cout)
    st = load().mh3d_unet_conv_input_grad(ctypes.byref(d), c_void_p(g.data_ptr()), c_void_p(W.data_ptr()),
                                          c_void_p(gin.data_ptr()), c_void_p(_stream_ptr(stream)))
    if st != 0:
        raise MH3DError(st, "mh3d_unet_conv_input_grad")


def mh3d_unet_conv_weight_grad(n, cin, cout, g, gW, gb, src=None, skip=None, src_f32=None, up=0, stream=None):
    import torch

    nx, ny, nz = n
    V = nx * ny * nz
    Vs = V // 8 if up else V
    _need(src, torch.bfloat16, Vs * cin, "src")
    _need(skip, torch.bfloat16, Vs * cin, "skip")
    _need(src_f32, torch.float32, V, "src_f32")
    _dev_ptr(g, torch.bfloat16, V * cout, "g")
    _dev_ptr(gW, torch.float32, cout * 27 * cin, "gW")
    _dev_ptr(gb, torch.float32, cout, "gb")
    d = _desc(n, cin, cout, src, skip, src_f32, up)
    st = load().mh3d_unet_conv_weight_grad(ctypes.byref(d), c_void_p(g.data_ptr()), c_void_p(gW.data_ptr()),
                                           c_void_p(gb.data_ptr()), c_void_p(_stream_ptr(stream)))
    if st != 0:
        raise MH3DError(st, "mh3d_unet_conv_weight_grad")
