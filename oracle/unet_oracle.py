"""Plain FP64 reference of the learned warm-start network (test
infrastructure only: imported by tests/ and the benchmark's CPU leg, never
by the product library).

The network maps the normalised back-projection A^T d (one channel) to a
warm start for CG.  It is a small 3D U-Net with additive skips of L levels
(channels C_0 .. C_{L-1}, L >= 2), written out layer by layer with numpy so
a reader can check it by eye.  For L = 3:

    e0a = relu(conv(in,        W0a))      C0 channels, full resolution
    e0  = relu(conv(e0a,       W0b))      C0            (skip 0)
    e1a = relu(conv(pool(e0),  W1a))      C1, half resolution
    e1  = relu(conv(e1a,       W1b))      C1            (skip 1)
    ba  = relu(conv(pool(e1),  W2a))      C2, quarter resolution
    b   = relu(conv(ba,        W2b))      C2
    u1  = relu(conv(up(b),     W3a))      C1, half
    d1  = relu(conv(u1 + e1,   W3b))      C1
    u0  = relu(conv(up(d1),    W4a))      C0, full
    d0  = relu(conv(u0 + e0,   W4b))      C0
    out = conv(d0, W5)                    1 channel, no activation

In general: encoder levels l = 0 .. L-1 (W{l}a, W{l}b; the input of level
l > 0 is pool(e_{l-1}), the last level is the bottleneck), decoder levels
l = L-2 .. 0 (W{2L-2-l}a on up(d_{l+1}), d_{L-1} = the bottleneck output,
and W{2L-2-l}b on u_l + e_l), then W{2L-1} to one channel.

conv: 3x3x3 cross-correlation with zero padding ("same"), weights
[Cout][3][3][3][Cin] (taps ordered dz, dy, dx), plus a bias per output
channel.  pool: mean over 2x2x2 blocks.  up: nearest-neighbour x2.
Volumes are channels-last [D][H][W][C].  Loss: L = sum((out - t)^2) / (2 V).

bf16=True rounds to bfloat16 (round to nearest even) exactly where the GPU
stores bfloat16: the weights, the network input, every stored activation,
the pooled volumes and the sums u + e.  Products and sums in between are
FP64 here (FP32 on the GPU).  The backward pass is plain FP64 (the
gradient the GPU's mixed-precision backward approximates).
"""
from __future__ import annotations

import numpy as np

LAYERS = ("W0a", "W0b", "W1a", "W1b", "W2a", "W2b", "W3a", "W3b", "W4a", "W4b", "W5")


def layer_shapes(*ch: int):
    """(name, Cin, Cout) of every convolution, in parameter order, for the
    network with channels ch = (C_0, .., C_{L-1})."""
    L = len(ch)
    assert L >= 2
    out = []
    for l in range(L):
        out += [(f"W{l}a", 1 if l == 0 else ch[l - 1], ch[l]), (f"W{l}b", ch[l], ch[l])]
    for l in range(L - 2, -1, -1):
        i = 2 * L - 2 - l
        out += [(f"W{i}a", ch[l + 1], ch[l]), (f"W{i}b", ch[l], ch[l])]
    out.append((f"W{2 * L - 1}", ch[0], 1))
    return out


def param_count(*ch: int) -> int:
    return sum(co * 27 * ci + co for _, ci, co in layer_shapes(*ch))


def unflatten(theta: np.ndarray, *ch: int) -> dict:
    """Flat parameter vector -> {name: (W [Cout,3,3,3,Cin], b [Cout])}.
    Layout: per layer in order, W row-major then b."""
    out, o = {}, 0
    for name, ci, co in layer_shapes(*ch):
        n = co * 27 * ci
        W = np.asarray(theta[o:o + n], dtype=np.float64).reshape(co, 3, 3, 3, ci)
        o += n
        b = np.asarray(theta[o:o + co], dtype=np.float64)
        o += co
        out[name] = (W, b)
    assert o == theta.size
    return out


def flatten(grads: dict, *ch: int) -> np.ndarray:
    parts = []
    for name, _, _ in layer_shapes(*ch):
        gW, gb = grads[name]
        parts += [gW.ravel(), gb.ravel()]
    return np.concatenate(parts)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Goes through float32 first, as the GPU's FP32 values do."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shifted(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """s[z, y, x] = x[z + dz, y + dy, x + dx], zero outside."""
    D, H, W = x.shape[:3]
    p = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    return p[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[v, co] = b[co] + sum_taps sum_ci W[co, tap, ci] x[v + tap, ci]."""
    co = W.shape[0]
    y = np.broadcast_to(b, x.shape[:3] + (co,)).astype(np.float64).copy()
    for t, (dz, dy, dx) in enumerate(_taps()):
        y += _shifted(x, dz, dy, dx) @ W.reshape(co, 27, -1)[:, t, :].T
    return y


def conv_input_grad(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Gradient of conv w.r.t. its input: gx[v, ci] = sum_taps sum_co
    W[co, tap, ci] g[v - tap, co] (the transposed correlation)."""
    ci = W.shape[-1]
    out = np.zeros(g.shape[:3] + (ci,))
    for t, (dz, dy, dx) in enumerate(_taps()):
        out += _shifted(g, -dz, -dy, -dx) @ W.reshape(W.shape[0], 27, ci)[:, t, :]
    return out


def conv_weight_grad(x: np.ndarray, g: np.ndarray):
    """gW[co, tap, ci] = sum_v g[v, co] x[v + tap, ci];  gb[co] = sum_v g[v, co]."""
    co, ci = g.shape[-1], x.shape[-1]
    gW = np.zeros((co, 27, ci))
    g2 = g.reshape(-1, co)
    for t, (dz, dy, dx) in enumerate(_taps()):
        gW[:, t, :] = g2.T @ _shifted(x, dz, dy, dx).reshape(-1, ci)
    return gW.reshape(co, 3, 3, 3, ci), g2.sum(axis=0)


def pool(x: np.ndarray) -> np.ndarray:
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool_grad(g: np.ndarray) -> np.ndarray:
    return up(g) / 8.0


def up(x: np.ndarray) -> np.ndarray:
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def up_grad(g: np.ndarray) -> np.ndarray:
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def _levels(params: dict) -> int:
    """L from the parameter names: 4 L - 1 convolutions."""
    n = len(params)
    assert (n + 1) % 4 == 0, n
    return (n + 1) // 4


def forward(params: dict, inp: np.ndarray, bf16: bool = False):
    """inp: [D, H, W] float.  Returns (out [D, H, W], cache of activations).
    The number of levels follows from the parameters."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    P = {k: (r(W), np.asarray(b, dtype=np.float64)) for k, (W, b) in params.items()}
    L = _levels(P)
    c = {"in": r(inp)[..., None]}
    x = c["in"]
    for l in range(L):                       # encoder; level L-1 is the bottleneck
        if l > 0:
            x = c[f"p{l - 1}"] = r(pool(c[f"e{l - 1}"]))
        c[f"x{l}"] = x
        c[f"e{l}a"] = r(relu(conv(x, *P[f"W{l}a"])))
        c[f"e{l}"] = r(relu(conv(c[f"e{l}a"], *P[f"W{l}b"])))
    c[f"d{L - 1}"] = c[f"e{L - 1}"]
    for l in range(L - 2, -1, -1):           # decoder
        i = 2 * L - 2 - l
        c[f"ud{l}"] = up(c[f"d{l + 1}"])
        c[f"u{l}"] = r(relu(conv(c[f"ud{l}"], *P[f"W{i}a"])))
        c[f"s{l}"] = r(c[f"u{l}"] + c[f"e{l}"])
        c[f"d{l}"] = r(relu(conv(c[f"s{l}"], *P[f"W{i}b"])))
    out = conv(c["d0"], *P[f"W{2 * L - 1}"])[..., 0]
    c["P"] = P
    return out, c


def loss_and_grad(params: dict, inp: np.ndarray, target: np.ndarray, bf16: bool = False):
    """L = sum((out - target)^2) / (2 V) and dL/dparams (FP64 backward
    through the forward's stored values)."""
    out, c = forward(params, inp, bf16)
    P = c["P"]
    L = _levels(P)
    V = out.size
    diff = out - target
    loss = float(np.sum(diff * diff) / (2 * V))
    G = {}

    def back_conv(name, x, g):
        G[name] = conv_weight_grad(x, g)
        return conv_input_grad(g, P[name][0])

    def mask(g, y):
        return g * (y > 0)

    g = (diff / V)[..., None]
    g_d = back_conv(f"W{2 * L - 1}", c["d0"], g)       # gradient w.r.t. d0
    g_s = {}
    for l in range(L - 1):                             # decoder, top to bottom
        i = 2 * L - 2 - l
        g_s[l] = back_conv(f"W{i}b", c[f"s{l}"], mask(g_d, c[f"d{l}"]))
        g = back_conv(f"W{i}a", c[f"ud{l}"], mask(g_s[l], c[f"u{l}"]))
        g_d = up_grad(g)                               # gradient w.r.t. d_{l+1}
    g_e = g_d                                          # the bottleneck: e_{L-1} = d_{L-1}
    for l in range(L - 1, -1, -1):                     # encoder, bottom to top
        g = back_conv(f"W{l}b", c[f"e{l}a"], mask(g_e, c[f"e{l}"]))
        g_x = back_conv(f"W{l}a", c[f"x{l}"], mask(g, c[f"e{l}a"]))
        if l > 0:
            g_e = g_s[l - 1] + pool_grad(g_x)          # e_{l-1}: skip and pool paths
    return loss, G, out
