"""Pins of the warm-start network's FP64 oracle (oracle/unet_oracle.py)
against things that are not the oracle: a brute-force loop, scipy's
correlate, adjoint identities of each layer, central finite differences of
the whole loss, and torch's own bfloat16 rounding."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def _rng(seed):
    return np.random.default_rng(seed)


def test_conv_matches_brute_force_loop():
    r = _rng(1)
    D, H, W, ci, co = 3, 4, 5, 2, 3
    x = r.standard_normal((D, H, W, ci))
    Wt = r.standard_normal((co, 3, 3, 3, ci))
    b = r.standard_normal(co)
    y = U.conv(x, Wt, b)
    ref = np.zeros((D, H, W, co))
    for z in range(D):
        for yy in range(H):
            for xx in range(W):
                for o in range(co):
                    acc = b[o]
                    for a in range(3):
                        for c in range(3):
                            for e in range(3):
                                zz, y2, x2 = z + a - 1, yy + c - 1, xx + e - 1
                                if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                    acc += np.dot(Wt[o, a, c, e], x[zz, y2, x2])
                    ref[z, yy, xx, o] = acc
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_conv_matches_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    r = _rng(2)
    x = r.standard_normal((6, 5, 7, 3))
    Wt = r.standard_normal((2, 3, 3, 3, 3))
    y = U.conv(x, Wt, np.zeros(2))
    for o in range(2):
        ref = sum(ndimage.correlate(x[..., i], Wt[o, ..., i], mode="constant", cval=0.0) for i in range(3))
        assert np.allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_conv_input_grad_is_the_adjoint():
    r = _rng(3)
    x = r.standard_normal((4, 6, 5, 3))
    g = r.standard_normal((4, 6, 5, 2))
    Wt = r.standard_normal((2, 3, 3, 3, 3))
    lhs = np.sum(U.conv(x, Wt, np.zeros(2)) * g)
    rhs = np.sum(x * U.conv_input_grad(g, Wt))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_conv_weight_grad_identity():
    """<conv(x, W, b), g> = <W, gW> + <b, gb> (conv is linear in (W, b))."""
    r = _rng(4)
    x = r.standard_normal((5, 4, 6, 2))
    g = r.standard_normal((5, 4, 6, 3))
    Wt = r.standard_normal((3, 3, 3, 3, 2))
    b = r.standard_normal(3)
    gW, gb = U.conv_weight_grad(x, g)
    lhs = np.sum(U.conv(x, Wt, b) * g)
    rhs = np.sum(Wt * gW) + np.sum(b * gb)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_pool_and_up_adjoints():
    r = _rng(5)
    x = r.standard_normal((4, 6, 8, 2))
    g = r.standard_normal((2, 3, 4, 2))
    assert np.isclose(np.sum(U.pool(x) * g), np.sum(x * U.pool_grad(g)), rtol=1e-13)
    y = r.standard_normal((2, 3, 4, 2))
    h = r.standard_normal((4, 6, 8, 2))
    assert np.isclose(np.sum(U.up(y) * h), np.sum(y * U.up_grad(h)), rtol=1e-13)
    assert np.allclose(U.pool(U.up(y)), y)


def test_loss_gradient_matches_central_differences():
    c0, c1, c2 = 2, 3, 4
    r = _rng(6)
    n = U.param_count(c0, c1, c2)
    theta = r.standard_normal(n) * 0.4
    inp = r.standard_normal((4, 8, 4))
    tgt = r.standard_normal((4, 8, 4))
    params = U.unflatten(theta, c0, c1, c2)
    _, G, _ = U.loss_and_grad(params, inp, tgt)
    g = U.flatten(G, c0, c1, c2)
    idx = r.choice(n, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        Lp = U.loss_and_grad(U.unflatten(tp, c0, c1, c2), inp, tgt)[0]
        Lm = U.loss_and_grad(U.unflatten(tm, c0, c1, c2), inp, tgt)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_param_layout_round_trip():
    c0, c1, c2 = 2, 3, 4
    theta = np.arange(U.param_count(c0, c1, c2), dtype=np.float64)
    P = U.unflatten(theta, c0, c1, c2)
    assert np.array_equal(U.flatten(P, c0, c1, c2), theta)
    assert P["W0a"][0].shape == (2, 3, 3, 3, 1) and P["W5"][0].shape == (1, 3, 3, 3, 2)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    r = _rng(7)
    x = np.concatenate([r.standard_normal(10000) * 10.0 ** r.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0, 1e-30]])
    x32 = x.astype(np.float32)
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(x32), ref)
    assert U.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0          # tie -> even
    assert U.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


@pytest.mark.parametrize("ch,shape", [((2, 3, 4, 5), (8, 8, 8)), ((2, 3), (4, 6, 2))])
def test_loss_gradient_matches_central_differences_other_depths(ch, shape):
    """Four levels (and two): the generic encoder/decoder loops against
    central differences of the loss."""
    r = _rng(16)
    n = U.param_count(*ch)
    theta = r.standard_normal(n) * 0.4
    inp = r.standard_normal(shape)
    tgt = r.standard_normal(shape)
    _, G, _ = U.loss_and_grad(U.unflatten(theta, *ch), inp, tgt)
    g = U.flatten(G, *ch)
    h = 1e-6
    for i in r.choice(n, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (U.loss_and_grad(U.unflatten(tp, *ch), inp, tgt)[0] - U.loss_and_grad(U.unflatten(tm, *ch), inp, tgt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_four_level_layout():
    """(16, 32, 64, 128): 15 convolutions, the bottleneck at 128 channels,
    1,314,849 parameters."""
    sh = U.layer_shapes(16, 32, 64, 128)
    assert len(sh) == 15 and sh[7] == ("W3b", 128, 128) and sh[8] == ("W4a", 128, 64) and sh[-1] == ("W7", 16, 1)
    assert U.param_count(16, 32, 64, 128) == sum(co * 27 * ci + co for _, ci, co in sh) == 1314849
