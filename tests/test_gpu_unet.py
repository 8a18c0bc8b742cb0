"""GPU parity of the warm-start network's kernels with the FP64 oracle
(oracle/unet_oracle.py), through the C ABI of include/mh3d_unet.h.

Layer primitives take bfloat16-exact inputs and weights, so both sides see
the same numbers and only the accumulation differs (FP32 on the tensor
cores, over at most 27 * 64 = 1728 products per output, or the voxel count
per weight): relative L2 <= 1e-5.

The whole network stores every activation as bfloat16 at the same points
on both sides (the oracle rounds where the GPU stores).  A rounding can
still flip by one bfloat16 ulp (2^-8 relative) where the FP32 and FP64 sums
straddle a rounding boundary, which happens for a small fraction of values
and propagates: output relative L2 <= 5e-3.  The GPU backward stores its
gradients in bfloat16 as well; against the oracle's FP64 backward, every
layer's weight gradient agrees to relative L2 <= 5e-2 and the whole
gradient's direction to cosine >= 0.999.
"""
import numpy as np
import pytest

from oracle import unet_oracle as U
from tests._cases import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_SMALL = (14, 10, 6)   # nx, ny, nz: V = 840, not a multiple of the 128-voxel tile; partial 8x4x4 blocks


@pytest.fixture(params=["umma", "umma_r1", "umma_r4", "umma_nopair", "umma_nb2", "umma_ws", "default", "tiled",
                        "gather"], autouse=True)
def conv_path(request, monkeypatch):
    """Every test runs with every convolution the tcgen05/TMEM kernel takes
    on it (MH3D_UNET_UMMA=1: the FP32 input, 8..32 bfloat16 channels in
    multiples of 8, up to 64 outputs; the others go to the mma.sync
    kernels) with two output rows per tile (the default), one and four
    (MH3D_UMMA_ROWS), without the paired taps of 8-channel sources
    (MH3D_UMMA_PAIR=0), on its double-buffered form (MH3D_UMMA_NB=2), on its
    warp-specialised pipelined form (MH3D_UMMA_WS=1), with
    the default choice (tcgen05 for sources with rows of 96 voxels
    or more), on the halo-tiled mma.sync kernel alone (MH3D_UNET_UMMA=0)
    and on the gather kernel (MH3D_UNET_UMMA=0, MH3D_UNET_GATHER=1)."""
    for v in ("MH3D_UNET_GATHER", "MH3D_UNET_UMMA", "MH3D_UMMA_NB", "MH3D_UMMA_ROWS", "MH3D_UMMA_WS",
              "MH3D_UMMA_PAIR"):
        monkeypatch.delenv(v, raising=False)
    if request.param.startswith("umma"):
        monkeypatch.setenv("MH3D_UNET_UMMA", "1")
        if request.param == "umma_nb2":
            monkeypatch.setenv("MH3D_UMMA_NB", "2")
        elif request.param == "umma_ws":
            monkeypatch.setenv("MH3D_UMMA_WS", "1")
        elif request.param == "umma_nopair":
            monkeypatch.setenv("MH3D_UMMA_PAIR", "0")
        elif request.param in ("umma_r1", "umma_r4"):
            monkeypatch.setenv("MH3D_UMMA_ROWS", request.param[-1])
    elif request.param in ("tiled", "gather"):
        monkeypatch.setenv("MH3D_UNET_UMMA", "0")
        if request.param == "gather":
            monkeypatch.setenv("MH3D_UNET_GATHER", "1")
    return request.param


def _bf(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16)


def _w(cout, cin, seed):
    g = torch.Generator().manual_seed(seed)
    W = (torch.randn(cout, 27 * cin, generator=g) * (2.0 / (27 * cin)) ** 0.5).to(torch.bfloat16).float()
    b = (torch.randn(cout, generator=g) * 0.1).float()
    return W, b


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


CONV_CASES = [
    # cin, cout, mode
    (1, 16, "f32"),
    (16, 16, "plain"),
    (16, 32, "plain"),
    (32, 64, "plain"),
    (64, 32, "up"),
    (32, 32, "skip"),
    (16, 1, "plain"),
    (8, 24, "plain"),
    (12, 16, "plain"),    # channels not a multiple of 8: scalar gathers
    (8, 16, "skip"),
    (64, 64, "plain"),    # weights beyond the tiled kernel's shared memory: gather kernel
]


def _sources(n, cin, mode, seed):
    nx, ny, nz = n
    if mode == "f32":
        x = torch.randn((nz, ny, nx), generator=torch.Generator().manual_seed(seed)).float()
        return dict(src_f32=x.cuda()), U.bf16_round(_np(x))[..., None]   # the gather rounds to bfloat16
    if mode == "up":
        a = _bf((nz // 2, ny // 2, nx // 2, cin), seed)
        return dict(src=a.cuda(), up=1), U.up(_np(a))
    a = _bf((nz, ny, nx, cin), seed)
    if mode == "skip":
        b = _bf((nz, ny, nx, cin), seed + 1)
        return dict(src=a.cuda(), skip=b.cuda()), U.bf16_round(_np(a) + _np(b))
    return dict(src=a.cuda()), _np(a)


@pytest.mark.parametrize("cin,cout,mode", CONV_CASES)
@pytest.mark.parametrize("relu", [False, True])
def test_conv_forward_matches_oracle(cin, cout, mode, relu):
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_forward

    n = N_SMALL
    kw, x = _sources(n, cin, mode, 10 * cin + cout)
    W, b = _w(cout, cin, cin * 7 + cout)
    out = torch.empty(n[2] * n[1] * n[0] * cout, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_forward(n, cin, cout, W.cuda(), b.cuda(), out, relu=relu, **kw)
    ref = U.conv(x, _np(W).reshape(cout, 3, 3, 3, cin), _np(b))
    if relu:
        ref = U.relu(ref)
    got = out.cpu().numpy().reshape(ref.shape)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


@pytest.mark.parametrize("n,cin,cout,mode", [
    ((136, 6, 4), 16, 16, "plain"),   # two 128-voxel x tiles, the second ragged
    ((130, 4, 4), 32, 48, "skip"),    # 48 outputs in 64 accumulator columns
    ((128, 6, 4), 1, 16, "f32"),
    ((260, 4, 2), 8, 8, "up"),        # three x tiles, upsampled source
])
def test_conv_forward_multi_tile_rows(n, cin, cout, mode):
    """Rows longer than one 128-voxel tile, with ragged last tiles."""
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_forward

    kw, x = _sources(n, cin, mode, 3 * cin + cout)
    W, b = _w(cout, cin, cin * 5 + cout)
    out = torch.empty(n[2] * n[1] * n[0] * cout, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_forward(n, cin, cout, W.cuda(), b.cuda(), out, relu=True, **kw)
    ref = U.relu(U.conv(x, _np(W).reshape(cout, 3, 3, 3, cin), _np(b)))
    got = out.cpu().numpy().reshape(ref.shape)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


@pytest.mark.parametrize("cin,cout,mode", [(8, 8, "plain"), (16, 8, "up"), (8, 8, "skip"), (8, 1, "plain")])
def test_conv_forward_at_the_bench_size(cin, cout, mode, conv_path):
    """The warm-start network's full-resolution layers at 128x128x64 (the
    size the learned benchmark runs), element by element against the
    oracle, on the tcgen05 kernel (default and forced) and the mma.sync
    tiles."""
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_forward

    if conv_path not in ("default", "umma", "umma_ws", "tiled"):
        pytest.skip("the full-size layers run on the default, tcgen05 and tiled paths")

    n = (128, 128, 64)
    kw, x = _sources(n, cin, mode, 40 * cin + cout)
    W, b = _w(cout, cin, cin * 3 + cout)
    out = torch.empty(n[2] * n[1] * n[0] * cout, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_forward(n, cin, cout, W.cuda(), b.cuda(), out, relu=True, **kw)
    ref = U.relu(U.conv(x, _np(W).reshape(cout, 3, 3, 3, cin), _np(b)))
    got = out.cpu().numpy().reshape(ref.shape)
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


@pytest.mark.parametrize("cin,cout", [(1, 16), (16, 16), (16, 32), (64, 32), (16, 1), (12, 16), (32, 8)])
def test_conv_input_grad_matches_oracle(cin, cout):
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_input_grad

    n = N_SMALL
    nx, ny, nz = n
    g = _bf((nz, ny, nx, cout), 3 * cin + cout)
    W, _ = _w(cout, cin, cin + 5 * cout)
    gin = torch.empty(nz * ny * nx * cin, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_input_grad(n, cin, cout, g.cuda(), W.cuda(), gin)
    ref = U.conv_input_grad(_np(g), _np(W).reshape(cout, 3, 3, 3, cin))
    assert rel_l2(gin.cpu().numpy().reshape(ref.shape), ref) <= 1e-5


@pytest.mark.parametrize("cin,cout,mode", [(1, 16, "f32"), (16, 16, "plain"), (32, 64, "plain"), (64, 32, "up"),
                                           (32, 32, "skip"), (16, 1, "plain"), (12, 16, "plain")])
def test_conv_weight_grad_matches_oracle(cin, cout, mode):
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_weight_grad

    n = N_SMALL
    nx, ny, nz = n
    kw, x = _sources(n, cin, mode, 20 * cin + cout)
    g = _bf((nz, ny, nx, cout), 9 * cin + cout)
    gW = torch.empty(cout * 27 * cin, dtype=torch.float32, device="cuda")
    gb = torch.empty(cout, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_weight_grad(n, cin, cout, g.cuda(), gW, gb, **kw)
    rW, rb = U.conv_weight_grad(x, _np(g))
    assert rel_l2(gW.cpu().numpy(), rW.ravel()) <= 1e-5
    assert rel_l2(gb.cpu().numpy(), rb) <= 1e-5


def test_weight_grad_over_many_chunks():
    """A volume of several 4096-voxel chunks (the split-K partial sums)."""
    from paper_2503_13802_gb300.unet import mh3d_unet_conv_weight_grad

    n = (32, 24, 20)   # V = 15360: 4 chunks, the last one partial
    nx, ny, nz = n
    cin, cout = 16, 32
    a = _bf((nz, ny, nx, cin), 31)
    g = _bf((nz, ny, nx, cout), 32)
    gW = torch.empty(cout * 27 * cin, dtype=torch.float32, device="cuda")
    gb = torch.empty(cout, dtype=torch.float32, device="cuda")
    mh3d_unet_conv_weight_grad(n, cin, cout, g.cuda(), gW, gb, src=a.cuda())
    rW, rb = U.conv_weight_grad(_np(a), _np(g))
    assert rel_l2(gW.cpu().numpy(), rW.ravel()) <= 1e-5
    assert rel_l2(gb.cpu().numpy(), rb) <= 1e-5


CH = (16, 32, 64)
N_NET = (16, 12, 8)


def _theta(seed, ch=CH):
    rng = np.random.default_rng(seed)
    parts = []
    for _, ci, co in U.layer_shapes(*ch):
        W = rng.standard_normal(co * 27 * ci) * np.sqrt(2.0 / (27 * ci))
        parts += [U.bf16_round(W), (rng.standard_normal(co) * 0.05).astype(np.float32).astype(np.float64)]
    return np.concatenate(parts)


def _net_inputs(seed):
    nx, ny, nz = N_NET
    rng = np.random.default_rng(seed)
    inp = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    tgt = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    return inp, tgt


def _gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).cuda()


def test_network_forward_matches_oracle():
    from paper_2503_13802_gb300.unet import UNet

    theta = _theta(1)
    inp, _ = _net_inputs(2)
    net = UNet(N_NET, *CH)
    assert net.nparam == theta.size == U.param_count(*CH)
    net.set_params(_gpu(theta))
    out = torch.empty(net.V, dtype=torch.float32, device="cuda")
    net.forward(_gpu(inp), out)
    ref, _ = U.forward(U.unflatten(theta, *CH), inp, bf16=True)
    got = out.cpu().numpy().reshape(ref.shape)
    assert rel_l2(got, ref) <= 5e-3, rel_l2(got, ref)


def test_network_gradient_matches_oracle():
    from paper_2503_13802_gb300.unet import UNet

    theta = _theta(3)
    inp, tgt = _net_inputs(4)
    net = UNet(N_NET, *CH)
    net.set_params(_gpu(theta))
    grad = torch.empty(net.nparam, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(_gpu(inp), _gpu(tgt), grad)
    Lr, G, _ = U.loss_and_grad(U.unflatten(theta, *CH), inp, tgt, bf16=True)
    assert abs(loss - Lr) <= 1e-3 * Lr, (loss, Lr)
    g = grad.cpu().numpy().astype(np.float64)
    gr = U.flatten(G, *CH)
    cos = float(np.dot(g, gr) / (np.linalg.norm(g) * np.linalg.norm(gr)))
    assert cos >= 0.999, cos
    o = 0
    for name, ci, co in U.layer_shapes(*CH):
        nW = co * 27 * ci
        assert rel_l2(g[o:o + nW], gr[o:o + nW]) <= 5e-2, (name, rel_l2(g[o:o + nW], gr[o:o + nW]))
        o += nW + co


CH4 = (8, 16, 32, 128)   # four levels; the bottleneck's 128 channels: gather kernels, two output tiles
N_NET4 = (32, 32, 16)


def test_four_level_network_forward_and_gradient_match_oracle():
    """The network with four levels (encoder and decoder loops of any
    depth) against the oracle: forward to 5e-3, the gradient to cosine
    0.999 and every layer's weight gradient to 5e-2, as for three levels."""
    from paper_2503_13802_gb300.unet import UNet

    theta = _theta(11, CH4)
    nx, ny, nz = N_NET4
    rng = np.random.default_rng(12)
    inp = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    tgt = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
    net = UNet(N_NET4, *CH4)
    assert net.nparam == theta.size == U.param_count(*CH4)
    net.set_params(_gpu(theta))
    out = torch.empty(net.V, dtype=torch.float32, device="cuda")
    net.forward(_gpu(inp), out)
    ref, _ = U.forward(U.unflatten(theta, *CH4), inp, bf16=True)
    got = out.cpu().numpy().reshape(ref.shape)
    assert rel_l2(got, ref) <= 5e-3, rel_l2(got, ref)
    grad = torch.empty(net.nparam, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(_gpu(inp), _gpu(tgt), grad)
    Lr, G, _ = U.loss_and_grad(U.unflatten(theta, *CH4), inp, tgt, bf16=True)
    assert abs(loss - Lr) <= 1e-3 * Lr, (loss, Lr)
    g = grad.cpu().numpy().astype(np.float64)
    gr = U.flatten(G, *CH4)
    cos = float(np.dot(g, gr) / (np.linalg.norm(g) * np.linalg.norm(gr)))
    assert cos >= 0.999, cos
    o = 0
    for name, ci, co in U.layer_shapes(*CH4):
        nW = co * 27 * ci
        assert rel_l2(g[o:o + nW], gr[o:o + nW]) <= 5e-2, (name, rel_l2(g[o:o + nW], gr[o:o + nW]))
        o += nW + co


def test_training_steps_reduce_the_loss():
    from paper_2503_13802_gb300.unet import UNet

    theta = _theta(5)
    inp, _ = _net_inputs(6)
    tgt = np.roll(inp, 1, axis=2) * 0.5       # a learnable linear map of the input
    net = UNet(N_NET, *CH)
    net.set_params(_gpu(theta))
    x, t = _gpu(inp), _gpu(tgt)
    first = net.loss_grad(x, t)
    for _ in range(60):
        net.adam_step(2e-3)
        net.loss_grad(x, t, want_loss=False)
    last = net.loss_grad(x, t)
    assert last < 0.5 * first, (first, last)
