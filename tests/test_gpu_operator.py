"""GPU parity of the forward operator, the adjoint and the normal operator
against the FP64 oracle, through the C ABI (libmh3d.so via the binding).

Tolerance: relative L2 <= 1e-5 for FP32 operators (the benchmark spec's bound),
also checked per harmonic.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import OP_CASES, gpu_plan, oracle_geom, rel_l2, sens_map

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(params=["specialised", "warpsplit", "warp1", "ctalevel", "generic", "alternatives", "cluster4"])
def kernel_path(request, monkeypatch):
    """Run each operator test on the default kernels (the compile-time
    specialised ones for the common lengths, with the warp-centric
    drive-axis passes at n_x = 128, s = 2, the forward and normal ones opted in, two
    warps per row group, the adjoint fused with T_z^T in y-slab clusters at
    n_z = 64), again with four warps per row group and the adjoint's T_z^T
    as a separate launch (MH3D_XWARP_KS=4, MH3D_XWARP_ZX=0), with one warp
    per row group and the alternative T-pass radix schedules the autotuner
    may pick (MH3D_XWARP_KS=1, MH3D_TPASS_RADIX=1), on the CTA-level drive-axis
    passes those replace (MH3D_XWARP=0: y-slab cluster passes, pipelined
    adjoint, 16-row normal pass), again with MH3D_GENERIC=1, which forces the
    runtime-general kernels for every size, and on the measured alternatives
    of the CTA-level path: the bulk-copy normal pass, the adjoint without
    copy pipelining, the 16-row forward pass with uneven harmonic groups of
    three per CTA, and the separate T_z and drive-axis passes instead of the
    y-slab cluster passes; and once more with those cluster passes on
    clusters of four CTAs (MH3D_ZX_CLUSTER=4) and the pipelined adjoint in
    rounds of two harmonics (MH3D_XADJ_KB=2)."""
    for v in ("MH3D_GENERIC", "MH3D_XNRM_BULK", "MH3D_XADJ_BULK", "MH3D_XNRM_PAIRS", "MH3D_XADJ_PAIRS",
              "MH3D_XFWD_KPC", "MH3D_XFWD_PAIRS", "MH3D_FUSE_ZX", "MH3D_ZX_CLUSTER", "MH3D_XADJ_KB", "MH3D_XWARP",
              "MH3D_XWARP_FWD", "MH3D_XWARP_KS", "MH3D_XWARP_ZX", "MH3D_XWARP_NRM", "MH3D_TPASS_RADIX"):
        monkeypatch.delenv(v, raising=False)
    if request.param == "specialised":
        monkeypatch.setenv("MH3D_XWARP_FWD", "1")    # the opt-in warp forward and normal passes too
        monkeypatch.setenv("MH3D_XWARP_NRM", "1")
    elif request.param == "warpsplit":
        monkeypatch.setenv("MH3D_XWARP_FWD", "1")
        monkeypatch.setenv("MH3D_XWARP_KS", "4")
        monkeypatch.setenv("MH3D_XWARP_ZX", "0")     # the warp adjoint and T_z^T as two launches
    elif request.param == "warp1":
        monkeypatch.setenv("MH3D_XWARP_FWD", "1")
        monkeypatch.setenv("MH3D_XWARP_KS", "1")
        monkeypatch.setenv("MH3D_TPASS_RADIX", "1")  # the alternative T-pass schedules (64: 4x16, 128: 8x16)
    elif request.param == "generic":
        monkeypatch.setenv("MH3D_GENERIC", "1")
    elif request.param == "ctalevel":
        monkeypatch.setenv("MH3D_XWARP", "0")
    elif request.param == "alternatives":
        monkeypatch.setenv("MH3D_XWARP", "0")
        monkeypatch.setenv("MH3D_XNRM_BULK", "1")
        monkeypatch.setenv("MH3D_XADJ_BULK", "0")
        monkeypatch.setenv("MH3D_XFWD_KPC", "3")
        monkeypatch.setenv("MH3D_XFWD_PAIRS", "8")
        monkeypatch.setenv("MH3D_FUSE_ZX", "0")
    elif request.param == "cluster4":
        monkeypatch.setenv("MH3D_XWARP", "0")
        monkeypatch.setenv("MH3D_ZX_CLUSTER", "4")
        monkeypatch.setenv("MH3D_XADJ_KB", "2")
    return request.param


@pytest.mark.parametrize("name", ["ds2_theta", "spec96", "spec192", "cube32_k4"])
def test_adjoint_32_row_pipelined_pass_matches_oracle(name, monkeypatch):
    """The 32-row pipelined drive-axis adjoint (MH3D_XADJ_PAIRS=16)."""
    monkeypatch.setenv("MH3D_XADJ_PAIRS", "16")
    p = OP_CASES[name]
    g = oracle_geom(p)
    b = sens_map(p)
    y = W.random_portraits(g.portrait_shape, 202)
    ref = oracle.adjoint(g, y, b)
    plan = gpu_plan(p, b)
    from paper_2503_13802_gb300 import mh3d_adjoint

    rho = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_adjoint(plan, _dev(y, torch.complex64), rho)
    assert rel_l2(rho.cpu().numpy(), ref) <= TOL, rel_l2(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("name", ["ds2_theta", "spec96", "cube32_k4"])
@pytest.mark.parametrize("mode", [0, 1])
def test_normal_32_row_pass_matches_oracle(name, mode, monkeypatch):
    """The 32-row, 256-thread drive-axis normal pass (MH3D_XNRM_PAIRS=16)."""
    monkeypatch.setenv("MH3D_XNRM_PAIRS", "16")
    p = OP_CASES[name]
    g = oracle_geom(p)
    b = sens_map(p)
    x = W.random_volume(g.shape, 301)
    oo = oracle.SolveOpts(lam=2e-2, reg_kind=0)
    ref = oracle.normal_apply(g, x, b, oo)
    plan = gpu_plan(p, b)
    from paper_2503_13802_gb300 import make_opts, mh3d_normal

    q = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_normal(plan, _dev(x, torch.float32), q, make_opts(lam=2e-2, normal_mode=mode))
    assert rel_l2(q.cpu().numpy(), ref) <= TOL, rel_l2(q.cpu().numpy(), ref)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("name", list(OP_CASES))
def test_forward_matches_oracle(name, kernel_path):
    p = OP_CASES[name]
    g = oracle_geom(p)
    b = sens_map(p)
    rho = W.random_volume(g.shape, 100)
    ref = oracle.forward(g, rho, b)
    plan = gpu_plan(p, b)
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    from paper_2503_13802_gb300 import mh3d_forward

    mh3d_forward(plan, _dev(rho, torch.float32), d)
    got = d.cpu().numpy()
    assert rel_l2(got, ref) <= TOL, rel_l2(got, ref)
    for k in range(g.K):
        assert rel_l2(got[k], ref[k]) <= 3 * TOL, (k, rel_l2(got[k], ref[k]))


@pytest.mark.parametrize("name", list(OP_CASES))
def test_adjoint_matches_oracle(name, kernel_path):
    p = OP_CASES[name]
    g = oracle_geom(p)
    b = sens_map(p)
    y = W.random_portraits(g.portrait_shape, 200)
    ref = oracle.adjoint(g, y, b)
    plan = gpu_plan(p, b)
    rho = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    from paper_2503_13802_gb300 import mh3d_adjoint

    mh3d_adjoint(plan, _dev(y, torch.complex64), rho)
    assert rel_l2(rho.cpu().numpy(), ref) <= TOL, rel_l2(rho.cpu().numpy(), ref)


@pytest.mark.parametrize("name", ["cube32_k4", "ds2_theta", "ds3_radix3", "odd_nx27", "tall_z", "zx128", "zx64"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("reg_kind", [0, 1])
def test_normal_matches_oracle(name, mode, reg_kind, kernel_path):
    p = OP_CASES[name]
    g = oracle_geom(p)
    b = sens_map(p)
    x = W.random_volume(g.shape, 300)
    oo = oracle.SolveOpts(lam=2e-2, reg_kind=reg_kind, alpha=4.0, shell=2)
    ref = oracle.normal_apply(g, x, b, oo)
    plan = gpu_plan(p, b)
    from paper_2503_13802_gb300 import make_opts, mh3d_normal

    q = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_normal(plan, _dev(x, torch.float32), q, make_opts(lam=2e-2, reg_kind=reg_kind, alpha=4.0, shell=2,
                                                           normal_mode=mode))
    assert rel_l2(q.cpu().numpy(), ref) <= TOL, rel_l2(q.cpu().numpy(), ref)


def test_delta_phantom_reproduces_psf_on_gpu():
    """A point source at voxel 0 (b = 1, s = 1, theta = 0) gives the sampled
    PSF of every harmonic (Eq. MH3Dcont with rho = delta)."""
    p = OP_CASES["cube32_k4"]
    g = oracle_geom(p)
    X, Y, Z = oracle.psf_tables(g)
    rho = np.zeros(g.shape)
    rho[0, 0, 0] = 1.0
    plan = gpu_plan(p, None)
    from paper_2503_13802_gb300 import mh3d_forward

    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, _dev(rho, torch.float32), d)
    got = d.cpu().numpy()
    for k in range(g.K):
        h = Z[:, None, None] * Y[None, :, None] * X[k][None, None, :]
        assert rel_l2(got[k].real, h) <= TOL
        assert np.abs(got[k].imag).max() == 0.0


def test_gpu_adjoint_identity_fp64_dots():
    """Re<A x, y> = <x, A^T y> for the FP32 GPU operators, dots in FP64."""
    p = OP_CASES["ds2_theta"]
    g = oracle_geom(p)
    b = sens_map(p)
    plan = gpu_plan(p, b)
    from paper_2503_13802_gb300 import mh3d_adjoint, mh3d_forward

    x = W.random_volume(g.shape, 7)
    y = W.random_portraits(g.portrait_shape, 8)
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    r = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_forward(plan, _dev(x, torch.float32), d)
    mh3d_adjoint(plan, _dev(y, torch.complex64), r)
    lhs = np.real(np.vdot(d.cpu().numpy().astype(np.complex128), y))
    rhs = float(np.sum(x * r.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(x) * np.linalg.norm(y) * 0.1


def test_full_size_128x128x64_forward_adjoint(kernel_path):
    """The 128x128x64, K = 8 (k = 2..9), s = 2 workload with a Gaussian
    sensitivity map, at full size in the launch configuration the benchmark
    uses: whole-array comparison with the oracle."""
    from tests._cases import params

    p = params((128, 128, 64), s=2, kmin=2, kmax=9)
    g = oracle_geom(p)
    b = sens_map(p)
    rho = W.phantom((128, 128, 64), (1, 1, 1), 3, 40, 3)
    plan = gpu_plan(p, b)
    from paper_2503_13802_gb300 import mh3d_adjoint, mh3d_forward

    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, _dev(rho, torch.float32), d)
    ref = oracle.forward(g, rho, b)
    assert rel_l2(d.cpu().numpy(), ref) <= TOL
    y = W.random_portraits(g.portrait_shape, 5)
    r = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_adjoint(plan, _dev(y, torch.complex64), r)
    assert rel_l2(r.cpu().numpy(), oracle.adjoint(g, y, b)) <= TOL


def test_unsupported_and_invalid_sizes_are_rejected():
    from paper_2503_13802_gb300 import MH3DError
    from tests._cases import params

    with pytest.raises(MH3DError) as e:
        gpu_plan(params((35, 8, 8)))               # prime factor 5 and 7
    assert "UNSUPPORTED_SIZE" in str(e.value)
    with pytest.raises(MH3DError) as e:
        gpu_plan(params((32, 8, 8), s=3))           # nx not a multiple of s
    assert "UNSUPPORTED_SIZE" in str(e.value)
    with pytest.raises(MH3DError) as e:
        gpu_plan(params((32, 8, 8), kmin=1))
    assert "INVALID_ARG" in str(e.value)
    with pytest.raises(MH3DError) as e:
        gpu_plan(params((32, 8, 8), gammaA=3.2))    # |gamma A| >= pi (Theorem 1)
    assert "INVALID_ARG" in str(e.value)
