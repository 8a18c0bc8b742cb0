"""Boundary image padding (Sec. 3.x): the model on the field of view
extended by pad voxels per side, portraits cropped to the field of view,
against the FP64 oracle's padded operators (oracle.padded_forward,
padded_adjoint, padded_cg), through the C ABI.

Tolerances: the FP32 operators to relative L2 1e-5, the solve at a fixed
iteration count to 1e-4, as for the unpadded plans.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import gpu_plan, oracle_geom, params, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5
CASES = {
    # field of view, padding (px a multiple of s); specialised and general lengths
    "ds2_pad": (params((48, 20, 12), s=2, r=1, kmin=2, kmax=6, theta=[0.3, -0.8, 1.9, 2.4, -1.3]), (8, 2, 2)),
    "s1_pad": (params((24, 12, 8), s=1, kmin=2, kmax=4), (4, 2, 4)),
    "cube_pad": (params((56, 56, 24), s=2, kmin=2, kmax=9), (4, 4, 4)),   # 64 x 64 x 32 padded
}


def _sens_ext(g_ext):
    nx, ny, nz = g_ext.n
    return W.sensitivity((nx, ny, nz), g_ext.voxel_mm, kind="gaussian")


def _plan(p, pad, b_ext):
    from paper_2503_13802_gb300 import Plan

    return Plan(p["n"], voxel_mm=p["voxel"], ds_factor=p["s"], ds_offset=p["r"], k_min=p["kmin"], k_max=p["kmax"],
                gamma_per_mm=p["gamma"], gammaA=p["gammaA"], transverse_ratio=p["tratio"], theta=p["theta"],
                sensitivity=b_ext, pad=pad)


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("name", list(CASES))
def test_padded_forward_and_adjoint_match_oracle(name):
    from paper_2503_13802_gb300 import mh3d_adjoint, mh3d_forward

    p, pad = CASES[name]
    g = oracle_geom(p)
    ge = oracle.padded_geometry(g, pad)
    b = _sens_ext(ge)
    plan = _plan(p, pad, b)
    assert plan.shape == ge.shape and plan.portrait_shape == g.portrait_shape
    rho = W.random_volume(ge.shape, 501)
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, _dev(rho, torch.float32), d)
    ref = oracle.padded_forward(g, pad, rho, b)
    assert rel_l2(d.cpu().numpy(), ref) <= TOL, rel_l2(d.cpu().numpy(), ref)
    y = W.random_portraits(g.portrait_shape, 502)
    r = torch.empty(ge.shape, dtype=torch.float32, device="cuda")
    mh3d_adjoint(plan, _dev(y, torch.complex64), r)
    ref_a = oracle.padded_adjoint(g, pad, y.astype(np.complex64).astype(np.complex128), b)
    assert rel_l2(r.cpu().numpy(), ref_a) <= TOL, rel_l2(r.cpu().numpy(), ref_a)


@pytest.mark.parametrize("name", ["ds2_pad", "s1_pad"])
def test_padded_normal_operator_matches_oracle(name):
    """mh3d_normal on a padded plan is A_p^T A_p + lambda I, whatever
    normal_mode the options name."""
    from paper_2503_13802_gb300 import make_opts, mh3d_normal

    p, pad = CASES[name]
    g = oracle_geom(p)
    ge = oracle.padded_geometry(g, pad)
    b = _sens_ext(ge)
    plan = _plan(p, pad, b)
    x = W.random_volume(ge.shape, 503)
    lam = 2e-2
    ref = oracle.padded_adjoint(g, pad, oracle.padded_forward(g, pad, x, b), b) + lam * x
    for mode in (0, 1):
        q = torch.empty(ge.shape, dtype=torch.float32, device="cuda")
        mh3d_normal(plan, _dev(x, torch.float32), q, make_opts(lam=lam, normal_mode=mode))
        assert rel_l2(q.cpu().numpy(), ref) <= TOL, (mode, rel_l2(q.cpu().numpy(), ref))


@pytest.mark.parametrize("variant", [0, 1])
def test_padded_solve_matches_oracle_at_fixed_iterations(variant):
    from paper_2503_13802_gb300 import make_opts, mh3d_solve

    p, pad = CASES["ds2_pad"]
    g = oracle_geom(p)
    ge = oracle.padded_geometry(g, pad)
    b = _sens_ext(ge)
    plan = _plan(p, pad, b)
    rho = W.phantom(g.n, g.voxel_mm, 31, 8, 1)
    rho_ext = np.zeros(ge.shape)
    px, py, pz = pad
    nx, ny, nz = g.n
    rho_ext[pz:pz + nz, py:py + ny, px:px + nx] = rho
    d = oracle.padded_forward(g, pad, rho_ext, b)
    d = d + 0.02 * math.sqrt(float(np.mean(np.abs(d) ** 2))) * W.unit_complex_noise(d.shape, 31)
    d64 = d.astype(np.complex64)
    lam, iters = 5e-2, 25
    x = torch.empty(ge.shape, dtype=torch.float32, device="cuda")
    info = mh3d_solve(plan, _dev(d64, torch.complex64),
                      make_opts(lam=lam, rel_tol=0.0, max_iter=iters, fixed_iters=True, cg_variant=variant), x)
    assert info["iters"] == iters
    ref = oracle.padded_cg(g, pad, d64.astype(np.complex128), b, lam, iters)
    assert rel_l2(x.cpu().numpy(), ref) <= 1e-4, rel_l2(x.cpu().numpy(), ref)


def test_padding_removes_wraparound_of_an_edge_phantom():
    """The paper's padding experiment, synthetically: blobs at the field of
    view's edges, data from the model on a grid padded well beyond the PSF
    (no wrap-around reaches the field of view), reconstructed without
    padding (the circular model on the field of view) and with 8 / 4 / 4
    voxels of padding.  The reference is the same regularised solve with the
    wrap-free model (FP64 oracle); inside the field of view the padded
    reconstruction is the closer one."""
    from paper_2503_13802_gb300 import make_opts, mh3d_solve

    p = params((32, 16, 8), s=2, kmin=2, kmax=5)
    g = oracle_geom(p)
    nx, ny, nz = g.n
    big = (16, 8, 8)                        # data model: (64, 32, 24) voxels
    gb = oracle.padded_geometry(g, big)
    rho = np.zeros(g.shape)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for (cx, cy, cz) in [(1.0, 8.0, 4.0), (30.5, 5.0, 3.0), (15.0, 0.5, 4.0), (12.0, 12.0, 7.0)]:
        rho += np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2) / (2 * 1.5 ** 2))
    rho_big = np.zeros(gb.shape)
    rho_big[big[2]:big[2] + nz, big[1]:big[1] + ny, big[0]:big[0] + nx] = rho
    d = oracle.padded_forward(g, big, rho_big)
    d = (d + 1e-3 * math.sqrt(float(np.mean(np.abs(d) ** 2))) * W.unit_complex_noise(d.shape, 7)).astype(np.complex64)
    lam = 1e-3 * oracle.operator_norm2(g)   # one absolute weight for every solve
    ref_big = oracle.padded_cg(g, big, d.astype(np.complex128), None, lam, 400)
    ref = ref_big[big[2]:big[2] + nz, big[1]:big[1] + ny, big[0]:big[0] + nx]
    errs = {}
    for pad in [(0, 0, 0), (8, 4, 4)]:
        plan = _plan(p, pad, None)
        x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
        info = mh3d_solve(plan, _dev(d, torch.complex64), make_opts(lam=lam, rel_tol=1e-5, max_iter=5000), x)
        assert info["status"] == 0, (pad, info)
        px, py, pz = pad
        xf = x.cpu().numpy()[pz:pz + nz, py:py + ny, px:px + nx]
        errs[pad] = rel_l2(xf, ref)
    print(f"\nfield-of-view error against the wrap-free reconstruction: {errs}")
    assert errs[(8, 4, 4)] < 0.5 * errs[(0, 0, 0)], errs


def test_padded_plan_argument_checks():
    from paper_2503_13802_gb300 import MH3DError, Plan, make_opts, mh3d_mhad, mh3d_solve_batched

    with pytest.raises(MH3DError) as e:
        Plan((32, 8, 8), ds_factor=2, k_min=2, k_max=3, pad=(3, 0, 0))   # px not a multiple of s
    assert "INVALID_ARG" in str(e.value)
    with pytest.raises(MH3DError) as e:
        Plan((32, 8, 8), ds_factor=2, k_min=2, k_max=3, pad=(2, 1, 0))   # 10 in y: factor 5
    assert "UNSUPPORTED_SIZE" in str(e.value)
    plan = Plan((32, 8, 8), ds_factor=2, k_min=2, k_max=3, pad=(2, 2, 0))
    d = torch.zeros(plan.portrait_shape, dtype=torch.complex64, device="cuda")
    x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(MH3DError) as e:
        mh3d_solve_batched([plan], [d], make_opts(lam=1e-3), [x])
    assert "INVALID_ARG" in str(e.value)
    K, nz, ny, mx = plan.portrait_shape
    with pytest.raises(MH3DError) as e:
        mh3d_mhad(plan, d, 1e-2, torch.empty(nz * ny * mx, dtype=torch.float32, device="cuda"))
    assert "INVALID_ARG" in str(e.value)
