"""The general model on the GPU (mh3d_general_set_psf / _forward / _adjoint):
three receive components with the tensor PSF's harmonic PSFs (Sec. 3.2,
Eq. MH3Dcont, Eq. matrixModel; appendix, Eq. PSF, Eq. skMD), against the
FP64 oracle (oracle/vector_model.py) on the same float32 PSF samples,
densities, sensitivities and portraits.  Tolerance: relative L2 1e-5, as for
the separable operators (FP32 transforms of a few hundred points)."""
import numpy as np
import pytest

import oracle
from oracle import vector_model as vm
from tests._cases import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5
CASES = {
    "s2_r1_vector_b": (dict(n=(16, 8, 8), s=2, r=1, kmin=2, kmax=5), True),
    "s1_drive_b": (dict(n=(24, 12, 8), s=1, r=0, kmin=2, kmax=4), False),
    "s2_r0_vector_b": (dict(n=(32, 16, 8), s=2, r=0, kmin=2, kmax=6), True),
    # s = 3 (the fold's s <= 4 register form) and s = 6 (its any-s form)
    "s3_r2_vector_b": (dict(n=(24, 8, 6), s=3, r=2, kmin=2, kmax=4), True),
    "s6_r5_drive_b": (dict(n=(36, 8, 4), s=6, r=5, kmin=2, kmax=3), False),
    # lengths 128 and 64 on the compile-time pencil kernel: x (b_j rho fused
    # in its load), y and the portrait x (the unphasing fused); then z (the
    # phase fused in its store)
    "ct_lengths_vector_b": (dict(n=(128, 64, 8), s=2, r=1, kmin=2, kmax=5), True),
    "ct_z64_drive_b": (dict(n=(16, 8, 64), s=2, r=0, kmin=2, kmax=4), False),
    # odd n_z and n_y: the half-spectrum fold's mirror planes without a middle plane
    "odd_nz9_vector_b": (dict(n=(16, 9, 9), s=2, r=1, kmin=2, kmax=4), True),
}


def _theta(c, seed):
    return list(np.random.default_rng(seed).uniform(-3.0, 3.0, c["kmax"] - c["kmin"] + 1))


def _geom(c, theta):
    return oracle.Geometry(n=c["n"], ds_factor=c["s"], ds_offset=c["r"], k_min=c["kmin"], k_max=c["kmax"],
                           theta=theta)


def _plan(c, theta):
    from paper_2503_13802_gb300 import Plan

    return Plan(c["n"], ds_factor=c["s"], ds_offset=c["r"], k_min=c["kmin"], k_max=c["kmax"], theta=theta)


@pytest.mark.parametrize("kernels", ["default", "runtime"])
@pytest.mark.parametrize("name", list(CASES))
def test_general_forward_and_adjoint_match_oracle(name, kernels, monkeypatch):
    """kernels = runtime: every pencil pass on the runtime-schedule kernel
    (MH3D_GEN_RUNTIME=1), the weighting, phase and unphasing as separate
    kernels."""
    if kernels == "runtime":
        monkeypatch.setenv("MH3D_GEN_RUNTIME", "1")
    else:
        monkeypatch.delenv("MH3D_GEN_RUNTIME", raising=False)
    from paper_2503_13802_gb300 import mh3d_general_adjoint, mh3d_general_forward, mh3d_general_set_psf

    c, use_b = CASES[name]
    theta = _theta(c, 7)
    g = _geom(c, theta)
    H = vm.general_psf(g).astype(np.float32)
    plan = _plan(c, theta)
    mh3d_general_set_psf(plan, H)
    rng = np.random.default_rng(17)
    rho = rng.standard_normal(g.shape).astype(np.float32)
    bvec = (0.3 + rng.random((3,) + tuple(g.shape))).astype(np.float32) if use_b else None
    bt = torch.as_tensor(bvec).cuda().contiguous() if use_b else None
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_general_forward(plan, torch.as_tensor(rho).cuda().contiguous(), d, bt)
    b64 = None if bvec is None else bvec.astype(np.float64)
    ref = vm.general_forward(g, rho.astype(np.float64), b64, H.astype(np.float64))
    assert rel_l2(d.cpu().numpy(), ref) <= TOL, rel_l2(d.cpu().numpy(), ref)
    y = (rng.standard_normal(g.portrait_shape) + 1j * rng.standard_normal(g.portrait_shape)).astype(np.complex64)
    out = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_general_adjoint(plan, torch.as_tensor(y).cuda().contiguous(), out, bt)
    ref_a = vm.general_adjoint(g, y.astype(np.complex128), b64, H.astype(np.float64))
    assert rel_l2(out.cpu().numpy(), ref_a) <= TOL, rel_l2(out.cpu().numpy(), ref_a)


def test_general_argument_checks():
    from paper_2503_13802_gb300 import MH3DError, Plan, mh3d_general_forward, mh3d_general_set_psf

    c, _ = CASES["s2_r1_vector_b"]
    plan = _plan(c, None)
    K, nz, ny, mx = plan.portrait_shape
    d = torch.empty(plan.portrait_shape, dtype=torch.complex64, device="cuda")
    rho = torch.zeros(plan.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(MH3DError) as e:      # no PSF set yet
        mh3d_general_forward(plan, rho, d)
    assert "INVALID_ARG" in str(e.value)
    padded = Plan((32, 8, 8), ds_factor=2, k_min=2, k_max=3, pad=(2, 2, 0))
    with pytest.raises(MH3DError) as e:
        mh3d_general_set_psf(padded, np.zeros(padded.K * 3 * padded.N, dtype=np.float32))
    assert "INVALID_ARG" in str(e.value)


def _lam_for(g, H, bvec, rel=1e-2):
    """An absolute lambda of rel times ||A||_2^2 (power iteration with the
    oracle's general normal operator, lambda = 0)."""
    v = np.random.default_rng(3).standard_normal(g.shape)
    lam = 0.0
    for _ in range(60):
        w = vm.general_normal_apply(g, v, 0.0, bvec, H)
        lam = float(np.vdot(v, w) / np.vdot(v, v))
        v = w / np.linalg.norm(w)
    return rel * lam


@pytest.mark.parametrize("name", ["s2_r1_vector_b", "s2_r0_vector_b"])
def test_general_solve_matches_oracle_cg(name):
    """CG on the general model (Sec. 4.3 with A of Eq. matrixModel), through
    mh3d_general_solve, against the oracle's general CG (pinned against the
    dense FP64 solve of the normal equations), with the comparisons of
    reading r2 (FP32 and FP64 CG follow different rounding paths): (a) after
    a fixed 10 iterations from zero, the residual histories agreeing while
    far above FP32 resolution; (b) both to a common relative residual of
    1e-6, against the oracle solved to 1e-11; (c) from a warm start that is
    the solution, which stops at once."""
    from paper_2503_13802_gb300 import make_opts, mh3d_general_set_psf, mh3d_general_solve

    c, use_b = CASES[name]
    theta = _theta(c, 11)
    g = _geom(c, theta)
    H = vm.general_psf(g).astype(np.float32)
    H64 = H.astype(np.float64)
    plan = _plan(c, theta)
    mh3d_general_set_psf(plan, H)
    rng = np.random.default_rng(23)
    bvec = (0.3 + rng.random((3,) + tuple(g.shape))).astype(np.float32) if use_b else None
    b64 = None if bvec is None else bvec.astype(np.float64)
    rho = np.abs(rng.standard_normal(g.shape))
    d = vm.general_forward(g, rho, b64, H64)
    d = d + 0.05 * np.abs(d).max() * (rng.standard_normal(d.shape) + 1j * rng.standard_normal(d.shape))
    lam = _lam_for(g, H64, b64)
    bt = torch.as_tensor(bvec).cuda().contiguous() if use_b else None
    dd = torch.as_tensor(d.astype(np.complex64)).cuda().contiguous()
    x = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    # (a)
    xo, it = vm.general_cg(g, d, lam, 10, b64, H64)
    info = mh3d_general_solve(plan, dd, make_opts(lam=lam, max_iter=10, fixed_iters=True), x, bt)
    assert info["iters"] == 10 and info["status"] == 0, info
    assert rel_l2(x.cpu().numpy(), xo) <= 1e-4, rel_l2(x.cpu().numpy(), xo)
    rhs = vm.general_adjoint(g, d, b64, H64)
    r = rhs.copy()
    p = r.copy()
    hist = [1.0]
    for _ in range(6):     # the oracle's own recurrence residuals, textbook CG
        q = vm.general_normal_apply(g, p, lam, b64, H64)
        a = float(np.vdot(r, r)) / float(np.vdot(p, q))
        rn = r - a * q
        p = rn + float(np.vdot(rn, rn)) / float(np.vdot(r, r)) * p
        r = rn
        hist.append(float(np.linalg.norm(r) / np.linalg.norm(rhs)))
    np.testing.assert_allclose(info["history"][:7], hist, rtol=1e-4)
    # (b)
    tight, _ = vm.general_cg(g, d, lam, 5000, b64, H64, rel_tol=1e-11)
    xo6, _ = vm.general_cg(g, d, lam, 5000, b64, H64, rel_tol=1e-6)
    info = mh3d_general_solve(plan, dd, make_opts(lam=lam, rel_tol=1e-6, max_iter=5000), x, bt)
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-5, info
    assert rel_l2(x.cpu().numpy(), tight) <= 1e-4, rel_l2(x.cpu().numpy(), tight)
    assert rel_l2(x.cpu().numpy(), xo6) <= 1e-4, rel_l2(x.cpu().numpy(), xo6)
    # (c)
    x0 = torch.as_tensor(tight.astype(np.float32)).cuda().contiguous()
    info = mh3d_general_solve(plan, dd, make_opts(lam=lam, rel_tol=1e-4, max_iter=100, x0=x0), x, bt)
    assert info["status"] == 0 and info["iters"] <= 1, info


def test_general_solve_rejects_unsupported_options():
    from paper_2503_13802_gb300 import MH3DError, make_opts, mh3d_general_set_psf, mh3d_general_solve

    c, _ = CASES["s1_drive_b"]
    g = _geom(c, None)
    plan = _plan(c, None)
    d = torch.zeros(plan.portrait_shape, dtype=torch.complex64, device="cuda")
    x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(MH3DError) as e:          # no PSF yet
        mh3d_general_solve(plan, d, make_opts(lam=1e-2), x)
    assert "INVALID_ARG" in str(e.value)
    mh3d_general_set_psf(plan, vm.general_psf(g).astype(np.float32))
    for bad in (make_opts(lam=1e-2, lam_relative=True), make_opts(lam=1e-2, solver=1),
                make_opts(lam=1e-2, reg_kind=1), make_opts(lam=0.0)):
        with pytest.raises(MH3DError) as e:
            mh3d_general_solve(plan, d, bad, x)
        assert "INVALID_ARG" in str(e.value)
    info = mh3d_general_solve(plan, d, make_opts(lam=1e-2), x)    # zero data: zero at once
    assert info["status"] == 0 and info["iters"] == 0
    assert float(torch.abs(x).max()) == 0.0
