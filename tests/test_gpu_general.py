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
}


def _theta(c, seed):
    return list(np.random.default_rng(seed).uniform(-3.0, 3.0, c["kmax"] - c["kmin"] + 1))


def _geom(c, theta):
    return oracle.Geometry(n=c["n"], ds_factor=c["s"], ds_offset=c["r"], k_min=c["kmin"], k_max=c["kmax"],
                           theta=theta)


def _plan(c, theta):
    from paper_2503_13802_gb300 import Plan

    return Plan(c["n"], ds_factor=c["s"], ds_offset=c["r"], k_min=c["kmin"], k_max=c["kmax"], theta=theta)


@pytest.mark.parametrize("name", list(CASES))
def test_general_forward_and_adjoint_match_oracle(name):
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
