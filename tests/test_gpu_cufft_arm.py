"""The benchmark's cuFFT comparison arm computes the same operators as the
library (so its timings compare like with like): A and A^T through
torch.fft from the plan's exported spectra agree with mh3d_forward /
mh3d_adjoint to FP32 accuracy, and the exported spectra are the FFTs of the
oracle's PSF samples."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import gpu_plan, oracle_geom, params, rel_l2, sens_map

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("p", [params((64, 32, 16), s=2, r=1, kmin=2, kmax=6, theta=[0.3, -1.1, 2.0, 0.5, 1.4]),
                               params((128, 128, 64), s=2, kmin=2, kmax=9)])
def test_cufft_arm_matches_library(p):
    import bench
    from paper_2503_13802_gb300 import mh3d_adjoint, mh3d_forward

    g = oracle_geom(p)
    b = sens_map(p)
    plan = gpu_plan(p, b)
    bt = torch.as_tensor(b, dtype=torch.float32, device="cuda").contiguous()
    cf = bench.CufftOperators(plan, bt)
    rho = torch.as_tensor(W.random_volume(g.shape, 3), dtype=torch.float32, device="cuda").contiguous()
    d0 = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    d1 = torch.empty_like(d0)
    mh3d_forward(plan, rho, d0)
    cf.forward(rho, d1)
    assert rel_l2(d1.cpu().numpy(), d0.cpu().numpy()) <= 1e-5
    y = torch.as_tensor(W.random_portraits(g.portrait_shape, 4).astype(np.complex64), device="cuda").contiguous()
    r0 = torch.empty_like(rho)
    r1 = torch.empty_like(rho)
    mh3d_adjoint(plan, y, r0)
    cf.adjoint(y, r1)
    assert rel_l2(r1.cpu().numpy(), r0.cpu().numpy()) <= 1e-5


def test_exported_spectra_are_dfts_of_oracle_samples():
    from paper_2503_13802_gb300 import mh3d_plan_spectra

    p = params((48, 24, 12), s=3, r=2, kmin=2, kmax=5)
    g = oracle_geom(p)
    plan = gpu_plan(p, None)
    X, Y, Z, ph = mh3d_plan_spectra(plan)
    Xo, Yo, Zo = oracle.psf_tables(g)
    nx, ny, nz = p["n"]
    # drive samples shifted by the row offset r: X'_k[o] = X_k[o + r]
    Xs = np.roll(Xo, -p["r"], axis=1)
    assert rel_l2(X.cpu().numpy(), np.fft.fft(Xs, axis=1) / nx) <= 1e-6
    assert rel_l2(Y.cpu().numpy(), np.fft.fft(Yo) / ny) <= 1e-6
    assert rel_l2(Z.cpu().numpy(), np.fft.fft(Zo) / nz) <= 1e-6
    assert np.allclose(ph.cpu().numpy(), 1.0)
