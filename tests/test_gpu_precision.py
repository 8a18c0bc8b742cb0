"""Precision of the FP32 operators at scale: 256x256x128, K = 16 (k = 2..17),
s = 1, uniform sensitivity, 200 blobs with amplitudes 10^U(-3,0).

The GPU evaluates the whole volume; the FP64 oracle evaluates a 64^3 output
crop directly in space (forward_crop / adjoint_crop).  Reported per result
and per harmonic:

* whole-crop relative L2 error <= 1e-5 (the FP32 operator tolerance);
* per harmonic, the error of harmonic k is bounded by FP32 round-off of
  the three FFT passes: every pass of length n adds at most about
  eps * (log2 n + 1) relative to the L2 norm of its input, and the
  spectral gains that follow scale it, so
      ||err_k|| <= C eps (sum_a log2 n_a + 3) |X^_k|_inf |Y^|_inf |Z^|_inf ||b rho||,
  taken over the crop by its share sqrt(crop / volume) of a spread-out
  error, with eps = 2^-24 and C = 4.  High harmonics have small outputs
  for a smooth phantom next to their spectral gain, so their relative
  error is larger; this bound is what FP32 arithmetic allows them.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24
CROP_FWD = ((96, 64), (96, 64), (32, 64))   # (i along drive), y, z
CROP_ADJ = ((96, 64), (96, 64), (32, 64))   # x, y, z


def _setup(seed=0):
    wl = W.WORKLOADS["precision_256x256x128_k16"]
    g = oracle.Geometry(n=wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
    rho = W.phantom(wl.n, wl.voxel_mm, seed, wl.n_blobs, wl.n_lines, wl.log_amplitudes)
    return wl, g, rho


def _spectral_gains(g, tables):
    X, Y, Z = tables
    gx = np.abs(np.fft.fft(X, axis=-1)).max(axis=-1)   # per harmonic
    return gx, np.abs(np.fft.fft(Y)).max(), np.abs(np.fft.fft(Z)).max()


def test_precision_forward_per_harmonic_256x256x128_k16():
    wl, g, rho = _setup(0)
    from paper_2503_13802_gb300 import Plan, mh3d_forward

    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, torch.as_tensor(rho, dtype=torch.float32, device="cuda").contiguous(), d)
    (i0, ni), (y0, nyc), (z0, nzc) = CROP_FWD
    got = d[:, z0:z0 + nzc, y0:y0 + nyc, i0:i0 + ni].cpu().numpy().astype(np.complex128)
    del d
    tables = oracle.psf_tables(g)
    ref = oracle.forward_crop(g, rho, CROP_FWD, None, tables)
    total = rel_l2(got, ref)
    gx, gy, gz = _spectral_gains(g, tables)
    nx, ny, nz = wl.n
    stages = math.log2(nx) + math.log2(ny) + math.log2(nz) + 3
    share = math.sqrt(ni * nyc * nzc / (nx * ny * nz))
    rho_norm = float(np.linalg.norm(rho))
    print(f"\nforward 256x256x128 K=16: whole-crop rel L2 = {total:.3e}")
    print(" k   rel L2 err    bound     |d_k|/|d|")
    dn = np.linalg.norm(ref)
    for j in range(g.K):
        e = rel_l2(got[j], ref[j])
        nk = float(np.linalg.norm(ref[j]))
        bound = 4 * EPS32 * stages * gx[j] * gy * gz * rho_norm * share / nk
        print(f"{g.k_min + j:3d}  {e:.3e}   {bound:.3e}   {nk / dn:.3e}")
        assert e <= bound, (g.k_min + j, e, bound)
    assert total <= 1e-5, total


def test_precision_adjoint_256x256x128_k16():
    wl, g, _ = _setup(0)
    from paper_2503_13802_gb300 import Plan, mh3d_adjoint

    y = W.random_portraits(g.portrait_shape, 41)
    plan = Plan(wl.n, voxel_mm=wl.voxel_mm, ds_factor=wl.ds_factor, k_min=wl.k_min, k_max=wl.k_max)
    r = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    mh3d_adjoint(plan, torch.as_tensor(y.astype(np.complex64), device="cuda").contiguous(), r)
    (x0, nxc), (y0, nyc), (z0, nzc) = CROP_ADJ
    got = r[z0:z0 + nzc, y0:y0 + nyc, x0:x0 + nxc].cpu().numpy().astype(np.float64)
    ref = oracle.adjoint_crop(g, y, CROP_ADJ, None)
    e = rel_l2(got, ref)
    print(f"\nadjoint 256x256x128 K=16 on white portraits: crop rel L2 = {e:.3e}")
    assert e <= 1e-5, e
