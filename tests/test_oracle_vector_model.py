"""Pins of the general-model oracle (oracle/vector_model.py): the vector
convolution model with the tensor PSF (Sec. 3.2, Eq. MH3Dcont, Eq.
matrixModel; appendix, Eq. PSF and Eq. skMD).

* On the drive axis the tensor PSF's drive row reduces to gamma L'(gamma x),
  so the harmonic PSF equals the separable model's drive-axis table exactly,
  and the transverse components vanish.
* Off the axis, the Taylor-mode derivatives equal a 40-digit numerical
  differentiation of the closed form (mpmath), an independent computation.
* Parities that the closed form fixes: the y component is odd in y, the z
  component odd in z, the drive component even in both; along the drive
  axis the drive component has parity (-1)^(k-1) and the others (-1)^k.
* The convolution, row selector and phase: with the separable PSF placed in
  the drive component and b = (b, 0, 0), the FFT-based forward equals the
  pinned separable oracle (C, direct sums); on a tiny grid it equals a
  brute-force sum; and the adjoint satisfies Re<A x, y> = <x, A^T y>.
* CG on the normal equations reaches the dense FP64 solution of
  (A^T A + lambda I) x = A^T d, the matrix built column by column from the
  forward operator on a tiny grid.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import vector_model as vm

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _geom(n=(16, 8, 8), s=1, r=0, kmin=2, kmax=6, theta=None, voxel=(1.0, 1.0, 1.0)):
    return oracle.Geometry(n=n, voxel_mm=voxel, ds_factor=s, ds_offset=r, k_min=kmin, k_max=kmax, theta=theta)


def test_drive_axis_equals_the_separable_table():
    g = _geom(kmin=2, kmax=9)
    H = vm.general_psf(g)
    X, _, _ = oracle.psf_tables(g)
    np.testing.assert_allclose(H[:, 0, 0, 0, :], X, rtol=1e-15, atol=0.0)
    assert np.abs(H[:, 1:, 0, 0, :]).max() == 0.0


def test_off_axis_derivatives_match_high_precision_differentiation():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    g = _geom(kmin=2, kmax=7)
    gam = g.gamma_per_mm
    gt = gam * g.transverse_ratio

    def h0j(j, xd, y, z):
        u = [gam * xd, gt * mp.mpf(y), gt * mp.mpf(z)]
        r = mp.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
        L = mp.coth(r) - 1 / r
        Lp = 1 / r ** 2 - 1 / mp.sinh(r) ** 2
        gj = [gam, gt, gt][j]
        return gj * ((Lp - L / r) * u[0] * u[j] / r ** 2 + (L / r if j == 0 else 0))

    pts = [(0.7, 1.0, 0.0), (-1.3, 0.5, 2.0), (2.0, -1.0, -1.0), (0.0, 2.0, 1.0), (3.0, 0.0, -1.0)]
    h = vm.harmonic_psf_at(g, [p[0] for p in pts], [p[1] for p in pts], [p[2] for p in pts])
    for pi, (xd, y, z) in enumerate(pts):
        for kk, k in enumerate(range(g.k_min, g.k_max + 1)):
            for j in range(3):
                d = mp.diff(lambda t: h0j(j, t, y, z), mp.mpf(xd), k - 1)
                ref = float(d) * g.gammaA ** k * gam ** (-k) / math.factorial(k - 1)
                assert h[kk, j, pi] == pytest.approx(ref, rel=1e-10, abs=1e-14), (pts[pi], k, j)


def test_parities_of_the_harmonic_psfs():
    g = _geom(n=(16, 8, 8), kmin=2, kmax=6)
    H = vm.general_psf(g)
    nx, ny, nz = g.n
    iy = np.arange(1, ny // 2)
    iz = np.arange(1, nz // 2)
    ix = np.arange(1, nx // 2)
    for kk, k in enumerate(range(g.k_min, g.k_max + 1)):
        h0, h1, h2 = H[kk]
        # y: the y component odd, the others even
        np.testing.assert_allclose(h1[:, iy, :], -h1[:, ny - iy, :], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h0[:, iy, :], h0[:, ny - iy, :], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h2[:, iy, :], h2[:, ny - iy, :], rtol=1e-12, atol=1e-15)
        # z: the z component odd, the others even
        np.testing.assert_allclose(h2[iz], -h2[nz - iz], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h0[iz], h0[nz - iz], rtol=1e-12, atol=1e-15)
        # drive axis: (-1)^(k-1) for the drive component, (-1)^k for the others
        sd = (-1.0) ** (k - 1)
        np.testing.assert_allclose(h0[:, :, ix], sd * h0[:, :, nx - ix], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h1[:, :, ix], -sd * h1[:, :, nx - ix], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h2[:, :, ix], -sd * h2[:, :, nx - ix], rtol=1e-12, atol=1e-15)


def test_separable_psf_in_the_drive_component_reproduces_the_separable_oracle():
    g = _geom(n=(16, 8, 4), s=2, r=1, kmin=2, kmax=5, theta=[0.3, -1.1, 2.0, 0.7])
    X, Y, Z = oracle.psf_tables(g)
    H = np.zeros((g.K, 3) + tuple(g.shape))
    H[:, 0] = Z[None, :, None, None] * Y[None, None, :, None] * X[:, None, None, :]
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(g.shape)
    b = 0.5 + rng.random(g.shape)
    bvec = np.zeros((3,) + tuple(g.shape))
    bvec[0] = b
    bvec[1] = rng.standard_normal(g.shape)   # ignored: its PSF component is zero
    d = vm.general_forward(g, rho, bvec, H)
    ref = oracle.forward(g, rho, b)
    np.testing.assert_allclose(d, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_fft_forward_equals_a_brute_force_sum_on_a_tiny_grid():
    g = _geom(n=(6, 4, 4), s=2, r=0, kmin=2, kmax=4, theta=[0.4, -0.9, 1.7])
    H = vm.general_psf(g)
    rng = np.random.default_rng(9)
    rho = rng.standard_normal(g.shape)
    bvec = rng.standard_normal((3,) + tuple(g.shape))
    d = vm.general_forward(g, rho, bvec, H)
    nx, ny, nz = g.n
    th = g.theta_array()
    ref = np.zeros(g.portrait_shape, dtype=np.complex128)
    for kk in range(g.K):
        for z in range(nz):
            for y in range(ny):
                for ip in range(nx // g.ds_factor):
                    x = g.ds_factor * ip + g.ds_offset
                    acc = 0.0
                    for j in range(3):
                        for zp in range(nz):
                            for yp in range(ny):
                                for xp in range(nx):
                                    acc += (H[kk, j, (z - zp) % nz, (y - yp) % ny, (x - xp) % nx]
                                            * bvec[j, zp, yp, xp] * rho[zp, yp, xp])
                    ref[kk, z, y, ip] = np.exp(1j * th[kk]) * acc
    np.testing.assert_allclose(d, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_adjoint_identity():
    g = _geom(n=(16, 8, 8), s=2, r=1, kmin=2, kmax=6, theta=[0.2, 1.4, -2.2, 0.9, -0.4])
    H = vm.general_psf(g)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(g.shape)
    bvec = rng.standard_normal((3,) + tuple(g.shape))
    y = rng.standard_normal(g.portrait_shape) + 1j * rng.standard_normal(g.portrait_shape)
    lhs = float(np.real(np.vdot(y, vm.general_forward(g, x, bvec, H))))
    rhs = float(np.dot(x.ravel(), vm.general_adjoint(g, y, bvec, H).ravel()))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_cg_reaches_the_dense_normal_equations_solution():
    g = _geom(n=(6, 4, 2), s=2, r=1, kmin=2, kmax=4, theta=[0.5, -0.3, 1.2])
    H = vm.general_psf(g)
    rng = np.random.default_rng(21)
    bvec = 0.2 + rng.random((3,) + tuple(g.shape))
    d = rng.standard_normal(g.portrait_shape) + 1j * rng.standard_normal(g.portrait_shape)
    N = int(np.prod(g.shape))
    # A as a real matrix on (Re d, Im d), one column per unit voxel
    cols = []
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        f = vm.general_forward(g, e.reshape(g.shape), bvec, H).ravel()
        cols.append(np.concatenate([f.real, f.imag]))
    A = np.stack(cols, axis=1)
    lam = 1e-2 * float(np.linalg.norm(A, 2) ** 2)
    dv = np.concatenate([d.ravel().real, d.ravel().imag])
    x_dense = np.linalg.solve(A.T @ A + lam * np.eye(N), A.T @ dv)
    x, it = vm.general_cg(g, d, lam, 500, bvec, H, rel_tol=1e-13)
    assert it < 500
    np.testing.assert_allclose(x.ravel(), x_dense, rtol=1e-9, atol=1e-10 * np.abs(x_dense).max())
