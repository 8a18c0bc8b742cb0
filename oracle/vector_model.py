"""FP64 CPU oracle for the general MH3D model: the vector (three-component)
convolution model with the tensor PSF (Sec. 3.2, Eq. MH3Dcont and Eq.
matrixModel; appendix derivation, Eq. PSF and Eq. skMD).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by
``tests/`` only; it shares no code with the CUDA path (general.cu), which
``tests/test_gpu_general.py`` compares with it.  These functions are pinned
by ``tests/test_oracle_vector_model.py``.

Axes follow the separable oracle: arrays are [nz][ny][nx], the drive axis is
x (the paper's z, e_3), and components are ordered (drive, y, z).  With
g = (gamma, gamma_t, gamma_t) the diagonal of G / H_sat (gamma_t = ratio
gamma) and u = (gamma x_d, gamma_t y, gamma_t z), r = |u|, the drive row of
the PSF tensor of Eq. PSF is

    h_0j(x) = g_j [ (L'(r) - L(r)/r) u_0 u_j / r^2 + delta_0j L(r)/r ],

and the harmonic PSFs of Eq. skMD (the gridding filter g taken as the
identity, as in the separable model) are

    (h_k)_j = A^k / (k-1)!  d^{k-1}/dx_d^{k-1} h_0j
            = (gamma A)^k gamma^{-k} [coefficient k-1 of the Taylor series of
              h_0j in the drive offset].

The derivatives are exact up to rounding: h_0j is evaluated in truncated
Taylor arithmetic in the drive offset (products, reciprocals and square
roots of series, and L composed with the series of r through its
derivatives L^(m)(r_0)).  On the drive axis (y = z = 0) the row reduces to
h_00 = gamma L'(gamma x_d), h_01 = h_02 = 0, so (h_k)_0 = c_k L^(k)(gamma x_d):
the separable model's drive-axis table.

The forward model of Eq. matrixModel with the row selector and phase of the
separable model:

    d_k[z][y][i'] = e^{i theta_k} sum_j (H_kj * (b_j rho))[z][y][s i' + r],

H_kj the 3D circular convolution with the samples of (h_k)_j at the minimal
image offsets of the grid; numpy's FFT is the library step for it.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as _orc


def _offsets(n: int) -> np.ndarray:
    i = np.arange(n)
    return np.where(2 * i < n, i, i - n).astype(np.float64)


def langevin0(x: np.ndarray) -> np.ndarray:
    """L(x) = coth x - 1/x (Sec. 2), with its Taylor series near 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-2
    xs = x[small]
    out[small] = xs / 3.0 - xs ** 3 / 45.0 + 2.0 * xs ** 5 / 945.0
    xl = x[~small]
    out[~small] = 1.0 / np.tanh(xl) - 1.0 / xl
    return out


# -- truncated Taylor series: arrays [n_terms, points] ----------------------

def _mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    n = a.shape[0]
    c = np.zeros_like(a)
    for m in range(n):
        for i in range(m + 1):
            c[m] += a[i] * b[m - i]
    return c


def _recip(a: np.ndarray) -> np.ndarray:
    n = a.shape[0]
    b = np.zeros_like(a)
    b[0] = 1.0 / a[0]
    for m in range(1, n):
        acc = np.zeros_like(a[0])
        for i in range(1, m + 1):
            acc += a[i] * b[m - i]
        b[m] = -acc / a[0]
    return b


def _sqrt(a: np.ndarray) -> np.ndarray:
    n = a.shape[0]
    s = np.zeros_like(a)
    s[0] = np.sqrt(a[0])
    for m in range(1, n):
        acc = np.zeros_like(a[0])
        for i in range(1, m):
            acc += s[i] * s[m - i]
        s[m] = (a[m] - acc) / (2.0 * s[0])
    return s


def _compose(fder: np.ndarray, d: np.ndarray) -> np.ndarray:
    """f(r_0 + d(delta)) for d with d[0] = 0; fder[m] = f^(m)(r_0)."""
    n = d.shape[0]
    out = np.zeros_like(d)
    out[0] = fder[0]
    p = np.zeros_like(d)
    p[0] = 1.0
    for m in range(1, n):
        p = _mul(p, d)
        out += (fder[m] / math.factorial(m)) * p
    return out


def _langevin_derivs(r0: np.ndarray, mmax: int) -> np.ndarray:
    """[mmax + 1, points]: L^(m)(r0), m = 0..mmax."""
    out = np.zeros((mmax + 1, r0.size))
    out[0] = langevin0(r0)
    for m in range(1, mmax + 1):
        out[m] = _orc.langevin_deriv(m, r0)
    return out


def drive_row_series(xd, y, z, gamma: float, gamma_t: float, nterms: int) -> np.ndarray:
    """Taylor coefficients [3, nterms, points] of h_0j(x_d + delta, y, z) in
    delta, for off-axis points ((y, z) != 0)."""
    xd, y, z = (np.atleast_1d(np.asarray(v, dtype=np.float64)).ravel() for v in (xd, y, z))
    P = xd.size
    rho2 = gamma_t ** 2 * (y ** 2 + z ** 2)
    assert np.all(rho2 > 0.0), "off-axis points only"
    u0 = np.zeros((nterms, P))
    u0[0] = gamma * xd
    if nterms > 1:
        u0[1] = gamma
    r2 = _mul(u0, u0)
    r2[0] += rho2
    r = _sqrt(r2)
    d = r.copy()
    d[0] = 0.0
    Lm = _langevin_derivs(r[0], nterms)
    L = _compose(Lm[:nterms], d)
    Lp = _compose(Lm[1:nterms + 1], d)
    rinv = _recip(r)
    r2inv = _recip(r2)
    L_over_r = _mul(L, rinv)
    radial = _mul(Lp - L_over_r, r2inv)   # (L'(r) - L(r)/r) / r^2
    g = (gamma, gamma_t, gamma_t)
    uj = [u0, np.zeros((nterms, P)), np.zeros((nterms, P))]
    uj[1][0] = gamma_t * y
    uj[2][0] = gamma_t * z
    out = np.zeros((3, nterms, P))
    for j in range(3):
        t = _mul(radial, _mul(u0, uj[j]))
        if j == 0:
            t = t + L_over_r
        out[j] = g[j] * t
    return out


def harmonic_psf_at(g: "_orc.Geometry", xd, y, z) -> np.ndarray:
    """(h_k)_j at physical points (mm): [K, 3, points]."""
    gamma = g.gamma_per_mm
    gamma_t = gamma * g.transverse_ratio
    xd, y, z = (np.atleast_1d(np.asarray(v, dtype=np.float64)).ravel() for v in (xd, y, z))
    P = xd.size
    out = np.zeros((g.K, 3, P))
    axis = (y == 0.0) & (z == 0.0)
    if np.any(axis):
        for kk, k in enumerate(range(g.k_min, g.k_max + 1)):
            out[kk, 0, axis] = _orc.ck(k, g.gammaA) * _orc.langevin_deriv(k, gamma * xd[axis])
    off = ~axis
    if np.any(off):
        ser = drive_row_series(xd[off], y[off], z[off], gamma, gamma_t, g.k_max)
        for kk, k in enumerate(range(g.k_min, g.k_max + 1)):
            scale = g.gammaA ** k * gamma ** (-k)
            out[kk, :, off] = (scale * ser[:, k - 1, :]).T
    return out


def general_psf(g: "_orc.Geometry") -> np.ndarray:
    """Samples of (h_k)_j at the grid's minimal-image offsets: [K, 3, nz, ny, nx]."""
    nx, ny, nz = g.n
    dx, dy, dz = g.voxel_mm
    Z, Y, X = np.meshgrid(_offsets(nz) * dz, _offsets(ny) * dy, _offsets(nx) * dx, indexing="ij")
    h = harmonic_psf_at(g, X.ravel(), Y.ravel(), Z.ravel())
    return h.reshape(g.K, 3, nz, ny, nx)


def _bvec(g, bvec) -> np.ndarray:
    if bvec is None:
        b = np.zeros((3,) + tuple(g.shape))
        b[0] = 1.0
        return b
    b = np.asarray(bvec, dtype=np.float64)
    assert b.shape == (3,) + tuple(g.shape)
    return b


def general_forward(g: "_orc.Geometry", rho, bvec=None, H=None) -> np.ndarray:
    """d = A rho for the vector model, complex128 [K, nz, ny, nx/s]; bvec
    [3, nz, ny, nx] (default (1, 0, 0)); H [K, 3, nz, ny, nx] (default
    general_psf)."""
    H = general_psf(g) if H is None else np.asarray(H, dtype=np.float64)
    b = _bvec(g, bvec)
    rho = np.asarray(rho, dtype=np.float64).reshape(g.shape)
    W = [np.fft.fftn(b[j] * rho) for j in range(3)]
    s, r = g.ds_factor, g.ds_offset
    th = g.theta_array()
    out = np.zeros(g.portrait_shape, dtype=np.complex128)
    for kk in range(g.K):
        acc = np.zeros(g.shape, dtype=np.complex128)
        for j in range(3):
            acc += np.fft.fftn(H[kk, j]) * W[j]
        c = np.real(np.fft.ifftn(acc))
        out[kk] = np.exp(1j * th[kk]) * c[:, :, r::s]
    return out


def general_adjoint(g: "_orc.Geometry", d, bvec=None, H=None) -> np.ndarray:
    """A^T d for the real inner product (Re<A x, d> = <x, A^T d>)."""
    H = general_psf(g) if H is None else np.asarray(H, dtype=np.float64)
    b = _bvec(g, bvec)
    d = np.asarray(d, dtype=np.complex128).reshape(g.portrait_shape)
    s, r = g.ds_factor, g.ds_offset
    th = g.theta_array()
    V = [np.zeros(g.shape, dtype=np.complex128) for _ in range(3)]
    for kk in range(g.K):
        e = np.zeros(g.shape)
        e[:, :, r::s] = np.real(np.exp(-1j * th[kk]) * d[kk])
        E = np.fft.fftn(e)
        for j in range(3):
            V[j] += np.conj(np.fft.fftn(H[kk, j])) * E
    out = np.zeros(g.shape)
    for j in range(3):
        out += b[j] * np.real(np.fft.ifftn(V[j]))
    return out


def general_normal_apply(g: "_orc.Geometry", p, lam: float, bvec=None, H=None) -> np.ndarray:
    """(A^T A + lambda I) p for the vector model."""
    H = general_psf(g) if H is None else H
    return general_adjoint(g, general_forward(g, p, bvec, H), bvec, H) + lam * np.asarray(p, dtype=np.float64)


def general_cg(g: "_orc.Geometry", d, lam: float, iters: int, bvec=None, H=None, rel_tol: float = 0.0):
    """Conjugate gradients on (A^T A + lambda I) x = A^T d from x = 0 (Hestenes-
    Stiefel, the steps in the textbook order); stops after iters iterations or
    when ||r|| <= rel_tol ||A^T d||.  Returns (x, iterations)."""
    H = general_psf(g) if H is None else H
    rhs = general_adjoint(g, d, bvec, H)
    x = np.zeros(g.shape)
    r = rhs.copy()
    p = r.copy()
    rr = float(np.vdot(r, r))
    bn = rr
    it = 0
    while it < iters and rr > 0.0 and not (rel_tol > 0.0 and rr <= rel_tol ** 2 * bn):
        q = general_normal_apply(g, p, lam, bvec, H)
        alpha = rr / float(np.vdot(p, q))
        x += alpha * p
        r -= alpha * q
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it
