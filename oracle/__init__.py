"""FP64 CPU oracle for the MH3D portrait model (arXiv 2503.13802).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.  The arithmetic lives in
``mh3d_oracle.c`` (plain C, FP64, OpenMP); this module compiles it with gcc on
first use and wraps it with numpy arrays.

Functions and the passages they follow:

* ``langevin_deriv(k, x)``: L^(k)(x), L(x) = coth x - 1/x (Sec. 2).
* ``ck(k, gammaA)``: (gamma A)^k / (k-1)! (Theorem 1).
* ``psf_tables(geom)``: separable harmonic PSF samples h_k ~ c_k L^(k)(gamma x)
  (Sec. 3.3, Eq. hkapprox) on the drive axis, 3 L'(gamma_t y) across it.
* ``forward / forward_full3d``: d = A rho, A = P H B (Eq. portz, Eq. dN), with
  the phase e^{i theta_k} of Sec. 4.4.
* ``adjoint``: A^T for the real inner product.
* ``reg_apply``: R = I, or T^T T + alpha P_a^T P_a (Sec. 4.3, Eq. finalR).
* ``normal_apply``: (A^T A + lambda R) p.
* ``operator_norm2``: ||A||_2^2 with b = 1, the scale relative weights refer to,
  by Lanczos on the oracle's own A^T A.
* ``cg``: conjugate gradients on the normal equations.
* ``apg``: the paper's accelerated projected gradient (Sec. 4.3, runtime
  subsection).
* ``mhad``: the multi-harmonic anti-differentiation native image (appendix
  MHAD, Eq. mhadM); numpy's FFT is the library step.
* ``vector_model`` (its own module): the general model of Sec. 3.2 (Eq.
  MH3Dcont, Eq. matrixModel) with the tensor PSF's harmonic PSFs (appendix,
  Eq. PSF, Eq. skMD); numpy's FFT is the library step of its convolutions.
* ``padded_forward / padded_adjoint / padded_cg``: boundary image padding
  (Sec. 3.x): the model on the field of view extended by ``pad`` voxels per
  side, its portraits cropped to the field of view; the adjoint zero-pads;
  CG on (A^T A + lambda I) x = A^T d with those two.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mh3d_oracle.c")
_LIB = os.path.join(_HERE, "libmh3d_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no fast-math, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    lib.orc_langevin_deriv.restype = d
    lib.orc_langevin_deriv.argtypes = [i, d]
    lib.orc_ck.restype = d
    lib.orc_ck.argtypes = [i, d]
    lib.orc_psf_tables.restype = None
    lib.orc_psf_tables.argtypes = [i, i, i, d, d, d, i, i, d, d, d, P, P, P]
    op_args = [i, i, i, i, i, i, P, P, P, P, P, P, P]
    lib.orc_forward.restype = None
    lib.orc_forward.argtypes = op_args
    lib.orc_forward_full3d.restype = None
    lib.orc_forward_full3d.argtypes = op_args
    lib.orc_adjoint.restype = None
    lib.orc_adjoint.argtypes = op_args
    crop_args = [i, i, i, i, i, i, P, P, P, P, P, P, P, P]
    lib.orc_forward_crop.restype = None
    lib.orc_forward_crop.argtypes = crop_args
    lib.orc_adjoint_crop.restype = None
    lib.orc_adjoint_crop.argtypes = crop_args
    lib.orc_reg_apply.restype = None
    lib.orc_reg_apply.argtypes = [i, i, i, i, d, i, P, P]
    lib.orc_normal_apply.restype = None
    lib.orc_normal_apply.argtypes = [i, i, i, i, i, i, P, P, P, P, P, d, i, d, i, P, P]
    lib.orc_cg.restype = i
    lib.orc_cg.argtypes = [i, i, i, i, i, i, P, P, P, P, P, d, i, d, i, P, d, i, P, P]
    lib.orc_apg.restype = None
    lib.orc_apg.argtypes = [i, i, i, i, i, i, P, P, P, P, P, d, i, d, i, P, d, i, P]
    lib.orc_normal_lambda_max.restype = d
    lib.orc_normal_lambda_max.argtypes = [i, i, i, i, i, i, P, P, P, P, P, d, i, d, i, P, d, i, P]
    lib.orc_num_threads.restype = i
    lib.orc_set_threads.argtypes = [i]
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


@dataclass
class Geometry:
    """Grid and model parameters.  n = (nx, ny, nz); arrays are [nz][ny][nx]."""

    n: Sequence[int]
    voxel_mm: Sequence[float] = (1.0, 1.0, 1.0)
    ds_factor: int = 1
    ds_offset: int = 0
    k_min: int = 2
    k_max: int = 5
    gamma_per_mm: float = 1.387016
    gammaA: float = 2.0
    transverse_ratio: float = 0.5
    theta: Optional[Sequence[float]] = None

    @property
    def K(self) -> int:
        return self.k_max - self.k_min + 1

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def portrait_shape(self):
        nx, ny, nz = self.n
        return (self.K, nz, ny, nx // self.ds_factor)

    def theta_array(self) -> np.ndarray:
        if self.theta is None:
            return np.zeros(self.K)
        t = _f64(self.theta)
        assert t.shape == (self.K,)
        return t


def langevin_deriv(k: int, x) -> np.ndarray:
    lib = _load()
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.array([lib.orc_langevin_deriv(int(k), float(v)) for v in xs.ravel()])
    return out.reshape(np.shape(x)) if np.ndim(x) else out[0]


def ck(k: int, gammaA: float) -> float:
    return _load().orc_ck(int(k), float(gammaA))


def psf_tables(g: Geometry):
    """Return (X [K, nx], Y [ny], Z [nz]) PSF sample tables (FP64)."""
    nx, ny, nz = g.n
    X = np.zeros((g.K, nx))
    Y = np.zeros(ny)
    Z = np.zeros(nz)
    dx, dy, dz = g.voxel_mm
    _load().orc_psf_tables(nx, ny, nz, dx, dy, dz, g.k_min, g.k_max, g.gamma_per_mm, g.gammaA,
                           g.transverse_ratio, _ptr(X), _ptr(Y), _ptr(Z))
    return X, Y, Z


def _op(fn, g: Geometry, tables, b, src, out):
    nx, ny, nz = g.n
    X, Y, Z = tables
    th = g.theta_array()
    fn(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z), _ptr(th),
       _ptr(b), _ptr(src), _ptr(out))
    return out


def forward(g: Geometry, rho, b=None, tables=None) -> np.ndarray:
    """d = A rho as complex128 [K, nz, ny, nx/s]."""
    tables = tables or psf_tables(g)
    rho = _f64(rho).reshape(g.shape)
    b = None if b is None else _f64(b).reshape(g.shape)
    out = np.zeros(g.portrait_shape + (2,))
    _op(_load().orc_forward, g, tables, b, rho, out)
    return out[..., 0] + 1j * out[..., 1]


def forward_full3d(g: Geometry, rho, b=None, tables=None) -> np.ndarray:
    tables = tables or psf_tables(g)
    rho = _f64(rho).reshape(g.shape)
    b = None if b is None else _f64(b).reshape(g.shape)
    out = np.zeros(g.portrait_shape + (2,))
    _op(_load().orc_forward_full3d, g, tables, b, rho, out)
    return out[..., 0] + 1j * out[..., 1]


def _complex_in(g: Geometry, d) -> np.ndarray:
    d = np.asarray(d).reshape(g.portrait_shape)
    return np.ascontiguousarray(np.stack([d.real, d.imag], axis=-1), dtype=np.float64)


def adjoint(g: Geometry, d, b=None, tables=None) -> np.ndarray:
    """rho = A^T d (real inner product), float64 [nz, ny, nx]."""
    tables = tables or psf_tables(g)
    b = None if b is None else _f64(b).reshape(g.shape)
    out = np.zeros(g.shape)
    _op(_load().orc_adjoint, g, tables, b, _complex_in(g, d), out)
    return out


def _crop_arg(crop):
    """crop = ((a0, na), (y0, ny), (z0, nz)) along (drive, y, z)."""
    (a0, na), (y0, ny), (z0, nz) = crop
    return np.ascontiguousarray([a0, na, y0, ny, z0, nz], dtype=np.int32)


def _op_crop(fn, g: Geometry, tables, b, src, crop, out):
    nx, ny, nz = g.n
    X, Y, Z = tables
    th = g.theta_array()
    c = _crop_arg(crop)
    fn(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z), _ptr(th),
       _ptr(b), _ptr(src), _ptr(c), _ptr(out))
    return out


def forward_crop(g: Geometry, rho, crop, b=None, tables=None) -> np.ndarray:
    """d = A rho on an output crop ((i0, ni), (y0, ny_c), (z0, nz_c)) of the
    portrait mesh (i along the downsampled drive axis): complex128
    [K, nz_c, ny_c, ni].  Only the crop's outputs are evaluated, so large
    grids stay tractable."""
    tables = tables or psf_tables(g)
    rho = _f64(rho).reshape(g.shape)
    b = None if b is None else _f64(b).reshape(g.shape)
    (_, ni), (_, nyc), (_, nzc) = crop
    out = np.zeros((g.K, nzc, nyc, ni, 2))
    _op_crop(_load().orc_forward_crop, g, tables, b, rho, crop, out)
    return out[..., 0] + 1j * out[..., 1]


def adjoint_crop(g: Geometry, d, crop, b=None, tables=None) -> np.ndarray:
    """rho = A^T d on an image crop ((x0, nx_c), (y0, ny_c), (z0, nz_c)):
    float64 [nz_c, ny_c, nx_c]."""
    tables = tables or psf_tables(g)
    b = None if b is None else _f64(b).reshape(g.shape)
    (_, nxc), (_, nyc), (_, nzc) = crop
    out = np.zeros((nzc, nyc, nxc))
    _op_crop(_load().orc_adjoint_crop, g, tables, b, _complex_in(g, d), crop, out)
    return out


def reg_apply(g: Geometry, p, kind: int = 0, alpha: float = 0.0, shell: int = 2) -> np.ndarray:
    nx, ny, nz = g.n
    p = _f64(p).reshape(g.shape)
    out = np.zeros(g.shape)
    _load().orc_reg_apply(nx, ny, nz, int(kind), float(alpha), int(shell), _ptr(p), _ptr(out))
    return out


def operator_norm2(g: Geometry, tables=None, rel_tol: float = 1e-13, max_iter: int = 400) -> float:
    """||A||_2^2 for b = 1: the largest eigenvalue of A^T A.

    Plain Lanczos (FP64, in C) on the oracle's own normal operator with
    lambda = 0 and uniform sensitivity: nothing about the operator's
    structure is used.  The start vector is seeded normal noise; the process
    stops once the largest Ritz value has changed by at most ``rel_tol``
    (relative) in three successive steps.  The result is cached per grid,
    offsets, phases and PSF tables, since relative regularisation weights
    call it on every solve."""
    tables = tables or psf_tables(g)
    key = (tuple(g.n), g.ds_factor, g.ds_offset, tuple(np.round(g.theta_array(), 15)), rel_tol, max_iter,
           b"".join(np.ascontiguousarray(t, dtype=np.float64).tobytes() for t in tables))
    if key not in _NORM2_CACHE:
        _NORM2_CACHE[key] = _lambda_max(g, None, 0.0, 0, 0.0, 1, tables, rel_tol, max_iter)
    return _NORM2_CACHE[key]


_NORM2_CACHE: dict = {}


def _lambda_max(g: Geometry, b, lam: float, kind: int, alpha: float, shell: int, tables, rel_tol: float,
                max_iter: int) -> float:
    X, Y, Z = tables or psf_tables(g)
    nx, ny, nz = g.n
    b = None if b is None else _f64(b).reshape(g.shape)
    v0 = np.random.default_rng(20250317).standard_normal(g.shape)
    it = ctypes.c_int(0)
    return float(_load().orc_normal_lambda_max(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z),
                                               _ptr(g.theta_array()), _ptr(b), float(lam), int(kind), float(alpha),
                                               int(shell), _ptr(v0), float(rel_tol), int(max_iter),
                                               ctypes.byref(it)))


def normal_lambda_max(g: Geometry, b=None, opts: "SolveOpts" = None, tables=None, rel_tol: float = 1e-13,
                      max_iter: int = 400) -> float:
    """lambda_max(A^T A + lambda R) with sensitivity b, by the same Lanczos
    process: the reciprocal is the APG step of Sec. 4.3 (tau = 1 / ||M||^2)."""
    opts = opts or SolveOpts()
    return _lambda_max(g, b, opts.lam_eff(g, tables), opts.reg_kind, opts.alpha, opts.shell, tables, rel_tol,
                       max_iter)


@dataclass
class SolveOpts:
    """lam is the weight of R; with lam_relative it is multiplied by
    operator_norm2(g) (the PSF's overall scale is a free constant)."""
    lam: float = 1e-3
    reg_kind: int = 0
    alpha: float = 0.0
    shell: int = 2
    rel_tol: float = 1e-4
    max_iter: int = 1000
    lam_relative: bool = False

    def lam_eff(self, g: Geometry, tables=None) -> float:
        return self.lam * operator_norm2(g, tables) if self.lam_relative else self.lam


def normal_apply(g: Geometry, p, b=None, opts: SolveOpts = SolveOpts(), tables=None) -> np.ndarray:
    tables = tables or psf_tables(g)
    nx, ny, nz = g.n
    X, Y, Z = tables
    th = g.theta_array()
    b = None if b is None else _f64(b).reshape(g.shape)
    p = _f64(p).reshape(g.shape)
    out = np.zeros(g.shape)
    _load().orc_normal_apply(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z),
                             _ptr(th), _ptr(b), opts.lam_eff(g, tables), opts.reg_kind, opts.alpha, opts.shell,
                             _ptr(p), _ptr(out))
    return out


def cg(g: Geometry, d, b=None, opts: SolveOpts = SolveOpts(), x0=None, tables=None):
    """Returns (x, iters, history) for CG on (A^T A + lambda R) x = A^T d."""
    tables = tables or psf_tables(g)
    nx, ny, nz = g.n
    X, Y, Z = tables
    th = g.theta_array()
    b = None if b is None else _f64(b).reshape(g.shape)
    x = np.zeros(g.shape) if x0 is None else _f64(x0).reshape(g.shape).copy()
    hist = np.zeros(opts.max_iter + 1)
    it = _load().orc_cg(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z),
                        _ptr(th), _ptr(b), opts.lam_eff(g, tables), opts.reg_kind, opts.alpha, opts.shell,
                        _ptr(_complex_in(g, d)), opts.rel_tol, opts.max_iter, _ptr(x), _ptr(hist))
    return x, it, hist[: it + 1]


def apg(g: Geometry, d, tau: float, iters: int, b=None, opts: SolveOpts = SolveOpts(), x0=None,
        tables=None) -> np.ndarray:
    """The paper's accelerated projected gradient, fixed iteration count."""
    tables = tables or psf_tables(g)
    nx, ny, nz = g.n
    X, Y, Z = tables
    th = g.theta_array()
    b = None if b is None else _f64(b).reshape(g.shape)
    x = np.zeros(g.shape) if x0 is None else _f64(x0).reshape(g.shape).copy()
    _load().orc_apg(nx, ny, nz, g.ds_factor, g.ds_offset, g.K, _ptr(X), _ptr(Y), _ptr(Z),
                    _ptr(th), _ptr(b), opts.lam_eff(g, tables), opts.reg_kind, opts.alpha, opts.shell,
                    _ptr(_complex_in(g, d)), float(tau), int(iters), _ptr(x))
    return x


def mhad(d_list, ck_list, lam: float, axis: int = -1, k_min: int = 2) -> np.ndarray:
    """MHAD native image (appendix MHAD, Eq. mhadM) along one axis.

    d_list[k'] is the portrait of harmonic k = k'+k_min (real), ck_list[k']
    its coefficient c_k.  With f = [0, -1, 0, ..., 0, 1] (so (f*u)[j] =
    u[j+1] - u[j-1]) and f^{m} its m-fold self-convolution,
    rho_N = F^{-1}[ sum_k c_k^{-1} conj(F f^{k-1}) F d_k / (sum_k |F f^{k-1}|^2 + lambda) ].
    """
    d0 = np.asarray(d_list[0])
    n = d0.shape[axis]
    f = np.zeros(n)
    f[1 % n] += -1.0
    f[(n - 1) % n] += 1.0
    fh = np.fft.fft(f)
    shape = [1] * d0.ndim
    shape[axis] = n
    num = 0.0
    den = lam
    for j, (dk, c) in enumerate(zip(d_list, ck_list)):
        k = j + k_min
        fk = (fh ** (k - 1)).reshape(shape)
        num = num + np.conj(fk) * np.fft.fft(np.asarray(dk, dtype=np.float64), axis=axis) / c
        den = den + np.abs(fk) ** 2
    return np.real(np.fft.ifft(num / den, axis=axis))


# ---------------------------------------------------------------------------
# Boundary image padding (Sec. 3.x): the forward model runs on the field of
# view extended by pad voxels on each side; the data cover the field of view
# only, so the padded forward crops the extended portraits and its adjoint
# zero-pads the field of view's portraits.
# ---------------------------------------------------------------------------
def padded_geometry(g_fov: Geometry, pad) -> Geometry:
    """The geometry of the extended grid (pad = (px, py, pz) per side; px a
    multiple of the downsampling factor)."""
    px, py, pz = pad
    nx, ny, nz = g_fov.n
    assert px % g_fov.ds_factor == 0
    return Geometry(n=(nx + 2 * px, ny + 2 * py, nz + 2 * pz), voxel_mm=g_fov.voxel_mm, ds_factor=g_fov.ds_factor,
                    ds_offset=g_fov.ds_offset, k_min=g_fov.k_min, k_max=g_fov.k_max,
                    gamma_per_mm=g_fov.gamma_per_mm, gammaA=g_fov.gammaA, transverse_ratio=g_fov.transverse_ratio,
                    theta=g_fov.theta)


def _fov_slices(g_fov: Geometry, pad):
    px, py, pz = pad
    _, nzf, nyf, mxf = g_fov.portrait_shape
    pm = px // g_fov.ds_factor
    return (slice(None), slice(pz, pz + nzf), slice(py, py + nyf), slice(pm, pm + mxf))


def padded_forward(g_fov: Geometry, pad, rho_ext, b_ext=None, tables=None) -> np.ndarray:
    """d = C A_ext rho on the field of view's portrait mesh."""
    g = padded_geometry(g_fov, pad)
    return forward(g, rho_ext, b_ext, tables)[_fov_slices(g_fov, pad)]


def padded_adjoint(g_fov: Geometry, pad, d_fov, b_ext=None, tables=None) -> np.ndarray:
    """rho_ext = A_ext^T C^T d (the field of view's portraits zero-padded)."""
    g = padded_geometry(g_fov, pad)
    y = np.zeros(g.portrait_shape, dtype=np.complex128)
    y[_fov_slices(g_fov, pad)] = np.asarray(d_fov)
    return adjoint(g, y, b_ext, tables)


def padded_cg(g_fov: Geometry, pad, d_fov, b_ext, lam: float, iters: int, tables=None) -> np.ndarray:
    """Plain CG on (A^T A + lam I) x = A^T d for the padded operator, from
    x = 0, a fixed number of iterations (test sizes only)."""
    g = padded_geometry(g_fov, pad)
    tables = tables or psf_tables(g)

    def nop(v):
        return padded_adjoint(g_fov, pad, padded_forward(g_fov, pad, v, b_ext, tables), b_ext, tables) + lam * v

    rhs = padded_adjoint(g_fov, pad, d_fov, b_ext, tables)
    x = np.zeros(g.shape)
    r = rhs.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(iters):
        if rr == 0.0:   # solved exactly (small systems): nothing left to do
            break
        q = nop(p)
        a = rr / float(np.sum(p * q))
        x += a * p
        r -= a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


# ---------------------------------------------------------------------------
# Portrait phase calibration (Sec. 4.4).  The measured portrait of harmonic
# k is e^{i theta_k} times a real field.
#  * theta_k modulo pi: the direction of the high-SNR samples (|d_k| >= frac
#    max |d_k|) in the complex plane, 1/2 arg sum d_k^2 (the samples are
#    +-|d| e^{i theta}, so their squares all point along 2 theta);
#  * the remaining pi, when the portraits are not downsampled (s = 1): the
#    single-harmonic back-projections B_k = A_k^T Re(e^{-i theta_k} d_k)
#    correlate positively for the true signs (along the drive axis
#    <B_j, B_k> sums |X_j|^2 |X_k|^2 |U|^2 over the frequencies, U the
#    filtered density), which fixes every sign relative to the harmonic with
#    the largest ||B_k||; the common sign is the one whose short CG
#    reconstruction (30 iterations, lambda = 1e-2 relative) is positively
#    skewed (sum x^3 > 0), as the image of a sparse non-negative density is;
#  * with s > 1 the row selector's aliases break the correlation argument
#    and theta_k is returned modulo pi.
# Returns (theta, resolved): theta in (-pi, pi]; resolved = 1 for every
# harmonic when s = 1, else 0.
# ---------------------------------------------------------------------------
def estimate_phase(g: Geometry, d, frac: float = 0.5, b=None, tables=None):
    d = np.asarray(d, dtype=np.complex128)
    K = g.K
    th = np.zeros(K)
    for j in range(K):
        a = np.abs(d[j])
        sj = a >= frac * a.max() if a.max() > 0 else np.zeros(a.shape, dtype=bool)
        th[j] = 0.5 * np.angle(np.sum(d[j][sj] ** 2))
    resolved = np.zeros(K, dtype=np.int32)
    if g.ds_factor == 1:
        tables = tables or psf_tables(g)
        g0 = Geometry(n=g.n, voxel_mm=g.voxel_mm, ds_factor=1, ds_offset=0, k_min=g.k_min, k_max=g.k_max,
                      gamma_per_mm=g.gamma_per_mm, gammaA=g.gammaA, transverse_ratio=g.transverse_ratio)
        B = []
        for j in range(K):
            y = np.zeros(g.portrait_shape, dtype=np.complex128)
            y[j] = np.real(np.exp(-1j * th[j]) * d[j])
            B.append(adjoint(g0, y, b, tables))
        r = int(np.argmax([float(np.sum(x * x)) for x in B]))
        sig = np.array([1.0 if j == r else (1.0 if float(np.sum(B[j] * B[r])) >= 0 else -1.0) for j in range(K)])
        y = np.array([sig[j] * np.real(np.exp(-1j * th[j]) * d[j]) for j in range(K)]).astype(np.complex128)
        x, _, _ = cg(g0, y, b, SolveOpts(lam=1e-2, lam_relative=True, rel_tol=0.0, max_iter=30), tables=tables)
        if float(np.sum(x ** 3)) < 0:
            sig = -sig
        th = np.where(sig < 0, th + np.pi, th)
        resolved[:] = 1
    return np.angle(np.exp(1j * th)), resolved
