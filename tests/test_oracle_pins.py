"""Pins of the FP64 oracle against mathematics that is not the oracle itself.

Each test states what fixes the expected value: a closed form, an
independent high-precision computation (mpmath), an independent library
routine applied to the defining formula (numpy FFT, dense linear algebra,
scipy NNLS), an identity (adjoint, shift covariance) or a brute-force sum.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

mp = pytest.importorskip("mpmath")


def _mp_langevin_deriv(k, x, dps=60):
    """k-th derivative of coth(t) - 1/t by mpmath numerical differentiation."""
    with mp.workdps(dps):
        f = lambda t: mp.coth(t) - 1 / t
        if x == 0:
            # removable singularity: use the series-free limit via a tiny offset pair
            return float((mp.diff(f, mp.mpf("1e-20"), k) + mp.diff(f, mp.mpf("-1e-20"), k)) / 2)
        return float(mp.diff(f, mp.mpf(x), k))


# --------------------------------------------------------------------------
# Langevin derivatives (Sec. 2, Eq. hkapprox; appendix, poles of L at i n pi)
# --------------------------------------------------------------------------

def test_langevin_odd_derivatives_at_zero_match_bernoulli():
    """L(x) = sum_n 2^{2n} B_{2n} x^{2n-1} / (2n)!  =>  L^{(2n-1)}(0) = 2^{2n} B_{2n} / (2n):
    1/3, -2/15, 16/63, -16/15, ... (exact rationals from sympy's Bernoulli numbers)."""
    sympy = pytest.importorskip("sympy")
    for n in range(1, 9):
        exact = float(sympy.Rational(2) ** (2 * n) * sympy.bernoulli(2 * n) / (2 * n))
        got = oracle.langevin_deriv(2 * n - 1, 0.0)
        assert got == pytest.approx(exact, rel=1e-13), (n, got, exact)
    assert oracle.langevin_deriv(1, 0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert oracle.langevin_deriv(3, 0.0) == pytest.approx(-2.0 / 15.0, rel=1e-14)


def test_langevin_even_derivatives_vanish_at_zero():
    """L is odd, so every even-order derivative is odd and vanishes at 0."""
    for k in range(0, 18, 2):
        assert abs(oracle.langevin_deriv(k, 0.0)) < 1e-15


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 8, 9, 12, 17])
def test_langevin_deriv_matches_mpmath(k):
    """Against mpmath differentiation of coth(t) - 1/t at 60 digits, on both
    sides of each of the oracle's internal branch points (|x| = 1, 1.5, 8)
    and far in the tail."""
    xs = [-9.1, -7.99, -2.5, -1.5, -1.499, -0.7, 0.05, 0.3, 0.999, 1.0, 1.499, 1.5, 1.97,
          3.3, 7.999, 8.0, 25.0, 60.0]
    for x in xs:
        ref = _mp_langevin_deriv(k, x)
        got = oracle.langevin_deriv(k, x)
        scale = max(abs(ref), 1e-300)
        # relative accuracy, with an absolute floor relative to the derivative's size at 0-ish
        floor = 1e-14 * max(abs(_mp_langevin_deriv(k, 0.5)), 1e-30)
        assert abs(got - ref) <= 5e-12 * scale + floor, (k, x, got, ref)


def test_langevin_first_derivative_closed_form():
    """L'(x) = 1/x^2 - 1/sinh^2 x (direct differentiation)."""
    for x in [0.5, 1.0, 2.5, 4.0, 10.0]:
        assert oracle.langevin_deriv(1, x) == pytest.approx(1 / x**2 - 1 / math.sinh(x) ** 2, rel=1e-12)


def test_langevin_integral_of_first_derivative_is_two():
    """int_R L'(x) dx = L(+inf) - L(-inf) = 2 (Riemann sum on a fine grid)."""
    h = 0.01
    xs = np.arange(-4000, 4001) * h
    vals = oracle.langevin_deriv(1, xs)
    tail = 2.0 / 40.0                         # int_{|x|>40} 1/x^2 dx
    assert np.sum(vals) * h + tail == pytest.approx(2.0, abs=2e-4)


# --------------------------------------------------------------------------
# c_k against Theorem 1 (harmonic expansion of the received signal)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("gammaA,x0", [(1.0, 0.0), (2.0, 0.0), (2.0, 0.4), (2.8, -0.3)])
def test_ck_matches_harmonic_expansion_of_signal(gammaA, x0):
    """Proposition 1 gives the unfiltered 1D signal of a point source at x0 as
    s0(t) = m gamma xi'(t) L'(gamma (xi(t) - x0)).  For the complex drive
    xi(t) = A e^{i 2 pi f0 t} (Delta_t = 0), Theorem 1 says the k-th harmonic
    coefficient is i 2 pi m f0 c_k L^{(k)}(-gamma x0) with
    c_k = (gamma A)^k / (k-1)!.  Compute the Fourier coefficients of s0 over
    one period numerically (mpmath, complex coth) and compare with the
    oracle's c_k * L^(k).  Units: gamma = 1, m = 1, f0 = 1."""
    M = 1024                                  # (gamma A / radius)^M far below 1e-12: no aliasing
    with mp.workdps(30):
        vals = []
        for j in range(M):
            th = 2 * mp.pi * j / M
            xi = gammaA * mp.e ** (1j * th)
            dxi = 1j * 2 * mp.pi * xi
            arg = xi - x0
            Lp = 1 / arg**2 - 1 / mp.sinh(arg) ** 2
            vals.append(complex(dxi * Lp))
    coef = np.fft.fft(np.array(vals)) / M     # coef[k] multiplies e^{i 2 pi k t}
    for k in range(1, 9):
        expect = 1j * 2 * math.pi * oracle.ck(k, gammaA) * oracle.langevin_deriv(k, -x0)
        assert abs(coef[k] - expect) <= 1e-9 * max(1.0, abs(expect)), (k, coef[k], expect)


# --------------------------------------------------------------------------
# PSF tables and the forward operator
# --------------------------------------------------------------------------

def _geom(n, s=1, r=0, kmin=2, kmax=5, theta=None, gamma=1.387016, gammaA=2.0, voxel=(1.0, 1.0, 1.0)):
    return oracle.Geometry(n=n, voxel_mm=voxel, ds_factor=s, ds_offset=r, k_min=kmin, k_max=kmax,
                           gamma_per_mm=gamma, gammaA=gammaA, theta=theta)


def test_psf_tables_minimal_image_and_values():
    """Entries are c_k L^(k)(gamma o dx) at minimal-image offsets o, with
    index n/2 taken as -n/2; transverse entries 3 L'(gamma_t o)."""
    g = _geom((8, 6, 5), kmin=2, kmax=4, voxel=(1.0, 1.5, 2.0))
    X, Y, Z = oracle.psf_tables(g)
    offs8 = [0, 1, 2, 3, -4, -3, -2, -1]
    for kk, k in enumerate(range(2, 5)):
        ck = gA = 2.0 ** k / math.factorial(k - 1)
        for i, o in enumerate(offs8):
            ref = ck * _mp_langevin_deriv(k, 1.387016 * o * 1.0)
            assert X[kk, i] == pytest.approx(ref, rel=1e-11, abs=1e-14)
    for i, o in enumerate([0, 1, 2, -3, -2, -1]):
        assert Y[i] == pytest.approx(3 * _mp_langevin_deriv(1, 0.5 * 1.387016 * o * 1.5), rel=1e-11)
    for i, o in enumerate([0, 1, 2, -2, -1]):
        assert Z[i] == pytest.approx(3 * _mp_langevin_deriv(1, 0.5 * 1.387016 * o * 2.0), rel=1e-11)
    assert Y[0] == pytest.approx(1.0) and Z[0] == pytest.approx(1.0)   # phi(0) = 3 * 1/3


def test_delta_phantom_reproduces_psf():
    """A point source at voxel 0 with b = 1, s = 1, theta = 0 gives d_k = h_k
    exactly (Eq. MH3Dcont with rho = delta; appendix: d_k = rho_b * h_k)."""
    g = _geom((12, 8, 6), kmin=2, kmax=5)
    X, Y, Z = oracle.psf_tables(g)
    rho = np.zeros(g.shape)
    rho[0, 0, 0] = 1.0
    d = oracle.forward(g, rho)
    for kk in range(g.K):
        h = Z[:, None, None] * Y[None, :, None] * X[kk][None, None, :]
        np.testing.assert_allclose(d[kk].real, h, rtol=0, atol=1e-15)
        assert np.all(d[kk].imag == 0)


def test_delta_at_offset_shifts_psf():
    """A point source at voxel (x0, y0, z0) gives the PSF circularly shifted by
    (x0, y0, z0): shift covariance of a convolution."""
    g = _geom((10, 6, 4), kmin=2, kmax=3)
    X, Y, Z = oracle.psf_tables(g)
    rho = np.zeros(g.shape)
    rho[1, 4, 7] = 1.0                         # z0=1, y0=4, x0=7
    d = oracle.forward(g, rho)
    for kk in range(g.K):
        h = Z[:, None, None] * Y[None, :, None] * X[kk][None, None, :]
        np.testing.assert_allclose(d[kk].real, np.roll(h, (1, 4, 7), axis=(0, 1, 2)), atol=1e-15)


@pytest.mark.parametrize("n,s,r", [((6, 4, 5), 1, 0), ((6, 4, 3), 2, 1), ((9, 3, 4), 3, 2), ((8, 5, 2), 2, 0)])
def test_forward_separable_equals_full_triple_sum(n, s, r):
    """The separable evaluation equals the brute-force triple sum over all
    source voxels (random rho, b, theta)."""
    g = _geom(n, s=s, r=r, kmin=2, kmax=4, theta=[0.3, -1.1, 2.0])
    rho = W.random_volume(g.shape, 11)
    b = 0.5 + np.abs(W.random_volume(g.shape, 12))
    d1 = oracle.forward(g, rho, b)
    d2 = oracle.forward_full3d(g, rho, b)
    np.testing.assert_allclose(d1, d2, rtol=1e-12, atol=1e-12 * np.abs(d2).max())


@pytest.mark.parametrize("n,s,r", [((16, 8, 6), 1, 0), ((12, 6, 4), 2, 1), ((12, 5, 3), 3, 0), ((9, 4, 6), 3, 1)])
def test_forward_matches_fft_convolution(n, s, r):
    """Independent computation through numpy's FFT: circular convolution of
    b.rho with the 3D kernel h_k = X_k (x) Y (x) Z, rows i = r mod s kept,
    times e^{i theta_k}."""
    theta = [0.7, -0.2, 1.9]
    g = _geom(n, s=s, r=r, kmin=3, kmax=5, theta=theta)
    X, Y, Z = oracle.psf_tables(g)
    rho = W.random_volume(g.shape, 5)
    b = 0.5 + np.abs(W.random_volume(g.shape, 6))
    d = oracle.forward(g, rho, b)
    U = np.fft.fftn(b * rho)
    for kk in range(g.K):
        h = Z[:, None, None] * Y[None, :, None] * X[kk][None, None, :]
        full = np.real(np.fft.ifftn(np.fft.fftn(h) * U))
        ref = np.exp(1j * theta[kk]) * full[:, :, r::s]
        np.testing.assert_allclose(d[kk], ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n,s,r", [((8, 6, 5), 1, 0), ((12, 4, 3), 2, 1), ((9, 5, 4), 3, 2), ((16, 1, 1), 4, 3)])
def test_adjoint_identity(n, s, r):
    """Re<A x, y> = <x, A^T y> to 1e-12 relative (random x, y, b, theta)."""
    g = _geom(n, s=s, r=r, kmin=2, kmax=6, theta=list(np.linspace(-2, 2, 5)))
    x = W.random_volume(g.shape, 21)
    y = W.random_portraits(g.portrait_shape, 22)
    b = 0.3 + np.abs(W.random_volume(g.shape, 23))
    lhs = np.real(np.vdot(oracle.forward(g, x, b), y))
    rhs = float(np.sum(x * oracle.adjoint(g, y, b)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10, (lhs, rhs)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_forward_is_linear():
    g = _geom((8, 4, 4), s=2, r=0, kmin=2, kmax=3, theta=[0.4, 1.0])
    a = W.random_volume(g.shape, 1)
    c = W.random_volume(g.shape, 2)
    np.testing.assert_allclose(oracle.forward(g, 2.0 * a - 3.0 * c),
                               2.0 * oracle.forward(g, a) - 3.0 * oracle.forward(g, c), atol=1e-12)


def test_downsample_shift_covariance():
    """Shifting rho by s voxels along the drive axis shifts every portrait by
    one portrait sample (P keeps every s-th row)."""
    g = _geom((12, 4, 3), s=3, r=1, kmin=2, kmax=4)
    rho = W.random_volume(g.shape, 9)
    d0 = oracle.forward(g, rho)
    d1 = oracle.forward(g, np.roll(rho, 3, axis=2))
    np.testing.assert_allclose(d1, np.roll(d0, 1, axis=3), atol=1e-13)


def test_drive_axis_sum_rules():
    """Integral of L^(k) is 0 for k >= 2 (appendix, information per harmonic).
    Even k: L^(k) is odd, so the minimal-image samples cancel in pairs except
    the unpaired -n/2 sample.  Odd k: by Poisson summation the sampled sum is
    the aliased continuous transform,
        sum_o L^(k)(gamma o) = (1/gamma) sum_{m != 0} F_k(2 pi m / gamma),
    with F_k(w) = (i w)^{k-1} F_1(w) and F_1(w) = 2 pi |w| / (e^{pi |w|} - 1)
    the Fourier transform of L' (from FT[1/x^2] = -pi|w| and
    FT[1/sinh^2 x] = -pi w coth(pi w / 2)).  n = 4096 makes the truncation of
    the lattice sum negligible."""
    gamma, n = 1.387016, 4096
    g = _geom((n, 1, 1), kmin=2, kmax=9, gamma=gamma)
    X, _, _ = oracle.psf_tables(g)
    for kk, k in enumerate(range(2, 10)):
        tot = X[kk].sum()
        if k % 2 == 0:
            assert abs(tot - X[kk, n // 2]) <= 1e-13 * np.abs(X[kk]).max()
        else:
            pred = 0.0
            for m in list(range(-6, 0)) + list(range(1, 7)):
                w = 2 * math.pi * m / gamma
                pred += ((1j * w) ** (k - 1) * 2 * math.pi * abs(w) / math.expm1(math.pi * abs(w))).real
            pred *= oracle.ck(k, 2.0) / gamma
            assert tot == pytest.approx(pred, rel=1e-6), (k, tot, pred)


def test_constant_density_gives_dc_eigenvalue():
    """A constant density is an eigenvector of every circulant: with b = 1
    each portrait sample equals (sum X_k)(sum Y)(sum Z) times the constant,
    i.e. the aliased DC response that the sum-rule test pins near zero (the
    missing background of Sec. 4.3)."""
    g = _geom((32, 6, 4), s=2, r=1, kmin=2, kmax=5, theta=[0.1, 0.2, 0.3, 0.4])
    X, Y, Z = oracle.psf_tables(g)
    d = oracle.forward(g, 2.5 * np.ones(g.shape))
    for kk in range(g.K):
        ref = 2.5 * X[kk].sum() * Y.sum() * Z.sum() * np.exp(1j * g.theta[kk])
        np.testing.assert_allclose(d[kk], ref, rtol=1e-10, atol=1e-14)


# --------------------------------------------------------------------------
# Regulariser (Sec. 4.3, Eq. finalR; Table ops: T^T T diagonal in Fourier)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [(8, 6, 5), (4, 1, 7), (2, 3, 4)])
def test_reg_second_order_matches_fourier_symbol(n):
    """T^T T = F^{-1} |T^|^2 F with |T^|^2 = sum_a (2 - 2 cos w_a)^2 for the
    periodic second difference (Table ops), plus alpha on the boundary shell."""
    g = _geom(n)
    p = W.random_volume(g.shape, 4)
    alpha, shell = 4.0, 1
    got = oracle.reg_apply(g, p, kind=1, alpha=alpha, shell=shell)
    nz, ny, nx = g.shape
    wz, wy, wx = np.meshgrid(*(2 * np.pi * np.fft.fftfreq(m) for m in (nz, ny, nx)), indexing="ij")
    sym = (2 - 2 * np.cos(wx)) ** 2 + (2 - 2 * np.cos(wy)) ** 2 + (2 - 2 * np.cos(wz)) ** 2
    ref = np.real(np.fft.ifftn(sym * np.fft.fftn(p)))
    zi, yi, xi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    shellmask = ((xi < shell) | (yi < shell) | (zi < shell) | (xi >= nx - shell)
                 | (yi >= ny - shell) | (zi >= nz - shell))
    ref = ref + alpha * shellmask * p
    np.testing.assert_allclose(got, ref, atol=1e-11)
    np.testing.assert_array_equal(oracle.reg_apply(g, p, kind=0), p)


# --------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------

def _dense_normal(g, b, opts):
    N = int(np.prod(g.shape))
    M = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = oracle.normal_apply(g, e, b, opts).ravel()
    return M


@pytest.mark.parametrize("kind,s", [(0, 1), (0, 2), (1, 2)])
def test_cg_matches_dense_cholesky(kind, s):
    """CG (tol 1e-13) against a dense FP64 Cholesky solve of the normal
    equations assembled column by column (N <= 192)."""
    g = _geom((8, 4, 6), s=s, r=s - 1, kmin=2, kmax=4, theta=[0.2, -0.5, 1.1])
    b = 0.4 + np.abs(W.random_volume(g.shape, 31))
    opts = oracle.SolveOpts(lam=1e-2, reg_kind=kind, alpha=4.0, shell=1, rel_tol=1e-13, max_iter=2000)
    d = oracle.forward(g, W.random_volume(g.shape, 32), b) + 0.1 * W.random_portraits(g.portrait_shape, 33)
    M = _dense_normal(g, b, opts)
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    L = np.linalg.cholesky(M)
    rhs = oracle.adjoint(g, d, b).ravel()
    ref = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
    x, it, hist = oracle.cg(g, d, b, opts)
    assert it < opts.max_iter
    assert hist[-1] <= 1e-13
    np.testing.assert_allclose(x.ravel(), ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("kind,s", [(0, 1), (1, 2)])
def test_normal_lambda_max_matches_dense_eigenvalues(kind, s):
    """lambda_max(A^T A + lambda R) with a non-uniform sensitivity, by the
    oracle's Lanczos process, equals the largest eigenvalue of the dense
    normal matrix assembled column by column (numpy eigvalsh)."""
    g = _geom((8, 4, 6), s=s, r=s - 1, kmin=2, kmax=4, theta=[0.2, -0.5, 1.1])
    b = 0.4 + np.abs(W.random_volume(g.shape, 34))
    opts = oracle.SolveOpts(lam=3e-2, reg_kind=kind, alpha=4.0, shell=1)
    ref = float(np.linalg.eigvalsh(_dense_normal(g, b, opts)).max())
    assert oracle.normal_lambda_max(g, b, opts) == pytest.approx(ref, rel=1e-11)


def test_cg_matches_fourier_closed_form():
    """b uniform, s = 1, R = I: the normal matrix is diagonal in Fourier and
    rho^ = sum_k conj(h^_k) D^_k / (sum_k |h^_k|^2 + lambda), D_k =
    Re(e^{-i theta_k} d_k) (the algebra of the MHAD closed form)."""
    theta = [0.3, 1.2, -0.7, 2.5]
    g = _geom((16, 12, 8), kmin=2, kmax=5, theta=theta)
    X, Y, Z = oracle.psf_tables(g)
    lam = 5e-3
    d = W.random_portraits(g.portrait_shape, 41)
    num = 0.0
    den = lam
    for kk in range(g.K):
        h = Z[:, None, None] * Y[None, :, None] * X[kk][None, None, :]
        H = np.fft.fftn(h)
        D = np.fft.fftn(np.real(np.exp(-1j * theta[kk]) * d[kk]))
        num = num + np.conj(H) * D
        den = den + np.abs(H) ** 2
    ref = np.real(np.fft.ifftn(num / den))
    x, it, _ = oracle.cg(g, d, None, oracle.SolveOpts(lam=lam, rel_tol=1e-13, max_iter=5000))
    np.testing.assert_allclose(x, ref, atol=1e-8 * np.abs(ref).max())


@pytest.mark.parametrize("n,s,r", [((12, 6, 4), 1, 0), ((12, 6, 4), 2, 1), ((18, 4, 3), 3, 2)])
def test_operator_norm2_matches_power_iteration(n, s, r):
    """||A||_2^2 (b = 1) by the oracle's Lanczos process equals the limit of
    a plain power iteration with the oracle's own A^T A (lambda = 0)."""
    g = _geom(n, s=s, r=r, kmin=2, kmax=5, theta=[0.1, 0.2, 0.3, 0.4])
    v = W.random_volume(g.shape, 5)
    o = oracle.SolveOpts(lam=0.0)
    lam = 0.0
    for _ in range(400):
        w = oracle.normal_apply(g, v, None, o)
        lam = float(np.sum(v * w) / np.sum(v * v))
        v = w / np.linalg.norm(w)
    assert oracle.operator_norm2(g) == pytest.approx(lam, rel=1e-9)


def _norm2_alias_blocks(g):
    """The closed form of ||A||_2^2 for a separable PSF and b = 1:
    A^T A = (drive part) (x) Y^T Y (x) Z^T Z, the transverse factors are
    circulant (eigenvalues |DFT|^2) and the drive part couples frequency m
    only with its aliases m + a n/s: with the kernels shifted by the kept-row
    offset r, the block is B_m[a][b] = (1/s) sum_k conj(x_k[m + aM]) x_k[m + bM]."""
    X, Y, Z = oracle.psf_tables(g)
    s, r = g.ds_factor, g.ds_offset
    M = g.n[0] // s
    xh = np.fft.fft(np.roll(X, -r, axis=1), axis=1)
    lam_x = 0.0
    for m in range(M):
        v = xh[:, m + M * np.arange(s)]
        lam_x = max(lam_x, float(np.linalg.eigvalsh((np.conj(v).T @ v) / s).max()))
    return lam_x * float(np.max(np.abs(np.fft.fft(Y)) ** 2)) * float(np.max(np.abs(np.fft.fft(Z)) ** 2))


@pytest.mark.parametrize("n,s,r,k", [((16, 8, 6), 1, 0, (2, 5)), ((24, 12, 8), 2, 1, (2, 9)),
                                     ((18, 6, 4), 3, 2, (3, 6)), ((32, 16, 8), 2, 0, (2, 9))])
def test_operator_norm2_matches_alias_block_closed_form(n, s, r, k):
    """The Lanczos value equals the Fourier alias-block closed form (written
    here, not in the oracle) to near FP64 precision."""
    g = _geom(n, s=s, r=r, kmin=k[0], kmax=k[1], theta=list(np.linspace(0.1, 0.9, k[1] - k[0] + 1)))
    assert oracle.operator_norm2(g) == pytest.approx(_norm2_alias_blocks(g), rel=1e-11)


def test_relative_lambda_scales_regulariser():
    g = _geom((8, 4, 4), s=2, kmin=2, kmax=3)
    p = W.random_volume(g.shape, 1)
    sig2 = oracle.operator_norm2(g)
    a = oracle.normal_apply(g, p, None, oracle.SolveOpts(lam=1e-3, lam_relative=True))
    b = oracle.normal_apply(g, p, None, oracle.SolveOpts(lam=1e-3 * sig2))
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(b).max())


def test_cg_fixed_iterations_and_history():
    g = _geom((8, 4, 4), kmin=2, kmax=3)
    d = W.random_portraits(g.portrait_shape, 3)
    x, it, hist = oracle.cg(g, d, None, oracle.SolveOpts(lam=1e-3, rel_tol=0.0, max_iter=7))
    assert it == 7 and len(hist) == 8 and hist[0] == pytest.approx(1.0)
    assert hist[-1] < hist[0]


def test_apg_matches_nnls():
    """The paper's accelerated projected gradient converges to the
    nonnegative least-squares minimiser; the reference is scipy's NNLS
    (Lawson-Hanson) on the stacked real system [A; sqrt(lambda) I]."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    g = _geom((8, 3, 3), s=2, r=0, kmin=2, kmax=4, theta=[0.4, -0.3, 0.9])
    b = 0.5 + np.abs(W.random_volume(g.shape, 51))
    lam = 0.2                                 # well conditioned: APG converges to 1e-8 in 20000 steps
    opts = oracle.SolveOpts(lam=lam)
    rho_true = np.maximum(W.random_volume(g.shape, 52), 0.0)
    d = oracle.forward(g, rho_true, b) + 0.05 * W.random_portraits(g.portrait_shape, 53)
    N = int(np.prod(g.shape))
    cols = []
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        dk = oracle.forward(g, e.reshape(g.shape), b)
        th = np.array([0.4, -0.3, 0.9])[:, None, None, None]
        cols.append(np.real(np.exp(-1j * th) * dk).ravel())
    A = np.array(cols).T
    th = np.array([0.4, -0.3, 0.9])[:, None, None, None]
    rhs = np.real(np.exp(-1j * th) * d).ravel()
    Ms = np.vstack([A, math.sqrt(lam) * np.eye(N)])
    bs = np.concatenate([rhs, np.zeros(N)])
    ref, _ = scipy_opt.nnls(Ms, bs, maxiter=50 * N)
    Nm = Ms.T @ Ms
    tau = 1.0 / np.linalg.eigvalsh(Nm).max()
    x = oracle.apg(g, d, tau, 20000, b, opts)
    assert np.all(x >= 0)
    assert np.sum(ref == 0) > 0               # the constraint is active somewhere
    np.testing.assert_allclose(x.ravel(), ref, atol=1e-7 * max(np.abs(ref).max(), 1))


def test_mhad_matches_dense_least_squares():
    """MHAD (appendix, Eq. mhadM) equals the dense minimiser of
    sum_k ||f^{k-1} * rho - c_k^{-1} d_k||^2 + lambda ||rho||^2 assembled
    from circulant matrices of the difference filter."""
    n, lam = 24, 0.05
    ks = [2, 3, 4, 5]
    cks = [oracle.ck(k, 2.0) for k in ks]
    rng_d = [W.random_volume((n,), 60 + k) for k in ks]
    got = oracle.mhad(rng_d, cks, lam)
    F = np.zeros((n, n))
    for j in range(n):                        # (f * u)[j] = u[j+1] - u[j-1]
        F[j, (j + 1) % n] += 1.0
        F[j, (j - 1) % n] -= 1.0
    rows, rhs = [], []
    for k, c, dk in zip(ks, cks, rng_d):
        rows.append(np.linalg.matrix_power(F, k - 1))
        rhs.append(dk / c)
    Ms = np.vstack(rows + [math.sqrt(lam) * np.eye(n)])
    bs = np.concatenate(rhs + [np.zeros(n)])
    ref = np.linalg.lstsq(Ms, bs, rcond=None)[0]
    np.testing.assert_allclose(got, ref, atol=1e-10)


# --------------------------------------------------------------------------
# Input generator
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    """SplitMix64 with seed 0: the first outputs published with the
    generator's reference implementation."""
    z = W.splitmix64(0, 0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generator_statistics_and_determinism():
    a = W.Stream(7).normal(200000)
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1) < 0.01
    n = W.unit_complex_noise((1000, 100), 3)
    assert abs(np.mean(np.abs(n) ** 2) - 1.0) < 0.02
    p1 = W.phantom((32, 24, 16), (1, 1, 1), 5, 5, 2)
    p2 = W.phantom((32, 24, 16), (1, 1, 1), 5, 5, 2)
    np.testing.assert_array_equal(p1, p2)
    assert p1.min() >= 0 and p1.max() > 0.1
    b = W.sensitivity((32, 24, 16))
    assert b.max() <= 1.0 and b.min() > 0.3   # corners: exp(-3 (0.5/0.6)^2 / 2) = 0.35


# --------------------------------------------------------------------------
# Golden fixtures (tests/golden/): values fixed by the paper's printed
# formulas and by the Taylor series of the Langevin function
# --------------------------------------------------------------------------

def _golden_rows(name):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(v) for v in line.split()])
    return rows


def test_golden_ck_theorem1():
    """c_k = (gamma A)^k / (k-1)! at gamma A = 2 (Theorem 1), k = 1..17."""
    rows = _golden_rows("ck_theorem1.txt")
    assert len(rows) == 17
    for k, num, den in rows:
        assert oracle.ck(k, 2.0) == pytest.approx(num / den, rel=1e-15), k


def test_golden_langevin_taylor_at_zero():
    """L^(k)(0) for odd k from the Taylor series of coth x - 1/x."""
    rows = _golden_rows("langevin_taylor_at_zero.txt")
    assert [r[0] for r in rows] == [1, 3, 5, 7, 9, 11]
    for k, num, den in rows:
        assert oracle.langevin_deriv(k, 0.0) == pytest.approx(num / den, rel=1e-13), k


# --------------------------------------------------------------------------
# Output crops (for grids too large for the whole-volume oracle)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,s,r", [((12, 10, 8), 1, 0), ((16, 6, 9), 2, 1), ((18, 7, 6), 3, 2)])
def test_forward_crop_equals_window_of_full_forward(n, s, r):
    """The crop evaluation is the same circular sum restricted to the outputs
    asked for: it must equal the matching window of the whole forward model
    (itself pinned against numpy's FFT convolution and the triple sum)."""
    g = _geom(n, s=s, r=r, kmin=2, kmax=5, theta=[0.2, -1.0, 2.5, 0.7])
    rho = W.random_volume(g.shape, 11)
    b = W.sensitivity(n, (1.0, 1.0, 1.0))
    full = oracle.forward(g, rho, b)
    mx = n[0] // s
    crop = ((1, mx - 2), (2, n[1] - 3), (1, n[2] - 2))
    got = oracle.forward_crop(g, rho, crop, b)
    ref = full[:, 1:1 + n[2] - 2, 2:2 + n[1] - 3, 1:1 + mx - 2]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(full).max()


@pytest.mark.parametrize("n,s,r", [((12, 10, 8), 1, 0), ((16, 6, 9), 2, 1), ((18, 7, 6), 3, 2)])
def test_adjoint_crop_equals_window_of_full_adjoint(n, s, r):
    g = _geom(n, s=s, r=r, kmin=2, kmax=5, theta=[0.2, -1.0, 2.5, 0.7])
    y = W.random_portraits(g.portrait_shape, 12)
    b = W.sensitivity(n, (1.0, 1.0, 1.0))
    full = oracle.adjoint(g, y, b)
    crop = ((3, n[0] - 5), (1, n[1] - 2), (2, n[2] - 4))
    got = oracle.adjoint_crop(g, y, crop, b)
    ref = full[2:2 + n[2] - 4, 1:1 + n[1] - 2, 3:3 + n[0] - 5]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(full).max()


# --------------------------------------------------------------------------
# Boundary image padding (Sec. 3.x)
# --------------------------------------------------------------------------

def test_padded_operators_are_adjoint_and_reduce_to_the_plain_ones():
    """Re<A_p x, y> = <x, A_p^T y> for the cropped forward and zero-padding
    adjoint, and with no padding they are the plain operators."""
    g = _geom((8, 4, 6), s=2, r=1, kmin=2, kmax=4, theta=[0.4, -1.0, 2.0])
    pad = (2, 1, 3)
    ge = oracle.padded_geometry(g, pad)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(ge.shape)
    b = 0.5 + rng.random(ge.shape)
    y = rng.standard_normal(g.portrait_shape) + 1j * rng.standard_normal(g.portrait_shape)
    lhs = np.real(np.vdot(y, oracle.padded_forward(g, pad, x, b)))
    rhs = float(np.sum(x * oracle.padded_adjoint(g, pad, y, b)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    x0 = rng.standard_normal(g.shape)
    np.testing.assert_array_equal(oracle.padded_forward(g, (0, 0, 0), x0), oracle.forward(g, x0))
    np.testing.assert_array_equal(oracle.padded_adjoint(g, (0, 0, 0), y), oracle.adjoint(g, y))


def test_padded_cg_matches_dense_normal_equations():
    """padded_cg solves (A_p^T A_p + lambda I) x = A_p^T d: against the dense
    matrix of A_p assembled column by column from unit vectors."""
    g = _geom((4, 2, 2), s=2, kmin=2, kmax=3)
    pad = (2, 1, 1)
    ge = oracle.padded_geometry(g, pad)
    n = int(np.prod(ge.shape))
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        dj = oracle.padded_forward(g, pad, e.reshape(ge.shape)).ravel()
        cols.append(np.concatenate([dj.real, dj.imag]))
    A = np.array(cols).T
    rng = np.random.default_rng(12)
    d = rng.standard_normal(g.portrait_shape) + 1j * rng.standard_normal(g.portrait_shape)
    lam = 0.05
    rhs = A.T @ np.concatenate([d.real.ravel(), d.imag.ravel()])
    ref = np.linalg.solve(A.T @ A + lam * np.eye(n), rhs)
    x = oracle.padded_cg(g, pad, d, None, lam, 100)
    np.testing.assert_allclose(x.ravel(), ref, atol=1e-9 * np.abs(ref).max())


# --------------------------------------------------------------------------
# Portrait phase calibration (Sec. 4.4)
# --------------------------------------------------------------------------

def test_phase_modulo_pi_is_the_principal_axis():
    """Samples e^{i theta} a_j with real a_j of both signs: the estimate is
    theta modulo pi exactly (closed form: every a_j^2 e^{2 i theta} points
    along 2 theta)."""
    rng = np.random.default_rng(21)
    for theta in (-2.9, -1.2, 0.0, 0.7, 1.5707, 3.1):
        a = rng.standard_normal((1, 3, 4, 5))
        d = np.exp(1j * theta) * a
        g = _geom((5, 4, 3), kmin=2, kmax=2)
        est, _ = oracle.estimate_phase(g, d, frac=1e-9)
        diff = np.angle(np.exp(2j * (est[0] - theta))) / 2
        assert abs(diff) <= 1e-12, (theta, est)


@pytest.mark.parametrize("n,s,kmin,kmax", [((48, 16, 12), 1, 3, 6), ((32, 24, 16), 1, 2, 7), ((64, 12, 8), 2, 2, 9)])
def test_phase_recovers_the_generating_phases(n, s, kmin, kmax):
    """Noise-free portraits of a non-negative phantom made with known phases:
    with s = 1 every theta_k is resolved and equals the generating one; with
    s = 2 none is resolved and each equals it modulo pi."""
    K = kmax - kmin + 1
    theta = np.random.default_rng(kmin + K).uniform(-np.pi, np.pi, K)
    g = _geom(n, s=s, kmin=kmin, kmax=kmax, theta=list(theta))
    rho = W.phantom(n, (1.0, 1.0, 1.0), 3, 6, 1)
    d = oracle.forward(g, rho)
    est, res = oracle.estimate_phase(g, d)
    assert res.all() if s == 1 else not res.any()
    err = np.angle(np.exp(1j * (est - theta)))
    err_pi = np.angle(np.exp(2j * (est - theta))) / 2
    if res.any():
        assert np.abs(err[res == 1]).max() <= 1e-10, err
    assert np.abs(err_pi).max() <= 1e-10, err_pi
