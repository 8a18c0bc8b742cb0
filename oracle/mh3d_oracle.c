/*
 * mh3d_oracle.c -- plain, slow FP64 reference of the MH3D portrait model.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (arXiv 2503.13802, "Multi-Harmonic Gridded 3D
 * Deconvolution"):
 *
 *   Langevin function  L(x) = coth(x) - 1/x                 (Sec. 2, signal model)
 *   harmonic PSF       h_k(x) ~ c_k L^(k)(gamma x)          (Sec. 3.3, Eq. hkapprox)
 *   coefficients       c_k = (gamma A)^k / (k-1)!           (Theorem 1; App. MHAD)
 *   portrait model     d_k = h_k * (b_z . rho)              (Sec. 3.2, Eq. portz)
 *   downsampled model  A = P H B                            (Sec. 4.1, Eq. dN)
 *   phase              d~_k = e^{i theta_k} d_k             (Sec. 4.4)
 *   regulariser        R = ||T rho||^2 + alpha ||P_a rho||^2 (Sec. 4.3, Eq. finalR)
 *
 * Readings taken where the paper is silent:
 *   - the 3D PSF is separable: along the drive axis c_k L^(k)(gamma o_x);
 *     across it phi(o) = 3 L'(gamma_t o) on each transverse axis, with
 *     gamma_t = transverse_ratio * gamma (the transverse gradient is half the
 *     drive-axis gradient, Sec. 2);
 *   - samples sit at minimal-image integer offsets of the periodic grid; for
 *     even n the index n/2 is the offset -n/2;
 *   - the convolution is circular (FFT-periodic, Sec. 4.2 and Table ops);
 *   - the row selector P keeps drive-axis indices i = r (mod s);
 *   - A maps real rho to complex portraits, d_k = e^{i theta_k} (real); its
 *     adjoint is taken for the real inner product Re<.,.>;
 *   - T stacks periodic second differences along each axis; P_a keeps the
 *     voxels within `shell` of a face.
 *
 * Layout: volumes are C-order [nz][ny][nx] (x, the drive axis, contiguous);
 * portraits are [K][nz][ny][mx] complex (interleaved re, im), mx = nx / s.
 *
 * Every function is a direct transcription of a definition: circular sums
 * evaluated in space, O(n) per output sample along each axis.  Separable
 * evaluation of a separable kernel is exact up to rounding order; the
 * function orc_forward_full3d evaluates the full triple sum instead and the
 * tests pin the two against each other.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Langevin derivatives                                                      */
/* ------------------------------------------------------------------------ */

/* zeta(2m) for m >= 1: direct sum of j^{-2m} for j < J plus the
 * Euler-Maclaurin tail J^{1-s}/(s-1) + J^{-s}/2 + s J^{-s-1}/12
 * - s(s+1)(s+2) J^{-s-3}/720.  With J = 2000 the remainder is far below
 * double precision for every s >= 2. */
static double orc_zeta_even(int m)
{
    const double s = 2.0 * m;
    const int J = 2000;
    double sum = 0.0;
    for (int j = J - 1; j >= 1; --j) sum += pow((double)j, -s);
    const double Jd = (double)J;
    sum += pow(Jd, 1.0 - s) / (s - 1.0) + 0.5 * pow(Jd, -s) + s * pow(Jd, -s - 1.0) / 12.0
         - s * (s + 1.0) * (s + 2.0) * pow(Jd, -s - 3.0) / 720.0;
    return sum;
}

#define ORC_TAYLOR_TERMS 420
static double orc_zeta_tab[ORC_TAYLOR_TERMS + 1];
static int orc_zeta_ready = 0;

static void orc_init_zeta(void)
{
    if (orc_zeta_ready) return;
    for (int m = 1; m <= ORC_TAYLOR_TERMS; ++m) orc_zeta_tab[m] = orc_zeta_even(m);
    orc_zeta_ready = 1;
}

/* Taylor series about 0 (radius pi, poles of coth at i n pi):
 *   L(x) = sum_{n>=1} (-1)^{n+1} 2 zeta(2n) x^{2n-1} / pi^{2n}
 * (this is 2^{2n} B_{2n} / (2n)! written through zeta), differentiated k
 * times term by term. */
static double orc_langevin_taylor(int k, double x)
{
    double sum = 0.0;
    const double xr = x / ORC_PI;
    for (int n = 1; n <= ORC_TAYLOR_TERMS; ++n) {
        const int p = 2 * n - 1;          /* power of x before differentiation */
        if (p < k) continue;
        double ff = 1.0;                  /* falling factorial p (p-1) ... (p-k+1) */
        for (int i = 0; i < k; ++i) ff *= (double)(p - i);
        const double sign = (n & 1) ? 1.0 : -1.0;
        /* x^{p-k} / pi^{2n} = (x/pi)^{p-k} / pi^{k+1} */
        const double term = sign * 2.0 * orc_zeta_tab[n] * ff * pow(xr, (double)(p - k))
                          / pow(ORC_PI, (double)(k + 1));
        sum += term;
    }
    return sum;
}

/* For x > 0: coth x = 1 + 2 sum_{m>=1} e^{-2 m x}, so
 *   D^k coth x = 2 sum_{m>=1} (-2m)^k e^{-2 m x}  (k >= 1),
 * and D^k (1/x) = (-1)^k k! / x^{k+1}. */
static double orc_langevin_large(int k, double x)
{
    double dk = (k == 0) ? 1.0 : 0.0;
    for (int m = 1; m <= 400; ++m) {
        const double t = 2.0 * pow(-2.0 * m, (double)k) * exp(-2.0 * m * x);
        dk += t;
        if (fabs(t) < 1e-300) break;
    }
    double kfact = 1.0;
    for (int i = 2; i <= k; ++i) kfact *= (double)i;
    const double inv = ((k & 1) ? -1.0 : 1.0) * kfact / pow(x, (double)(k + 1));
    return dk - inv;
}

/* Mittag-Leffler pole expansion coth x - 1/x = sum_{n>=1} [1/(x - i n pi) + 1/(x + i n pi)]
 * (poles of coth at i n pi), differentiated k times:
 *   L^{(k)}(x) = sum_{n>=1} 2 Re[ (-1)^k k! / (x - i n pi)^{k+1} ].
 * With x - i n pi = r e^{i phi}: Re[(x - i n pi)^{-(k+1)}] = cos((k+1) phi) / r^{k+1}.
 * Used for k >= 6, where the terms fall like n^{-(k+1)} and 4000 terms leave
 * a tail below 1e-20 of the first term. */
static double orc_langevin_poles(int k, double x)
{
    double kfact = 1.0;
    for (int i = 2; i <= k; ++i) kfact *= (double)i;
    const double sgn = (k & 1) ? -1.0 : 1.0;
    double sum = 0.0;
    for (int n = 4000; n >= 1; --n) {          /* smallest terms first */
        const double im = -n * ORC_PI;
        const double r = sqrt(x * x + im * im);
        const double phi = atan2(im, x);
        sum += 2.0 * sgn * kfact * cos((k + 1) * phi) / pow(r, (double)(k + 1));
    }
    return sum;
}

/* L^{(k)}(x), the k-th derivative of the Langevin function, k >= 0.
 * Branches (each an exact expansion of the same function, chosen where its
 * rounding error is smallest): Taylor about 0 for |x| < 1.5 (|x| < 1 when
 * k >= 6); the pole expansion for k >= 6 and |x| < 8; the exponential
 * expansion of coth elsewhere. */
double orc_langevin_deriv(int k, double x)
{
    orc_init_zeta();
    const double ax = fabs(x);
    if (ax < 1.0 || (k < 6 && ax < 1.5)) return orc_langevin_taylor(k, x);
    if (k >= 6 && ax < 8.0) return orc_langevin_poles(k, x);
    /* L is odd, so L^{(k)}(-x) = (-1)^{k+1} L^{(k)}(x). */
    if (x < 0.0) return ((k & 1) ? 1.0 : -1.0) * orc_langevin_large(k, -x);
    return orc_langevin_large(k, x);
}

/* ------------------------------------------------------------------------ */
/* PSF sample tables                                                         */
/* ------------------------------------------------------------------------ */

/* Minimal-image offset of index i on a periodic axis of length n. */
static int orc_offset(int i, int n) { return (2 * i < n) ? i : i - n; }

/* c_k = (gamma A)^k / (k-1)!  (Theorem 1). */
double orc_ck(int k, double gammaA)
{
    double f = 1.0;
    for (int i = 2; i <= k - 1; ++i) f *= (double)i;
    return pow(gammaA, (double)k) / f;
}

/* X[(k-kmin)*nx + i] = c_k L^(k)(gamma * o_i * dx)      (drive axis)
 * Y[i] = 3 L'(gamma_t * o_i * dy),  Z[i] = 3 L'(gamma_t * o_i * dz). */
void orc_psf_tables(int nx, int ny, int nz, double dx, double dy, double dz,
                    int kmin, int kmax, double gamma, double gammaA, double tratio,
                    double* X, double* Y, double* Z)
{
    orc_init_zeta();
    const double gt = gamma * tratio;
    for (int k = kmin; k <= kmax; ++k) {
        const double ck = orc_ck(k, gammaA);
        for (int i = 0; i < nx; ++i)
            X[(size_t)(k - kmin) * nx + i] = ck * orc_langevin_deriv(k, gamma * orc_offset(i, nx) * dx);
    }
    for (int i = 0; i < ny; ++i) Y[i] = 3.0 * orc_langevin_deriv(1, gt * orc_offset(i, ny) * dy);
    for (int i = 0; i < nz; ++i) Z[i] = 3.0 * orc_langevin_deriv(1, gt * orc_offset(i, nz) * dz);
}

/* ------------------------------------------------------------------------ */
/* Forward A = P H B and adjoint                                            */
/* ------------------------------------------------------------------------ */

static int orc_mod(long a, int n) { long m = a % n; return (int)(m < 0 ? m + n : m); }

/* Circular convolution along z then y of a volume (in place into out). */
static void orc_conv_yz(int nx, int ny, int nz, const double* Y, const double* Z,
                        const double* u, double* out, int correlate)
{
    const size_t N = (size_t)nx * ny * nz;
    double* v = (double*)malloc(N * sizeof(double));
    /* along z:  v[z] = sum_z' Z[z - z'] u[z']   (correlation: Z[z' - z]) */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double acc = 0.0;
                for (int zp = 0; zp < nz; ++zp) {
                    const int o = correlate ? orc_mod((long)zp - z, nz) : orc_mod((long)z - zp, nz);
                    acc += Z[o] * u[((size_t)zp * ny + y) * nx + x];
                }
                v[((size_t)z * ny + y) * nx + x] = acc;
            }
    /* along y */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double acc = 0.0;
                for (int yp = 0; yp < ny; ++yp) {
                    const int o = correlate ? orc_mod((long)yp - y, ny) : orc_mod((long)y - yp, ny);
                    acc += Y[o] * v[((size_t)z * ny + yp) * nx + x];
                }
                out[((size_t)z * ny + y) * nx + x] = acc;
            }
    free(v);
}

/* d_k[z][y][i'] = e^{i theta_k} sum_x' X_k[(s i' + r - x') mod nx] w[z][y][x'],
 * w = Y *_y (Z *_z (b . rho)).  b == NULL means b = 1. */
void orc_forward(int nx, int ny, int nz, int s, int r, int K,
                 const double* X, const double* Y, const double* Z, const double* theta,
                 const double* b, const double* rho, double* d)
{
    const size_t N = (size_t)nx * ny * nz;
    const int mx = nx / s;
    double* u = (double*)malloc(N * sizeof(double));
    double* w = (double*)malloc(N * sizeof(double));
    for (size_t i = 0; i < N; ++i) u[i] = (b ? b[i] : 1.0) * rho[i];
    orc_conv_yz(nx, ny, nz, Y, Z, u, w, 0);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int kk = 0; kk < K; ++kk)
        for (int zy = 0; zy < nz * ny; ++zy) {
            const double c = cos(theta ? theta[kk] : 0.0), sn = sin(theta ? theta[kk] : 0.0);
            const double* row = w + (size_t)zy * nx;
            const double* Xk = X + (size_t)kk * nx;
            for (int ip = 0; ip < mx; ++ip) {
                double acc = 0.0;
                for (int xp = 0; xp < nx; ++xp)
                    acc += Xk[orc_mod((long)s * ip + r - xp, nx)] * row[xp];
                double* o = d + 2 * (((size_t)kk * nz * ny + zy) * mx + ip);
                o[0] = c * acc;
                o[1] = sn * acc;
            }
        }
    free(u);
    free(w);
}

/* The same operator as the full triple sum over every source voxel:
 * d_k[z][y][i'] = e^{i theta_k} sum_{z',y',x'} X_k[s i'+r-x'] Y[y-y'] Z[z-z'] b rho.
 * O(N K M); for tiny grids only. */
void orc_forward_full3d(int nx, int ny, int nz, int s, int r, int K,
                        const double* X, const double* Y, const double* Z, const double* theta,
                        const double* b, const double* rho, double* d)
{
    const int mx = nx / s;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int kk = 0; kk < K; ++kk)
        for (int zy = 0; zy < nz * ny; ++zy) {
            const int z = zy / ny, y = zy % ny;
            const double c = cos(theta ? theta[kk] : 0.0), sn = sin(theta ? theta[kk] : 0.0);
            for (int ip = 0; ip < mx; ++ip) {
                double acc = 0.0;
                for (int zp = 0; zp < nz; ++zp)
                    for (int yp = 0; yp < ny; ++yp)
                        for (int xp = 0; xp < nx; ++xp) {
                            const size_t j = ((size_t)zp * ny + yp) * nx + xp;
                            const double h = X[(size_t)kk * nx + orc_mod((long)s * ip + r - xp, nx)]
                                           * Y[orc_mod((long)y - yp, ny)] * Z[orc_mod((long)z - zp, nz)];
                            acc += h * (b ? b[j] : 1.0) * rho[j];
                        }
                double* o = d + 2 * (((size_t)kk * nz * ny + zy) * mx + ip);
                o[0] = c * acc;
                o[1] = sn * acc;
            }
        }
}

/* Adjoint for Re<.,.>:
 * rho[z][y][x] = b . corr_y corr_z ( sum_k sum_i' X_k[s i' + r - x] Re(e^{-i theta_k} d_k[z][y][i']) ). */
void orc_adjoint(int nx, int ny, int nz, int s, int r, int K,
                 const double* X, const double* Y, const double* Z, const double* theta,
                 const double* b, const double* d, double* rho)
{
    const size_t N = (size_t)nx * ny * nz;
    const int mx = nx / s;
    double* g = (double*)malloc(N * sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int zy = 0; zy < nz * ny; ++zy) {
        for (int x = 0; x < nx; ++x) {
            double acc = 0.0;
            for (int kk = 0; kk < K; ++kk) {
                const double c = cos(theta ? theta[kk] : 0.0), sn = sin(theta ? theta[kk] : 0.0);
                const double* Xk = X + (size_t)kk * nx;
                for (int ip = 0; ip < mx; ++ip) {
                    const double* dv = d + 2 * (((size_t)kk * nz * ny + zy) * mx + ip);
                    const double proj = c * dv[0] + sn * dv[1];
                    acc += Xk[orc_mod((long)s * ip + r - x, nx)] * proj;
                }
            }
            g[(size_t)zy * nx + x] = acc;
        }
    }
    orc_conv_yz(nx, ny, nz, Y, Z, g, rho, 1);
    if (b) for (size_t i = 0; i < N; ++i) rho[i] *= b[i];
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Output crops of the forward and adjoint operators (large grids)          */
/* ------------------------------------------------------------------------ */

/* The forward model of orc_forward, evaluated only on the output crop
 * z in [c[4], c[4]+c[5]), y in [c[2], c[2]+c[3]), i' in [c[0], c[0]+c[1])
 * (c = {i0, ni, y0, ny_c, z0, nz_c}); d_crop is [K][nz_c][ny_c][ni] complex.
 * Same definition, the circular sums restricted to the outputs asked for:
 *   v[z][y'][x'] = sum_z' Z[z - z'] b rho[z'][y'][x']      (z in the crop)
 *   w[z][y][x']  = sum_y' Y[y - y'] v[z][y'][x']           (y in the crop)
 *   d_k[z][y][i'] = e^{i theta_k} sum_x' X_k[s i' + r - x'] w[z][y][x']. */
void orc_forward_crop(int nx, int ny, int nz, int s, int r, int K,
                      const double* X, const double* Y, const double* Z, const double* theta,
                      const double* b, const double* rho, const int* c, double* d)
{
    const int i0 = c[0], ni = c[1], y0 = c[2], nyc = c[3], z0 = c[4], nzc = c[5];
    double* v = (double*)malloc((size_t)nzc * ny * nx * sizeof(double));
    double* w = (double*)malloc((size_t)nzc * nyc * nx * sizeof(double));
    #pragma omp parallel for collapse(2) schedule(static)
    for (int zc = 0; zc < nzc; ++zc)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double acc = 0.0;
                for (int zp = 0; zp < nz; ++zp) {
                    const size_t j = ((size_t)zp * ny + y) * nx + x;
                    acc += Z[orc_mod((long)(z0 + zc) - zp, nz)] * (b ? b[j] : 1.0) * rho[j];
                }
                v[((size_t)zc * ny + y) * nx + x] = acc;
            }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int zc = 0; zc < nzc; ++zc)
        for (int yc = 0; yc < nyc; ++yc)
            for (int x = 0; x < nx; ++x) {
                double acc = 0.0;
                for (int yp = 0; yp < ny; ++yp)
                    acc += Y[orc_mod((long)(y0 + yc) - yp, ny)] * v[((size_t)zc * ny + yp) * nx + x];
                w[((size_t)zc * nyc + yc) * nx + x] = acc;
            }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int kk = 0; kk < K; ++kk)
        for (int zy = 0; zy < nzc * nyc; ++zy) {
            const double cs = cos(theta ? theta[kk] : 0.0), sn = sin(theta ? theta[kk] : 0.0);
            const double* row = w + (size_t)zy * nx;
            const double* Xk = X + (size_t)kk * nx;
            for (int ic = 0; ic < ni; ++ic) {
                const long ip = i0 + ic;
                double acc = 0.0;
                for (int xp = 0; xp < nx; ++xp) acc += Xk[orc_mod((long)s * ip + r - xp, nx)] * row[xp];
                double* o = d + 2 * (((size_t)kk * nzc * nyc + zy) * ni + ic);
                o[0] = cs * acc;
                o[1] = sn * acc;
            }
        }
    free(v);
    free(w);
}

/* The adjoint of orc_adjoint, evaluated only on the image crop
 * z in [c[4], c[4]+c[5]), y in [c[2], c[2]+c[3]), x in [c[0], c[0]+c[1]);
 * rho_crop is [nz_c][ny_c][nx_c]:
 *   g[z'][y'][x] = sum_k sum_i' X_k[s i' + r - x] Re(e^{-i theta_k} d_k[z'][y'][i'])   (x in the crop)
 *   v[z][y'][x]  = sum_z' Z[z' - z] g[z'][y'][x]                                        (z in the crop)
 *   rho[z][y][x] = b sum_y' Y[y' - y] v[z][y'][x]                                       (y in the crop) */
void orc_adjoint_crop(int nx, int ny, int nz, int s, int r, int K,
                      const double* X, const double* Y, const double* Z, const double* theta,
                      const double* b, const double* d, const int* c, double* rho)
{
    const int x0 = c[0], nxc = c[1], y0 = c[2], nyc = c[3], z0 = c[4], nzc = c[5];
    const int mx = nx / s;
    double* g = (double*)malloc((size_t)nz * ny * nxc * sizeof(double));
    double* v = (double*)malloc((size_t)nzc * ny * nxc * sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int zy = 0; zy < nz * ny; ++zy)
        for (int xc = 0; xc < nxc; ++xc) {
            double acc = 0.0;
            for (int kk = 0; kk < K; ++kk) {
                const double cs = cos(theta ? theta[kk] : 0.0), sn = sin(theta ? theta[kk] : 0.0);
                const double* Xk = X + (size_t)kk * nx;
                for (int ip = 0; ip < mx; ++ip) {
                    const double* dv = d + 2 * (((size_t)kk * nz * ny + zy) * mx + ip);
                    acc += Xk[orc_mod((long)s * ip + r - (x0 + xc), nx)] * (cs * dv[0] + sn * dv[1]);
                }
            }
            g[(size_t)zy * nxc + xc] = acc;
        }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int zc = 0; zc < nzc; ++zc)
        for (int y = 0; y < ny; ++y)
            for (int xc = 0; xc < nxc; ++xc) {
                double acc = 0.0;
                for (int zp = 0; zp < nz; ++zp)
                    acc += Z[orc_mod((long)zp - (z0 + zc), nz)] * g[((size_t)zp * ny + y) * nxc + xc];
                v[((size_t)zc * ny + y) * nxc + xc] = acc;
            }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int zc = 0; zc < nzc; ++zc)
        for (int yc = 0; yc < nyc; ++yc)
            for (int xc = 0; xc < nxc; ++xc) {
                double acc = 0.0;
                for (int yp = 0; yp < ny; ++yp)
                    acc += Y[orc_mod((long)yp - (y0 + yc), ny)] * v[((size_t)zc * ny + yp) * nxc + xc];
                const size_t j = ((size_t)(z0 + zc) * ny + (y0 + yc)) * nx + (x0 + xc);
                rho[((size_t)zc * nyc + yc) * nxc + xc] = (b ? b[j] : 1.0) * acc;
            }
    free(g);
    free(v);
}

/* ------------------------------------------------------------------------ */
/* Regulariser and normal operator                                          */
/* ------------------------------------------------------------------------ */

/* Periodic second difference along axis a: (D p)[i] = p[i-e] - 2 p[i] + p[i+e]. */
static void orc_second_diff(int nx, int ny, int nz, int axis, const double* p, double* out)
{
    const int n[3] = {nx, ny, nz};
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c[3] = {x, y, z};
                int lo[3] = {x, y, z}, hi[3] = {x, y, z};
                lo[axis] = orc_mod((long)c[axis] - 1, n[axis]);
                hi[axis] = orc_mod((long)c[axis] + 1, n[axis]);
                const size_t i0 = ((size_t)z * ny + y) * nx + x;
                const size_t il = ((size_t)lo[2] * ny + lo[1]) * nx + lo[0];
                const size_t ih = ((size_t)hi[2] * ny + hi[1]) * nx + hi[0];
                out[i0] = p[il] - 2.0 * p[i0] + p[ih];
            }
}

/* 1 if voxel (x,y,z) lies within `shell` voxels of a face of the grid. */
static int orc_in_shell(int x, int y, int z, int nx, int ny, int nz, int shell)
{
    return x < shell || y < shell || z < shell || x >= nx - shell || y >= ny - shell || z >= nz - shell;
}

/* out = R p with R = I (kind 0) or R = T^T T + alpha P_a^T P_a (kind 1). */
void orc_reg_apply(int nx, int ny, int nz, int kind, double alpha, int shell,
                   const double* p, double* out)
{
    const size_t N = (size_t)nx * ny * nz;
    if (kind == 0) { memcpy(out, p, N * sizeof(double)); return; }
    double* t1 = (double*)malloc(N * sizeof(double));
    double* t2 = (double*)malloc(N * sizeof(double));
    memset(out, 0, N * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        orc_second_diff(nx, ny, nz, a, p, t1);   /* D_a p        */
        orc_second_diff(nx, ny, nz, a, t1, t2);  /* D_a^T D_a p  (D_a is symmetric) */
        for (size_t i = 0; i < N; ++i) out[i] += t2[i];
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (orc_in_shell(x, y, z, nx, ny, nz, shell)) {
                    const size_t i = ((size_t)z * ny + y) * nx + x;
                    out[i] += alpha * p[i];
                }
    free(t1);
    free(t2);
}

/* out = A^T A p + lambda R p. */
void orc_normal_apply(int nx, int ny, int nz, int s, int r, int K,
                      const double* X, const double* Y, const double* Z, const double* theta,
                      const double* b, double lambda, int kind, double alpha, int shell,
                      const double* p, double* out)
{
    const size_t N = (size_t)nx * ny * nz;
    const size_t Md = (size_t)K * nz * ny * (nx / s) * 2;
    double* d = (double*)malloc(Md * sizeof(double));
    double* rp = (double*)malloc(N * sizeof(double));
    orc_forward(nx, ny, nz, s, r, K, X, Y, Z, theta, b, p, d);
    orc_adjoint(nx, ny, nz, s, r, K, X, Y, Z, theta, b, d, out);
    orc_reg_apply(nx, ny, nz, kind, alpha, shell, p, rp);
    for (size_t i = 0; i < N; ++i) out[i] += lambda * rp[i];
    free(d);
    free(rp);
}

/* ------------------------------------------------------------------------ */
/* ||A||_2^2: the largest eigenvalue of A^T A                               */
/* ------------------------------------------------------------------------ */

/* Number of eigenvalues below mu of the symmetric tridiagonal matrix with
 * diagonal a[0..m) and off-diagonal b[0..m-1): the count of negative pivots
 * of the LDL^T factorisation of T - mu I (Sylvester's law of inertia). */
static int orc_tridiag_count_below(const double* a, const double* b, int m, double mu)
{
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double off = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - mu) - ((i > 0) ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;       /* mu hit an eigenvalue of a leading block: count it as below */
        if (d < 0.0) ++c;
    }
    return c;
}

/* Largest eigenvalue of that tridiagonal matrix, by bisection between its
 * Gershgorin bounds. */
static double orc_tridiag_max_eig(const double* a, const double* b, int m)
{
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        const double rad = ((i > 0) ? fabs(b[i - 1]) : 0.0) + ((i < m - 1) ? fabs(b[i]) : 0.0);
        if (a[i] - rad < lo) lo = a[i] - rad;
        if (a[i] + rad > hi) hi = a[i] + rad;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-16 * (fabs(lo) + fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (orc_tridiag_count_below(a, b, m, mid) == m) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* The largest eigenvalue of the symmetric positive semi-definite normal
 * operator A^T A + lambda R (sensitivity b, NULL = 1), applied by
 * orc_normal_apply -- nothing about the operator's structure is used.  With
 * b = NULL and lambda = 0 it is ||A||_2^2; the paper's APG step is its
 * reciprocal (Sec. 4.3).  The Lanczos process (three-term recurrence, FP64)
 * starts from v0 (N values, not all zero); after each step the largest
 * eigenvalue of the Lanczos tridiagonal matrix (a lower bound that rises
 * towards the answer) is taken by bisection.  Stops once that value has
 * changed by at most rel_tol relative in three successive steps, when the
 * Krylov space is exhausted, or after max_iter steps.  *iters_out (may be
 * NULL) receives the number of steps. */
double orc_normal_lambda_max(int nx, int ny, int nz, int s, int r, int K,
                             const double* X, const double* Y, const double* Z, const double* theta,
                             const double* b, double lambda, int kind, double alpha, int shell,
                             const double* v0, double rel_tol, int max_iter, int* iters_out)
{
    const size_t N = (size_t)nx * ny * nz;
    double* q = (double*)malloc(N * sizeof(double));
    double* qp = (double*)calloc(N, sizeof(double));
    double* w = (double*)malloc(N * sizeof(double));
    double* al = (double*)malloc((size_t)(max_iter + 1) * sizeof(double));
    double* be = (double*)malloc((size_t)(max_iter + 1) * sizeof(double));
    double nv = 0.0;
    for (size_t i = 0; i < N; ++i) nv += v0[i] * v0[i];
    nv = sqrt(nv);
    for (size_t i = 0; i < N; ++i) q[i] = v0[i] / nv;
    double theta_max = 0.0, prev = 0.0;
    int stable = 0, m = 0;
    for (int j = 0; j < max_iter; ++j) {
        orc_normal_apply(nx, ny, nz, s, r, K, X, Y, Z, theta, b, lambda, kind, alpha, shell, q, w);
        double a = 0.0;
        for (size_t i = 0; i < N; ++i) a += q[i] * w[i];
        const double bprev = (j > 0) ? be[j - 1] : 0.0;
        double bn = 0.0;
        for (size_t i = 0; i < N; ++i) {
            w[i] -= a * q[i] + bprev * qp[i];
            bn += w[i] * w[i];
        }
        bn = sqrt(bn);
        al[j] = a;
        be[j] = bn;
        m = j + 1;
        theta_max = orc_tridiag_max_eig(al, be, m);
        if (j > 0 && fabs(theta_max - prev) <= rel_tol * fabs(theta_max)) {
            if (++stable >= 3) break;
        } else {
            stable = 0;
        }
        prev = theta_max;
        if (!(bn > 1e-300)) break;        /* invariant subspace: T_m holds the answer */
        for (size_t i = 0; i < N; ++i) {
            qp[i] = q[i];
            q[i] = w[i] / bn;
        }
    }
    if (iters_out) *iters_out = m;
    free(q); free(qp); free(w); free(al); free(be);
    return theta_max;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients on (A^T A + lambda R) rho = A^T d                    */
/* ------------------------------------------------------------------------ */

static double orc_dot(const double* a, const double* b, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Plain CG (Hestenes-Stiefel).  rhs = A^T d.  x holds x0 on entry (zeros for
 * a zero start) and the solution on exit.  Stops when
 * ||r_k|| <= rel_tol * ||A^T d|| (recurrence residual, zero-start
 * denominator), or after max_iter iterations; rel_tol <= 0 runs exactly
 * max_iter iterations.  history (may be NULL) receives ||r_k||/||A^T d|| for
 * k = 0..iters.  Returns the iteration count. */
int orc_cg(int nx, int ny, int nz, int s, int r, int K,
           const double* X, const double* Y, const double* Z, const double* theta,
           const double* b, double lambda, int kind, double alpha, int shell,
           const double* d, double rel_tol, int max_iter, double* x, double* history)
{
    const size_t N = (size_t)nx * ny * nz;
    double* rhs = (double*)malloc(N * sizeof(double));
    double* res = (double*)malloc(N * sizeof(double));
    double* p = (double*)malloc(N * sizeof(double));
    double* q = (double*)malloc(N * sizeof(double));
    orc_adjoint(nx, ny, nz, s, r, K, X, Y, Z, theta, b, d, rhs);
    const double bnorm = sqrt(orc_dot(rhs, rhs, N));
    orc_normal_apply(nx, ny, nz, s, r, K, X, Y, Z, theta, b, lambda, kind, alpha, shell, x, q);
    for (size_t i = 0; i < N; ++i) { res[i] = rhs[i] - q[i]; p[i] = res[i]; }
    double gam = orc_dot(res, res, N);
    if (history) history[0] = (bnorm > 0) ? sqrt(gam) / bnorm : 0.0;
    int it = 0;
    while (it < max_iter) {
        if (rel_tol > 0 && sqrt(gam) <= rel_tol * bnorm) break;
        orc_normal_apply(nx, ny, nz, s, r, K, X, Y, Z, theta, b, lambda, kind, alpha, shell, p, q);
        const double delta = orc_dot(p, q, N);
        const double a = gam / delta;
        for (size_t i = 0; i < N; ++i) { x[i] += a * p[i]; res[i] -= a * q[i]; }
        const double gnew = orc_dot(res, res, N);
        const double beta = gnew / gam;
        gam = gnew;
        for (size_t i = 0; i < N; ++i) p[i] = res[i] + beta * p[i];
        ++it;
        if (history) history[it] = (bnorm > 0) ? sqrt(gam) / bnorm : 0.0;
    }
    free(rhs); free(res); free(p); free(q);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Accelerated projected gradient (Sec. 4.3, the paper's solver)             */
/* ------------------------------------------------------------------------ */

/* y^k = rho^k + (k-1)/(k+2) (rho^k - rho^{k-1});
 * rho^{k+1} = max(y^k - tau M^*(M y^k - b), 0), with M^*(M y - b) =
 * (A^T A + lambda R) y - A^T d.  k starts at 1; rho^0 = rho^1 = x (input). */
void orc_apg(int nx, int ny, int nz, int s, int r, int K,
             const double* X, const double* Y, const double* Z, const double* theta,
             const double* b, double lambda, int kind, double alpha, int shell,
             const double* d, double tau, int iters, double* x)
{
    const size_t N = (size_t)nx * ny * nz;
    double* rhs = (double*)malloc(N * sizeof(double));
    double* prev = (double*)malloc(N * sizeof(double));
    double* yv = (double*)malloc(N * sizeof(double));
    double* g = (double*)malloc(N * sizeof(double));
    orc_adjoint(nx, ny, nz, s, r, K, X, Y, Z, theta, b, d, rhs);
    memcpy(prev, x, N * sizeof(double));
    for (int k = 1; k <= iters; ++k) {
        const double mom = (double)(k - 1) / (double)(k + 2);
        for (size_t i = 0; i < N; ++i) yv[i] = x[i] + mom * (x[i] - prev[i]);
        orc_normal_apply(nx, ny, nz, s, r, K, X, Y, Z, theta, b, lambda, kind, alpha, shell, yv, g);
        memcpy(prev, x, N * sizeof(double));
        for (size_t i = 0; i < N; ++i) {
            const double v = yv[i] - tau * (g[i] - rhs[i]);
            x[i] = v > 0.0 ? v : 0.0;
        }
    }
    free(rhs); free(prev); free(yv); free(g);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
