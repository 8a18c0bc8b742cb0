// Host-side construction of the harmonic PSF spectra, in FP64.
//
// The drive-axis PSF of harmonic k is c_k L^(k)(gamma x) with L the Langevin
// function and c_k = (gamma A)^k / (k-1)! (Sec. 3.3, Eq. hkapprox; Theorem 1).
// Across the drive axis the PSF is phi(t) = 3 L'(gamma_t t) on each
// transverse axis (separable reading of the 3D PSF; gamma_t = ratio * gamma).
// Samples sit at minimal-image offsets of the periodic grid.  The operator
// applies circular convolutions through their DFTs (Table ops), so the plan
// stores the DFT of every sampled 1D kernel, computed here by a direct
// O(n^2) sum with exactly reduced angles, then rounded once to FP32.
#include "mh3d_internal.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

namespace mh3d {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

// Sum over the poles of coth at i n pi (Mittag-Leffler):
//   L^(k)(x) = sum_{n>=1} 2 Re[(-1)^k k! (x - i n pi)^{-(k+1)}],
// the first NP terms explicitly and the rest by the Euler-Maclaurin midpoint
// form  sum_{n>NP} g(n) = int_a^inf g(t) dt - g'(a)/24 + O(g'''(a)),
// a = NP + 1/2, with
//   int_a^inf (x - i pi t)^{-(k+1)} dt = i (x - i pi a)^{-k} / (k pi)   (k >= 1),
//   d/dt (x - i pi t)^{-(k+1)} = i pi (k+1) (x - i pi t)^{-(k+2)}.
// For k = 0 the real part of the integrand is 2x/(x^2 + pi^2 t^2), whose
// tail integral is (2/pi) atan(x / (pi a)).
double langevin_pole_sum(int k, double x)
{
    const int NP = 1500;
    const double kf = factorial(k);
    const double sgn = (k & 1) ? -1.0 : 1.0;
    double acc = 0.0;
    for (int n = NP; n >= 1; --n) {
        const double re = x, im = -kPi * n;
        const double mod = std::hypot(re, im);
        const double ang = std::atan2(im, re);
        acc += 2.0 * sgn * kf * std::cos(-(k + 1) * ang) * std::pow(mod, -(double)(k + 1));
    }
    const double a = NP + 0.5;
    double tail;
    if (k == 0) {
        tail = (2.0 / kPi) * std::atan(x / (kPi * a));
    } else {
        // 2 Re[(-1)^k k! * i (x - i pi a)^{-k} / (k pi)]
        const double mod = std::hypot(x, -kPi * a);
        const double ang = std::atan2(-kPi * a, x);
        const double pr = std::pow(mod, -(double)k);
        const double c = std::cos(-k * ang) * pr, s = std::sin(-k * ang) * pr;  // (x - i pi a)^{-k}
        // i * (c + i s) = -s + i c  -> real part -s
        tail = 2.0 * sgn * kf * (-s) / (k * kPi);
    }
    {   // - g'(a) / 24 with g'(a) = 2 Re[(-1)^k k! i pi (k+1) (x - i pi a)^{-(k+2)}]
        const double mod = std::hypot(x, -kPi * a);
        const double ang = std::atan2(-kPi * a, x);
        const double pr = std::pow(mod, -(double)(k + 2));
        const double s = std::sin(-(k + 2) * ang) * pr;   // Im (x - i pi a)^{-(k+2)}
        const double gp = 2.0 * sgn * kf * kPi * (k + 1) * (-s);
        tail -= gp / 24.0;
    }
    return acc + tail;
}

// For |x| >= 12 the exponential expansion coth x = 1 + 2 sum_m e^{-2 m x} is
// short: L^(k)(x) = 2 sum_m (-2m)^k e^{-2mx} (+1 when k = 0) - (-1)^k k!/x^{k+1}
// for x > 0, and L^(k)(-x) = (-1)^{k+1} L^(k)(x).
double langevin_far(int k, double x)
{
    const double ax = std::fabs(x);
    double e = (k == 0) ? 1.0 : 0.0;
    for (int m = 1; m <= 60; ++m) e += 2.0 * std::pow(-2.0 * m, k) * std::exp(-2.0 * m * ax);
    const double v = e - ((k & 1) ? -1.0 : 1.0) * factorial(k) / std::pow(ax, k + 1);
    return (x < 0) ? ((k & 1) ? v : -v) : v;
}

}  // namespace

double langevin_deriv_host(int k, double x)
{
    if (std::fabs(x) >= 12.0) return langevin_far(k, x);
    return langevin_pole_sum(k, x);
}

static int min_image(int i, int n) { return (2 * i < n) ? i : i - n; }

// DFT of a real kernel sampled on a periodic axis: H[w] = sum_i h[i] e^{-2 pi i w i / n}.
static void dft_real(const std::vector<double>& h, std::vector<cplx>& H)
{
    const int n = (int)h.size();
    H.assign(n, cplx(0, 0));
    for (int w = 0; w < n; ++w) {
        double re = 0, im = 0;
        for (int i = 0; i < n; ++i) {
            const long m = ((long)w * i) % n;
            const double ang = -2.0 * kPi * (double)m / (double)n;
            re += h[i] * std::cos(ang);
            im += h[i] * std::sin(ang);
        }
        H[w] = cplx(re, im);
    }
}

// Drive-axis samples of c_k L^(k)(gamma o dx), shifted by the row offset r:
// X'_k[o] = X_k[o + r], so that portrait row i' = model row s i' + r.
static std::vector<double> drive_samples(int n, double dx, int k, double gamma, double gammaA, int r)
{
    std::vector<double> v(n);
    const double ck = std::pow(gammaA, k) / factorial(k - 1);
    for (int i = 0; i < n; ++i) {
        const int j = (i + r) % n;
        v[i] = ck * langevin_deriv_host(k, gamma * min_image(j, n) * dx);
    }
    return v;
}

static std::vector<double> transverse_samples(int n, double d, double gt)
{
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) v[i] = 3.0 * langevin_deriv_host(1, gt * min_image(i, n) * d);
    return v;
}

// Process-wide cache of FP64 spectra keyed by every parameter they depend on
// (batched plans share size classes).
namespace {
std::mutex g_cache_mu;
std::map<std::tuple<int, double, int, double, double, int>, std::vector<cplx>> g_drive_cache;
std::map<std::tuple<int, double, double>, std::vector<cplx>> g_trans_cache;
}  // namespace

std::vector<cplx> drive_spectrum(int n, double dx, int k, double gamma, double gammaA, int r)
{
    auto key = std::make_tuple(n, dx, k, gamma, gammaA, r);
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_drive_cache.find(key);
        if (it != g_drive_cache.end()) return it->second;
    }
    std::vector<cplx> H;
    dft_real(drive_samples(n, dx, k, gamma, gammaA, r), H);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_drive_cache[key] = H;
    return H;
}

std::vector<cplx> transverse_spectrum(int n, double d, double gt)
{
    auto key = std::make_tuple(n, d, gt);
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_trans_cache.find(key);
        if (it != g_trans_cache.end()) return it->second;
    }
    std::vector<cplx> H;
    dft_real(transverse_samples(n, d, gt), H);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_trans_cache[key] = H;
    return H;
}

// Largest eigenvalue of a small Hermitian positive semidefinite matrix
// (row-major s x s) by the cyclic Jacobi method on its real 2s x 2s
// symmetric embedding [[Re, -Im], [Im, Re]] (each eigenvalue appears twice).
double hermitian_lambda_max(const std::vector<cplx>& H, int s)
{
    if (s == 1) return H[0].real();
    const int n = 2 * s;
    std::vector<double> a((size_t)n * n);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) {
            const cplx h = H[(size_t)i * s + j];
            a[(size_t)i * n + j] = h.real();
            a[(size_t)i * n + j + s] = -h.imag();
            a[(size_t)(i + s) * n + j] = h.imag();
            a[(size_t)(i + s) * n + j + s] = h.real();
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {   // rotate columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - sn * akq;
                    a[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rotate rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - sn * aqk;
                    a[(size_t)q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    double mx = a[0];
    for (int i = 1; i < n; ++i) mx = std::max(mx, a[(size_t)i * n + i]);
    return mx;
}

// Twiddles W_n^t = e^{-2 pi i t / n}, t = 0..n-1, from exactly reduced angles.
std::vector<cplx> twiddles(int n)
{
    std::vector<cplx> w(n);
    for (int t = 0; t < n; ++t) {
        const double ang = -2.0 * kPi * (double)t / (double)n;
        w[t] = cplx(std::cos(ang), std::sin(ang));
    }
    return w;
}

// Radix schedule for a length: factors 8, 4, 2, 3 only.  The default puts
// large radices first; the autotuner may pick another permutation.
bool radix_plan(int n, RadixPlan& pl, int variant)
{
    pl.n = n;
    pl.nst = 0;
    int m = n, p2 = 0, p3 = 0;
    while (m % 2 == 0) { m /= 2; ++p2; }
    while (m % 3 == 0) { m /= 3; ++p3; }
    if (m != 1 || n < 1 || n > kMaxLen) return false;
    int rs[kMaxStages];
    int ns = 0;
    // variant 0: 8s first; variant 1: 4s (then a trailing 8/2); variant 2: 8s last.
    int e = p2;
    if (variant == 1) {
        while (e >= 2 && ns < kMaxStages) { rs[ns++] = 4; e -= 2; }
        if (e == 1) rs[ns++] = 2;
    } else {
        while (e >= 3 && ns < kMaxStages) { rs[ns++] = 8; e -= 3; }
        if (e == 2) rs[ns++] = 4;
        if (e == 1) rs[ns++] = 2;
        if (variant == 2) {   // reverse the power-of-two part
            for (int i = 0; i < ns / 2; ++i) { int t = rs[i]; rs[i] = rs[ns - 1 - i]; rs[ns - 1 - i] = t; }
        }
    }
    for (int i = 0; i < p3; ++i) {
        if (ns >= kMaxStages) return false;
        rs[ns++] = 3;
    }
    pl.nst = ns;
    for (int i = 0; i < ns; ++i) pl.radix[i] = rs[i];
    for (int i = ns; i < kMaxStages; ++i) pl.radix[i] = 1;
    return true;
}

}  // namespace mh3d
