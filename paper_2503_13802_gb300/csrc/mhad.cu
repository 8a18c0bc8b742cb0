// MHAD native image (App. D, Eq. mhad2 / mhadM) and a warm start built on it.
//
// Along the drive axis of every portrait row (z, y), the closed form
//   rho_N = IDFT[ sum_k c_k^{-1} conj(F f^{k-1}) DFT(D_k) / (sum_k |F f^{k-1}|^2 + lambda) ]
// with D_k = Re(e^{-i theta_k} d_k), f the circular central difference of
// the portrait mesh ((f * u)[j] = u[j+1] - u[j-1]) and c_k = (gamma A)^k /
// (k-1)!, is one per-frequency filter per harmonic, applied to that
// harmonic's de-phased rows and summed over harmonics before one inverse
// transform.  That is the drive-axis adjoint pass with other tables: it
// transforms each harmonic's rows Re(e^{-i theta_k} y_k), multiplies bin by
// bin by conj(table_k), sums over k and runs one inverse DFT.  This file
// builds the MHAD tables (FP64, rounded once) and runs that pass; every
// arithmetic step is in the existing pencil kernels.
//
// Upsampled image: with table length nx and the table zero outside the
// portrait mesh's band (|w| < mx/2; the Nyquist bin split between +-mx/2),
// the same pass returns the band-limited interpolation of the image onto
// the model grid, portrait row i' landing on model row s i' + ds_offset.
//
// Warm start: u = upsampled image / b (b the sensitivity, where b > 0),
// x0 = alpha u with alpha = Re<A u, d> / ||A u||^2, the least-squares scale
// on the data, reduced on the device (compensated float pairs, FP64 totals).
#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "mh3d_internal.h"
#include "solve_internal.h"

namespace mh3d {
namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

constexpr int kDotBlocks = 1024;   // CTAs of the scale reduction

// W_k(m) = c_k^{-1} conj(Fhat(m)^{k-1}) / (sum_j |Fhat(m)^{j-1}|^2 + lambda),
// m in [0, mx), for the plan's harmonics k_min..k_max (Eq. mhadM).
std::vector<cd> mhad_filter(const Plan& P, double lambda)
{
    const int mx = P.mx, K = P.K;
    std::vector<cd> W((size_t)K * mx);
    std::vector<cd> pw(K);
    for (int m = 0; m < mx; ++m) {
        // DFT of f: -e^{-2 pi i m/mx} + e^{+2 pi i m/mx} = 2 i sin(2 pi m/mx)
        const cd fh(0.0, 2.0 * std::sin(2.0 * kPi * m / mx));
        double den = lambda;
        for (int j = 0; j < K; ++j) {
            pw[j] = std::pow(fh, P.kmin + j - 1);
            den += std::norm(pw[j]);
        }
        for (int j = 0; j < K; ++j) {
            const int k = P.kmin + j;
            double fact = 1.0;
            for (int i = 2; i < k; ++i) fact *= i;
            const double ck = std::pow(P.gammaA, k) / fact;
            W[(size_t)j * mx + m] = std::conj(pw[j]) / (ck * den);
        }
    }
    return W;
}

// Tables for the adjoint pass (which multiplies by the conjugate of the
// table and runs an unnormalised inverse DFT).
std::vector<float2> mhad_tables(const Plan& P, double lambda, int upsample)
{
    const int mx = P.mx, nx = P.nx, K = P.K, s = P.s, r = P.r;
    const std::vector<cd> W = mhad_filter(P, lambda);
    const int len = upsample ? nx : mx;
    std::vector<float2> t((size_t)K * len);
    for (int j = 0; j < K; ++j)
        for (int w = 0; w < len; ++w) {
            cd g = 0.0;
            if (!upsample) {
                g = W[(size_t)j * mx + w] / (double)mx;
            } else {
                const int ws = (2 * w <= nx) ? w : w - nx;   // signed bin of the model grid
                const int aw = ws < 0 ? -ws : ws;
                double wt = 0.0;
                if (2 * aw < mx) wt = 1.0;
                else if (2 * aw == mx) wt = (s == 1) ? 1.0 : 0.5;   // Nyquist of the portrait mesh
                if (wt != 0.0) {
                    const int m = ((ws % mx) + mx) % mx;
                    const double ph = -2.0 * kPi * (double)ws * r / nx;
                    g = wt * W[(size_t)j * mx + m] * cd(std::cos(ph), std::sin(ph)) / (double)mx;
                }
            }
            t[(size_t)j * len + w] = make_float2((float)g.real(), (float)-g.imag());
        }
    return t;
}

mh3d_status fail(Plan& P, const std::string& msg, mh3d_status s)
{
    P.err = msg;
    return s;
}

#define MHAD_CK(P, call)                                                                    \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((P), std::string(#call) + ": " + cudaGetErrorString(e_), MH3D_ERR_CUDA); \
    } while (0)

mh3d_status mhad_run(Plan& P, const float2* d, double lambda, int upsample, float* out, cudaStream_t st)
{
    if (P.padded) return fail(P, "mh3d_mhad: padded plans are not supported", MH3D_ERR_INVALID_ARG);
    if (!(lambda > 0.0) || !std::isfinite(lambda))
        return fail(P, "mh3d_mhad: lambda must be finite and > 0", MH3D_ERR_INVALID_ARG);
    if (!P.mhad_tab)
        MHAD_CK(P, dev_malloc(&P.mhad_tab, sizeof(float2) * (size_t)P.K * (P.nx > P.mx ? P.nx : P.mx)));
    if (P.mhad_lambda != lambda || P.mhad_up != upsample) {
        const std::vector<float2> t = mhad_tables(P, lambda, upsample);
        // pageable source: the copy is staged before the call returns; it is
        // ordered on `st` after every earlier use of the table on `st`
        MHAD_CK(P, cudaMemcpyAsync(P.mhad_tab, t.data(), sizeof(float2) * t.size(), cudaMemcpyHostToDevice, st));
        P.mhad_lambda = lambda;
        P.mhad_up = upsample;
    }
    XArgs a = xpass_args(P);
    a.Xhat = P.mhad_tab;
    a.din = d;
    a.vout = out;
    if (!upsample) {   // the image on the portrait mesh: a length-mx pass with s = 1
        a.nx = P.mx;
        a.s = 1;
        a.twx = P.am.tw;
        a.rpx = P.am.rp;
    }
    MHAD_CK(P, run_xadj(a, st));
    return MH3D_OK;
}

// u[i] /= b[i] where b[i] > 0, else 0.
__global__ void __launch_bounds__(256) k_mhad_unweight(float* __restrict__ u, const float* __restrict__ b, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float bb = b[i];
        u[i] = bb > 0.f ? u[i] / bb : 0.f;
    }
}

// Per-CTA partials of Re<a, d> and ||a||^2 over n complex values.
__global__ void __launch_bounds__(256) k_mhad_dots(const float2* __restrict__ a, const float2* __restrict__ d,
                                                   long long n, double* __restrict__ part)
{
    __shared__ double red[34];
    DotAcc ad, aa;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 x = a[i], y = d[i];
        ad.add(x.x, y.x);
        ad.add(x.y, y.y);
        aa.add(x.x, x.x);
        aa.add(x.y, x.y);
    }
    const double t1 = block_sum_acc(ad, red);
    const double t2 = block_sum_acc(aa, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = t1;
        part[2 * blockIdx.x + 1] = t2;
    }
}

// alpha = (sum of the first partials) / (sum of the second), 0 if the latter
// is 0; one CTA, a fixed summation order.
__global__ void __launch_bounds__(256) k_mhad_alpha(const double* __restrict__ part, int nb,
                                                    double* __restrict__ alpha)
{
    __shared__ double red[34];
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        s1 += part[2 * i];
        s2 += part[2 * i + 1];
    }
    const double t1 = block_sum_f64(s1, red);
    const double t2 = block_sum_f64(s2, red);
    if (threadIdx.x == 0) *alpha = t2 > 0.0 ? t1 / t2 : 0.0;
}

__global__ void __launch_bounds__(256) k_mhad_scale(float* __restrict__ x, long long N, const double* __restrict__ alpha)
{
    const float al = (float)*alpha;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        x[i] *= al;
}

}  // namespace

void mhad_free(Plan& P)
{
    if (P.mhad_tab) cudaFree(P.mhad_tab);
    if (P.mhad_scratch) cudaFree(P.mhad_scratch);
    if (P.mhad_red) cudaFree(P.mhad_red);
    P.mhad_tab = nullptr;
    P.mhad_scratch = nullptr;
    P.mhad_red = nullptr;
}

}  // namespace mh3d

using namespace mh3d;

struct mh3d_plan_s : public Plan {};

extern "C" {

mh3d_status mh3d_mhad(mh3d_plan P, const void* d, double lambda, int upsample, float* out, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d || !out) return fail(*P, "mh3d_mhad: null pointer", MH3D_ERR_INVALID_ARG);
    P->err.clear();
    return mhad_run(*P, (const float2*)d, lambda, upsample ? 1 : 0, out, (cudaStream_t)stream);
}

mh3d_status mh3d_mhad_warm_start(mh3d_plan P, const void* d, double lambda, float* x0, double* alpha_dev,
                                 void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d || !x0) return fail(*P, "mh3d_mhad_warm_start: null pointer", MH3D_ERR_INVALID_ARG);
    P->err.clear();
    const cudaStream_t st = (cudaStream_t)stream;
    mh3d_status s = mhad_run(*P, (const float2*)d, lambda, 1, x0, st);
    if (s != MH3D_OK) return s;
    const long long KM = (long long)P->K * P->M;
    if (!P->mhad_scratch) MHAD_CK(*P, dev_malloc(&P->mhad_scratch, sizeof(float2) * (size_t)KM));
    if (!P->mhad_red) MHAD_CK(*P, dev_malloc(&P->mhad_red, sizeof(double) * (2 * kDotBlocks + 1)));
    const int nU = (int)std::min<long long>((P->N + 255) / 256, 4096);
    if (P->sens) {
        k_mhad_unweight<<<nU, 256, 0, st>>>(x0, P->sens, P->N);
        MHAD_CK(*P, cudaGetLastError());
    }
    MHAD_CK(*P, launch_forward(*P, x0, P->mhad_scratch, P->w.t1, P->w.t2, st));
    k_mhad_dots<<<kDotBlocks, 256, 0, st>>>(P->mhad_scratch, (const float2*)d, KM, P->mhad_red);
    MHAD_CK(*P, cudaGetLastError());
    double* alpha = alpha_dev ? alpha_dev : P->mhad_red + 2 * kDotBlocks;
    k_mhad_alpha<<<1, 256, 0, st>>>(P->mhad_red, kDotBlocks, alpha);
    MHAD_CK(*P, cudaGetLastError());
    k_mhad_scale<<<nU, 256, 0, st>>>(x0, P->N, alpha);
    MHAD_CK(*P, cudaGetLastError());
    return MH3D_OK;
}

}  // extern "C"
