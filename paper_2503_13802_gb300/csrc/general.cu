// The general MH3D model on the GPU: the three-component convolution model
// d_k = e^{i theta_k} S_s( sum_j h_kj * (b_j rho) )  (Sec. 3.2, Eq. MH3Dcont,
// Eq. matrixModel), with PSFs that need not be separable -- the harmonic
// PSFs of the tensor PSF (appendix, Eq. PSF, Eq. skMD) or simulated ones.
// The caller supplies the PSF samples (h_k)_j at the grid's minimal-image
// offsets; the plan keeps their spectra, DFT(h)/N, as K * 3 complex volumes.
//
// Forward: the weighted volumes b_j rho go through complex pencil passes
// along x, y and z (the Stockham engine of fft_smem.cuh, no spectral step);
// one pointwise kernel forms every harmonic's portrait-grid spectrum
//   D_k(w') = sum_{a < s} e^{2 pi i (w' + a m_x) r / n_x} sum_j H_kj W_j (w' + a m_x)
// (the row selector x = s i' + r is exactly this alias sum with the offset
// phase) in the output buffer, and inverse passes along x (length m_x), y and
// z over all K portraits return c_k[z][y][s i' + r]; d_k = e^{i theta_k} Re c
// in place.  Adjoint: the real parts Re(e^{-i theta_k} d_k) of every
// harmonic are inserted at x = s i' + r into K volumes, the K volumes are
// transformed together, V_j = sum_k conj(H_kj) E_k, and the inverse passes
// and sum_j b_j Re V_j finish.  Each pass covers every harmonic (or
// component) in one launch: 9 launches a call, whatever K.  Unnormalised
// transforms throughout; the 1/N sits in the stored spectra.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "fft_smem.cuh"
#include "mh3d_internal.h"

namespace mh3d {
namespace {

constexpr int kGP = 8;      // pencils per CTA
constexpr int kGT = 128;    // threads per CTA
constexpr int kGB = 256;    // threads per CTA of the pointwise kernels

// Pencils of `vols` complex volumes [nz][ny][W] (x fastest), vstride
// float2 apart: axis 0 walks x (pencil p = row z ny + y), 1 walks y
// (p = z W + x), 2 walks z (p = y W + x); pencil p of the whole set is
// pencil p % per_vol() of volume p / per_vol().
struct Pencils {
    int axis, W, ny, nz;
    int vols = 1;
    long long vstride = 0;
    __host__ __device__ long long per_vol() const
    {
        return axis == 0 ? (long long)ny * nz : (axis == 1 ? (long long)W * nz : (long long)W * ny);
    }
    __host__ __device__ long long count() const { return per_vol() * vols; }
    __device__ __forceinline__ long long base(long long pg) const
    {
        const long long pv = per_vol(), c = pg / pv, p = pg - c * pv;
        if (axis == 0) return c * vstride + p * W;
        const long long x = p % W, q = p / W;
        return c * vstride + (axis == 1 ? q * ny * W + x : q * W + x);
    }
    __device__ __forceinline__ long long stride() const
    {
        return axis == 0 ? 1 : (axis == 1 ? (long long)W : (long long)W * ny);
    }
};

// Element e of the CTA's pencil p: base[p] + e * stride (base < 0: a pencil
// past the end, read as zero and not written).  The bases are computed once
// per CTA, so the per-element address is one multiply-add.
struct GenLd {
    const float2* v;
    const long long* base;
    long long stride;
    __device__ __forceinline__ float2 operator()(int e, int p) const
    {
        const long long b = base[p];
        return b < 0 ? make_float2(0.f, 0.f) : v[b + e * stride];
    }
};
struct GenSt {
    float2* v;
    const long long* base;
    long long stride;
    __device__ __forceinline__ void operator()(int e, int p, float2 x) const
    {
        const long long b = base[p];
        if (b >= 0) v[b + e * stride] = x;
    }
};

// One transform along an axis, in place: every CTA owns kGP whole pencils;
// the first stage reads all of them before the last stage writes.  PF: the
// first and last stages walk pencils fastest (axes y and z, where the kGP
// pencils are neighbours in memory); along x they walk elements fastest.
template <bool INV, bool PF>
__global__ void __launch_bounds__(kGT) k_gen_line(float2* v, Pencils g, RadixPlan pl, const float2* __restrict__ tw)
{
    extern __shared__ float2 gsm[];
    __shared__ long long sbase[kGP];
    float2* s0 = gsm;
    float2* s1 = gsm + (size_t)pl.n * kGP;
    const long long p0 = (long long)blockIdx.x * kGP, np = g.count();
    if (threadIdx.x < kGP) sbase[threadIdx.x] = p0 + threadIdx.x < np ? g.base(p0 + threadIdx.x) : -1;
    __syncthreads();
    const long long sd = g.stride();
    fft_run<INV, PF, PF>(pl, GenLd{v, sbase, sd}, GenSt{v, sbase, sd}, s0, s1, kGP, kGP, tw);
}

__global__ void k_gen_spectra_in(const float* __restrict__ h, float2* __restrict__ H, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        H[i] = make_float2(h[i], 0.f);
}

__global__ void k_gen_scale(float2* __restrict__ H, long long n, float sc)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = H[i];
        H[i] = make_float2(v.x * sc, v.y * sc);
    }
}

// W_j = b_j rho (b = (1, 0, 0) when bvec is null: one component)
__global__ void k_gen_weight(const float* __restrict__ rho, const float* __restrict__ bvec, float2* __restrict__ W,
                             long long N, int nc)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N * nc;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v = i % N;
        const float b = bvec ? bvec[i] : 1.f;
        W[i] = make_float2(b * rho[v], 0.f);
    }
}

// Portrait-grid spectra of every harmonic: D[k][q], q over [nz][ny][mx]:
// D_k(w) = sum_a e^{2 pi i f r / nx} sum_j H_kj(f) W_j(f), f = w + a mx (the
// row selector x = s i' + r as an alias sum).
__global__ void k_gen_fold(const float2* __restrict__ H, const float2* __restrict__ W, float2* __restrict__ D,
                           int nx, int ny, int nz, int mx, int s, int r, int nc, int K, long long N,
                           const float2* __restrict__ twx)
{
    const long long Q = (long long)nz * ny * mx;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < Q * K;
         g += (long long)gridDim.x * blockDim.x) {
        const long long k = g / Q, q = g - k * Q;
        const float2* __restrict__ Hk = H + k * 3 * N;
        const int w = (int)(q % mx);
        const long long row = q / mx;   // z ny + y
        float2 acc = make_float2(0.f, 0.f);
        for (int a = 0; a < s; ++a) {
            const int f = w + a * mx;
            const long long i = row * nx + f;
            float2 t = make_float2(0.f, 0.f);
            for (int j = 0; j < nc; ++j) t = c_add(t, c_mul(Hk[(long long)j * N + i], W[(long long)j * N + i]));
            // e^{+2 pi i f r / nx} = conj(W_nx^{f r mod nx})
            const float2 tw = twx[(int)(((long long)f * r) % nx)];
            acc = c_add(acc, c_mul(t, make_float2(tw.x, -tw.y)));
        }
        D[g] = acc;
    }
}

// d_k = e^{i theta_k} Re(D_k) for every harmonic (ph[k] = e^{i theta_k})
__global__ void k_gen_phase(const float2* D, float2* d, long long Q, int K,
                            const float2* __restrict__ ph)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < Q * K; g += (long long)gridDim.x * blockDim.x) {
        const float2 p = ph[g / Q];
        const float c = D[g].x;
        d[g] = make_float2(p.x * c, p.y * c);
    }
}

// E_k = Re(e^{-i theta_k} d_k) at x = s i' + r, zero elsewhere, every harmonic
__global__ void k_gen_insert(const float2* __restrict__ d, float2* __restrict__ E, int nx, int mx, int s, int r,
                             long long N, long long Q, int K, const float2* __restrict__ ph)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N * K; g += (long long)gridDim.x * blockDim.x) {
        const long long k = g / N, i = g - k * N;
        const int x = (int)(i % nx);
        const long long row = i / nx;
        float v = 0.f;
        if (x >= r && (x - r) % s == 0) {
            const float2 dv = d[k * Q + row * mx + (x - r) / s];
            const float2 p = ph[k];
            v = p.x * dv.x + p.y * dv.y;
        }
        E[g] = make_float2(v, 0.f);
    }
}

// V_j = sum_k conj(H_kj) E_k
__global__ void k_gen_acc(const float2* __restrict__ H, const float2* __restrict__ E, float2* __restrict__ V,
                          long long N, int nc, int K)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N * nc;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / N, v = i - j * N;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < K; ++k) {
            const float2 h = H[((long long)k * 3 + j) * N + v];
            acc = c_add(acc, c_mul(make_float2(h.x, -h.y), E[(long long)k * N + v]));
        }
        V[i] = acc;
    }
}

// out = sum_j b_j Re V_j
__global__ void k_gen_out(const float2* __restrict__ V, const float* __restrict__ bvec, float* __restrict__ out,
                          long long N, int nc)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int j = 0; j < nc; ++j) acc = fmaf(bvec ? bvec[(long long)j * N + i] : 1.f, V[(long long)j * N + i].x, acc);
        out[i] = acc;
    }
}

int gen_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kGB - 1) / kGB, 8192)); }

mh3d_status gen_fail(Plan& P, const std::string& msg, mh3d_status s)
{
    P.err = msg;
    return s;
}

#define GEN_CK(P, call)                                                                                 \
    do {                                                                                                \
        const cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return gen_fail((P), std::string(#call) + ": " + cudaGetErrorString(e_), \
                                               MH3D_ERR_CUDA);                                         \
    } while (0)

// The pencil kernels' dynamic shared-memory limit, raised once per device
// (the attribute belongs to the current device) to what the longest
// supported axis needs; the status is checked where it is set.
constexpr int kGenMaxDevices = 64;
std::mutex g_gen_attr_mu;
bool g_gen_attr_done[kGenMaxDevices] = {};

cudaError_t gen_set_attributes()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kGenMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_gen_attr_mu);
    if (g_gen_attr_done[dev]) return cudaSuccess;
    const int smem = (int)(sizeof(float2) * 2 * (size_t)kMaxLen * kGP);
    e = cudaFuncSetAttribute(k_gen_line<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gen_line<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gen_line<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gen_line<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) g_gen_attr_done[dev] = true;
    return e;
}

// In-place transform of every pencil of `vols` volumes (rows of width W,
// vstride float2 apart) along `axis`.
cudaError_t gen_line(float2* v, int axis, int W, int ny, int nz, int vols, long long vstride, const AxisPlan& ap,
                     bool inv, cudaStream_t st)
{
    Pencils g{axis, W, ny, nz};
    g.vols = vols;
    g.vstride = vstride;
    const long long np = g.count();
    const size_t smem = sizeof(float2) * 2 * (size_t)ap.n * kGP;
    const int grid = (int)((np + kGP - 1) / kGP);
    const bool pf = axis != 0;
    if (inv && pf) k_gen_line<true, true><<<grid, kGT, smem, st>>>(v, g, ap.rp, ap.tw);
    else if (inv) k_gen_line<true, false><<<grid, kGT, smem, st>>>(v, g, ap.rp, ap.tw);
    else if (pf) k_gen_line<false, true><<<grid, kGT, smem, st>>>(v, g, ap.rp, ap.tw);
    else k_gen_line<false, false><<<grid, kGT, smem, st>>>(v, g, ap.rp, ap.tw);
    return cudaGetLastError();
}

// 3D transform of `count` consecutive volumes [nz][ny][W], W = the x length
// of `axp`: three launches, each over every volume's pencils.
cudaError_t gen_fft3(const Plan& P, float2* v, int count, const AxisPlan& axp, bool inv, cudaStream_t st)
{
    const long long vol = (long long)axp.n * P.ny * P.nz;
    cudaError_t e;
    if ((e = gen_line(v, 0, axp.n, P.ny, P.nz, count, vol, axp, inv, st)) != cudaSuccess) return e;
    if ((e = gen_line(v, 1, axp.n, P.ny, P.nz, count, vol, P.ay, inv, st)) != cudaSuccess) return e;
    return gen_line(v, 2, axp.n, P.ny, P.nz, count, vol, P.az, inv, st);
}

mh3d_status gen_check(Plan& P, const char* who)
{
    const cudaError_t ea = gen_set_attributes();
    if (ea != cudaSuccess)
        return gen_fail(P, std::string(who) + ": kernel attributes: " + cudaGetErrorString(ea), MH3D_ERR_CUDA);
    if (P.padded) return gen_fail(P, std::string(who) + ": padded plans are not supported", MH3D_ERR_INVALID_ARG);
    if (!P.gen_H) return gen_fail(P, std::string(who) + ": no PSF spectra (call mh3d_general_set_psf)",
                                  MH3D_ERR_INVALID_ARG);
    return MH3D_OK;
}

}  // namespace

void general_free(Plan& P)
{
    if (P.gen_H) cudaFree(P.gen_H);
    if (P.gen_work) cudaFree(P.gen_work);
    P.gen_H = nullptr;
    P.gen_work = nullptr;
}

}  // namespace mh3d

using namespace mh3d;

struct mh3d_plan_s : public Plan {};

extern "C" {

mh3d_status mh3d_general_set_psf(mh3d_plan Pp, const float* h_host)
{
    if (!Pp) return MH3D_ERR_INVALID_ARG;
    Plan& P = *Pp;
    if (!h_host) return gen_fail(P, "mh3d_general_set_psf: null pointer", MH3D_ERR_INVALID_ARG);
    if (P.padded) return gen_fail(P, "mh3d_general_set_psf: padded plans are not supported", MH3D_ERR_INVALID_ARG);
    P.err.clear();
    GEN_CK(P, gen_set_attributes());
    const long long N = P.N, n3 = 3LL * P.K * N;
    if (!P.gen_H) GEN_CK(P, dev_malloc(&P.gen_H, sizeof(float2) * (size_t)n3));
    // work area: 3 component volumes + one inserted volume per harmonic
    if (!P.gen_work) GEN_CK(P, dev_malloc(&P.gen_work, sizeof(float2) * (size_t)((3 + P.K) * N)));
    // the real samples are staged in the work area (>= 4N float2 >= 3N floats per harmonic)
    float* stage = reinterpret_cast<float*>(P.gen_work);
    const cudaStream_t st = 0;
    for (int k = 0; k < P.K; ++k) {
        float2* Hk = P.gen_H + (long long)k * 3 * N;
        GEN_CK(P, cudaMemcpy(stage, h_host + (long long)k * 3 * N, sizeof(float) * (size_t)(3 * N),
                             cudaMemcpyHostToDevice));
        k_gen_spectra_in<<<gen_blocks(3 * N), kGB, 0, st>>>(stage, Hk, 3 * N);
        GEN_CK(P, cudaGetLastError());
        GEN_CK(P, cudaStreamSynchronize(st));   // the stage is reused by the next harmonic
        GEN_CK(P, gen_fft3(P, Hk, 3, P.ax, false, st));
    }
    k_gen_scale<<<gen_blocks(n3), kGB, 0, st>>>(P.gen_H, n3, (float)(1.0 / (double)N));
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, cudaStreamSynchronize(st));
    return MH3D_OK;
}

mh3d_status mh3d_general_forward(mh3d_plan Pp, const float* rho, const float* bvec, void* d, void* stream)
{
    if (!Pp) return MH3D_ERR_INVALID_ARG;
    Plan& P = *Pp;
    if (!rho || !d) return gen_fail(P, "mh3d_general_forward: null pointer", MH3D_ERR_INVALID_ARG);
    mh3d_status s = gen_check(P, "mh3d_general_forward");
    if (s != MH3D_OK) return s;
    P.err.clear();
    const cudaStream_t st = (cudaStream_t)stream;
    const long long N = P.N, Q = (long long)P.nz * P.ny * P.mx;
    const int nc = bvec ? 3 : 1;
    float2* W = P.gen_work;   // nc volumes
    float2* D = (float2*)d;   // the portrait-grid spectra, transformed and phased in place
    k_gen_weight<<<gen_blocks(N * nc), kGB, 0, st>>>(rho, bvec, W, N, nc);
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, gen_fft3(P, W, nc, P.ax, false, st));
    k_gen_fold<<<gen_blocks(Q * P.K), kGB, 0, st>>>(P.gen_H, W, D, P.nx, P.ny, P.nz, P.mx, P.s, P.r, nc, P.K, N,
                                                    P.ax.tw);
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, gen_fft3(P, D, P.K, P.am, true, st));
    k_gen_phase<<<gen_blocks(Q * P.K), kGB, 0, st>>>(D, D, Q, P.K, P.phase);
    GEN_CK(P, cudaGetLastError());
    return MH3D_OK;
}

mh3d_status mh3d_general_adjoint(mh3d_plan Pp, const void* d, const float* bvec, float* out, void* stream)
{
    if (!Pp) return MH3D_ERR_INVALID_ARG;
    Plan& P = *Pp;
    if (!d || !out) return gen_fail(P, "mh3d_general_adjoint: null pointer", MH3D_ERR_INVALID_ARG);
    mh3d_status s = gen_check(P, "mh3d_general_adjoint");
    if (s != MH3D_OK) return s;
    P.err.clear();
    const cudaStream_t st = (cudaStream_t)stream;
    const long long N = P.N, Q = (long long)P.nz * P.ny * P.mx;
    const int nc = bvec ? 3 : 1;
    float2* V = P.gen_work;          // nc accumulators
    float2* E = P.gen_work + 3 * N;  // the harmonics' inserted volumes
    k_gen_insert<<<gen_blocks(N * P.K), kGB, 0, st>>>((const float2*)d, E, P.nx, P.mx, P.s, P.r, N, Q, P.K, P.phase);
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, gen_fft3(P, E, P.K, P.ax, false, st));
    k_gen_acc<<<gen_blocks(N * nc), kGB, 0, st>>>(P.gen_H, E, V, N, nc, P.K);
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, gen_fft3(P, V, nc, P.ax, true, st));
    k_gen_out<<<gen_blocks(N), kGB, 0, st>>>(V, bvec, out, N, nc);
    GEN_CK(P, cudaGetLastError());
    return MH3D_OK;
}

}  // extern "C"
