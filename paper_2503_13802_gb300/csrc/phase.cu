// Portrait phase calibration (Sec. 4.4): theta_k of portraits measured as
// e^{i theta_k} times a real field.
//
//  * theta_k modulo pi: 1/2 arg sum d_k^2 over the high-SNR samples
//    (|d_k| >= frac max |d_k|): the samples are +-|d| e^{i theta}, so their
//    squares all point along 2 theta.
//  * the remaining pi, when the portraits are not downsampled (s = 1): the
//    single-harmonic back-projections B_k = A_k^T Re(e^{-i theta_k} d_k)
//    correlate positively for the true signs (along the drive axis <B_j,
//    B_k> sums |X_j|^2 |X_k|^2 |U|^2 over the frequencies), which fixes
//    every sign relative to the harmonic with the largest ||B_k||; the
//    common sign is the one whose short CG reconstruction (30 iterations,
//    lambda = 1e-2 relative) is positively skewed (sum x^3 > 0), as the
//    image of a sparse non-negative density is.
//  * with s > 1 the row selector's aliases break the correlation argument,
//    and theta_k stays modulo pi (reported).
//
// The sums run in FP64 (per-CTA partials, added on the host in a fixed
// order); back-projections and the reconstruction use the library's adjoint
// and solver.  The call is a calibration step: it allocates its scratch,
// synchronises and frees it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mh3d_internal.h"

namespace mh3d {
namespace {

constexpr int kPhBlocks = 128;   // CTAs per harmonic for the sums
constexpr double kPi = 3.14159265358979323846;

// per harmonic (blockIdx.y): max |d| as float bits (non-negative floats
// order like their bit patterns, so the atomic max is exact)
__global__ void __launch_bounds__(256) k_phase_max(const float2* __restrict__ d, long long M, unsigned* maxbits)
{
    const float2* dk = d + (long long)blockIdx.y * M;
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = dk[i];
        m = fmaxf(m, sqrtf(v.x * v.x + v.y * v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits + blockIdx.y, __float_as_uint(m));
}

// per harmonic (blockIdx.y) over the samples with |d| >= thr[k]: sum d^2
// (re, im) as per-CTA partials part[(k * gridDim.x + block) * 2 + {0, 1}]
__global__ void __launch_bounds__(256) k_phase_sums(const float2* __restrict__ d, long long M, const float* thr,
                                                    double* part)
{
    __shared__ double red[2][8];
    const int k = blockIdx.y;
    const float2* dk = d + (long long)k * M;
    const float t = thr[k];
    double a0 = 0.0, a1 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = dk[i];
        if (sqrtf(v.x * v.x + v.y * v.y) < t) continue;
        const double x = v.x, y = v.y;
        a0 += x * x - y * y;
        a1 += 2.0 * x * y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = a0;
        red[1][w] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
        }
        part[((long long)k * gridDim.x + blockIdx.x) * 2] = s0;
        part[((long long)k * gridDim.x + blockIdx.x) * 2 + 1] = s1;
    }
}

// y_k = f_k d_k (f_k = 0 leaves harmonic k out)
__global__ void __launch_bounds__(256) k_phase_rotate(const float2* __restrict__ d, float2* __restrict__ y, long long M,
                                                      int K, const float2* f)
{
    const long long n = (long long)K * M;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 a = f[i / M], v = d[i];
        y[i] = make_float2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
    }
}

// per-CTA partials of sum a b (b = nullptr: sum a^3)
__global__ void __launch_bounds__(256) k_phase_dot(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                                   double* part)
{
    __shared__ double red[8];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = a[i];
        acc += b ? v * (double)b[i] : v * v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        part[blockIdx.x] = s;
    }
}

// Device scratch of one call, freed when the call returns (cudaFree waits
// for the work that uses it).
struct Scratch {
    std::vector<void*> p;
    ~Scratch()
    {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    cudaError_t get(T** out, size_t bytes)
    {
        void* q = nullptr;
        cudaError_t e = dev_malloc(&q, bytes);
        if (e == cudaSuccess) p.push_back(q);
        *out = static_cast<T*>(q);
        return e;
    }
};

}  // namespace
}  // namespace mh3d

using namespace mh3d;

struct mh3d_plan_s : public Plan {};

#define PH_CK(call)                                                                 \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            P->err = std::string("mh3d_estimate_phase: ") + #call + ": " + cudaGetErrorString(e_); \
            return e_ == cudaErrorMemoryAllocation ? MH3D_ERR_OOM : MH3D_ERR_CUDA;  \
        }                                                                           \
    } while (0)

extern "C" {

mh3d_status mh3d_estimate_phase(mh3d_plan P, const void* d_dev, double frac, double* theta_out, int* resolved_out,
                                void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d_dev || !theta_out || !(frac > 0.0 && frac <= 1.0)) {
        P->err = "mh3d_estimate_phase: null pointer, or frac outside (0, 1]";
        return MH3D_ERR_INVALID_ARG;
    }
    P->err.clear();
    const cudaStream_t st = (cudaStream_t)stream;
    const int K = P->K;
    const long long Mf = P->Mf;   // samples per harmonic of the caller's portraits
    const float2* d = (const float2*)d_dev;
    Scratch S;
    unsigned* maxbits = nullptr;
    float* thr = nullptr;
    double* part = nullptr;
    PH_CK(S.get(&maxbits, sizeof(unsigned) * K));
    PH_CK(S.get(&thr, sizeof(float) * K));
    PH_CK(S.get(&part, sizeof(double) * 2 * (size_t)K * kPhBlocks));
    std::vector<double> hpart(2 * (size_t)K * kPhBlocks);
    auto sum_parts = [&](int k, int c) {
        double s = 0.0;
        for (int b = 0; b < kPhBlocks; ++b) s += hpart[((size_t)k * kPhBlocks + b) * 2 + c];
        return s;
    };

    // 1. the high-SNR threshold of every harmonic
    PH_CK(cudaMemsetAsync(maxbits, 0, sizeof(unsigned) * K, st));
    k_phase_max<<<dim3(kPhBlocks, K), 256, 0, st>>>(d, Mf, maxbits);
    PH_CK(cudaGetLastError());
    std::vector<unsigned> hmax(K);
    PH_CK(cudaMemcpyAsync(hmax.data(), maxbits, sizeof(unsigned) * K, cudaMemcpyDeviceToHost, st));
    PH_CK(cudaStreamSynchronize(st));
    std::vector<float> hthr(K);
    for (int k = 0; k < K; ++k) {
        float m;
        std::memcpy(&m, &hmax[k], sizeof m);
        hthr[k] = m > 0.f ? (float)(frac * m) : 1.f;   // an all-zero harmonic selects nothing
    }
    PH_CK(cudaMemcpyAsync(thr, hthr.data(), sizeof(float) * K, cudaMemcpyHostToDevice, st));

    // 2. theta modulo pi: 1/2 arg sum d^2
    k_phase_sums<<<dim3(kPhBlocks, K), 256, 0, st>>>(d, Mf, thr, part);
    PH_CK(cudaGetLastError());
    PH_CK(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * hpart.size(), cudaMemcpyDeviceToHost, st));
    PH_CK(cudaStreamSynchronize(st));
    std::vector<double> th(K);
    for (int k = 0; k < K; ++k) th[k] = 0.5 * std::atan2(sum_parts(k, 1), sum_parts(k, 0));

    // 3. the pi (s = 1): signs relative to the strongest back-projection,
    // then the common sign from the skewness of a short reconstruction
    std::vector<int> flip(K, 0), resolved(K, 0);
    if (P->s == 1) {
        float2* y = nullptr;
        float* imgs = nullptr;
        float* x = nullptr;
        float2* f = nullptr;
        double* dpart = nullptr;
        PH_CK(S.get(&y, sizeof(float2) * (size_t)K * Mf));
        PH_CK(S.get(&imgs, sizeof(float) * (size_t)K * P->N));
        PH_CK(S.get(&x, sizeof(float) * (size_t)P->N));
        PH_CK(S.get(&f, sizeof(float2) * K));
        PH_CK(S.get(&dpart, sizeof(double) * kPhBlocks));
        if (P->padded && ensure_portrait(*P) != MH3D_OK) return MH3D_ERR_OOM;
        const int nb = (int)std::min<long long>(((long long)K * Mf + 255) / 256, 4096);
        // y = the de-phased portraits of the harmonics with weight w_j != 0,
        // times w_j, expressed for the plan's own phase (the adjoint and the
        // solver remove e^{i theta_plan})
        auto rotate = [&](const std::vector<double>& w) -> cudaError_t {
            std::vector<float2> hf(K);
            for (int j = 0; j < K; ++j) {
                const double a = P->theta[j] - th[j];
                hf[j] = make_float2((float)(w[j] * std::cos(a)), (float)(w[j] * std::sin(a)));
            }
            cudaError_t e = cudaMemcpyAsync(f, hf.data(), sizeof(float2) * K, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            k_phase_rotate<<<nb, 256, 0, st>>>(d, y, Mf, K, f);
            return cudaGetLastError();
        };
        auto backproject = [&](float* out) -> cudaError_t {
            if (P->padded) {
                cudaError_t e = pad_portraits(*P, y, P->w.portrait, st);
                if (e != cudaSuccess) return e;
                return launch_adjoint(*P, P->w.portrait, out, P->w.t1, P->w.t2, st);
            }
            return launch_adjoint(*P, y, out, P->w.t1, P->w.t2, st);
        };
        auto dot = [&](const float* a, const float* b, double* outv) -> cudaError_t {
            k_phase_dot<<<kPhBlocks, 256, 0, st>>>(a, b, P->N, dpart);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            std::vector<double> hd(kPhBlocks);
            if ((e = cudaMemcpyAsync(hd.data(), dpart, sizeof(double) * kPhBlocks, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
            double c = 0.0;
            for (double v : hd) c += v;
            *outv = c;
            return cudaSuccess;
        };
        std::vector<double> w(K), energy(K);
        for (int j = 0; j < K; ++j) {
            std::fill(w.begin(), w.end(), 0.0);
            w[j] = 1.0;
            PH_CK(rotate(w));
            PH_CK(backproject(imgs + (size_t)j * P->N));
            PH_CK(dot(imgs + (size_t)j * P->N, imgs + (size_t)j * P->N, &energy[j]));
        }
        const int r = (int)(std::max_element(energy.begin(), energy.end()) - energy.begin());
        std::vector<double> sig(K, 1.0);
        for (int j = 0; j < K; ++j) {
            if (j == r) continue;
            double c = 0.0;
            PH_CK(dot(imgs + (size_t)j * P->N, imgs + (size_t)r * P->N, &c));
            sig[j] = c >= 0.0 ? 1.0 : -1.0;
        }
        PH_CK(rotate(sig));
        mh3d_solve_opts o{};
        o.reg_kind = 0;
        o.lambda = 1e-2;
        o.lambda_relative = 1;
        o.shell = 1;
        o.solver = 0;
        o.rel_tol = 0.0;
        o.max_iter = 30;
        o.fixed_iters = 1;
        o.normal_mode = 0;
        o.cg_variant = 0;
        mh3d_status sv = mh3d_solve(P, y, &o, x, nullptr, stream);
        if (sv != MH3D_OK) return sv;
        double skew = 0.0;
        PH_CK(dot(x, nullptr, &skew));
        for (int j = 0; j < K; ++j) {
            flip[j] = (skew < 0.0 ? -sig[j] : sig[j]) < 0.0;
            resolved[j] = 1;
        }
    }
    PH_CK(cudaStreamSynchronize(st));
    for (int j = 0; j < K; ++j) {
        double t = th[j] + (flip[j] ? kPi : 0.0);
        t = std::atan2(std::sin(t), std::cos(t));
        theta_out[j] = t;
        if (resolved_out) resolved_out[j] = resolved[j];
    }
    return MH3D_OK;
}

}  // extern "C"
