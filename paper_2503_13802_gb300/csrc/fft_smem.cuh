// Shared-memory Stockham FFT engine for batches of short pencils (sm_103a).
//
// A batch is P pencils of one length n (2^a 3^b, n <= 1024).  Element e of
// pencil p lives at buf[e * ld + p] (pencil index fastest), so consecutive
// threads touch consecutive float2 words: a half warp covers 128 contiguous
// bytes, which is bank-conflict free for 64-bit accesses.  ld = P + 1 keeps
// column walks (j-fast mapping, below) at most two-way conflicted.
//
// Each radix-R stage is the self-sorting (Stockham) step: butterfly j reads
// elements j + r n/R (r < R), multiplies by the twiddles W_{Ns R}^{r (j mod Ns)},
// applies the length-R DFT in registers and writes elements
// (j - j mod Ns) R + j mod Ns + r Ns.  Stages alternate between two scratch
// buffers; the first stage reads through a loader functor and the last
// writes through a storer functor, so global loads, spectral multiplies,
// folds and epilogues fuse into the first or last stage.  Every stage ends
// with __syncthreads().
//
// Thread mappings: PFAST puts the pencil index fastest (butterfly idx ->
// p = idx % P, j = idx / P); !PFAST puts the butterfly index fastest, which
// makes the first stage read and the last stage write consecutive elements
// of one pencil -- the mapping used where a pencil is a contiguous row in
// global memory.
//
// Twiddle tables (W_n^t, t < n) come from the host, computed in FP64 and
// rounded once; the DFT kernels use only the exact constants 1/2, sqrt(3)/2
// and sqrt(1/2).
#pragma once

#include <cuda_runtime.h>

#include "mh3d_internal.h"

namespace mh3d {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// Multiply by -i (forward transform) or +i (inverse transform).
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of length R with sign -1 (forward) or +1 (INV).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<2, false>(float2* v)
{
    const float2 a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
}
template <>
__device__ __forceinline__ void dft<2, true>(float2* v) { dft<2, false>(v); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* v)
{
    constexpr float kS = 0.86602540378443864676f;   // sqrt(3)/2
    const float2 t1 = c_add(v[1], v[2]);
    const float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
    const float2 d = c_scale(c_sub(v[1], v[2]), kS);
    const float2 md = c_rot<INV>(d);
    v[0] = c_add(v[0], t1);
    v[1] = c_add(t2, md);
    v[2] = c_sub(t2, md);
}
template <>
__device__ __forceinline__ void dft<3, false>(float2* v) { dft3<false>(v); }
template <>
__device__ __forceinline__ void dft<3, true>(float2* v) { dft3<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft4(float2* v)
{
    const float2 a = c_add(v[0], v[2]), b = c_sub(v[0], v[2]);
    const float2 c = c_add(v[1], v[3]), d = c_rot<INV>(c_sub(v[1], v[3]));
    v[0] = c_add(a, c);
    v[2] = c_sub(a, c);
    v[1] = c_add(b, d);
    v[3] = c_sub(b, d);
}
template <>
__device__ __forceinline__ void dft<4, false>(float2* v) { dft4<false>(v); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* v) { dft4<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* v)
{
    constexpr float kH = 0.70710678118654752440f;   // sqrt(1/2)
    // y_{2q} = DFT4(v_m + v_{m+4}),  y_{2q+1} = DFT4((v_m - v_{m+4}) W8^m)
    float2 a[4], b[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        a[m] = c_add(v[m], v[m + 4]);
        b[m] = c_sub(v[m], v[m + 4]);
    }
    // W8^1 = (1 -+ i)/sqrt2, W8^2 = -+i, W8^3 = (-1 -+ i)/sqrt2  (upper sign forward)
    {
        const float2 t = b[1];
        const float2 r = c_rot<INV>(t);                    // -+ i t
        b[1] = make_float2(kH * (t.x + r.x), kH * (t.y + r.y));
    }
    b[2] = c_rot<INV>(b[2]);
    {
        const float2 t = b[3];
        const float2 r = c_rot<INV>(t);
        b[3] = make_float2(kH * (r.x - t.x), kH * (r.y - t.y));
    }
    dft4<INV>(a);
    dft4<INV>(b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[2 * q] = a[q];
        v[2 * q + 1] = b[q];
    }
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* v) { dft8<true>(v); }

// Plain shared-memory buffer access.
struct BufLd {
    const float2* b;
    int ld;
    __device__ __forceinline__ float2 operator()(int e, int p) const { return b[e * ld + p]; }
};
struct BufSt {
    float2* b;
    int ld;
    __device__ __forceinline__ void operator()(int e, int p, float2 v) const { b[e * ld + p] = v; }
};

// One radix-R Stockham stage over P pencils of length n.
template <int R, bool INV, bool PFAST, class LD, class ST>
__device__ __forceinline__ void fft_stage(const LD& ld, const ST& st, int n, int Ns, int P,
                                          const float2* __restrict__ tw)
{
    const int nb = n / R;
    const int total = nb * P;
    const int tstep = n / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int p, j;
        if (PFAST) {
            p = idx % P;
            j = idx / P;
        } else {
            j = idx % nb;
            p = idx / nb;
        }
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * nb, p);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * k * tstep];
                if (INV) w.y = -w.y;
                v[r] = c_mul(v[r], w);
            }
        }
        dft<R, INV>(v);
        const int dst = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) st(dst + r * Ns, p, v[r]);
    }
}

template <bool INV, bool PFAST, class LD, class ST>
__device__ __forceinline__ void fft_stage_dispatch(int R, const LD& ld, const ST& st, int n, int Ns, int P,
                                                   const float2* tw)
{
    switch (R) {
        case 8: fft_stage<8, INV, PFAST>(ld, st, n, Ns, P, tw); break;
        case 4: fft_stage<4, INV, PFAST>(ld, st, n, Ns, P, tw); break;
        case 2: fft_stage<2, INV, PFAST>(ld, st, n, Ns, P, tw); break;
        case 3: fft_stage<3, INV, PFAST>(ld, st, n, Ns, P, tw); break;
        default: break;
    }
}

// Full transform of P pencils: first stage reads `first`, last stage writes
// `last`, intermediate stages use scratch buffers s0 (written by stage 0,
// 2, ...) and s1 (stage 1, 3, ...), both with leading dimension lds >= P.
// `last` may target either scratch buffer only if that buffer is not read by
// the last stage: the caller guarantees it (see fft_result_buf).
// FIRST_PFAST / LAST_PFAST choose the mapping of the first / last stage
// (a single-stage transform uses LAST_PFAST).  Length 1 copies.
template <bool INV, bool FIRST_PFAST, bool LAST_PFAST, class LD, class ST>
__device__ __forceinline__ void fft_run(const RadixPlan& pl, const LD& first, const ST& last, float2* s0,
                                        float2* s1, int lds, int P, const float2* tw)
{
    const int n = pl.n;
    if (pl.nst == 0) {
        for (int p = threadIdx.x; p < P; p += blockDim.x) last(0, p, first(0, p));
        __syncthreads();
        return;
    }
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.radix[s];
        const bool isFirst = (s == 0), isLast = (s == pl.nst - 1);
        float2* dstb = (s & 1) ? s1 : s0;
        const float2* srcb = (s & 1) ? s0 : s1;   // buffer written by stage s-1
        if (isFirst && isLast) {
            fft_stage_dispatch<INV, LAST_PFAST>(R, first, last, n, Ns, P, tw);
        } else if (isFirst) {
            fft_stage_dispatch<INV, FIRST_PFAST>(R, first, BufSt{dstb, lds}, n, Ns, P, tw);
        } else if (isLast) {
            fft_stage_dispatch<INV, LAST_PFAST>(R, BufLd{srcb, lds}, last, n, Ns, P, tw);
        } else {
            fft_stage_dispatch<INV, true>(R, BufLd{srcb, lds}, BufSt{dstb, lds}, n, Ns, P, tw);
        }
        Ns *= R;
        __syncthreads();
    }
}

// Index (0 -> s0, 1 -> s1) of the scratch buffer a transform of `nst`
// stages should write its last stage into when the result is to stay in
// scratch: stage s writes s_(s & 1), so the last stage (nst - 1) reads
// s_(nst & 1) and may write s_((nst + 1) & 1).  A transform that then reads
// this result must run with its scratch pair swapped: (s0', s1') =
// (s_(res ^ 1), s_res), so that its stage 0 does not overwrite its input.
__host__ __device__ __forceinline__ int fft_result_index(int nst) { return (nst + 1) & 1; }

// ----------------------------------------------------------------------------
// FP64-grade dot-product accumulation with FP32 arithmetic.
// GB300's FP64 pipe is narrow, so each thread accumulates its products as an
// unevaluated float pair (Dekker's exact product via fma, Knuth's TwoSum),
// and only the per-thread totals are combined in FP64.
// ----------------------------------------------------------------------------
struct DotAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = a * b;
        const float pe = fmaf(a, b, -p);          // exact: a*b = p + pe
        const float s = hi + p;                   // TwoSum(hi, p)
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += e + pe;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Block-wide FP64 sum (all threads participate; result valid in thread 0).
__device__ __forceinline__ double block_sum_f64(double v, double* sh /* >= 32 doubles */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        const int nw = (blockDim.x + 31) >> 5;
        t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// Block-wide sums of one or two compensated FP32 accumulators (all threads
// participate; results valid in thread 0).  The FP64 pipe is narrow on this
// part, so the warp levels add the (hi, lo) pairs in FP32: the high words
// by TwoSum (Knuth), whose exact rounding error joins the low words.  A
// pair carries about 48 bits, as each thread's accumulator did.  Each warp's
// total becomes one double, and thread 0 adds the warp totals in FP64 in
// warp order, so the result does not depend on timing.
__device__ __forceinline__ void warp_sum_acc(float& hi, float& lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + h2;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (h2 - bb);
        hi = s;
        lo = (lo + l2) + e;
    }
}

__device__ __forceinline__ double block_sum_acc(const DotAcc& a, double* sh /* >= 32 doubles */)
{
    float hi = a.hi, lo = a.lo;
    warp_sum_acc(hi, lo);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = (double)hi + (double)lo;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) t += sh[w];
    }
    return t;
}

__device__ __forceinline__ void block_sum_acc2(const DotAcc& a, const DotAcc& b, double* sh /* >= 32 doubles */,
                                               double* ta, double* tb)
{
    float ha = a.hi, la = a.lo, hb = b.hi, lb = b.lo;
    warp_sum_acc(ha, la);
    warp_sum_acc(hb, lb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[wid] = (double)ha + (double)la;
        sh[16 + wid] = (double)hb + (double)lb;
    }
    __syncthreads();
    double s0 = 0.0, s1 = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) {
            s0 += sh[w];
            s1 += sh[16 + w];
        }
    }
    *ta = s0;
    *tb = s1;
}

// Deterministic FP64 sum of n partials, identical in every block (same
// order): result returned to all threads of the block.
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int n, double* sh)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    v = block_sum_f64(v, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Grid-wide deterministic FP64 reduction.  Each block stores its partial
// (v valid in thread 0) at part[bid]; the last block to arrive (atomic
// ticket) sums part[0..nparts) in a fixed order (warp 0: lane l takes
// l, l + 32, ..., then a butterfly over the lanes) and stores the total in
// *out, then re-arms the ticket counter for the next launch.  Consumers
// read the single scalar.
__device__ __forceinline__ void grid_sum_finalize(double v, double* part, int bid, int nparts, unsigned int* counter,
                                                  double* out, double* sh)
{
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        part[bid] = v;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == (unsigned int)nparts - 1u);
    }
    __syncthreads();
    // warp 0 alone: a strided FP64 sum per lane, then the lanes in a fixed
    // butterfly (no block barrier on the last block's tail)
    if (am_last && threadIdx.x < 32) {
        __threadfence();
        double acc = 0.0;
        for (int i = threadIdx.x; i < nparts; i += 32) acc += __ldcg(part + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) {
            *out = acc;
            *counter = 0u;
            __threadfence();
        }
    }
}

// Two totals with one ticket: the last block sums both partial arrays.
__device__ __forceinline__ void grid_sum_finalize2(double v0, double v1, double* part0, double* part1, int bid,
                                                   int nparts, unsigned int* counter, double* out0, double* out1,
                                                   double* sh)
{
    __shared__ int am_last2;
    if (threadIdx.x == 0) {
        part0[bid] = v0;
        part1[bid] = v1;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        am_last2 = (t == (unsigned int)nparts - 1u);
    }
    __syncthreads();
    if (am_last2 && threadIdx.x < 32) {
        __threadfence();
        double a0 = 0.0, a1 = 0.0;
        for (int i = threadIdx.x; i < nparts; i += 32) {
            a0 += __ldcg(part0 + i);
            a1 += __ldcg(part1 + i);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (threadIdx.x == 0) {
            *out0 = a0;
            *out1 = a1;
            *counter = 0u;
            __threadfence();
        }
    }
}

}  // namespace mh3d
