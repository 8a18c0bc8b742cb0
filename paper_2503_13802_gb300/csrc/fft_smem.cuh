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
// unevaluated float pair (Dekker's exact product via fma, Knuth's TwoSum);
// the block and grid trees below add such pairs in FP32 too, and only a
// final total becomes a double.
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

// x = m 2^e for a positive normal double x: m in [1, 2) as a float (the
// leading 24 significand bits), e the unbiased exponent.  Integer operations
// only.  Returns false for zero, negative, subnormal, infinite or NaN x.
__device__ __forceinline__ bool dsplit(double x, float* m, int* e)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ffu);
    *e = ef - 1023;
    *m = __uint_as_float(0x3f800000u | (unsigned int)((b >> 29) & 0x7fffffu));
    return (b >> 63) == 0 && ef != 0 && ef != 0x7ff;
}

// x / y as a float for doubles x, y: the leading significand bits are
// divided in FP32 and the exponents subtracted.  Truncating each operand to
// 24 bits and rounding the quotient leave a relative error below 3e-7; the
// loop applies the quotient as a float anyway.  Falls back to the FP64
// division when either operand is not a positive normal number.
__device__ __forceinline__ float ddiv_to_float(double x, double y)
{
    float mx, my;
    int ex, ey;
    if (dsplit(x, &mx, &ex) && dsplit(y, &my, &ey)) return ldexpf(mx / my, ex - ey);
    return (float)(x / y);
}

__device__ __forceinline__ bool dbits_finite(double x)
{
    return ((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7ffu) != 0x7ffu;
}

__device__ __forceinline__ bool dbits_zero(double x)
{
    return (((unsigned long long)__double_as_longlong(x)) << 1) == 0ull;
}

// Sums of compensated FP32 accumulators.  The FP64 pipe is narrow on this
// part (one FP64 warp instruction holds it for many cycles, whatever its
// active lanes), so the whole reduction tree adds (hi, lo) pairs in FP32:
// the high words by TwoSum (Knuth), whose exact rounding error joins the
// low words.  A pair carries about 48 bits, as each thread's accumulator
// did, and only the final total is converted to FP64.  The trees are fixed
// (xor butterflies, lane order), so results do not depend on timing.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float h2, float l2)
{
    const float s = hi + h2;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (h2 - bb);
    hi = s;
    lo = (lo + l2) + e;
}

__device__ __forceinline__ void warp_sum_acc(float& hi, float& lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        pair_add(hi, lo, h2, l2);
    }
}

// Block-wide pair sums of one or two accumulators (all threads participate;
// results valid in thread 0).  sh: at least 4 floats per warp of the block.
__device__ __forceinline__ void block_pair_acc2(const DotAcc& a, const DotAcc* b, float* sh, float2* ta, float2* tb)
{
    float ha = a.hi, la = a.lo, hb = b ? b->hi : 0.f, lb = b ? b->lo : 0.f;
    warp_sum_acc(ha, la);
    if (b) warp_sum_acc(hb, lb);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float* shb = sh + 2 * nw;
    __syncthreads();
    if (lane == 0) {
        sh[2 * wid] = ha;
        sh[2 * wid + 1] = la;
        shb[2 * wid] = hb;
        shb[2 * wid + 1] = lb;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool in = (int)threadIdx.x < nw;
        ha = in ? sh[2 * threadIdx.x] : 0.f;
        la = in ? sh[2 * threadIdx.x + 1] : 0.f;
        warp_sum_acc(ha, la);
        *ta = make_float2(ha, la);
        if (b) {
            hb = in ? shb[2 * threadIdx.x] : 0.f;
            lb = in ? shb[2 * threadIdx.x + 1] : 0.f;
            warp_sum_acc(hb, lb);
            *tb = make_float2(hb, lb);
        }
    }
}

__device__ __forceinline__ float2 block_pair_acc(const DotAcc& a, double* sh /* >= 2 doubles per warp */)
{
    float2 t = make_float2(0.f, 0.f), u;
    block_pair_acc2(a, nullptr, reinterpret_cast<float*>(sh), &t, &u);
    return t;
}

// The block total as a double (valid in thread 0).
__device__ __forceinline__ double block_sum_acc(const DotAcc& a, double* sh /* >= 2 doubles per warp */)
{
    const float2 t = block_pair_acc(a, sh);
    return (double)t.x + (double)t.y;
}

// Grid-wide deterministic reduction of the blocks' pair sums.  Each block
// stores its pair (v valid in thread 0) in the 8-byte slot part[bid]; the
// last block to arrive (atomic ticket) adds part[0..nparts) in a fixed
// order (warp 0: lane l takes l, l + 32, ..., then a butterfly over the
// lanes), stores the total in *out as a double, and re-arms the ticket
// counter for the next launch.  Consumers read the single scalar.
__device__ __forceinline__ float2 grid_pairs_sum(const double* part, int nparts)
{
    const float2* pp = reinterpret_cast<const float2*>(part);
    float hi = 0.f, lo = 0.f;
    for (int i = threadIdx.x; i < nparts; i += 32) {
        const float2 v = __ldcg(pp + i);
        pair_add(hi, lo, v.x, v.y);
    }
    warp_sum_acc(hi, lo);
    return make_float2(hi, lo);
}

__device__ __forceinline__ void grid_sum_finalize(float2 v, double* part, int bid, int nparts, unsigned int* counter,
                                                  double* out)
{
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        reinterpret_cast<float2*>(part)[bid] = v;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == (unsigned int)nparts - 1u);
    }
    __syncthreads();
    if (am_last && threadIdx.x < 32) {
        __threadfence();
        const float2 t = grid_pairs_sum(part, nparts);
        if (threadIdx.x == 0) {
            *out = (double)t.x + (double)t.y;
            *counter = 0u;
            __threadfence();
        }
    }
}

// Two totals with one ticket: the last block sums both partial arrays.
__device__ __forceinline__ void grid_sum_finalize2(float2 v0, float2 v1, double* part0, double* part1, int bid,
                                                   int nparts, unsigned int* counter, double* out0, double* out1)
{
    __shared__ int am_last2;
    if (threadIdx.x == 0) {
        reinterpret_cast<float2*>(part0)[bid] = v0;
        reinterpret_cast<float2*>(part1)[bid] = v1;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        am_last2 = (t == (unsigned int)nparts - 1u);
    }
    __syncthreads();
    if (am_last2 && threadIdx.x < 32) {
        __threadfence();
        const float2 t0 = grid_pairs_sum(part0, nparts);
        const float2 t1 = grid_pairs_sum(part1, nparts);
        if (threadIdx.x == 0) {
            *out0 = (double)t0.x + (double)t0.y;
            *out1 = (double)t1.x + (double)t1.y;
            *counter = 0u;
            __threadfence();
        }
    }
}

}  // namespace mh3d
