// Compile-time specialised pencil FFT engine (sm_103a).
//
// Same Stockham formulation and shared-memory layout as fft_smem.cuh
// (element e of pencil p at buf[e * ld + p]), but the length, the radix
// schedule, the number of pencils P and the number of threads T are template
// parameters: index arithmetic folds to constants and shifts, every
// butterfly loop unrolls to its exact trip count, and each stage
// instantiates one radix only (small code, no instruction-cache stalls).
//
// Fusion across the spectral step.  In the last stage of a transform with
// radix R (Ns = n/R) butterfly j produces exactly the elements
// j + r n/R (r < R).  The first stage of a transform whose radix schedule
// starts with R' reads, for butterfly j, the elements j + r' n'/R'.  When
// n'/R' = n/R these are the same positions (or, for a fold over s aliases,
// positions m + a n/s held by the same thread), so a spectral product, an
// alias fold, a sum over harmonics or an alias-block product can be applied
// in registers between the two stages, without a shared-memory round trip.
// The helpers below expose the last-stage outputs and first-stage inputs of
// one butterfly for that purpose.
#pragma once

#include "fft_smem.cuh"

namespace mh3d {

// Radix 16 as 4 x 4: y_{q1 + 4 q2} = sum_{m2} W4^{q2 m2} [W16^{q1 m2} sum_{m1} W4^{q1 m1} v_{4 m1 + m2}].
template <bool INV>
__device__ __forceinline__ void dft16(float2* v)
{
    constexpr float kH = 0.70710678118654752440f;   // cos(pi/4)
    constexpr float kC = 0.92387953251128675613f;   // cos(pi/8)
    constexpr float kS = 0.38268343236508977173f;   // sin(pi/8)
    float2 a[4][4];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) {
        float2 t[4] = {v[m2], v[4 + m2], v[8 + m2], v[12 + m2]};
        dft4<INV>(t);
#pragma unroll
        for (int q1 = 0; q1 < 4; ++q1) a[q1][m2] = t[q1];
    }
    // twiddles W16^{q1 m2} (forward e^{-2 pi i q1 m2 / 16})
    const float sg = INV ? 1.f : -1.f;
    // q1 = 1: m2 = 1, 2, 3 -> angles pi/8, pi/4, 3pi/8
    a[1][1] = c_mul(a[1][1], make_float2(kC, sg * kS));
    a[1][2] = c_mul(a[1][2], make_float2(kH, sg * kH));
    a[1][3] = c_mul(a[1][3], make_float2(kS, sg * kC));
    // q1 = 2: angles pi/4, pi/2, 3pi/4
    a[2][1] = c_mul(a[2][1], make_float2(kH, sg * kH));
    a[2][2] = c_rot<INV>(a[2][2]);
    a[2][3] = c_mul(a[2][3], make_float2(-kH, sg * kH));
    // q1 = 3: angles 3pi/8, 3pi/4, 9pi/8
    a[3][1] = c_mul(a[3][1], make_float2(kS, sg * kC));
    a[3][2] = c_mul(a[3][2], make_float2(-kH, sg * kH));
    a[3][3] = c_mul(a[3][3], make_float2(-kC, -sg * kS));
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        dft4<INV>(a[q1]);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) v[q1 + 4 * q2] = a[q1][q2];
    }
}
template <>
__device__ __forceinline__ void dft<16, false>(float2* v) { dft16<false>(v); }
template <>
__device__ __forceinline__ void dft<16, true>(float2* v) { dft16<true>(v); }

namespace ct {

// ---------------------------------------------------------------------------
// Radix schedules as type lists
// ---------------------------------------------------------------------------
template <int... Rs>
struct RList {
    static constexpr int count = sizeof...(Rs);
};

template <class L>
struct RInfo;
template <int... Rs>
struct RInfo<RList<Rs...>> {
    static constexpr int nst = sizeof...(Rs);
    static constexpr int r[sizeof...(Rs)] = {Rs...};
    static constexpr int n()
    {
        int p = 1;
        for (int i = 0; i < nst; ++i) p *= r[i];
        return p;
    }
    static constexpr int ns(int s)   // product of the radices before stage s
    {
        int p = 1;
        for (int i = 0; i < s; ++i) p *= r[i];
        return p;
    }
    static constexpr int first() { return r[0]; }
    static constexpr int last() { return r[nst - 1]; }
};

template <int N, bool INV>
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int t, int stride)
{
    float2 w = tw[t * stride];
    if (INV) w.y = -w.y;
    return w;
}


// ---------------------------------------------------------------------------
// One Stockham stage with compile-time geometry.
//   N: transform length, R: radix, NS: product of earlier radices,
//   P: pencils, T: threads, TWS: stride into the twiddle table (the table
//   holds W_{N*TWS}^t, so W_N^t = table[t * TWS]).
// ---------------------------------------------------------------------------
template <int N, int R, int NS, int P, int T, int TWS, bool INV, bool PFAST, class LD, class ST>
__device__ __forceinline__ void stage(const LD& ld, const ST& st, const float2* __restrict__ tw)
{
    constexpr int NB = N / R;
    constexpr int TOTAL = NB * P;
    constexpr int TSTEP = N / (NS * R);
    constexpr int ITER = (TOTAL + T - 1) / T;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        if ((TOTAL % T) != 0 && idx >= TOTAL) break;
        int p, j;
        if (PFAST) {
            p = idx % P;
            j = idx / P;
        } else {
            j = idx % NB;
            p = idx / NB;
        }
        const int k = j % NS;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * NB, p);
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], twid<N, INV>(tw, r * k * TSTEP, TWS));
        }
        dft<R, INV>(v);
        const int dst = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) st(dst + r * NS, p, v[r]);
    }
}

// Stages [S0, SEND) of schedule L.  Stage S0 reads `first`; stage SEND-1
// writes `last`; the stages between alternate through b0 (written by S0),
// b1, b0, ...  A barrier follows every stage.
template <class L, int N, int S0, int S, int SEND, int P, int T, int TWS, bool INV, bool FPF, bool LPF, class LD,
          class ST>
struct Runner {
    __device__ __forceinline__ static void run(const LD& first, const ST& last, float2* b0, float2* b1, int ld,
                                               const float2* tw)
    {
        using I = RInfo<L>;
        constexpr int R = I::r[S];
        constexpr int NS = I::ns(S);
        constexpr int par = (S - S0) & 1;
        float2* dstb = par ? b1 : b0;
        const float2* srcb = par ? b0 : b1;   // written by stage S-1
        if constexpr (S + 1 == SEND) {
            if constexpr (S == S0) {
                stage<N, R, NS, P, T, TWS, INV, LPF>(first, last, tw);
            } else {
                stage<N, R, NS, P, T, TWS, INV, LPF>(BufLd{srcb, ld}, last, tw);
            }
            __syncthreads();
        } else {
            if constexpr (S == S0) {
                stage<N, R, NS, P, T, TWS, INV, FPF>(first, BufSt{dstb, ld}, tw);
            } else {
                stage<N, R, NS, P, T, TWS, INV, true>(BufLd{srcb, ld}, BufSt{dstb, ld}, tw);
            }
            __syncthreads();
            Runner<L, N, S0, S + 1, SEND, P, T, TWS, INV, FPF, LPF, LD, ST>::run(first, last, b0, b1, ld, tw);
        }
    }
};

template <class L, int S0, int SEND, int P, int T, int TWS, bool INV, bool FPF, bool LPF, class LD, class ST>
__device__ __forceinline__ void run_stages(const LD& first, const ST& last, float2* b0, float2* b1, int ld,
                                           const float2* tw)
{
    constexpr int N = RInfo<L>::n();
    if constexpr (S0 < SEND)
        Runner<L, N, S0, S0, SEND, P, T, TWS, INV, FPF, LPF, LD, ST>::run(first, last, b0, b1, ld, tw);
}

// Parity of the buffer holding stage SEND-1's output when a run that
// started at S0 writes its last stage into the alternating buffers too.
template <int S0, int SEND>
constexpr int result_parity() { return (SEND - 1 - S0) & 1; }

// Reversed radix schedule (the inverse transform of a fused pair).
template <class A, class B>
struct RevImpl;
template <int... Bs>
struct RevImpl<RList<>, RList<Bs...>> {
    using type = RList<Bs...>;
};
template <int A0, int... As, int... Bs>
struct RevImpl<RList<A0, As...>, RList<Bs...>> {
    using type = typename RevImpl<RList<As...>, RList<A0, Bs...>>::type;
};
template <class L>
using Reverse = typename RevImpl<L, RList<>>::type;

}  // namespace ct
}  // namespace mh3d
