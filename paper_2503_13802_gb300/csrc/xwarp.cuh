// Warp-centric drive-axis passes for n_x = 128, s = 2 (portrait rows of 64).
//
// The CTA-level passes of ops_ct.cuh spread a pencil's butterflies over the
// whole CTA, so every radix stage ends on a CTA barrier, and per harmonic the
// adjoint waits for its staged rows.  Here every warp owns 8 consecutive
// rows outright -- 4 pencils, each packing two real rows as one complex
// sequence, on 8 lanes -- and runs their transforms in registers with
// warp-private shared-memory transposes between the radix steps: no CTA
// barrier after the tables are loaded, so the warps of an SM interleave
// loads, transforms and stores freely.
//
// Lane (q, t) = (lane / 8, lane % 8) of a warp works on pencil q (rows
// 2q and 2q + 1 of the warp's 8).  Index maps (every transform unnormalised;
// W_n = e^{-2 pi i / n}):
//
//   forward, length 128, n = n1 + 16 n2, f = f1 + 8 f2:
//     X[f1 + 8 f2] = sum_n1 W16^{n1 f2} W128^{n1 f1} sum_n2 W8^{n2 f1} x[n1 + 16 n2]
//     lane t first takes n1 in {2t, 2t + 1} (two radix-8 DFTs), then, after
//     a transpose, f1 = t (one radix-16 DFT): it ends holding X at t + 8 f2.
//   fold by s = 2 and harmonic k (Sec. 4.1, Eq. dN: the row selector as a
//   spectral fold): F[m] = X^_k[m] X[m] + X^_k[m + 64] X[m + 64], m = t + 8 j
//     -- both aliases sit in the same lane.
//   inverse, length 64, m = m1 + 8 m2, n = n1 + 8 n2:
//     v[n1 + 8 n2] = sum_m1 e^{+2 pi i m1 n2 / 8} e^{+2 pi i m1 n1 / 64}
//                    sum_m2 e^{+2 pi i m2 n1 / 8} F[m1 + 8 m2]
//     lane t takes m1 = t, then after a transpose n1 = t: it ends holding the
//     portrait samples t + 8 n2 of both rows (real and imaginary part).
//   adjoint: the same maps run backwards -- per harmonic the length-64
//     forward transform of Re(e^{-i theta_k} y_k) of both rows (lane t ends
//     with frequencies t + 8 k1), times conj(X^_k) at those frequencies and
//     at their alias + 64 (zero insertion = periodisation), summed over k in
//     16 registers; then one length-128 inverse (16 x 8: lane t holds the
//     frequencies t + 8 m, a radix-16 step, a transpose, radix-8 steps).
//
// Transposes use padded strides so that each half-warp's 16 lanes hit 16
// distinct 8-byte bank pairs.
#pragma once

#include "ops_ct.cuh"

namespace mh3d {
namespace xw {

constexpr int kNX = 128, kMX = 64;
constexpr int kWarps = 4;                   // warps per CTA
constexpr int kRowsW = 8;                   // rows per warp (4 pencils of 8 lanes)
constexpr int kRowsCTA = kWarps * kRowsW;
// 16 x 8 transpose of the forward's first step: Z[n1][f1] at f1 * 18 + n1,
// pencils 145 float2 apart (writes and reads conflict-free)
constexpr int kRSF = 18, kQSF = 145;
// 8 x 8 transposes: [a][b] at a * 9 + b, pencils 72 float2 apart
constexpr int kRS8 = 9, kQS8 = 72;
// 16 x 8 transpose of the adjoint's inverse: [j][t] at j * 17 + t, pencils
// 280 float2 apart
constexpr int kRSU = 17, kQSU = 280;
constexpr int kScrF = 4 * kQSF;             // float2 of scratch per warp, forward
constexpr int kScrA = 4 * kQSU;             // adjoint

__host__ __device__ constexpr int tab_floats2(int K) { return kNX + ((K + 1) & ~1) + K * kNX; }
__host__ __device__ constexpr size_t fwd_smem(int K)
{
    return sizeof(float2) * (size_t)(tab_floats2(K) + kWarps * kScrF);
}
__host__ __device__ constexpr size_t adj_smem(int K)
{
    return sizeof(float2) * (size_t)(tab_floats2(K) + kWarps * kScrA);
}

// Twiddles W128^t, phases and the drive-axis spectra into shared memory.
__device__ __forceinline__ void load_tables(const XArgs& a, float2* tw, float2* ph, float2* xh)
{
    for (int i = threadIdx.x; i < kNX; i += blockDim.x) tw[i] = a.twx[i];
    for (int i = threadIdx.x; i < a.K; i += blockDim.x) ph[i] = a.phase[i];
    for (int i = threadIdx.x; i < a.K * kNX; i += blockDim.x) xh[i] = a.Xhat[i];
    __syncthreads();
}

// Forward length-128 transform of a pencil on 8 lanes: xe[n2] and xo[n2]
// hold x[2t + 16 n2] and x[2t + 1 + 16 n2]; X[j] receives the spectrum at
// t + 8 j.  z: the pencil's scratch (8 x 18 float2 used); the caller makes
// sure no lane still reads it.
__device__ __forceinline__ void wfwd128(float2 (&xe)[8], float2 (&xo)[8], float2* z, const float2* tw, int t,
                                        float2 (&X)[16])
{
    dft<8, false>(xe);
    dft<8, false>(xo);
    z[2 * t] = xe[0];
    z[2 * t + 1] = xo[0];
#pragma unroll
    for (int f1 = 1; f1 < 8; ++f1) {
        z[f1 * kRSF + 2 * t] = c_mul(xe[f1], tw[(2 * t) * f1]);
        z[f1 * kRSF + 2 * t + 1] = c_mul(xo[f1], tw[(2 * t + 1) * f1]);
    }
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) X[n1] = z[t * kRSF + n1];
    dft<16, false>(X);
}

// Inverse length-128 transform of a pencil on 8 lanes: V[m] holds the
// frequency t + 8 m; out[e][i] receives the sample t + 8 e + 16 i.  ub: the
// pencil's scratch (16 x 17 float2 used); the caller makes sure no lane still
// reads it.
__device__ __forceinline__ void winv128(float2 (&V)[16], float2* ub, const float2* tw, int t, float2 (&out)[2][8])
{
    dft<16, true>(V);
#pragma unroll
    for (int j = 1; j < 16; ++j) V[j] = c_mulc(V[j], tw[t * j]);   // e^{+2 pi i t j / 128}
#pragma unroll
    for (int j = 0; j < 16; ++j) ub[j * kRSU + t] = V[j];
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int j = t + 8 * e;
#pragma unroll
        for (int i = 0; i < 8; ++i) out[e][i] = ub[j * kRSU + i];
        dft<8, true>(out[e]);
    }
}

// One harmonic of the adjoint on a pencil: Re(e^{-i theta} y) of rows a
// (ya) and b (yb), samples t + 8 n2, through the length-64 forward transform
// (lane t ends with frequencies t + 8 k1), times conj(X^_k) at k1 and at its
// alias + 64, added into V.  hb: the pencil's 8 x 9 scratch; the warp
// barrier before it is written follows the first radix step, so the loads
// a caller issues just before (a warp barrier waits for them) overlap that
// step.
__device__ __forceinline__ void wadj_harmonic(const float2 (&ya)[8], const float2 (&yb)[8], float2 ph, float2* hb,
                                              const float2* tw, const float2* xk, int t, float2 (&V)[16])
{
    float2 w[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2)
        w[n2] = make_float2(fmaf(ph.x, ya[n2].x, ph.y * ya[n2].y), fmaf(ph.x, yb[n2].x, ph.y * yb[n2].y));
    dft<8, false>(w);
#pragma unroll
    for (int k2 = 1; k2 < 8; ++k2) w[k2] = c_mul(w[k2], tw[2 * t * k2]);   // W64^{t k2}
    __syncwarp();   // the previous harmonic's reads of hb are done
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) hb[k2 * kRS8 + t] = w[k2];
    __syncwarp();
    float2 Y[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) Y[n1] = hb[t * kRS8 + n1];
    dft<8, false>(Y);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        V[k1] = c_add(V[k1], c_mulc(Y[k1], xk[8 * k1]));
        V[k1 + 8] = c_add(V[k1 + 8], c_mulc(Y[k1], xk[8 * k1 + 64]));
    }
}

// d = Phi X_k (rows of a.vin): rows [rows][128] float -> portraits
// [K][rows][64] complex.  KS warps share a row group: each runs the
// length-128 transform of the group's rows and then the harmonics
// k = split, split + KS, ... (no communication between them).
template <int KS>
__global__ void __launch_bounds__(kWarps * 32) k_xfwd_w128(const XArgs a)
{
    static_assert(kWarps % KS == 0, "whole row groups per CTA");
    extern __shared__ __align__(16) float2 xw_sm[];
    const int K = a.K;
    float2* tw = xw_sm;
    float2* ph = tw + kNX;
    float2* xh = ph + ((K + 1) & ~1);
    float2* scr = xh + K * kNX;
    load_tables(a, tw, ph, xh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, t = lane & 7;
    const int group = (int)blockIdx.x * (kWarps / KS) + warp / KS, split = warp % KS;
    const int rbase = group * kRowsW;
    if (rbase >= a.rows) return;   // no CTA barrier follows
    float2* sc = scr + warp * kScrF;
    const int ra = rbase + 2 * q, rb = ra + 1;
    const bool va = ra < a.rows, vb = rb < a.rows;

    // forward length 128, first step: lane t takes n1 = 2t (xe) and 2t + 1 (xo)
    float2 xe[8], xo[8];
    {
        const float* pa = a.vin + (long long)ra * kNX + 2 * t;
        const float* pb = a.vin + (long long)rb * kNX + 2 * t;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            const float2 u = va ? __ldg(reinterpret_cast<const float2*>(pa + 16 * n2)) : make_float2(0.f, 0.f);
            const float2 v = vb ? __ldg(reinterpret_cast<const float2*>(pb + 16 * n2)) : make_float2(0.f, 0.f);
            xe[n2] = make_float2(u.x, v.x);
            xo[n2] = make_float2(u.y, v.y);
        }
    }
    float2 X[16];   // spectrum at t + 8 j
    wfwd128(xe, xo, sc + q * kQSF, tw, t, X);

    float2* hb = sc + q * kQS8;
    float2* dka = a.dout + (long long)ra * kMX + t;
    float2* dkb = a.dout + (long long)rb * kMX + t;
    for (int k = split; k < K; k += KS) {
        // fold by s = 2 times X^_k, then the length-64 inverse, first step (m1 = t)
        const float2* xk = xh + k * kNX + t;
        float2 F[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) F[j] = c_add(c_mul(X[j], xk[8 * j]), c_mul(X[j + 8], xk[8 * j + 64]));
        dft<8, true>(F);
#pragma unroll
        for (int n1 = 1; n1 < 8; ++n1) F[n1] = c_mulc(F[n1], tw[2 * t * n1]);   // e^{+2 pi i t n1 / 64}
        __syncwarp();   // the previous reads of this scratch are done
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) hb[n1 * kRS8 + t] = F[n1];
        __syncwarp();
        // second step: n1 = t, radix 8 over m1 -> samples t + 8 n2
        float2 g[8];
#pragma unroll
        for (int m1 = 0; m1 < 8; ++m1) g[m1] = hb[t * kRS8 + m1];
        dft<8, true>(g);
        const float2 p = ph[k];
        float2* oa = dka + (long long)k * a.M;
        float2* ob = dkb + (long long)k * a.M;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            if (va) oa[8 * n2] = make_float2(p.x * g[n2].x, p.y * g[n2].x);
            if (vb) ob[8 * n2] = make_float2(p.x * g[n2].y, p.y * g[n2].y);
        }
    }
}

// v = sum_k X_k^T Phi^T d: portraits [K][rows][64] complex -> rows
// [rows][128] float (the real inner product's adjoint).  KS warps share a
// row group, each summing the harmonics k = split, split + KS, ...; the
// group's first warp adds the others' sums (through their scratch, after a
// barrier of the group's KS warps only) and runs the length-128 inverse.
template <int KS>
__global__ void __launch_bounds__(kWarps * 32) k_xadj_w128(const XArgs a)
{
    static_assert(kWarps % KS == 0, "whole row groups per CTA");
    extern __shared__ __align__(16) float2 xw_sm[];
    const int K = a.K;
    float2* tw = xw_sm;
    float2* ph = tw + kNX;
    float2* xh = ph + ((K + 1) & ~1);
    float2* scr = xh + K * kNX;
    load_tables(a, tw, ph, xh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, t = lane & 7;
    const int gl = warp / KS, split = warp % KS;
    const int rbase = ((int)blockIdx.x * (kWarps / KS) + gl) * kRowsW;
    if (rbase >= a.rows) return;   // the group's KS warps all leave: nothing waits on them
    float2* sc = scr + warp * kScrA;
    const int ra = rbase + 2 * q, rb = ra + 1;
    const bool va = ra < a.rows, vb = rb < a.rows;
    const float2* sa = a.din + (long long)ra * kMX + t;
    const float2* sb = a.din + (long long)rb * kMX + t;
    const float2 zero = make_float2(0.f, 0.f);
    float2 ya[8], yb[8];
    {
        const long long off = (long long)split * a.M;
        const bool any = split < K;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            ya[n2] = (any && va) ? __ldg(sa + off + 8 * n2) : zero;
            yb[n2] = (any && vb) ? __ldg(sb + off + 8 * n2) : zero;
        }
    }
    float2 V[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) V[i] = zero;
    float2* hb = sc + q * kQS8;
    for (int k = split; k < K; k += KS) {
        // the next harmonic's rows are in flight while this one transforms
        float2 na[8], nb[8];
        const bool more = k + KS < K;
        const long long off = (long long)(k + KS) * a.M;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            na[n2] = (more && va) ? __ldg(sa + off + 8 * n2) : zero;
            nb[n2] = (more && vb) ? __ldg(sb + off + 8 * n2) : zero;
        }
        // Re(e^{-i theta_k} y) of both rows packed as one complex sequence,
        // its length-64 transform times conj(X^_k) periodised, into V
        wadj_harmonic(ya, yb, ph[k], hb, tw, xh + k * kNX + t, t, V);
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            ya[n2] = na[n2];
            yb[n2] = nb[n2];
        }
    }
    if constexpr (KS > 1) {
        // the group's sums meet in the first warp: the others leave theirs in
        // their own scratch (lane-major, conflict-free), then a barrier of
        // the group's KS warps (named barrier gl + 1)
        __syncwarp();
        if (split > 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) sc[i * 32 + lane] = V[i];
        }
        asm volatile("bar.sync %0, %1;" ::"r"(gl + 1), "r"(KS * 32) : "memory");
        if (split > 0) return;
#pragma unroll
        for (int w2 = 1; w2 < KS; ++w2) {
            const float2* o = scr + (warp + w2) * kScrA;
#pragma unroll
            for (int i = 0; i < 16; ++i) V[i] = c_add(V[i], o[i * 32 + lane]);
        }
    }
    // length-128 inverse: lane t holds frequencies t + 8 m
    __syncwarp();
    float2 g[2][8];   // samples t + 8 e + 16 i
    winv128(V, sc + q * kQSU, tw, t, g);
    float* outa = a.vout + (long long)ra * kNX;
    float* outb = a.vout + (long long)rb * kNX;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (va) outa[t + 8 * e + 16 * i] = g[e][i].x;
            if (vb) outb[t + 8 * e + 16 * i] = g[e][i].y;
        }
}


// ---------------------------------------------------------------------------
// The adjoint's first two steps in one launch: the warp-centric drive-axis
// adjoint, then the z-axis correlation (T_z^T), for one y-slab per cluster
// of two CTAs (the structure of ct::k_xzadj_ct, with the CTA-level
// drive-axis part replaced by the warp pass above):
//   phase 1: CTA c's warps run the drive-axis adjoint of rows
//            z in [c nz/2, (c+1) nz/2) (portrait rows z ny + y), KS warps per
//            group of 8 rows; the group's first warp stores every output
//            sample into the z-tile of the CTA that owns its x-column
//            (columns [c' 64, (c'+1) 64) belong to CTA c'), locally or through
//            distributed shared memory;
//   cluster barrier;
//   phase 2: CTA c runs the z correlation (T pass stages, multiplier Z^*) on
//            its 64 columns of every z and stores the box with one TMA store.
// No thread leaves before the second cluster barrier.
template <class LZ, int KS>
struct XzwGeom {
    static constexpr int NZ = ct::RInfo<LZ>::n(), ROWS = NZ / 2, GROUPS = ROWS / kRowsW, WARPS = GROUPS * KS;
    static constexpr int T = WARPS * 32;
    static constexpr int QX = kNX / 2, PZ = QX / 2;   // 64 columns (32 column pairs) per CTA
    static constexpr int XT = NZ * PZ;                  // float2: the z-tile
    static constexpr int WS = kScrA;                    // float2 per warp
    static constexpr int SCR = WARPS * WS;              // float2: phase-1 scratch
    static constexpr int UN = SCR > XT ? SCR : XT;      // phase 2: the z pass's second buffer
    static_assert(ROWS % kRowsW == 0 && T <= 1024 && GROUPS + 1 <= 16, "row groups of the slab");
    static __host__ __device__ int tab(int K) { return kNX + 2 * NZ + ((K + 1) & ~1) + K * kNX; }
    static __host__ __device__ int xt_off(int K) { return (tab(K) + 15) / 16 * 16; }   // 128-byte aligned
    static __host__ __device__ size_t smem(int K) { return sizeof(float2) * (size_t)(xt_off(K) + XT + UN) + 128; }
};

template <class LZ, int KS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(XzwGeom<LZ, KS>::T)
    k_xzadj_w(const __grid_constant__ ZXArgs a)
{
    using G = XzwGeom<LZ, KS>;
    using namespace ct;
    constexpr int NZ = G::NZ, ROWS = G::ROWS, T = G::T, QX = G::QX, PZ = G::PZ;
    constexpr int NSTZ = RInfo<LZ>::nst, RLZ = RInfo<LZ>::last();
    using LZI = Reverse<LZ>;
    static_assert(NSTZ >= 2, "two stages at least along z");
    extern __shared__ __align__(128) float2 xzw_raw[];
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(xzw_raw) + 127) & ~uintptr_t(127));
    const int K = a.x.K;
    float2* tw = sm;
    float2* twz = tw + kNX;
    float2* muz = twz + NZ;
    float2* ph = muz + NZ;
    float2* xh = ph + ((K + 1) & ~1);
    float2* xt = sm + G::xt_off(K);     // the z-tile [NZ][PZ], written by both CTAs of the cluster
    float2* un = xt + G::XT;
    const uint32_t rank = cluster_ctarank();
    const int y = (int)blockIdx.x / 2;
    for (int i = threadIdx.x; i < NZ; i += T) {
        twz[i] = a.twz[i];
        muz[i] = a.muz[i];
    }
    load_tables(a.x, tw, ph, xh);   // ends on a CTA barrier
    cluster_sync_all();             // every CTA of the cluster runs before any remote store

    // ---- phase 1: the drive-axis adjoint of this CTA's rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, t = lane & 7;
    const int gl = warp / KS, split = warp % KS;
    float2* sc = un + warp * G::WS;
    const int za = (int)rank * ROWS + gl * kRowsW + 2 * q, zb = za + 1;
    const float2* sa = a.x.din + ((long long)za * a.ny + y) * kMX + t;
    const float2* sb = a.x.din + ((long long)zb * a.ny + y) * kMX + t;
    const float2 zero = make_float2(0.f, 0.f);
    float2 V[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) V[i] = zero;
    float2* hb = sc + q * kQS8;
    float2 ya[8], yb[8];
    {
        const long long off = (long long)split * a.x.M;
        const bool any = split < K;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            ya[n2] = any ? __ldg(sa + off + 8 * n2) : zero;
            yb[n2] = any ? __ldg(sb + off + 8 * n2) : zero;
        }
    }
    for (int k = split; k < K; k += KS) {
        float2 na[8], nb[8];
        const bool more = k + KS < K;
        const long long off = (long long)(k + KS) * a.x.M;
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            na[n2] = more ? __ldg(sa + off + 8 * n2) : zero;
            nb[n2] = more ? __ldg(sb + off + 8 * n2) : zero;
        }
        wadj_harmonic(ya, yb, ph[k], hb, tw, xh + k * kNX + t, t, V);
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            ya[n2] = na[n2];
            yb[n2] = nb[n2];
        }
    }
    if constexpr (KS > 1) {
        __syncwarp();
        if (split > 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) sc[i * 32 + lane] = V[i];
        }
        asm volatile("bar.sync %0, %1;" ::"r"(gl + 1), "r"(KS * 32) : "memory");
        if (split == 0) {
#pragma unroll
            for (int w2 = 1; w2 < KS; ++w2) {
                const float2* o = un + (warp + w2) * G::WS;
#pragma unroll
                for (int i = 0; i < 16; ++i) V[i] = c_add(V[i], o[i * 32 + lane]);
            }
        }
    }
    if (split == 0) {
        __syncwarp();
        float2 g[2][8];   // samples t + 8 e + 16 i
        winv128(V, sc + q * kQSU, tw, t, g);
        float* xtf = reinterpret_cast<float*>(xt);
        const uint32_t peer = cluster_smem_addr(xtf, rank ^ 1u);
        // sample x = t + 8 e + 16 i: owner CTA i / 4, column t + 8 e + 16 (i % 4)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int col = t + 8 * e + 16 * (i & 3);
                const int oa = za * QX + col, ob = zb * QX + col;
                if ((uint32_t)(i >> 2) == rank) {
                    xtf[oa] = g[e][i].x;
                    xtf[ob] = g[e][i].y;
                } else {
                    st_cluster_f32(peer + 4u * (uint32_t)oa, g[e][i].x);
                    st_cluster_f32(peer + 4u * (uint32_t)ob, g[e][i].y);
                }
            }
    }
    cluster_sync_all();   // every column of this CTA's z-tile has landed

    // ---- phase 2: z correlation of this CTA's columns, one TMA store
    float2* tile = xt;
    float2* zb2 = un;
    constexpr int pf = result_parity<0, NSTZ - 1>();
    float2* fo = pf ? tile : zb2;
    float2* fx = pf ? zb2 : tile;
    run_stages<LZ, 0, NSTZ - 1, PZ, T, 1, false, true, true>(BufLd{tile, PZ}, BufSt{fo, PZ}, zb2, tile, PZ, twz);
    fused_conv_stage<NZ, RLZ, PZ, T>(BufLd{fo, PZ}, BufSt{fx, PZ}, muz, twz);
    __syncthreads();
    float2* stg = (NSTZ % 2 == 0) ? fo : fx;
    run_stages<LZI, 1, NSTZ, PZ, T, 1, true, true, true>(BufLd{fx, PZ}, BufSt{stg, PZ}, fo, fx, PZ, twz);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tma_store_3d(&a.tz, (int)rank * QX, y, 0, stg);
        bulk_commit();
        bulk_wait_all();   // the copy reads shared memory and must land before the CTA ends
    }
}


// ---------------------------------------------------------------------------
// The normal operator's last two steps in one launch (the CG loop's second
// kernel): T_z (multiplier |Z^|^2), then the drive-axis Fourier-block
// product, q = b w + lambda p, and the dot products p^T q and p^T p, for one
// y-slab per cluster of two CTAs (the structure of ct::k_zxnrm_ct, with the
// CTA-level drive-axis part replaced by warp-centric transforms):
//   phase 1: ct::zx_zconv -- CTA c convolves its 64 x-columns along z and
//            stores each row into the exchange buffer of the CTA that owns
//            it (rows [c nz/2, (c+1) nz/2));
//   cluster barrier;
//   phase 2: each warp takes 8 of the CTA's rows: the length-128 forward
//            transform (lane t ends with frequencies t + 8 j, so a frequency
//            and its alias + 64 sit in one lane), the s x s alias-block
//            product Q(m) of the normal operator's drive-axis part (Sec. 4.3,
//            the Fourier-block form of sum_k X_k^T P^T P X_k), the inverse,
//            then the epilogue on the lane's 32 samples (b and p loaded
//            before the transforms) and the CTA's pair-sum reduction.
// Host conditions: n_x = 128, s = 2, R = I, 16-byte aligned vectors.
template <class LZ>
struct ZxwGeom {
    static constexpr int NZ = ct::RInfo<LZ>::n(), ROWS = NZ / 2, WARPS = ROWS / kRowsW, T = WARPS * 32;
    static constexpr int QX = kNX / 2, PZ = QX / 2, NXP = kNX + 1;
    static_assert(ROWS % kRowsW == 0 && NZ % 2 == 0, "whole row groups per CTA");
    static constexpr int TAB = 2 * NZ + kNX + kMX * 4;          // float2: W_nz, z multiplier, W_128, Q blocks
    static constexpr int XB = ROWS * NXP;                        // floats: exchange rows
    static constexpr int OFF = (TAB + (XB + 1) / 2 + 15) / 16 * 16;   // float2 offset of the union (128 B)
    static constexpr int P1 = 2 * NZ * PZ;                       // phase 1: tile + second buffer
    static constexpr int P2 = WARPS * kScrA;                     // phase 2: warp scratch
    static constexpr int UN = P1 > P2 ? P1 : P2;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(OFF + UN) + 128; }
};

template <class LZ, bool EARLY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(ZxwGeom<LZ>::T)
    k_zxnrm_w(const __grid_constant__ ZXArgs a)
{
    using G = ZxwGeom<LZ>;
    using namespace ct;
    constexpr int NZ = G::NZ, ROWS = G::ROWS, T = G::T, NXP = G::NXP;
    extern __shared__ __align__(128) float2 zxw_raw[];
    __shared__ double red[34];
    __shared__ __align__(8) uint64_t bar;
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(zxw_raw) + 127) & ~uintptr_t(127));
    float2* twz = sm;
    float2* muz = twz + NZ;
    float2* twx = muz + NZ;           // W_128 (zx_zconv loads it)
    float2* qb = twx + kNX;           // [64][2][2] alias blocks
    float* xb = reinterpret_cast<float*>(qb + kMX * 4);
    float2* un = sm + G::OFF;         // 128-byte aligned: the TMA box lands at its start
    const uint32_t rank = cluster_ctarank();
    const int y = (int)blockIdx.x / 2;
    for (int i = threadIdx.x; i < kMX * 4; i += T) qb[i] = a.x.Q[i];
    cluster_sync_all();   // every CTA of the cluster runs before any remote store
    float dummy;
    if (a.x.cg_active && !cg_enter(a.x.cg, false, &dummy, red)) return;

    // ---- phase 1: z-axis convolution of this CTA's columns (ends on a CTA barrier)
    const bool ok = zx_zconv<LZ, kNX, 2, G::PZ, T>(a, a.muz, twz, muz, twx, xb, un, &bar, y, rank);
    cluster_sync_all();   // every part of every owned row has landed (local and remote stores)
    if (!ok) return;

    // ---- phase 2: rows rr = 8 warp + 2q (+1) of this CTA, z = rank ROWS + rr
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, t = lane & 7;
    const int rra = warp * kRowsW + 2 * q, rrb = rra + 1;
    const long long ia = ((long long)((int)rank * ROWS + rra) * a.ny + y) * kNX;
    const long long ib = ((long long)((int)rank * ROWS + rrb) * a.ny + y) * kNX;
    const float* __restrict__ bp = a.x.b;
    const float* __restrict__ pp = a.x.pin;
    // epilogue operands at the lane's samples x = t + 8 e + 16 i
    float ba[2][8], bb[2][8], pa[2][8], pb[2][8];
    auto load_bp = [&]() {
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int x = t + 8 * e + 16 * i;
                ba[e][i] = bp ? __ldg(bp + ia + x) : 1.f;
                bb[e][i] = bp ? __ldg(bp + ib + x) : 1.f;
                pa[e][i] = __ldg(pp + ia + x);
                pb[e][i] = __ldg(pp + ib + x);
            }
    };
    if constexpr (EARLY) load_bp();
    float2 xe[8], xo[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) {
        const int c = 2 * t + 16 * n2;
        xe[n2] = make_float2(xb[rra * NXP + c], xb[rrb * NXP + c]);
        xo[n2] = make_float2(xb[rra * NXP + c + 1], xb[rrb * NXP + c + 1]);
    }
    float2* sc = un + warp * kScrA;   // the phase-1 buffers are dead after the cluster barrier
    float2 X[16];   // spectrum at t + 8 j
    wfwd128(xe, xo, sc + q * kQSF, twx, t, X);
    // alias blocks: out(m + 64 a) = sum_b Q(m)[a][b] in(m + 64 b), m = t + 8 j
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2* qm = qb + (t + 8 * j) * 4;
        const float2 u0 = X[j], u1 = X[j + 8];
        X[j] = c_add(c_mul(qm[0], u0), c_mul(qm[1], u1));
        X[j + 8] = c_add(c_mul(qm[2], u0), c_mul(qm[3], u1));
    }
    __syncwarp();   // the forward's scratch reads are done
    float2 g[2][8];
    winv128(X, sc + q * kQSU, twx, t, g);
    if constexpr (!EARLY) load_bp();
    // epilogue: q = b w + lambda p, dots p^T q (and p^T p)
    float* __restrict__ qo = a.x.qout;
    const float lam = a.x.reg.lambda;
    DotAcc dacc, dacc2;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int x = t + 8 * e + 16 * i;
            const float qa = fmaf(ba[e][i], g[e][i].x, lam * pa[e][i]);
            const float qb2 = fmaf(bb[e][i], g[e][i].y, lam * pb[e][i]);
            qo[ia + x] = qa;
            qo[ib + x] = qb2;
            dacc.add(pa[e][i], qa);
            dacc.add(pb[e][i], qb2);
            if (a.x.part2) {
                dacc2.add(pa[e][i], pa[e][i]);
                dacc2.add(pb[e][i], pb[e][i]);
            }
        }
    if (a.x.part) {
        float2 t0, t2;
        block_pair_acc2(dacc, a.x.part2 ? &dacc2 : nullptr, reinterpret_cast<float*>(red), &t0, &t2);
        if (a.x.part2)
            grid_sum_finalize2(t0, t2, a.x.part, a.x.part2, blockIdx.x, gridDim.x, a.x.ticket, a.x.sum_out,
                               a.x.sum_out2);
        else
            grid_sum_finalize(t0, a.x.part, blockIdx.x, gridDim.x, a.x.ticket, a.x.sum_out);
    }
    if (a.x.count_iter) cg_count_iteration(a.x.cg);
}

}  // namespace xw
}  // namespace mh3d
