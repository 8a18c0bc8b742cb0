// Kernels of the learned warm-start network: a small 3D U-Net with additive
// skips whose 3x3x3 convolutions run as implicit GEMMs on the tensor cores
// (bfloat16 operands, FP32 accumulation, mma.sync m16n8k16).
//
// Activations are channels-last bfloat16 volumes [D][H][W][C].  A
// convolution "same" (zero padding) with weights W[co][tap][ci] (tap =
// 9 (dz+1) + 3 (dy+1) + (dx+1)) is the GEMM
//     out[v][co] = sum_k A[v][k] Wt[k][co],   k = tap * Cin + ci,
// where A[v][k] = in[v + tap][ci] is gathered on the fly (never stored).
// The gather also forms the two special inputs of the decoder: a nearest x2
// upsampling of a half-resolution source, and the sum of two sources (the
// additive skip), rounded to bfloat16 as a stored sum would be.  The same
// kernel with negated taps and re-laid-out weights computes the gradient
// with respect to the input; the weight gradient is the GEMM
//     dW^T[k][co] = sum_v A[v][k] dY[v][co]
// split over voxel chunks into FP32 partials that a second kernel adds in a
// fixed order.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mh3d {
namespace unet {

constexpr int kBM = 128;   // GEMM rows per CTA (voxels, or weight rows in wgrad)
constexpr int kBK = 32;    // reduction depth per shared-memory stage
constexpr int kThreads = 256;
constexpr int kWChunk = 4096;   // voxels per CTA in the weight gradient

// Source of a convolution's input (the GEMM's gathered operand).
struct ConvSrc {
    const __nv_bfloat16* a = nullptr;   // [.][.][.][C] bfloat16
    const __nv_bfloat16* b = nullptr;   // second addend (skip), same shape as a, or null
    const float* f32 = nullptr;         // single-channel FP32 source instead of a (network input)
    const float* f32_scale = nullptr;   // device scalar multiplying the FP32 source (null: 1)
    int D = 0, H = 0, W = 0;            // resolution of the convolution (output)
    int C = 0;                          // source channels
    int up = 0;                         // 1: a is at half resolution (nearest x2 upsampling)
    int flip = 0;                       // 1: taps negated (gradient w.r.t. the input)
};

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }

// A[v][k] for one voxel (z, y, x) and k = tap * C + ci; 0 outside the volume.
__device__ __forceinline__ float gather1(const ConvSrc& s, int z, int y, int x, int k)
{
    const int tap = k / s.C, ci = k - tap * s.C;
    int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    if (s.flip) {
        dz = -dz;
        dy = -dy;
        dx = -dx;
    }
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= s.D || yy < 0 || yy >= s.H || xx < 0 || xx >= s.W) return 0.f;
    if (s.f32) return s.f32[((size_t)zz * s.H + yy) * s.W + xx] * (s.f32_scale ? *s.f32_scale : 1.f);
    size_t off;
    if (s.up)
        off = (((size_t)(zz >> 1) * (s.H >> 1) + (yy >> 1)) * (s.W >> 1) + (xx >> 1)) * s.C + ci;
    else
        off = (((size_t)zz * s.H + yy) * s.W + xx) * s.C + ci;
    float v = bf2f(s.a[off]);
    if (s.b) v = bf2f(__float2bfloat16(v + bf2f(s.b[off])));
    return v;
}

// Eight consecutive k (one tap, ci .. ci+7; needs C % 8 == 0) as 16 bytes.
__device__ __forceinline__ uint4 gather8(const ConvSrc& s, int z, int y, int x, int k)
{
    const int tap = k / s.C, ci = k - tap * s.C;
    int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    if (s.flip) {
        dz = -dz;
        dy = -dy;
        dx = -dx;
    }
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    uint4 r = make_uint4(0, 0, 0, 0);
    if (zz < 0 || zz >= s.D || yy < 0 || yy >= s.H || xx < 0 || xx >= s.W) return r;
    size_t off;
    if (s.up)
        off = (((size_t)(zz >> 1) * (s.H >> 1) + (yy >> 1)) * (s.W >> 1) + (xx >> 1)) * s.C + ci;
    else
        off = (((size_t)zz * s.H + yy) * s.W + xx) * s.C + ci;
    r = *reinterpret_cast<const uint4*>(s.a + off);
    if (s.b) {
        const uint4 q = *reinterpret_cast<const uint4*>(s.b + off);
        __nv_bfloat162* pr = reinterpret_cast<__nv_bfloat162*>(&r);
        const __nv_bfloat162* pq = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 u = __bfloat1622float2(pr[i]), w = __bfloat1622float2(pq[i]);
            pr[i] = __floats2bfloat162_rn(u.x + w.x, u.y + w.y);
        }
    }
    return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One kBK-deep stage: warp w owns GEMM rows [16 w, 16 w + 16) and every
// column of the BN-wide tile.  sA is [kBM][kBK + 8] (row-major, m by k) or,
// with A_KMAJOR, [kBK][kBM + 8] (k by m); sB is [kBK][BN + 8] (k by n).
template <int BN, bool A_KMAJOR>
__device__ __forceinline__ void mma_stage(const __nv_bfloat16* sA, const __nv_bfloat16* sB, float (&acc)[BN / 8][4],
                                          int warp, int lane)
{
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
        uint32_t a[4];
        if (A_KMAJOR) {
            const int row = kk + (lane & 7) + (lane >> 4) * 8;
            const int col = 16 * warp + ((lane >> 3) & 1) * 8;
            ldsm_x4_t(a, sA + row * (kBM + 8) + col);
        } else {
            const int row = 16 * warp + (lane & 15);
            const int col = kk + (lane >> 4) * 8;
            ldsm_x4(a, sA + row * (kBK + 8) + col);
        }
#pragma unroll
        for (int j = 0; j < BN / 16; ++j) {
            uint32_t b[4];
            const int row = kk + (lane & 7) + ((lane >> 3) & 1) * 8;
            const int col = j * 16 + (lane >> 4) * 8;
            ldsm_x4_t(b, sB + row * (BN + 8) + col);
            mma_bf16(acc[2 * j], a, b[0], b[1]);
            mma_bf16(acc[2 * j + 1], a, b[2], b[3]);
        }
    }
}

// Loads rows [k0, k0 + kBK) x columns [n0, n0 + BN) of a [Kpad][Npad] bfloat16
// weight matrix (Kpad a multiple of kBK, Npad a multiple of BN).
template <int BN>
__device__ __forceinline__ void load_weights(__nv_bfloat16* sB, const __nv_bfloat16* Wt, int Npad, int k0, int n0)
{
    constexpr int CH = BN / 8;
    for (int i = threadIdx.x; i < kBK * CH; i += kThreads) {
        const int r = i / CH, c = i % CH;
        *reinterpret_cast<uint4*>(sB + r * (BN + 8) + c * 8) =
            *reinterpret_cast<const uint4*>(Wt + (size_t)(k0 + r) * Npad + n0 + c * 8);
    }
}

// Convolution as GEMM: out[v][n] (n < N) = sum_k A[v][k] Wt[k][n] (+ bias,
// times the device scalar *oscale when given, ReLU).  Kvalid = 27 C; Wt is
// [Kpad][Npad] with zero rows k >= Kvalid.  OutT = __nv_bfloat16 (stored
// activations) or float.  Split K (part != null): blockIdx.z takes
// k in [z kl, (z + 1) kl) and writes its FP32 sums to part[z][v][n], which
// k_splitk_finish adds in split order before the epilogue.
template <int BN, class OutT>
__global__ void __launch_bounds__(kThreads) k_conv(ConvSrc src, const __nv_bfloat16* __restrict__ Wt, int Kpad,
                                                   int Npad, int N, const float* __restrict__ bias, int relu,
                                                   const float* __restrict__ oscale, OutT* __restrict__ out,
                                                   int kl, float* __restrict__ part)
{
    __shared__ __align__(16) __nv_bfloat16 sA[kBM * (kBK + 8)];
    __shared__ __align__(16) __nv_bfloat16 sB[kBK * (BN + 8)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long V = (long long)src.D * src.H * src.W;
    const long long m0 = (long long)blockIdx.x * kBM;
    const int n0 = blockIdx.y * BN;
    const int Kvalid = 27 * src.C;
    const bool vec = (src.C % 8) == 0 && !src.f32;
    float acc[BN / 8][4];
#pragma unroll
    for (int t = 0; t < BN / 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    const int kbeg = blockIdx.z * kl, kend = kbeg + kl < Kpad ? kbeg + kl : Kpad;
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
        if (vec) {
            for (int i = threadIdx.x; i < kBM * (kBK / 8); i += kThreads) {
                const int r = i / (kBK / 8), c = i % (kBK / 8);
                const long long v = m0 + r;
                const int k = k0 + c * 8;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (v < V && k < Kvalid) {
                    const int x = (int)(v % src.W), y = (int)((v / src.W) % src.H), z = (int)(v / ((long long)src.W * src.H));
                    val = gather8(src, z, y, x, k);
                }
                *reinterpret_cast<uint4*>(sA + r * (kBK + 8) + c * 8) = val;
            }
        } else {
            for (int i = threadIdx.x; i < kBM * kBK; i += kThreads) {
                const int r = i / kBK, c = i % kBK;
                const long long v = m0 + r;
                const int k = k0 + c;
                float val = 0.f;
                if (v < V && k < Kvalid) {
                    const int x = (int)(v % src.W), y = (int)((v / src.W) % src.H), z = (int)(v / ((long long)src.W * src.H));
                    val = gather1(src, z, y, x, k);
                }
                sA[r * (kBK + 8) + c] = __float2bfloat16(val);
            }
        }
        load_weights<BN>(sB, Wt, Npad, k0, n0);
        __syncthreads();
        mma_stage<BN, false>(sA, sB, acc, warp, lane);
        __syncthreads();
    }
    // epilogue: fragment (row lane/4 [+8], columns 2 (lane%4) + {0, 1})
    if (part) {
        float* P = part + (size_t)blockIdx.z * V * N;
#pragma unroll
        for (int t = 0; t < BN / 8; ++t)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long v = m0 + 16 * warp + (lane >> 2) + 8 * h;
                if (v >= V) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int n = n0 + t * 8 + 2 * (lane & 3) + e;
                    if (n < N) P[v * N + n] = acc[t][2 * h + e];
                }
            }
        return;
    }
    const float osc = oscale ? *oscale : 1.f;
#pragma unroll
    for (int t = 0; t < BN / 8; ++t) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long v = m0 + 16 * warp + (lane >> 2) + 8 * h;
            if (v >= V) continue;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = n0 + t * 8 + 2 * (lane & 3) + e;
                if (n >= N) continue;
                float val = (acc[t][2 * h + e] + (bias ? bias[n] : 0.f)) * osc;
                if (relu) val = fmaxf(val, 0.f);
                if constexpr (sizeof(OutT) == 2)
                    out[v * N + n] = __float2bfloat16(val);
                else
                    out[v * N + n] = val;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled convolution: one CTA per 8 x 4 x 4 output block.  The block's input
// halo (10 x 6 x 6 voxels, all C channels) and the whole weight matrix are
// staged in shared memory once; the GEMM operand for tap t is then the halo
// shifted by t, read by ldmatrix with one row address per lane, so each
// input voxel leaves global memory about 2.8 times per block instead of 27.
// Halo voxels are padded to C + 8 elements (16 bytes) so that the eight
// rows an ldmatrix reads fall in distinct banks.  C = 1 (the network input,
// or a one-channel gradient) builds the 128 x 32 operand explicitly instead.
constexpr int kTX = 8, kTY = 4, kTZ = 4;
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2, kHV = kHX * kHY * kHZ;

template <int C>
__host__ __device__ constexpr int halo_stride() { return C == 1 ? 1 : C + 8; }

// Shared-memory bytes of k_conv_tile<C, BN> for a weight matrix of Kpad rows
// (weights, two halo buffers, a zero row, and for C == 1 the explicit
// operand tile).
template <int C, int BN>
constexpr size_t tile_smem(int Kpad)
{
    return sizeof(__nv_bfloat16) * ((size_t)Kpad * (BN + 8) + 2 * (((kHV * halo_stride<C>() + 7) / 8) * 8) + 8 +
                                    (C == 1 ? kBM * (kBK + 8) : 0));
}

// Halo elements a thread carries between tiles: uint4 (8 channels) for
// C >= 8, one value for C == 1.
template <int C>
struct HaloRegs {
    static constexpr int kItems = (C == 1) ? kHV : kHV * (C / 8);
    static constexpr int kPer = (kItems + kThreads - 1) / kThreads;
    uint4 v[kPer];
};

__device__ __forceinline__ void tile_origin(const ConvSrc& s, int t, int& x0, int& y0, int& z0)
{
    const int tilesX = (s.W + kTX - 1) / kTX, tilesY = (s.H + kTY - 1) / kTY;
    x0 = (t % tilesX) * kTX;
    t /= tilesX;
    y0 = (t % tilesY) * kTY;
    z0 = (t / tilesY) * kTZ;
}

// Global -> registers: the halo of the tile at (x0, y0, z0), zero outside,
// the skip addend summed and rounded as a stored sum would be.
template <int C>
__device__ __forceinline__ void halo_fetch(const ConvSrc& src, int x0, int y0, int z0, HaloRegs<C>& h)
{
    const int Hs = src.up ? (src.H >> 1) : src.H, Ws = src.up ? (src.W >> 1) : src.W;
#pragma unroll
    for (int j = 0; j < HaloRegs<C>::kPer; ++j) {
        const int i = threadIdx.x + j * kThreads;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (i < HaloRegs<C>::kItems) {
            const int hv = (C == 1) ? i : i / (C / 8), c8 = (C == 1) ? 0 : i % (C / 8);
            const int hx = hv % kHX, hy = (hv / kHX) % kHY, hz = hv / (kHX * kHY);
            const int z = z0 - 1 + hz, y = y0 - 1 + hy, x = x0 - 1 + hx;
            if (z >= 0 && z < src.D && y >= 0 && y < src.H && x >= 0 && x < src.W) {
                const size_t vox = src.up ? ((size_t)(z >> 1) * Hs + (y >> 1)) * Ws + (x >> 1)
                                          : ((size_t)z * src.H + y) * src.W + x;
                if constexpr (C == 1) {
                    float v;
                    if (src.f32) {
                        v = src.f32[((size_t)z * src.H + y) * src.W + x] * (src.f32_scale ? *src.f32_scale : 1.f);
                    } else {
                        v = bf2f(src.a[vox]);
                        if (src.b) v = bf2f(__float2bfloat16(v + bf2f(src.b[vox])));
                    }
                    r.x = __float_as_uint(v);
                } else {
                    const size_t off = vox * C + c8 * 8;
                    r = *reinterpret_cast<const uint4*>(src.a + off);
                    if (src.b) {
                        const uint4 q = *reinterpret_cast<const uint4*>(src.b + off);
                        __nv_bfloat162* pr = reinterpret_cast<__nv_bfloat162*>(&r);
                        const __nv_bfloat162* pq = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 u = __bfloat1622float2(pr[e]), w = __bfloat1622float2(pq[e]);
                            pr[e] = __floats2bfloat162_rn(u.x + w.x, u.y + w.y);
                        }
                    }
                }
            }
        }
        h.v[j] = r;
    }
}

// Registers -> one halo buffer.
template <int C>
__device__ __forceinline__ void halo_store(__nv_bfloat16* sH, const HaloRegs<C>& h)
{
    constexpr int CS = halo_stride<C>();
#pragma unroll
    for (int j = 0; j < HaloRegs<C>::kPer; ++j) {
        const int i = threadIdx.x + j * kThreads;
        if (i >= HaloRegs<C>::kItems) continue;
        if constexpr (C == 1) {
            sH[i] = __float2bfloat16(__uint_as_float(h.v[j].x));
        } else {
            const int hv = i / (C / 8), c8 = i % (C / 8);
            *reinterpret_cast<uint4*>(sH + hv * CS + c8 * 8) = h.v[j];
        }
    }
}

// Persistent: each CTA stages the weight matrix once and walks output
// blocks blockIdx.x, blockIdx.x + gridDim.x, ...; while it multiplies one
// block, the next block's halo is in flight to registers, and lands in the
// other halo buffer afterwards.
template <int C, int BN, class OutT>
__global__ void __launch_bounds__(kThreads, 2) k_conv_tile(ConvSrc src, const __nv_bfloat16* __restrict__ Wt, int Kpad,
                                                        int Npad, int N, const float* __restrict__ bias, int relu,
                                                        const float* __restrict__ oscale, OutT* __restrict__ out,
                                                        int ntiles)
{
    extern __shared__ __align__(16) unsigned char tile_raw[];
    constexpr int CS = halo_stride<C>();
    constexpr int HB = ((kHV * CS + 7) / 8) * 8;
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(tile_raw);   // [Kpad][BN + 8]
    __nv_bfloat16* sH0 = sW + (size_t)Kpad * (BN + 8);                 // two [kHV][CS] buffers
    __nv_bfloat16* sZ = sH0 + 2 * HB;                                  // 8 zeros
    __nv_bfloat16* sA = sZ + 8;                                        // C == 1: [kBM][kBK + 8]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * BN;
    const int sgn = src.flip ? -1 : 1;
    const float osc = oscale ? *oscale : 1.f;

    for (int i = threadIdx.x; i < Kpad * (BN / 8); i += kThreads) {
        const int r = i / (BN / 8), c = i % (BN / 8);
        *reinterpret_cast<uint4*>(sW + r * (BN + 8) + c * 8) =
            *reinterpret_cast<const uint4*>(Wt + (size_t)r * Npad + n0 + c * 8);
    }
    if (threadIdx.x < 8) sZ[threadIdx.x] = __float2bfloat16(0.f);
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    HaloRegs<C> h;
    int x0, y0, z0;
    tile_origin(src, tile, x0, y0, z0);
    halo_fetch<C>(src, x0, y0, z0, h);
    halo_store<C>(sH0, h);
    __syncthreads();
    int cur = 0;
    // this thread's fragment row
    const int m = 16 * warp + (lane & 15);
    const int hc = ((m / (kTX * kTY) + 1) * kHY + ((m / kTX) % kTY + 1)) * kHX + (m % kTX + 1);
    for (;;) {
        const int next = tile + gridDim.x;
        int nx0 = 0, ny0 = 0, nz0 = 0;
        if (next < ntiles) {
            tile_origin(src, next, nx0, ny0, nz0);
            halo_fetch<C>(src, nx0, ny0, nz0, h);
        }
        const __nv_bfloat16* sH = sH0 + cur * HB;
        float acc[BN / 8][4];
#pragma unroll
        for (int q = 0; q < BN / 8; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        if constexpr (C == 1) {
            for (int i = threadIdx.x; i < kBM * kBK; i += kThreads) {
                const int mm = i / kBK, k = i % kBK;
                __nv_bfloat16 v = __float2bfloat16(0.f);
                if (k < 27) {
                    const int tx = mm % kTX, ty = (mm / kTX) % kTY, tz = mm / (kTX * kTY);
                    const int dz = sgn * (k / 9 - 1), dy = sgn * ((k / 3) % 3 - 1), dx = sgn * (k % 3 - 1);
                    v = sH[((tz + 1 + dz) * kHY + (ty + 1 + dy)) * kHX + (tx + 1 + dx)];
                }
                sA[mm * (kBK + 8) + k] = v;
            }
            __syncthreads();
            mma_stage<BN, false>(sA, sW, acc, warp, lane);
        } else {
            const int KS = Kpad / 16;
            for (int ks = 0; ks < KS; ++ks) {
                const int k = ks * 16 + (lane >> 4) * 8;
                const int tap = k / C, ch = k % C;
                const __nv_bfloat16* pa = sZ;
                if (tap < 27) {
                    const int dz = sgn * (tap / 9 - 1), dy = sgn * ((tap / 3) % 3 - 1), dx = sgn * (tap % 3 - 1);
                    pa = sH + (hc + (dz * kHY + dy) * kHX + dx) * CS + ch;
                }
                uint32_t a[4];
                ldsm_x4(a, pa);
#pragma unroll
                for (int j = 0; j < BN / 16; ++j) {
                    uint32_t b[4];
                    const int row = ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                    const int col = j * 16 + (lane >> 4) * 8;
                    ldsm_x4_t(b, sW + row * (BN + 8) + col);
                    mma_bf16(acc[2 * j], a, b[0], b[1]);
                    mma_bf16(acc[2 * j + 1], a, b[2], b[3]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < BN / 8; ++q) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int mm = 16 * warp + (lane >> 2) + 8 * hh;
                const int x = x0 + mm % kTX, y = y0 + (mm / kTX) % kTY, z = z0 + mm / (kTX * kTY);
                if (x >= src.W || y >= src.H || z >= src.D) continue;
                const long long v = ((long long)z * src.H + y) * src.W + x;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int n = n0 + q * 8 + 2 * (lane & 3) + e;
                    if (n >= N) continue;
                    float val = (acc[q][2 * hh + e] + (bias ? bias[n] : 0.f)) * osc;
                    if (relu) val = fmaxf(val, 0.f);
                    if constexpr (sizeof(OutT) == 2)
                        out[v * N + n] = __float2bfloat16(val);
                    else
                        out[v * N + n] = val;
                }
            }
        }
        if (next >= ntiles) break;
        // the other buffer was last read two tiles ago, before the previous barrier
        halo_store<C>(sH0 + (cur ^ 1) * HB, h);
        __syncthreads();
        cur ^= 1;
        tile = next;
        x0 = nx0;
        y0 = ny0;
        z0 = nz0;
    }
}

// out[v][n] = epilogue(sum over the S splits, in order, of part[z][v][n]).
template <class OutT>
__global__ void k_splitk_finish(const float* __restrict__ part, int S, long long VN, int N,
                                const float* __restrict__ bias, int relu, const float* __restrict__ oscale,
                                OutT* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= VN) return;
    float a = 0.f;
    for (int z = 0; z < S; ++z) a += part[(size_t)z * VN + i];
    const int n = (int)(i % N);
    float val = (a + (bias ? bias[n] : 0.f)) * (oscale ? *oscale : 1.f);
    if (relu) val = fmaxf(val, 0.f);
    if constexpr (sizeof(OutT) == 2)
        out[i] = __float2bfloat16(val);
    else
        out[i] = val;
}

// Weight gradient, split over voxel chunks: part[chunk][k][n] =
// sum over the chunk's voxels of A[v][k] dY[v][n] (k < Kpad, n < N, dY is
// [V][N] bfloat16).  Grid (Kpad / kBM rounded up, chunks, N / BN rounded
// up): blockIdx.z takes outputs n0 = BN blockIdx.z .. n0 + BN - 1.
template <int BN>
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(ConvSrc src, const __nv_bfloat16* __restrict__ dY, int N,
                                                         int Kpad, float* __restrict__ part)
{
    __shared__ __align__(16) __nv_bfloat16 sA[kBK * (kBM + 8)];   // [v][k]
    __shared__ __align__(16) __nv_bfloat16 sB[kBK * (BN + 8)];    // [v][n]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long V = (long long)src.D * src.H * src.W;
    const int k0 = blockIdx.x * kBM, n0 = blockIdx.z * BN;
    const long long v0 = (long long)blockIdx.y * kWChunk;
    const long long v1 = v0 + kWChunk < V ? v0 + kWChunk : V;
    const int Kvalid = 27 * src.C;
    const bool vec = (src.C % 8) == 0 && !src.f32;
    const bool vecy = (N % 8) == 0;
    float acc[BN / 8][4];
#pragma unroll
    for (int t = 0; t < BN / 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    for (long long vb = v0; vb < v1; vb += kBK) {
        if (vec) {
            for (int i = threadIdx.x; i < kBK * (kBM / 8); i += kThreads) {
                const int r = i / (kBM / 8), c = i % (kBM / 8);
                const long long v = vb + r;
                const int k = k0 + c * 8;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (v < v1 && k < Kvalid) {
                    const int x = (int)(v % src.W), y = (int)((v / src.W) % src.H), z = (int)(v / ((long long)src.W * src.H));
                    val = gather8(src, z, y, x, k);
                }
                *reinterpret_cast<uint4*>(sA + r * (kBM + 8) + c * 8) = val;
            }
        } else {
            for (int i = threadIdx.x; i < kBK * kBM; i += kThreads) {
                const int r = i / kBM, c = i % kBM;
                const long long v = vb + r;
                const int k = k0 + c;
                float val = 0.f;
                if (v < v1 && k < Kvalid) {
                    const int x = (int)(v % src.W), y = (int)((v / src.W) % src.H), z = (int)(v / ((long long)src.W * src.H));
                    val = gather1(src, z, y, x, k);
                }
                sA[r * (kBM + 8) + c] = __float2bfloat16(val);
            }
        }
        if (vecy) {
            for (int i = threadIdx.x; i < kBK * (BN / 8); i += kThreads) {
                const int r = i / (BN / 8), c = i % (BN / 8);
                const long long v = vb + r;
                uint4 val = make_uint4(0, 0, 0, 0);
                if (v < v1 && n0 + c * 8 < N) val = *reinterpret_cast<const uint4*>(dY + v * N + n0 + c * 8);
                *reinterpret_cast<uint4*>(sB + r * (BN + 8) + c * 8) = val;
            }
        } else {
            for (int i = threadIdx.x; i < kBK * BN; i += kThreads) {
                const int r = i / BN, c = i % BN;
                const long long v = vb + r;
                sB[r * (BN + 8) + c] = (v < v1 && n0 + c < N) ? dY[v * N + n0 + c] : __float2bfloat16(0.f);
            }
        }
        __syncthreads();
        mma_stage<BN, true>(sA, sB, acc, warp, lane);
        __syncthreads();
    }
    float* P = part + (size_t)blockIdx.y * Kpad * N;
#pragma unroll
    for (int t = 0; t < BN / 8; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + 16 * warp + (lane >> 2) + 8 * h;
            if (k >= Kpad) continue;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = n0 + t * 8 + 2 * (lane & 3) + e;
                if (n < N) P[(size_t)k * N + n] = acc[t][2 * h + e];
            }
        }
}

// grad[n][k] (k < Kvalid: the parameter layout W[co][tap][ci]) = sum over
// chunks, in chunk order, of part[chunk][k][n].
__global__ void k_wgrad_reduce(const float* __restrict__ part, int chunks, int Kpad, int Kvalid, int N,
                               float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kvalid * N) return;
    const int k = i / N, n = i % N;
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += part[((size_t)c * Kpad + k) * N + n];
    grad[(size_t)n * Kvalid + k] = s;
}

// Bias gradient: part[b][n] = sum over block b's voxels of dY[v][n]; then
// grad[n] = sum over blocks in order.  The block reads its chunk of dY as one
// contiguous run: thread t (t < per, per the largest multiple of N within
// the block) always lands on channel t % N, and the threads of a channel are
// combined in thread order.
__global__ void k_bias_part(const __nv_bfloat16* __restrict__ dY, long long V, int N, float* __restrict__ part)
{
    __shared__ float red[kThreads];
    const long long v0 = (long long)blockIdx.x * kWChunk;
    const long long v1 = v0 + kWChunk < V ? v0 + kWChunk : V;
    const int per = (kThreads / N) * N;
    float s = 0.f;
    if ((int)threadIdx.x < per)
        for (long long i = v0 * N + threadIdx.x; i < v1 * N; i += per) s += bf2f(dY[i]);
    red[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < N) {
        float t = 0.f;
        for (int j = threadIdx.x; j < per; j += N) t += red[j];
        part[(size_t)blockIdx.x * N + threadIdx.x] = t;
    }
}

__global__ void k_bias_reduce(const float* __restrict__ part, int blocks, int N, float* __restrict__ grad)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < blocks; ++b) s += part[(size_t)b * N + n];
    grad[n] = s;
}

// 2x2x2 mean pool of [D][H][W][C] (D, H, W even) into [D/2][H/2][W/2][C].
__global__ void k_pool(const __nv_bfloat16* __restrict__ in, int D, int H, int W, int C,
                       __nv_bfloat16* __restrict__ out)
{
    const long long n = (long long)(D / 2) * (H / 2) * (W / 2) * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % (W / 2));
    v /= (W / 2);
    const int y = (int)(v % (H / 2));
    const int z = (int)(v / (H / 2));
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                s += bf2f(in[(((size_t)(2 * z + a) * H + (2 * y + b)) * W + (2 * x + e)) * C + c]);
    out[i] = __float2bfloat16(s * 0.125f);
}

// g[v][c] = skip[v][c] + gp[parent(v)][c] / 8: gradient of a volume that
// feeds both a 2x2x2 mean pool (gradient gp) and an additive skip (skip).
__global__ void k_pool_grad_add(const __nv_bfloat16* __restrict__ skip, const __nv_bfloat16* __restrict__ gp, int D,
                                int H, int W, int C, __nv_bfloat16* __restrict__ g)
{
    const long long n = (long long)D * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % W);
    v /= W;
    const int y = (int)(v % H);
    const int z = (int)(v / H);
    const size_t pi = (((size_t)(z >> 1) * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1)) * C + c;
    g[i] = __float2bfloat16(bf2f(skip[i]) + bf2f(gp[pi]) * 0.125f);
}

// Gradient of a nearest x2 upsampling: g[z][y][x][c] = sum of the 8 children
// of fine-grid gradient gf ([2D][2H][2W][C]).
__global__ void k_up_grad(const __nv_bfloat16* __restrict__ gf, int D, int H, int W, int C,
                          __nv_bfloat16* __restrict__ g)
{
    const long long n = (long long)D * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    long long v = i / C;
    const int x = (int)(v % W);
    v /= W;
    const int y = (int)(v % H);
    const int z = (int)(v / H);
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int e = 0; e < 2; ++e)
                s += bf2f(gf[(((size_t)(2 * z + a) * (2 * H) + (2 * y + b)) * (2 * W) + (2 * x + e)) * C + c]);
    g[i] = __float2bfloat16(s);
}

// out = g where y > 0 else 0 (ReLU gradient; g itself is kept, a skip may
// need it unmasked).
__global__ void k_relu_grad(__nv_bfloat16* __restrict__ out, const __nv_bfloat16* __restrict__ g,
                            const __nv_bfloat16* __restrict__ y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = bf2f(y[i]) > 0.f ? g[i] : __float2bfloat16(0.f);
}

// Loss sum((out - t)^2) / (2 V) per block in FP64 partials; gradient
// g = (out - t) / V as bfloat16.  The target is multiplied by the device
// scalar *tscale when given.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ t, const float* __restrict__ tscale,
                      long long V, __nv_bfloat16* __restrict__ g, double* __restrict__ part)
{
    __shared__ double red[kThreads];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < V) {
        const float d = out[i] - t[i] * (tscale ? *tscale : 1.f);
        g[i] = __float2bfloat16(d / (float)V);
        s = (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] / (2.0 * (double)V);
}

// Per-block FP64 partial sums of in[i]^2.
__global__ void k_sumsq_part(const float* __restrict__ in, long long V, double* __restrict__ part)
{
    __shared__ double red[kThreads];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        const double v = in[i];
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// r = RMS of the input from the partials (in block order); scales =
// {1 / r, r gain, 1 / (r gain)} (r = 1 for an all-zero input).
__global__ void k_scales(const double* __restrict__ part, int nb, long long V, float gain, float* __restrict__ scales)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    double r = sqrt(s / (double)V);
    if (!(r > 0.0)) r = 1.0;
    scales[0] = (float)(1.0 / r);
    scales[1] = (float)(r * gain);
    scales[2] = (float)(1.0 / (r * gain));
}

// Wt[k][n] (forward) = W[n][k] for k < 27 Cin, n < Cout; zero padding.
// With transpose_io (gradient w.r.t. the input): k = tap * Cout + co,
// n = ci, Wt[k][n] = W[co][tap][ci].
__global__ void k_prep_weights(const float* __restrict__ W, int Cin, int Cout, int Kpad, int Npad, int transpose_io,
                               __nv_bfloat16* __restrict__ Wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kpad * Npad) return;
    const int k = i / Npad, n = i % Npad;
    float v = 0.f;
    if (!transpose_io) {
        if (k < 27 * Cin && n < Cout) v = W[(size_t)n * 27 * Cin + k];
    } else {
        if (k < 27 * Cout && n < Cin) {
            const int tap = k / Cout, co = k % Cout;
            v = W[((size_t)co * 27 + tap) * Cin + n];
        }
    }
    Wt[i] = __float2bfloat16(v);
}

// Adam (FP32 master weights): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace unet
}  // namespace mh3d
