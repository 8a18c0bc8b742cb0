// 3x3x3 convolutions of the warm-start network on the fifth-generation
// tensor cores: tcgen05.mma (kind::f16, bfloat16 operands, FP32
// accumulation) reading both operands from shared memory through matrix
// descriptors and accumulating in tensor memory (TMEM); the epilogue reads
// the accumulators back with tcgen05.ld.
//
// The GEMM of one output tile.  A tile is R x rows of 128 consecutive
// voxels (z, y0 + r, x0 .. x0 + 127), r < R; row r's accumulator
// D_r[128][NP] (FP32, NP >= N output channels, a multiple of 16) lives in
// TMEM columns r NP .. r NP + NP - 1, lane m = voxel x0 + m.  For every row,
// tap (dz, dy, dx) and 16 input channels
//     D_r[m][n] += sum_{c < 16} in[z + dz][y0 + r + dy][x0 + m + dx][c] W[n][tap][c]
// is one tcgen05.mma with M = 128, N = NP, K = 16.
//
// Operand layout (no swizzle, K-major canonical layout: 8 rows x 16 bytes
// per core matrix, rows 16 bytes apart, core matrices along M 128 bytes
// apart, along K `LBO` bytes apart):
//   halo: the tile's 3 x (R + 2) neighbouring x rows, x0 - 1 .. x0 + 128,
//         staged as planes [chunk of 8 channels][dz][dy][kHP voxels][8]: a
//         plane is 136 x 16 bytes, so the A operand of tap (dz, dy, dx) for
//         row r is the plane (dz, r + dy) started dx + 1 rows in -- a
//         descriptor offset, no data movement -- and the tap's second 8
//         channels sit 3 (R + 2) planes on;
//   weights: [tap][chunk][NP][8], the B operand of (tap, chunk pair) one
//         descriptor, its second 8 channels NP rows on.
// Chunks are padded to an even count with zeros (8 channels: one zero
// chunk; the FP32 single-channel network input: channel 0 of chunk 0).
//
// Persistent CTAs of 128 threads: the weights are staged once; per tile the
// threads stage the halo (bounds, the nearest x2 upsampling and the rounded
// skip sum of the decoder inputs are applied here, as in the mma.sync
// kernel; stage_halo), one thread issues the 27 x (chunks / 2) MMAs and commits them to
// an mbarrier, and the four warps read their 32 TMEM lanes each.  The wait
// on the mbarrier is bounded (%globaltimer): on expiry the CTA records
// MH3D_ERR_TIMEOUT in *status, frees its TMEM and returns.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bulk.cuh"
#include "unet_kernels.cuh"

namespace mh3d {
namespace unet {
namespace umma {

constexpr int kM = 128;       // voxels per tile (TMEM lanes)
constexpr int kHP = 136;      // voxels per staged plane (130 used; 136 x 16 B = 17 x 128 B)
// R output rows per tile (y0 .. y0 + R - 1) share the staged planes: 3 dz
// x (R + 2) dy neighbour rows.
template <int R>
constexpr int planes() { return 3 * (R + 2); }
constexpr int kT = 128;       // threads per CTA

// NB halo buffers and accumulators (2: the next tile's halo is staged and
// the previous tile's epilogue runs while this tile's MMAs execute).
template <int C8P, int NP, int NB, int R = 1>
struct Geom {
    static_assert(C8P % 2 == 0 && NP % 16 == 0 && NP >= 16 && NP <= 128 && (NB == 1 || NB == 2), "operand shape");
    static_assert(R == 1 || (NB == 1 && (R == 2 || R == 4)), "rows per tile");
    static constexpr int kPl = planes<R>();
    static constexpr int kWBytes = 27 * C8P * NP * 16;
    static constexpr int kHBytes = C8P * kPl * kHP * 16;       // one halo buffer
    static constexpr int kAcc = NB * R * NP;                   // TMEM columns used
    static constexpr int kCols = kAcc <= 32 ? 32 : (kAcc <= 64 ? 64 : (kAcc <= 128 ? 128 : 256));   // allocated
    static constexpr size_t smem() { return 1024 + (size_t)kWBytes + (size_t)NB * kHBytes; }
};

// ---- tcgen05 primitives (inline PTX) ----------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) (+)= A (smem) B (smem); accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives once on the mbarrier when every MMA this thread issued so far has
// completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes (lane i: TMEM lane
// base + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D (bits 4-5 = 1), bfloat16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16
// at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- staging ---------------------------------------------------------------

// Asynchronous 16-byte copy global -> shared (cp.async, L2 only); src_bytes
// 0 fills the 16 bytes with zeros without reading.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stages the tile's halo: 16-byte units, channels 8 c .. 8 c + 7 of voxel
// (z + dz, y + dy, x0 - 1 + xi), zero outside the volume.  Only the cv
// chunks that carry channels are written (the padding chunks stay zero from
// the kernel's start).  Each thread takes whole voxels.  Plain and
// upsampled bfloat16 sources: one cp.async per unit, all in flight at once.
// The skip sum (rounded to bfloat16, as a stored sum would be; not
// upsampled) and the FP32 input (rounded to bfloat16, channel 0) need
// arithmetic: their units are loaded into registers in batches (all loads
// of a batch in flight), combined and stored.
template <int C8P, int R>
__device__ __forceinline__ void stage_halo(const ConvSrc& src, unsigned char* sH, int z, int y, int x0, int cv,
                                           int tid = threadIdx.x, int nthr = kT)
{
    constexpr int PL = planes<R>();
    constexpr int NV = PL * 130;
    constexpr size_t CST = (size_t)PL * kHP * 16;   // bytes between chunk planes
    auto voxel = [&](int vi, unsigned char*& d, long long& off) {
        const int plane = vi / 130, xi = vi - plane * 130;
        const int zz = z + plane / (R + 2) - 1, yy = y + plane % (R + 2) - 1, xx = x0 + xi - 1;
        d = sH + ((size_t)plane * kHP + xi) * 16;
        const bool in = zz >= 0 && zz < src.D && yy >= 0 && yy < src.H && xx >= 0 && xx < src.W;
        if (!in) {
            off = -1;
        } else if (src.up) {
            off = (((long long)(zz >> 1) * (src.H >> 1) + (yy >> 1)) * (src.W >> 1) + (xx >> 1)) * src.C;
        } else {
            off = (((long long)zz * src.H + yy) * src.W + xx) * (src.f32 ? 1 : src.C);
        }
    };
    if (!src.b && !src.f32) {
        for (int vi = tid; vi < NV; vi += nthr) {
            unsigned char* d;
            long long off;
            voxel(vi, d, off);
            const __nv_bfloat16* g = off >= 0 ? src.a + off : src.a;
#pragma unroll
            for (int c = 0; c < C8P; ++c)
                if (c < cv) cp_async16(d + c * CST, g + 8 * c, off >= 0 ? 16u : 0u);
        }
        return;   // the caller waits (cp_async_wait_all) before the halo is read
    }
    if (src.f32) {
        constexpr int kB = 8;
        const float fsc = src.f32_scale ? *src.f32_scale : 1.f;
        for (int v0 = tid; v0 < NV; v0 += kB * nthr) {
            unsigned char* d[kB];
            long long off[kB];
            float f[kB];
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                const int vi = v0 + i * nthr;
                if (vi < NV) voxel(vi, d[i], off[i]);
                else off[i] = -2;
            }
#pragma unroll
            for (int i = 0; i < kB; ++i) f[i] = off[i] >= 0 ? __ldg(src.f32 + off[i]) : 0.f;
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                if (off[i] == -2) continue;
                const __nv_bfloat16 b = __float2bfloat16(f[i] * fsc);
                *reinterpret_cast<uint4*>(d[i]) =
                    make_uint4(off[i] >= 0 ? (uint32_t)(*reinterpret_cast<const uint16_t*>(&b)) : 0u, 0, 0, 0);
            }
        }
        return;
    }
    constexpr int kB = 8 / C8P > 0 ? 8 / C8P : 1;   // voxels per batch: 8 chunk units
    for (int v0 = tid; v0 < NV; v0 += kB * nthr) {
        unsigned char* d[kB];
        long long off[kB];
        uint4 va[kB][C8P], vb[kB][C8P];
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int vi = v0 + i * nthr;
            if (vi < NV) voxel(vi, d[i], off[i]);
            else off[i] = -2;
        }
#pragma unroll
        for (int i = 0; i < kB; ++i)
#pragma unroll
            for (int c = 0; c < C8P; ++c) {
                const bool in = off[i] >= 0 && c < cv;
                va[i][c] = in ? __ldg(reinterpret_cast<const uint4*>(src.a + off[i] + 8 * c)) : make_uint4(0, 0, 0, 0);
                vb[i][c] = in ? __ldg(reinterpret_cast<const uint4*>(src.b + off[i] + 8 * c)) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            if (off[i] == -2) continue;
#pragma unroll
            for (int c = 0; c < C8P; ++c) {
                if (c >= cv) continue;
                __nv_bfloat162* pr = reinterpret_cast<__nv_bfloat162*>(&va[i][c]);
                const __nv_bfloat162* pq = reinterpret_cast<const __nv_bfloat162*>(&vb[i][c]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 a = __bfloat1622float2(pr[k]), b = __bfloat1622float2(pq[k]);
                    pr[k] = __floats2bfloat162_rn(a.x + b.x, a.y + b.y);
                }
                *reinterpret_cast<uint4*>(d[i] + c * CST) = va[i][c];
            }
        }
    }
}

// ---- the kernel --------------------------------------------------------------

// Epilogue of one tile: warp w holds TMEM lanes 32 w .. 32 w + 31 = voxels
// x0 + 32 w + lane, columns acc .. acc + NP - 1 = output channels.
template <int NP, class OutT>
__device__ __forceinline__ void epilogue(const ConvSrc& src, uint32_t acc, int z, int y, int x0, int N,
                                         const float* __restrict__ bias, int relu, float osc, OutT* __restrict__ out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = x0 + 32 * warp + lane;
    const long long v = ((long long)z * src.H + y) * src.W + x;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
        float a[16];
        tmem_ld16(acc + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, a);
        tmem_ld_wait();
        if (x >= src.W || y >= src.H) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = c0 + j;
            a[j] = (a[j] + ((bias && n < N) ? bias[n] : 0.f)) * osc;
            if (relu) a[j] = fmaxf(a[j], 0.f);
        }
        if constexpr (sizeof(OutT) == 2) {
            if (N % 8 == 0) {   // whole 16-byte groups of channels (the voxel's row is 16-byte aligned)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (c0 + 8 * h >= N) break;
                    uint4 pk;
                    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
                    for (int i = 0; i < 4; ++i) q[i] = __floats2bfloat162_rn(a[8 * h + 2 * i], a[8 * h + 2 * i + 1]);
                    *reinterpret_cast<uint4*>(out + v * N + c0 + 8 * h) = pk;
                }
                continue;
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = c0 + j;
            if (n >= N) break;
            if constexpr (sizeof(OutT) == 2)
                out[v * N + n] = __float2bfloat16(a[j]);
            else
                out[v * N + n] = a[j];
        }
    }
}

// The R x 27 x C8P / 2 MMAs of one tile (row r into the accumulator at
// column acc + r NP), committed to `bar` (one thread).
// The rows' MMAs are interleaved (tap by tap, each row in turn): an MMA's
// successor accumulates into another row's columns, so R chains of
// dependent MMAs are in flight instead of one.
//
// Paired taps (pair != 0; sources of at most 8 channels, whose second chunk
// is zero padding): one MMA takes two taps of the same (dz, dx) whose planes
// are neighbours -- plane offsets 0 and 1, the second chunk LBO = one plane
// on -- and a second MMA the third plane with a zero second chunk: 18 MMAs a
// row instead of 27.  The paired weights ([3 pz][3 px][2 g][2 c][NP][8],
// k_prep_umma_pair) are indexed by plane offsets, the flip folded in.
template <int C8P, int NP, int R>
__device__ __forceinline__ void issue_mmas(uint32_t acc, uint32_t sH_a, uint32_t sW_a, int sgn, uint64_t* bar,
                                           int pair = 0)
{
    constexpr uint32_t kIdesc = idesc_bf16(kM, NP);
    constexpr int PL = planes<R>();
    if (pair) {
        for (int pz = 0; pz < 3; ++pz)
            for (int px = 0; px < 3; ++px)
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const uint32_t b = sW_a + (uint32_t)((((pz * 3 + px) * 2 + g) * 2) * NP * 16);
                    const uint64_t bdesc = smem_desc(b, NP * 16, 128);
                    const uint32_t accumulate = (pz | px | g) != 0;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int plane = pz * (R + 2) + r + 2 * g;
                        const uint32_t a = sH_a + (uint32_t)((plane * kHP + px) * 16);
                        mma_f16(acc + (uint32_t)(r * NP), smem_desc(a, kHP * 16, 128), bdesc, kIdesc, accumulate);
                    }
                }
        mma_commit(bar);
        return;
    }
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = sgn * (tap / 9 - 1), dy = sgn * ((tap / 3) % 3 - 1), dx = sgn * (tap % 3 - 1);
#pragma unroll
        for (int ks = 0; ks < C8P / 2; ++ks) {
            const uint32_t b = sW_a + (uint32_t)((tap * C8P + 2 * ks) * NP * 16);
            const uint64_t bdesc = smem_desc(b, NP * 16, 128);
            const uint32_t accumulate = (tap | ks) != 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int plane = (dz + 1) * (R + 2) + (r + dy + 1);
                const uint32_t a = sH_a + (uint32_t)(((2 * ks * PL + plane) * kHP + dx + 1) * 16);
                mma_f16(acc + (uint32_t)(r * NP), smem_desc(a, PL * kHP * 16, 128), bdesc, kIdesc, accumulate);
            }
        }
    }
    mma_commit(bar);
}

// Wu: [27][C8P][NP][8] bfloat16 (k_prep_umma); out: [V][N] channels last.
template <int C8P, int NP, int NB, int R, class OutT>
__global__ void __launch_bounds__(kT) k_conv_umma(ConvSrc src, const __nv_bfloat16* __restrict__ Wu, int N,
                                                  const float* __restrict__ bias, int relu,
                                                  const float* __restrict__ oscale, OutT* __restrict__ out,
                                                  int ntiles, int* status, const __nv_bfloat16* __restrict__ Wpair)
{
    const int pair = (Wpair != nullptr && NB == 1) ? 1 : 0;   // paired taps (NB == 1 form only)
    using G = Geom<C8P, NP, NB, R>;
    extern __shared__ unsigned char umma_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_s;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(umma_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sW = base;                  // [27][C8P][NP][16 B]
    unsigned char* sH = base + G::kWBytes;     // NB x [C8P][9][kHP][16 B]
    const int warp = threadIdx.x >> 5;
    const int ntx = (src.W + kM - 1) / kM;
    const int sgn = src.flip ? -1 : 1;

    if (warp == 0) {
        tmem_alloc(&tmem_base_s, G::kCols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_barrier_init();
    }
    {
        const uint4* w4 = reinterpret_cast<const uint4*>(pair ? Wpair : Wu);
        uint4* s4 = reinterpret_cast<uint4*>(sW);
        const int n16 = pair ? 9 * 2 * 2 * NP : G::kWBytes / 16;   // the paired layout is smaller
        for (int i = threadIdx.x; i < n16; i += kT) s4[i] = w4[i];
    }
    // chunks carrying channels; the padding chunks of every halo buffer are
    // zeroed once and never staged
    const int cv = src.f32 ? 1 : (src.C + 7) / 8;
    for (int nb = 0; nb < NB; ++nb) {
        uint4* h4 = reinterpret_cast<uint4*>(sH + (size_t)nb * G::kHBytes + (size_t)cv * G::kPl * kHP * 16);
        const int n16 = (C8P - cv) * G::kPl * kHP;
        for (int i = threadIdx.x; i < n16; i += kT) h4[i] = make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async_smem();   // generic-proxy writes -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t sW_a = smem_u32(sW), sH_a = smem_u32(sH);
    const float osc = oscale ? *oscale : 1.f;
    const int nyb = (src.H + R - 1) / R;   // row groups per z slice
    auto origin = [&](int tile, int& z, int& y, int& x0) {
        const int tx = tile % ntx, row = tile / ntx;
        y = (row % nyb) * R;
        z = row / nyb;
        x0 = tx * kM;
    };

    if constexpr (NB == 1) {
        uint32_t phase = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            int z, y, x0;
            origin(tile, z, y, x0);
            stage_halo<C8P, R>(src, sH, z, y, x0, cv);
            cp_async_wait_all();
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after();
                issue_mmas<C8P, NP, R>(tmem, sH_a, sW_a, sgn, &mbar[0], pair);
            }
            // one thread waits on the MMAs' mbarrier; the block barrier
            // releases the others (no spinning warps taking issue slots)
            const bool ok = __syncthreads_and(threadIdx.x != 0 || mbar_wait(&mbar[0], phase, status));
            phase ^= 1;
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int r = 0; r < R; ++r) epilogue<NP>(src, tmem + (uint32_t)(r * NP), z, y + r, x0, N, bias, relu, osc, out);
            tc_fence_before();
            __syncthreads();   // TMEM read and halo consumed before the next tile reuses both
        }
    } else {
        // iteration i: the MMAs of tile i (halo and accumulator i & 1) run
        // while the threads stage tile i + 1 and write tile i - 1 out
        int tile = blockIdx.x, pz = 0, py = 0, px0 = 0;
        if (tile < ntiles) {
            int z, y, x0;
            origin(tile, z, y, x0);
            stage_halo<C8P, 1>(src, sH, z, y, x0, cv);
        }
        for (int i = 0; tile < ntiles; ++i, tile += gridDim.x) {
            const int b = i & 1;
            int z, y, x0;
            origin(tile, z, y, x0);
            cp_async_wait_all();
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after();
                issue_mmas<C8P, NP, 1>(tmem + (uint32_t)(b * NP), sH_a + (uint32_t)(b * G::kHBytes), sW_a, sgn,
                                       &mbar[b]);
            }
            if (i > 0) {   // tile i - 1's MMAs: done before its halo buffer is refilled
                if (!__syncthreads_and(threadIdx.x != 0 || mbar_wait(&mbar[b ^ 1], ((i - 1) >> 1) & 1, status)))
                    break;
                tc_fence_after();
            }
            const int next = tile + gridDim.x;
            if (next < ntiles) {
                int nz, ny, nx0;
                origin(next, nz, ny, nx0);
                stage_halo<C8P, 1>(src, sH + (size_t)(b ^ 1) * G::kHBytes, nz, ny, nx0, cv);
            }
            if (i > 0) {
                epilogue<NP>(src, tmem + (uint32_t)((b ^ 1) * NP), pz, py, px0, N, bias, relu, osc, out);
                tc_fence_before();
            }
            if (next >= ntiles) {   // the last tile: wait for its MMAs and write it
                if (!__syncthreads_and(threadIdx.x != 0 || mbar_wait(&mbar[b], (i >> 1) & 1, status))) break;
                tc_fence_after();
                epilogue<NP>(src, tmem + (uint32_t)(b * NP), z, y, x0, N, bias, relu, osc, out);
                tc_fence_before();
            }
            pz = z;
            py = y;
            px0 = x0;
        }
    }
    cp_async_wait_all();   // no copy lands after the CTA has gone
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, G::kCols);
    }
}

// ---- the warp-specialised form ---------------------------------------------
//
// One persistent CTA per SM, three roles over the same tile sequence
// (tiles of one x row), linked by mbarriers:
//   warps 4-7 (producers) stage tile i's halo into ring slot i % NS, after
//     slot i % NS is released (empty: the MMAs of tile i - NS completed),
//     keeping NS - 1 tiles of cp.async copies in flight; when a tile's copies
//     have landed each producer thread fences them for the async proxy and
//     arrives on full[slot] (128 arrivals);
//   warp 8, lane 0 (MMA) waits for full[slot] and for the accumulator i % 2
//     to be drained (acce), issues the tile's MMAs and commits them to
//     empty[slot] and accf[i % 2];
//   warps 0-3 (epilogue) wait for accf, read their 32 TMEM lanes, store and
//     arrive on acce (one arrival per warp).
// So the staging of the next tiles, this tile's MMAs and the previous
// tile's epilogue overlap inside the CTA.  Every wait is bounded; a timeout
// records MH3D_ERR_TIMEOUT, sets the CTA's abort flag, and every role leaves
// its loop (at the latest after its own bounded wait) before TMEM is freed.
constexpr int kWsT = 288;   // 4 epilogue warps, 4 producer warps, 1 MMA warp

template <int C8P, int NP, int NS>
struct GeomWs {
    static_assert(C8P % 2 == 0 && NP % 16 == 0 && NP >= 16 && NP <= 64 && NS >= 2 && NS <= 4, "operand shape");
    static constexpr int kWBytes = 27 * C8P * NP * 16;
    static constexpr int kHBytes = C8P * planes<1>() * kHP * 16;
    static constexpr int kCols = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : 128);
    static constexpr size_t smem() { return 1024 + (size_t)kWBytes + (size_t)NS * kHBytes; }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_commit_wait()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The 27 x C8P / 2 MMAs of one row tile into the accumulator at column acc
// (no commit).
template <int C8P, int NP>
__device__ __forceinline__ void issue_mmas_row(uint32_t acc, uint32_t sH_a, uint32_t sW_a, int sgn)
{
    constexpr uint32_t kIdesc = idesc_bf16(kM, NP);
    constexpr int PL = planes<1>();
    uint32_t accumulate = 0;
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = sgn * (tap / 9 - 1), dy = sgn * ((tap / 3) % 3 - 1), dx = sgn * (tap % 3 - 1);
        const int plane = (dz + 1) * 3 + (dy + 1);
#pragma unroll
        for (int ks = 0; ks < C8P / 2; ++ks) {
            const uint32_t a = sH_a + (uint32_t)(((2 * ks * PL + plane) * kHP + dx + 1) * 16);
            const uint32_t b = sW_a + (uint32_t)((tap * C8P + 2 * ks) * NP * 16);
            mma_f16(acc, smem_desc(a, PL * kHP * 16, 128), smem_desc(b, NP * 16, 128), kIdesc, accumulate);
            accumulate = 1;
        }
    }
}

template <int C8P, int NP, int NS, class OutT>
__global__ void __launch_bounds__(kWsT, 1) k_conv_umma_ws(ConvSrc src, const __nv_bfloat16* __restrict__ Wu, int N,
                                                          const float* __restrict__ bias, int relu,
                                                          const float* __restrict__ oscale, OutT* __restrict__ out,
                                                          int ntiles, int* status)
{
    using G = GeomWs<C8P, NP, NS>;
    extern __shared__ unsigned char umma_raw[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], accf[2], acce[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_s;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(umma_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sW = base;
    unsigned char* sH = base + G::kWBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (src.W + kM - 1) / kM;
    const int sgn = src.flip ? -1 : 1;
    const bool async_src = !src.b && !src.f32;   // staged by cp.async
    const int cv = src.f32 ? 1 : (src.C + 7) / 8;

    if (warp == 8) {
        tmem_alloc(&tmem_base_s, G::kCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 128);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], 4);
        }
        abort_s = 0;
        fence_barrier_init();
    }
    {
        const uint4* w4 = reinterpret_cast<const uint4*>(Wu);
        uint4* s4 = reinterpret_cast<uint4*>(sW);
        for (int i = tid; i < G::kWBytes / 16; i += kWsT) s4[i] = w4[i];
        for (int nb = 0; nb < NS; ++nb) {   // padding chunks: zero once, never staged
            uint4* h4 = reinterpret_cast<uint4*>(sH + (size_t)nb * G::kHBytes + (size_t)cv * planes<1>() * kHP * 16);
            const int n16 = (C8P - cv) * planes<1>() * kHP;
            for (int i = tid; i < n16; i += kWsT) h4[i] = make_uint4(0, 0, 0, 0);
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t sW_a = smem_u32(sW), sH_a = smem_u32(sH);
    auto origin = [&](int tile, int& z, int& y, int& x0) {
        const int tx = tile % ntx, row = tile / ntx;
        y = row % src.H;
        z = row / src.H;
        x0 = tx * kM;
    };

    if (warp >= 4 && warp < 8) {
        // producers: slot of tile i is i % NS; its full arrival comes NS - 1
        // tiles later (async sources) or at once (register-staged sources)
        const int pt = tid - 128;
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int sl = i % NS, k = i / NS;
            if (k > 0 && !mbar_wait(&empty[sl], (k - 1) & 1, status)) abort_s = 1;
            if (abort_s) break;
            int z, y, x0;
            origin(tile, z, y, x0);
            stage_halo<C8P, 1>(src, sH + (size_t)sl * G::kHBytes, z, y, x0, cv, pt, 128);
            if (async_src) {
                cp_async_commit();
                if (i >= NS - 1) {   // tile i - (NS - 1) has landed
                    cp_async_wait_group<NS - 1>();
                    fence_proxy_async_smem();
                    mbar_arrive(&full[(i - (NS - 1)) % NS]);
                }
            } else {
                fence_proxy_async_smem();
                mbar_arrive(&full[sl]);
            }
        }
        // the copies still in flight: land them and arrive for their tiles
        cp_async_wait_all();
        if (async_src && !abort_s) {
            fence_proxy_async_smem();
            for (int j = i - (NS - 1) > 0 ? i - (NS - 1) : 0; j < i; ++j) mbar_arrive(&full[j % NS]);
        }
    } else if (warp == 8) {
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int sl = i % NS, k = i / NS, a = i & 1, ka = i >> 1;
                if (!mbar_wait(&full[sl], k & 1, status) ||
                    (ka > 0 && !mbar_wait(&acce[a], (ka - 1) & 1, status)))
                    abort_s = 1;
                if (abort_s) break;
                tc_fence_after();
                issue_mmas_row<C8P, NP>(tmem + (uint32_t)(a * NP), sH_a + (uint32_t)(sl * G::kHBytes), sW_a, sgn);
                mma_commit(&empty[sl]);
                mma_commit(&accf[a]);
            }
        }
        __syncwarp();
    } else {
        const float osc = oscale ? *oscale : 1.f;
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int a = i & 1, ka = i >> 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&accf[a], ka & 1, status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) abort_s = 1;
            if (abort_s) break;
            tc_fence_after();
            int z, y, x0;
            origin(tile, z, y, x0);
            epilogue<NP>(src, tmem + (uint32_t)(a * NP), z, y, x0, N, bias, relu, osc, out);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[a]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tmem_dealloc(tmem, G::kCols);
    }
}

// The paired-tap weights of a source of at most 8 channels:
// Wp[pz][px][g][c][n][j], plane offsets (pz, p, px) of the halo, p = 0 and 1
// for g = 0 (c = 0, 1) and p = 2 for g = 1 (c = 0; c = 1 zero); the tap is
// the one applied at offset (pz - 1, p - 1, px - 1) = sgn (dz, dy, dx).
__global__ void k_prep_umma_pair(const __nv_bfloat16* __restrict__ Wt, int Npad, int Cs, int N, int NP, int sgn,
                                 __nv_bfloat16* __restrict__ Wp)
{
    const int total = 9 * 2 * 2 * NP * 8;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int j = i % 8, n = (i / 8) % NP, c = (i / (8 * NP)) % 2, g = (i / (16 * NP)) % 2, pzx = i / (32 * NP);
    const int pz = pzx / 3, px = pzx % 3;
    const int p = g == 0 ? c : (c == 0 ? 2 : -1);
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (p >= 0 && j < Cs && n < N) {
        const int dz = sgn * (pz - 1), dy = sgn * (p - 1), dx = sgn * (px - 1);
        const int tap = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
        v = Wt[(size_t)(tap * Cs + j) * Npad + n];
    }
    Wp[i] = v;
}

// Wu[tap][c][n][j] = Wt[(tap * Cs + 8 c + j) * Npad + n] (zero past Cs
// source channels or N output channels); Wt is the implicit-GEMM matrix
// [Kpad][Npad] of the mma.sync kernels (forward or input-gradient layout).
__global__ void k_prep_umma(const __nv_bfloat16* __restrict__ Wt, int Npad, int Cs, int N, int C8P, int NP,
                            __nv_bfloat16* __restrict__ Wu)
{
    const int total = 27 * C8P * NP * 8;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int j = i % 8, n = (i / 8) % NP, c = (i / (8 * NP)) % C8P, tap = i / (8 * NP * C8P);
    const int ci = 8 * c + j;
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (ci < Cs && n < N) v = Wt[(size_t)(tap * Cs + ci) * Npad + n];
    Wu[i] = v;
}

}  // namespace umma
}  // namespace unet
}  // namespace mh3d
