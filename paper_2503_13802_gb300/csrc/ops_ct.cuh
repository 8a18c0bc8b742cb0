// Compile-time specialised pencil kernels (the fast path for the common
// lengths; ops.cu keeps the runtime-general kernels for every other size).
//
// Each kernel is the same computation as its runtime counterpart in ops.cu;
// what changes is that the transform lengths, radix schedules, pencil count
// and thread count are template parameters, and the spectral step between a
// forward and an inverse transform runs in registers (fft_ct.cuh):
//   T pass   : forward last stage -> times the axis spectrum -> inverse first
//              stage, one butterfly per thread, no shared-memory round trip.
//   X forward: the drive-axis spectrum stays in registers across harmonics;
//              per harmonic, its fold over the s aliases times X^_k feeds the
//              first stage of the length-n/s inverse directly.
//   X adjoint: per harmonic, the last stage of the length-n/s transform adds
//              conj(X^_k) times its periodised output into registers that are
//              the inputs of the length-n inverse's first stage.
//   X normal : the s x s alias-block product sits between the forward's last
//              and the inverse's first stage, in registers.
#pragma once

#include <type_traits>

#include "bulk.cuh"
#include "fft_ct.cuh"
#include "ops_functors.cuh"

namespace mh3d {
namespace ct {

constexpr int kP = 16;    // pencils per CTA of the X passes: 16 row pairs
constexpr int kT = 128;   // threads per CTA
constexpr int kTN = 256;  // threads per CTA of the X normal pass (one butterfly each per stage)
constexpr int kKG = 2;    // harmonics per inverse batch in the X forward kernel

// Pencil stride (float2) of a [element][pencil] shared buffer read or
// written by a stage whose consecutive lanes take consecutive butterflies
// j (NB per pencil) of a few pencils.  The 16 lanes of a half-warp then
// span min(NB, 16) butterflies x 16 / min(NB, 16) pencils; with
// ld = 16 / nb (mod 32 / nb) the butterflies' rows start 32 / nb banks
// apart and every lane lands in its own bank.  Pencil-fast stages stay
// conflict-free with any stride.
constexpr int conflict_free_ld(int P, int NB)
{
    const int nb = NB < 16 ? NB : 16;
    if (nb <= 1) return P;
    int ld = P;
    while (ld % (32 / nb) != 16 / nb) ++ld;
    return ld;
}

// Forward last stage (radix R, Ns = N/R) -> per-element spectral multiplier
// -> inverse first stage (radix R, Ns = 1), for P pencils.
template <int N, int R, int P, int T, class LD, class ST>
__device__ __forceinline__ void fused_conv_stage(const LD& ld, const ST& st, const float2* __restrict__ mu,
                                                 const float2* __restrict__ tw)
{
    constexpr int NB = N / R, TOTAL = NB * P, ITER = (TOTAL + T - 1) / T;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        if ((TOTAL % T) != 0 && idx >= TOTAL) break;
        const int p = idx % P, j = idx / P;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * NB, p);
        if (NB > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw[r * j]);
        }
        dft<R, false>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = c_mul(v[r], mu[j + r * NB]);
        dft<R, true>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) st(j * R + r, p, v[r]);
    }
}

// T pass with bulk (copy-engine) tile I/O.  A tile is N rows (the axis
// elements, stride es) x 2P contiguous floats (P column pairs); row e of a
// tile lands in shared memory as the P float2 of pencil layout row e, so
// the FFT stages read it directly.  Tiles loaded, by loader mode:
//   plain      : in (and b when the input or output is weighted by b)
//   pupdate 1  : r, p, b            (p = r + beta p, input b p)
//   pupdate 2  : r, s, p, q, x, b   (single-reduction CG update, input b r)
//   epilogue   : in, p, b           (q = b w + lambda p, p^T q [, p^T p])
// Updated vectors are written back by bulk stores that overlap the FFT; the
// output leaves through a staging tile.  Host conditions: nx % 2P == 0,
// every pointer 16-byte aligned, regulariser R = I for the epilogue.
template <int N, int P>
struct TTiles {
    static constexpr int kTile = N * P;   // float2 per tile
};

template <class L, int P, int TT = kT>
__global__ void __launch_bounds__(TT) k_tpass_ct(const __grid_constant__ TArgs a)
{
    using I = RInfo<L>;
    constexpr int N = I::n(), NST = I::nst, RL = I::last();
    using LI = Reverse<L>;
    constexpr int T = TT, TILE = N * P;
    static_assert(NST >= 2, "the specialised T pass has at least two stages");
    extern __shared__ __align__(128) float2 sm_raw[];
    __shared__ double red[34];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float cgs[3];
    float beta = 0.f, alpha = 0.f;
    pdl_wait();   // a no-op unless launched with programmatic serialization
    if (a.cg.flags && !cg_enter_cta(a.cg, a.pupdate != 0, &beta, &alpha, cgs)) return;
    // 128-byte aligned start for the TMA boxes (the launcher adds the slack)
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~uintptr_t(127));
    float2* tw = sm;
    float2* mu = tw + N;
    float2* tiles = mu + N;   // six tile slots
    const int x0 = blockIdx.x * 2 * P;
    // tiles by loader mode (tensor-map slot of each)
    int tmap[6] = {0, 0, 0, 0, 0, 0};
    int nt = 0;
    const int mode = a.pupdate ? a.pupdate : (a.epilogue ? 3 : 0);
    const bool bw = (a.bin || a.bout);
    if (mode == 0) {
        tmap[nt++] = kTmIn;
    } else if (mode == 1) {
        tmap[nt++] = kTmR;
        tmap[nt++] = kTmP;
    } else if (mode == 2) {
        tmap[nt++] = kTmR;
        tmap[nt++] = kTmS;
        tmap[nt++] = kTmP;
        tmap[nt++] = kTmQ;
        tmap[nt++] = kTmX;
    } else {
        tmap[nt++] = kTmIn;
        tmap[nt++] = kTmPin;
    }
    if (bw) tmap[nt++] = kTmB;
    // box coordinates (x, y, z) of this tile
    const int cy = (a.axis == 1) ? 0 : (int)blockIdx.y;
    const int cz = (a.axis == 1) ? (int)blockIdx.y : 0;
    constexpr uint32_t TILEB = (uint32_t)(N * P * sizeof(float2));
    // The barrier must be initialised (and the initialisation fenced) before
    // any thread waits on it: the word may hold a previous CTA's state.
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, TILEB * nt + a.debug_extra_tx);
        for (int t = 0; t < nt; ++t) tma_load_3d(tiles + t * TILE, &a.tm.m[tmap[t]], x0, cy, cz, &bar);
    }
    // tables while the tile copies are in flight
    for (int i = threadIdx.x; i < N; i += T) {
        tw[i] = a.tw[i];
        mu[i] = a.mult[i];
    }
    // A copy that never completes would be a hardware fault; the bounded wait
    // records MH3D_ERR_TIMEOUT and the CTA skips its work instead of hanging.
    const bool ok = mbar_wait(&bar, 0, a.status);
    if (!__syncthreads_and(ok)) return;

    // ---- input to the first stage (tin), CG updates in place in the tiles.
    // tin overwrites, element by element, a tile that only its own thread
    // reads (in, r or s); the FFT's second buffer b0 is a free slot, or in
    // the CG update the b tile, which is dead once tin is formed.  Tiles being
    // written back (r, p, q, x) are never reused before the final wait.
    const float2* tb = bw ? tiles + (nt - 1) * TILE : nullptr;   // b is the last tile
    float2* tin = (mode == 2) ? tiles + TILE : tiles;
    float2* b1 = tin;
    float2* b0 = (mode == 2) ? tiles + 5 * TILE : tiles + nt * TILE;
    if (mode == 0 || mode == 3) {
        const float2* t0 = tiles;
        for (int i = threadIdx.x; i < TILE; i += T) {
            float2 v = t0[i];
            if (a.bin) {
                const float2 bb = tb[i];
                v.x *= bb.x;
                v.y *= bb.y;
            }
            tin[i] = v;
        }
    } else if (mode == 1) {
        float2* tr = tiles;
        float2* tp = tiles + TILE;
        for (int i = threadIdx.x; i < TILE; i += T) {
            const float2 r = tr[i], pp = tp[i];
            const float2 pn = make_float2(fmaf(beta, pp.x, r.x), fmaf(beta, pp.y, r.y));
            tp[i] = pn;
            const float2 bb = tb ? tb[i] : make_float2(1.f, 1.f);
            tin[i] = make_float2(pn.x * bb.x, pn.y * bb.y);
        }
    } else {
        float2* tr = tiles;
        const float2* ts = tiles + TILE;
        float2* tp = tiles + 2 * TILE;
        float2* tq = tiles + 3 * TILE;
        float2* tx = tiles + 4 * TILE;
        for (int i = threadIdx.x; i < TILE; i += T) {
            const float2 r = tr[i], sv = ts[i], pp = tp[i], qq = tq[i], xx = tx[i];
            const float2 pn = make_float2(fmaf(beta, pp.x, r.x), fmaf(beta, pp.y, r.y));
            const float2 qn = make_float2(fmaf(beta, qq.x, sv.x), fmaf(beta, qq.y, sv.y));
            const float2 rn = make_float2(fmaf(-alpha, qn.x, r.x), fmaf(-alpha, qn.y, r.y));
            tp[i] = pn;
            tq[i] = qn;
            tx[i] = make_float2(fmaf(alpha, pn.x, xx.x), fmaf(alpha, pn.y, xx.y));
            tr[i] = rn;
            const float2 bb = tb ? tb[i] : make_float2(1.f, 1.f);
            tin[i] = make_float2(rn.x * bb.x, rn.y * bb.y);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    // write the updated vectors back while the transform runs
    if ((mode == 1 || mode == 2) && threadIdx.x == 0) {
        if (mode == 1) {
            tma_store_3d(&a.tm.m[kTmP], x0, cy, cz, tiles + TILE);
        } else {
            tma_store_3d(&a.tm.m[kTmR], x0, cy, cz, tiles);
            tma_store_3d(&a.tm.m[kTmP], x0, cy, cz, tiles + 2 * TILE);
            tma_store_3d(&a.tm.m[kTmQ], x0, cy, cz, tiles + 3 * TILE);
            tma_store_3d(&a.tm.m[kTmX], x0, cy, cz, tiles + 4 * TILE);
        }
        bulk_commit();
    }

    // ---- convolution: forward stages, fused spectral step, inverse stages
    constexpr int pf = result_parity<0, NST - 1>();
    float2* fo = pf ? b1 : b0;   // output of forward stage NST-2
    float2* fx = pf ? b0 : b1;
    run_stages<L, 0, NST - 1, P, T, 1, false, true, true>(BufLd{tin, P}, BufSt{fo, P}, b0, b1, P, tw);
    fused_conv_stage<N, RL, P, T>(BufLd{fo, P}, BufSt{fx, P}, mu, tw);
    __syncthreads();
    // the last inverse stage writes the buffer it does not read
    float2* stg = (NST % 2 == 0) ? fo : fx;
    run_stages<LI, 1, NST, P, T, 1, true, true, true>(BufLd{fx, P}, BufSt{stg, P}, fo, fx, P, tw);

    // ---- output: b weighting / CG epilogue in the staging tile, bulk store
    DotAcc acc, acc2;
    if (mode == 3) {
        const float2* tpin = tiles + TILE;
        const float lam = a.reg.lambda;
        for (int i = threadIdx.x; i < TILE; i += T) {
            float2 w = stg[i];
            const float2 pv = tpin[i];
            if (a.bout) {
                const float2 bb = tb[i];
                w.x *= bb.x;
                w.y *= bb.y;
            }
            w.x = fmaf(lam, pv.x, w.x);
            w.y = fmaf(lam, pv.y, w.y);
            stg[i] = w;
            acc.add(pv.x, w.x);
            acc.add(pv.y, w.y);
            if (a.part2) {
                acc2.add(pv.x, pv.x);
                acc2.add(pv.y, pv.y);
            }
        }
    } else if (a.bout) {
        for (int i = threadIdx.x; i < TILE; i += T) {
            float2 w = stg[i];
            const float2 bb = tb[i];
            stg[i] = make_float2(w.x * bb.x, w.y * bb.y);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    // a dependent launch may now be scheduled; it reads nothing of this
    // kernel's before its griddepcontrol.wait (the whole grid's completion)
    pdl_trigger();
    if (threadIdx.x == 0) {
        tma_store_3d(&a.tm.m[kTmOut], x0, cy, cz, stg);
        bulk_commit();
        bulk_wait_all();   // the copies read shared memory and must land before the kernel ends
    }

    if (mode == 3 && a.part) {
        const int bid = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
        float2 t, t2;
        block_pair_acc2(acc, a.part2 ? &acc2 : nullptr, reinterpret_cast<float*>(red), &t, &t2);
        if (a.part2) grid_sum_finalize2(t, t2, a.part, a.part2, bid, nb, a.ticket, a.sum_out, a.sum_out2);
        else grid_sum_finalize(t, a.part, bid, nb, a.ticket, a.sum_out);
    }
    if (a.count_iter) cg_count_iteration(a.cg);
}

template <class L, int P>
constexpr size_t tpass_ct_smem()
{
    // tables, 6 tile slots, and 128 bytes of alignment slack
    return sizeof(float2) * (size_t)(2 * RInfo<L>::n() + 6 * RInfo<L>::n() * P) + 128;
}

// Portrait store of one inverse batch (pencil q = kk * P + p), skipping
// harmonics beyond the last one of the batch.
struct PortraitStK {
    float2* d;
    const float2* __restrict__ phase;
    long long M;
    int mx, row0, rows, kn;
    int P = kP;        // pencils per harmonic in the batch
    int rstride = 1;   // portrait rows between a pencil's two rows (and between pencils: 2 rstride)
    __device__ __forceinline__ void operator()(int m, int q, float2 val) const
    {
        const int kk = q / P, p = q - kk * P;
        if (kk >= kn) return;
        const float2 ph = __ldg(phase + kk);
        const int r = row0 + 2 * p * rstride;
        float2* dk = d + (long long)kk * M;
        if (r < rows) dk[(long long)r * mx + m] = make_float2(ph.x * val.x, ph.y * val.x);
        if (r + rstride < rows) dk[(long long)(r + rstride) * mx + m] = make_float2(ph.x * val.y, ph.y * val.y);
    }
};

// Pencil stride of the X forward kernel's inverse buffers (KG * PP pencils;
// the last inverse stage runs butterfly-fast).
template <class LI, int PP>
constexpr int xfwd_ldc()
{
    return conflict_free_ld(kKG * PP, RInfo<LI>::n() / RInfo<LI>::last());
}

// The drive-axis forward on 2P rows (LF = radix schedule of length nx, LI =
// schedule of the length mx = nx / S inverse, whose first radix is LF's last
// divided by S): the length-nx forward transform of the
// rows (loader ld: pencil p packs rows 2p and 2p + 1), then per batch of kKG
// harmonics in [kbeg, kend) the fold times X_k, the length-mx inverse, the
// phase and the portrait store (pst: every field but d, phase and kn).
// Shared memory: tw (W_nx, loaded) and a scratch region of
// max(2 nx P, 2 mx ldc) float2.
template <class LF, class LI, int S, int P, int T, class LD>
__device__ __forceinline__ void xfwd_rows(const LD& ld, const XArgs& a, PortraitStK pst, int kbeg, int kend,
                                          const float2* tw, float2* scratch)
{
    using IF = RInfo<LF>;
    using II = RInfo<LI>;
    constexpr int NX = IF::n(), MX = II::n(), NSTF = IF::nst, NSTI = II::nst, RL = IF::last(), R2 = II::first();
    static_assert(NX == MX * S && RL == R2 * S, "inconsistent X forward schedules");
    constexpr int KG = kKG, PB = KG * P;
    constexpr int NBL = NX / RL;   // = MX / R2
    constexpr int ITERL = (NBL * P + T - 1) / T;
    constexpr int LDC = xfwd_ldc<LI, P>();
    float2* b0 = scratch;
    float2* b1 = b0 + NX * P;
    float2* c0 = scratch;            // reused after the forward transform
    float2* c1 = c0 + MX * LDC;
    constexpr int pf = result_parity<0, NSTF - 1>();
    float2* fo = pf ? b1 : b0;
    if constexpr (NSTF > 1) run_stages<LF, 0, NSTF - 1, P, T, 1, false, false, true>(ld, BufSt{fo, P}, b0, b1, P, tw);
    // last forward stage into registers: F[it][r] = spectrum at j + r NX/RL
    float2 F[ITERL][RL];
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % P, j = idx / P;
        if ((NBL * P) % T != 0 && idx >= NBL * P) break;
#pragma unroll
        for (int r = 0; r < RL; ++r) F[it][r] = (NSTF > 1) ? fo[(j + r * NBL) * P + p] : ld(j + r * NBL, p);
        if (NBL > 1) {
#pragma unroll
            for (int r = 1; r < RL; ++r) F[it][r] = c_mul(F[it][r], tw[r * j]);
        }
        dft<RL, false>(F[it]);
    }
    __syncthreads();   // the c buffers alias the forward scratch
    for (int k0 = kbeg; k0 < kend; k0 += KG) {
        const int kn = min(KG, kend - k0);
        pst.d = a.dout + (long long)k0 * a.M;
        pst.phase = a.phase + k0;
        pst.kn = kn;
#pragma unroll
        for (int kk = 0; kk < KG; ++kk) {
            const float2* __restrict__ xk = a.Xhat + (long long)(k0 + (kk < kn ? kk : 0)) * NX;
#pragma unroll
            for (int it = 0; it < ITERL; ++it) {
                const int idx = (int)threadIdx.x + it * T;
                const int p = idx % P, j = idx / P;
                if ((NBL * P) % T != 0 && idx >= NBL * P) break;
                float2 G[R2];
#pragma unroll
                for (int r2 = 0; r2 < R2; ++r2) {
                    const int m = j + r2 * NBL;
                    float2 g = c_mul(F[it][r2], __ldg(xk + m));
#pragma unroll
                    for (int al = 1; al < S; ++al) g = c_add(g, c_mul(F[it][r2 + al * R2], __ldg(xk + m + al * MX)));
                    G[r2] = (kk < kn) ? g : make_float2(0.f, 0.f);
                }
                dft<R2, true>(G);
#pragma unroll
                for (int r2 = 0; r2 < R2; ++r2) {
                    if constexpr (NSTI > 1) c0[(j * R2 + r2) * LDC + kk * P + p] = G[r2];
                    else pst(j * R2 + r2, kk * P + p, G[r2]);
                }
            }
        }
        __syncthreads();
        if constexpr (NSTI > 1) run_stages<LI, 1, NSTI, PB, T, S, true, true, false>(BufLd{c0, LDC}, pst, c1, c0, LDC, tw);
    }
}

// X forward over consecutive rows.  Harmonics split over grid.y in groups
// of a.kpc (0: one group); every group recomputes the drive-axis spectrum of
// its rows (one more read of the L2-resident input per group).
template <class LF, class LI, int S, int PP = kP, int TT = kT>
__global__ void __launch_bounds__(TT) k_xfwd_ct(const XArgs a)
{
    constexpr int NX = RInfo<LF>::n(), MX = RInfo<LI>::n(), P = PP, T = TT;
    extern __shared__ float2 sm[];
    float2* tw = sm;                 // W_NX^t; W_MX^t = tw[t S]
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const int kpc = a.kpc > 0 ? a.kpc : a.K;
    const int kbeg = (int)blockIdx.y * kpc, kend = min(a.K, kbeg + kpc);
    const PortraitStK pst{nullptr, nullptr, a.M, MX, row0, a.rows, 0, P};
    xfwd_rows<LF, LI, S, P, T>(RowPairLd{a.vin, NX, row0, a.rows}, a, pst, kbeg, kend, tw, tw + NX);
}

template <class LF, class LI, int S, int PP = kP>
constexpr size_t xfwd_ct_smem()
{
    constexpr size_t nx = RInfo<LF>::n(), mx = RInfo<LI>::n();
    constexpr size_t b = 2 * nx * PP, c = 2 * mx * xfwd_ldc<LI, PP>();
    return sizeof(float2) * (nx + (b > c ? b : c));
}

// X adjoint: LF2 = schedule of the length-mx forward transforms (one per
// harmonic), LI = schedule of the length-nx inverse, first radix = LF2's
// last times S.
// Loader of the adjoint's first stage from a staged block of one harmonic's
// portrait rows, mxs float2 apart: pencil p packs Re(e^{-i theta} y) of
// rows p and p + P (rows at or beyond nrow read as zero).  With mxs = mx + 2
// the rows of a half-warp's pencils start 4 banks apart, so the
// pencil-fast first stage reads without bank conflicts.
struct PortraitSplitLd {
    const float2* blk;
    float2 ph;
    int mxs, P, nrow;
    __device__ __forceinline__ float2 operator()(int m, int p) const
    {
        float2 o = make_float2(0.f, 0.f);
        if (p < nrow) {
            const float2 y = blk[p * mxs + m];
            o.x = fmaf(ph.x, y.x, ph.y * y.y);
        }
        if (p + P < nrow) {
            const float2 y = blk[(p + P) * mxs + m];
            o.y = fmaf(ph.x, y.x, ph.y * y.y);
        }
        return o;
    }
};
// Output rows of that pairing: pencil p's real part is row row0 + p, its
// imaginary part row row0 + p + P.
struct RowSplitSt {
    float* v;
    int nx, row0, rows, P;
    __device__ __forceinline__ void operator()(int e, int p, float2 val) const
    {
        const int r = row0 + p;
        if (r < rows) v[(long long)r * nx + e] = val.x;
        if (r + P < rows) v[(long long)(r + P) * nx + e] = val.y;
    }
};

// Adjoint buffer geometry: pencil stride of the transform buffers (the last
// inverse stage runs butterfly-fast) and row stride of the staged portrait
// blocks.
template <class LI, int PP>
constexpr int xadj_ld()
{
    return conflict_free_ld(PP, RInfo<LI>::n() / RInfo<LI>::last());
}
template <class LF2>
constexpr int xadj_mxs()
{
    return RInfo<LF2>::n() + 2;
}

// Loader of the first stage of a round of KB harmonics (KB = 1 or 2) from
// their staged row blocks (blk_stride float2 apart, rows mxs float2 apart):
// pencil q = kk P + p packs Re(e^{-i theta} y) of rows p and p + P of
// harmonic kk of the round; rows at or beyond nrow, and harmonics at or
// beyond nk, read as zero.
struct PortraitRoundLd {
    const float2* blk;
    float2 ph0, ph1;
    int mxs, P, nrow, nk, blk_stride;
    __device__ __forceinline__ float2 operator()(int m, int q) const
    {
        const int kk = q >= P ? 1 : 0;
        const int p = q - kk * P;
        float2 o = make_float2(0.f, 0.f);
        if (kk >= nk) return o;
        const float2 ph = kk ? ph1 : ph0;
        const float2* b = blk + kk * blk_stride;
        if (p < nrow) {
            const float2 y = b[p * mxs + m];
            o.x = fmaf(ph.x, y.x, ph.y * y.y);
        }
        if (p + P < nrow) {
            const float2 y = b[(p + P) * mxs + m];
            o.y = fmaf(ph.x, y.x, ph.y * y.y);
        }
        return o;
    }
};

// Adjoint shared-memory geometry for P pencils and KB harmonics per round:
// each of the two transform buffers holds max(nx ld, mx KB P) float2.
template <class LF2, class LI, int P, int KB>
constexpr int xadj_buf()
{
    constexpr int a = RInfo<LI>::n() * xadj_ld<LI, P>(), b = RInfo<LF2>::n() * KB * P;
    return a > b ? a : b;
}
template <class LF2, int P, int KB>
constexpr int xadj_pb()   // two rounds of KB row blocks
{
    return 2 * KB * 2 * P * xadj_mxs<LF2>();
}

// The drive-axis adjoint of 2P rows, portrait row rbase + r rstride for row
// r of the CTA (r < nrow): per harmonic the length-mx forward transform of
// Re(e^{-i theta_k} y_k), times conj(X_k) periodised to length nx, summed
// over k in registers; then one length-nx inverse whose last stage goes to
// `st` (element, pencil, value).
// BULK: pencil p packs rows p and p + P; the harmonics go in rounds of KB,
// one first-stage run over the round's KB P pencils and one CTA barrier per
// round.  Each harmonic's rows reach a padded shared-memory block (rows of
// mx + 2 float2) by one 1D bulk copy per row; two round buffers with one
// mbarrier each take rounds t and t + 1, and a buffer is refilled with round
// t + 2 once round t's first stage has read it, so the copies run under the
// transforms.  Otherwise (KB = 1): rows 2p and 2p + 1, read from global
// memory (rstride 1).  Loads W_nx into tw.  Returns false if a bulk copy's
// bounded wait gave up (MH3D_ERR_TIMEOUT recorded; the rest skipped).
template <class LF2, class LI, int S, bool BULK, int P, int T, int KB, class ST>
__device__ __forceinline__ bool xadj_rows(const XArgs& a, int rbase, int rstride, int nrow, const ST& st, float2* tw,
                                          float2* b0, float2* b1, float2* pb, uint64_t* bars)
{
    using IF = RInfo<LF2>;
    using II = RInfo<LI>;
    constexpr int MX = IF::n(), NX = II::n(), NST2 = IF::nst, NSTI = II::nst, R = IF::last(), RI = II::first();
    static_assert(NX == MX * S && RI == R * S, "inconsistent X adjoint schedules");
    static_assert(KB == 1 || (KB == 2 && BULK), "rounds of two harmonics need the staged rows");
    constexpr int NBL = MX / R;    // = NX / RI
    constexpr int ITERL = (NBL * P + T - 1) / T;
    constexpr int LD = xadj_ld<LI, P>();
    constexpr int PB = KB * P;     // first-stage pencils per round (pencil stride PB)
    constexpr int MXS = xadj_mxs<LF2>();
    constexpr int BLK = 2 * P * MXS;
    constexpr uint32_t ROWB = (uint32_t)(MX * sizeof(float2));
    const uint32_t pbytes = (uint32_t)nrow * ROWB;
    const int nround = (a.K + KB - 1) / KB;
    // warp 0 stages round t's rows into round buffer t & 1, one copy per row
    auto stage_round = [&](int t) {
        const int k0 = t * KB, nk = min(KB, a.K - k0);
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&bars[t & 1], pbytes * (uint32_t)nk);
        __syncwarp();
        for (int kk = 0; kk < nk; ++kk) {
            const float2* src = a.din + (long long)(k0 + kk) * a.M;
            float2* dst = pb + ((t & 1) * KB + kk) * BLK;
            for (int r = (int)threadIdx.x; r < nrow; r += 32)
                bulk_g2s(dst + r * MXS, src + (long long)(rbase + r * rstride) * MX, ROWB, &bars[t & 1]);
        }
    };
    if constexpr (BULK) {
        if (threadIdx.x == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (threadIdx.x < 32)
            for (int t = 0; t < nround && t < 2; ++t) stage_round(t);
    }
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    __syncthreads();
    float2 acc[ITERL][RI];
#pragma unroll
    for (int it = 0; it < ITERL; ++it)
#pragma unroll
        for (int r = 0; r < RI; ++r) acc[it][r] = make_float2(0.f, 0.f);
    constexpr int pf = result_parity<0, NST2 - 1>();
    float2* fo = pf ? b1 : b0;
    for (int t = 0; t < nround; ++t) {
        const int k0 = t * KB, nk = min(KB, a.K - k0);
        if constexpr (BULK) {
            // a copy that never lands would be a hardware fault: bounded wait
            const bool ok = mbar_wait(&bars[t & 1], (uint32_t)((t >> 1) & 1), a.status);
            if (!__syncthreads_and(ok)) return false;
        }
        using LdT = typename std::conditional<BULK, PortraitRoundLd, PortraitLd>::type;
        LdT ld;
        if constexpr (BULK)
            ld = PortraitRoundLd{pb + (t & 1) * KB * BLK, __ldg(a.phase + k0), __ldg(a.phase + k0 + (nk > 1 ? 1 : 0)),
                                 MXS, P, nrow, nk, BLK};
        else
            ld = PortraitLd{a.din + (long long)k0 * a.M, a.phase + k0, a.M, MX, rbase, a.rows, P};
        if constexpr (NST2 > 1)
            run_stages<LF2, 0, NST2 - 1, PB, T, S, false, false, true>(ld, BufSt{fo, PB}, b0, b1, PB, tw);
#pragma unroll
        for (int kk = 0; kk < KB; ++kk) {
            if (kk >= nk) break;
            const float2* __restrict__ xk = a.Xhat + (long long)(k0 + kk) * NX;
#pragma unroll
            for (int it = 0; it < ITERL; ++it) {
                const int idx = (int)threadIdx.x + it * T;
                const int p = idx % P, j = idx / P;
                if ((NBL * P) % T != 0 && idx >= NBL * P) break;
                float2 v[R];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    v[r] = (NST2 > 1) ? fo[(j + r * NBL) * PB + kk * P + p] : ld(j + r * NBL, kk * P + p);
                if (NBL > 1) {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw[r * j * S]);
                }
                dft<R, false>(v);
#pragma unroll
                for (int r = 0; r < RI; ++r)
                    acc[it][r] = c_add(acc[it][r], c_mulc(v[r % R], __ldg(xk + j + r * NBL)));
            }
        }
        __syncthreads();
        if constexpr (BULK) {
            // round t's blocks have been read (barrier above): refill the
            // buffer with round t + 2; each issuing lane orders the CTA's
            // reads before its own async-proxy writes
            if (threadIdx.x < 32 && t + 2 < nround) {
                fence_proxy_async_smem();
                stage_round(t + 2);
            }
        }
    }
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % P, j = idx / P;
        if ((NBL * P) % T != 0 && idx >= NBL * P) break;
        dft<RI, true>(acc[it]);
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            if constexpr (NSTI > 1) b0[(j * RI + r) * LD + p] = acc[it][r];
            else st(j * RI + r, p, acc[it][r]);
        }
    }
    __syncthreads();
    if constexpr (NSTI > 1) run_stages<LI, 1, NSTI, P, T, 1, true, true, false>(BufLd{b0, LD}, st, b1, b0, LD, tw);
    return true;
}

template <class LF2, class LI, int S, bool BULK = false, int PP = kP, int TT = kT, int KB = 1>
__global__ void __launch_bounds__(TT) k_xadj_ct(const XArgs a)
{
    constexpr int NX = RInfo<LI>::n(), P = PP;
    constexpr int BUF = xadj_buf<LF2, LI, PP, KB>();
    extern __shared__ __align__(16) float2 sm[];
    __shared__ __align__(8) uint64_t bars[2];
    float2* tw = sm;               // W_NX^t; W_MX^t = tw[t S]
    float2* b0 = tw + NX;
    float2* b1 = b0 + BUF;
    float2* pb = b1 + BUF;         // BULK: two rounds of KB [2P][MXS] portrait blocks
    const int row0 = blockIdx.x * 2 * P;
    const int nrow = min(2 * P, a.rows - row0);
    using StT = typename std::conditional<BULK, RowSplitSt, RowPairSt>::type;
    StT st;
    if constexpr (BULK)
        st = RowSplitSt{a.vout, NX, row0, a.rows, P};
    else
        st = RowPairSt{a.vout, NX, row0, a.rows};
    xadj_rows<LF2, LI, S, BULK, P, TT, KB>(a, row0, 1, nrow, st, tw, b0, b1, pb, bars);
}

template <class LF2, class LI, int S, bool BULK = false, int PP = kP, int KB = 1>
constexpr size_t xadj_ct_smem()
{
    constexpr size_t nx = RInfo<LI>::n();
    return sizeof(float2) * (nx + 2 * xadj_buf<LF2, LI, PP, KB>() + (BULK ? xadj_pb<LF2, PP, KB>() : 0));
}

// Storer into a row-major staging tile: pencil p's real part is tile row
// 2p, its imaginary part row 2p + 1.
struct RowStageSt {
    float* stg;
    int nx;
    __device__ __forceinline__ void operator()(int e, int p, float2 v) const
    {
        stg[(2 * p) * nx + e] = v.x;
        stg[(2 * p + 1) * nx + e] = v.y;
    }
};

// Normal-operator epilogue over a staged tile of ROWS rows:
// q = b w + lambda R p, with p^T q (and p^T p) accumulated.
template <int NX, int ROWS, int T, int NXS = NX>
__device__ __forceinline__ void nrm_epilogue(const XArgs& a, int row0, const float* __restrict__ stg, DotAcc* acc,
                                             DotAcc* acc2)
{
    static_assert(NXS % 4 == 0, "staged rows start on 16-byte boundaries");
    constexpr int V = NX / 4;
    constexpr int TOTAL = ROWS * V;
    constexpr int ITER = (TOTAL + T - 1) / T;
    static_assert(NX % 4 == 0, "tile rows are read as float4");
    const float* __restrict__ bp = a.b;
    const float* __restrict__ pp = a.pin;
    float* __restrict__ qp = a.qout;
    if (!a.vec4 || a.reg.kind != 0) {
        for (int idx = threadIdx.x; idx < ROWS * NX; idx += T) {
            const int rr = idx / NX, x = idx - rr * NX;
            const int r = row0 + rr;
            if (r >= a.rows) continue;
            const long long i = (long long)r * NX + x;
            const float w = stg[rr * NXS + x];
            float q = bp ? bp[i] * w : w;
            const int z = r / a.reg.ny, y = r - z * a.reg.ny;
            q += reg_term(a.reg, pp, i, x, y, z);
            qp[i] = q;
            const float pv = pp[i];
            acc->add(pv, q);
            if (acc2) acc2->add(pv, pv);
        }
        return;
    }
    float4 W[ITER], B[ITER], Pv[ITER];
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int rr = idx / V, c = idx - rr * V;
        const int r = row0 + rr;
        if (((TOTAL % T) != 0 && idx >= TOTAL) || r >= a.rows) continue;
        const long long i = (long long)r * NX + 4 * c;
        W[it] = *reinterpret_cast<const float4*>(stg + rr * NXS + 4 * c);
        B[it] = bp ? __ldg(reinterpret_cast<const float4*>(bp + i)) : make_float4(1.f, 1.f, 1.f, 1.f);
        Pv[it] = __ldg(reinterpret_cast<const float4*>(pp + i));
    }
    const float lam = a.reg.lambda;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int rr = idx / V, c = idx - rr * V;
        const int r = row0 + rr;
        if (((TOTAL % T) != 0 && idx >= TOTAL) || r >= a.rows) continue;
        const long long i = (long long)r * NX + 4 * c;
        float4 q;
        q.x = fmaf(B[it].x, W[it].x, lam * Pv[it].x);
        q.y = fmaf(B[it].y, W[it].y, lam * Pv[it].y);
        q.z = fmaf(B[it].z, W[it].z, lam * Pv[it].z);
        q.w = fmaf(B[it].w, W[it].w, lam * Pv[it].w);
        *reinterpret_cast<float4*>(qp + i) = q;
        acc->add(Pv[it].x, q.x);
        acc->add(Pv[it].y, q.y);
        acc->add(Pv[it].z, q.z);
        acc->add(Pv[it].w, q.w);
        if (acc2) {
            acc2->add(Pv[it].x, Pv[it].x);
            acc2->add(Pv[it].y, Pv[it].y);
            acc2->add(Pv[it].z, Pv[it].z);
            acc2->add(Pv[it].w, Pv[it].w);
        }
    }
}

// X normal pass buffer geometry: the pencil stride of the transform
// buffers (the last inverse stage runs butterfly-fast), and the row stride
// of the staging tile, padded by 8 floats (rows 2p and 2p + 2 of one
// half-warp's store then start 16 banks apart) where the padded tile still
// fits in the buffer it overlays; the bulk-copy variant stores the tile
// with one contiguous copy and keeps it unpadded.
template <class LF, int PP>
constexpr int xnrm_ld()
{
    return conflict_free_ld(PP, RInfo<LF>::n() / RInfo<LF>::first());
}
template <class LF, bool BULK, int PP>
constexpr int xnrm_nxs()
{
    constexpr int nx = RInfo<LF>::n();
    return (!BULK && PP * (nx + 8) <= nx * xnrm_ld<LF, PP>()) ? nx + 8 : nx;
}

// X normal: LF = schedule of length nx whose last radix is divisible by S;
// the inverse runs the reversed schedule.
// The epilogue of the bulk-copy variant: q = b w + lambda p for the tile's
// nrow rows, with w, b and p read from shared memory and q written in place
// over w (each thread reads and then writes the same float4); dots p^T q
// (and p^T p) accumulate in the same order as nrm_epilogue's.
template <int NX, int ROWS, int T>
__device__ __forceinline__ void nrm_epilogue_tile(const XArgs& a, int nrow, float* stg, const float* tb,
                                                  const float* tp, DotAcc* acc, DotAcc* acc2)
{
    constexpr int V = NX / 4;
    constexpr int TOTAL = ROWS * V;
    constexpr int ITER = (TOTAL + T - 1) / T;
    const float lam = a.reg.lambda;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int rr = idx / V, c = idx - rr * V;
        if (((TOTAL % T) != 0 && idx >= TOTAL) || rr >= nrow) continue;
        const int o = rr * NX + 4 * c;
        const float4 W = *reinterpret_cast<const float4*>(stg + o);
        const float4 B = tb ? *reinterpret_cast<const float4*>(tb + o) : make_float4(1.f, 1.f, 1.f, 1.f);
        const float4 Pv = *reinterpret_cast<const float4*>(tp + o);
        float4 q;
        q.x = fmaf(B.x, W.x, lam * Pv.x);
        q.y = fmaf(B.y, W.y, lam * Pv.y);
        q.z = fmaf(B.z, W.z, lam * Pv.z);
        q.w = fmaf(B.w, W.w, lam * Pv.w);
        *reinterpret_cast<float4*>(stg + o) = q;
        acc->add(Pv.x, q.x);
        acc->add(Pv.y, q.y);
        acc->add(Pv.z, q.z);
        acc->add(Pv.w, q.w);
        if (acc2) {
            acc2->add(Pv.x, Pv.x);
            acc2->add(Pv.y, Pv.y);
            acc2->add(Pv.z, Pv.z);
            acc2->add(Pv.w, Pv.w);
        }
    }
}

// BULK: the CTA's 2P consecutive rows of the input, b and p are one
// contiguous block each, brought in by three 1D bulk copies on one
// mbarrier while the twiddles load; q leaves the same way from the staging
// tile.  Host conditions: 16-byte aligned vectors, R = I.
// PP row pairs per CTA (2 PP rows), TT threads.
template <class LF, int S, bool BULK, int PP = kP, int TT = kTN>
__global__ void __launch_bounds__(TT) k_xnrm_ct(const XArgs a)
{
    using IF = RInfo<LF>;
    using LI = Reverse<LF>;
    constexpr int NX = IF::n(), NST = IF::nst, R = IF::last(), R2 = R / S, MX = NX / S;
    static_assert(R % S == 0, "alias blocks must sit in one butterfly");
    constexpr int P = PP, T = TT;
    constexpr int NBL = NX / R;
    constexpr int ITERL = (NBL * P + T - 1) / T;
    constexpr int LD = xnrm_ld<LF, PP>();     // pencil stride of b0 / b1
    constexpr int NXS = xnrm_nxs<LF, BULK, PP>();   // row stride of the staging tile
    extern __shared__ __align__(16) float2 sm[];
    __shared__ double red[34];
    __shared__ __align__(8) uint64_t bar;
    float dummy;
    pdl_trigger();
    pdl_wait();   // no-ops unless launched with programmatic serialization
    if (a.cg_active && !cg_enter(a.cg, false, &dummy, red)) return;
    float2* tw = sm;
    float2* b0 = tw + NX;
    float2* b1 = b0 + NX * LD;
    float* tin = reinterpret_cast<float*>(b1 + NX * LD);   // BULK: [2P][NX] tiles of v, b, p
    float* tb = tin + 2 * P * NX;
    float* tp = tb + 2 * P * NX;
    const int row0 = blockIdx.x * 2 * P;
    const int nrow = min(2 * P, a.rows - row0);
    const uint32_t tbytes = (uint32_t)(nrow * NX * sizeof(float));
    if constexpr (BULK) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar, tbytes * (a.b ? 3u : 2u));
            const size_t off = (size_t)row0 * NX;
            bulk_g2s(tin, a.vin + off, tbytes, &bar);
            if (a.b) bulk_g2s(tb, a.b + off, tbytes, &bar);
            bulk_g2s(tp, a.pin + off, tbytes, &bar);
        }
    }
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    if constexpr (BULK) {
        // a copy that never lands would be a hardware fault: give up after
        // the bounded wait, record MH3D_ERR_TIMEOUT and skip the work
        const bool ok = mbar_wait(&bar, 0, a.status);
        if (!__syncthreads_and(ok)) return;
    } else {
        __syncthreads();
    }
    const RowPairLd ld{BULK ? tin : a.vin, NX, BULK ? 0 : row0, BULK ? nrow : a.rows};
    DotAcc dacc, dacc2;
    constexpr int pf = result_parity<0, NST - 1>();
    float2* fo = pf ? b1 : b0;
    float2* fx = pf ? b0 : b1;
    if constexpr (NST > 1) run_stages<LF, 0, NST - 1, P, T, 1, false, false, true>(ld, BufSt{fo, LD}, b0, b1, LD, tw);
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % P, j = idx / P;
        if ((NBL * P) % T != 0 && idx >= NBL * P) break;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = (NST > 1) ? fo[(j + r * NBL) * LD + p] : ld(j + r * NBL, p);
        if (NBL > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw[r * j]);
        }
        dft<R, false>(v);
        float2 g[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int al = r / R2, rr = r - al * R2;
            const int m = j + rr * NBL;
            const float2* __restrict__ q = a.Q + ((long long)m * S + al) * S;
            float2 s = c_mul(__ldg(q), v[rr]);
#pragma unroll
            for (int b = 1; b < S; ++b) s = c_add(s, c_mul(__ldg(q + b), v[rr + b * R2]));
            g[r] = s;
        }
        dft<R, true>(g);
#pragma unroll
        for (int r = 0; r < R; ++r) fx[(j * R + r) * LD + p] = g[r];
    }
    __syncthreads();
    // Last inverse stage into a row-major staging tile (2P rows x NX floats)
    // in the buffer that stage does not read, then the epilogue over the tile
    // with all of a thread's loads issued before its stores.
    float* stg = reinterpret_cast<float*>((NST % 2 == 0) ? fo : fx);
    run_stages<LI, 1, NST, P, T, 1, true, true, false>(BufLd{fx, LD}, RowStageSt{stg, NXS}, fo, fx, LD, tw);
    if constexpr (BULK) {
        nrm_epilogue_tile<NX, 2 * P, T>(a, nrow, stg, a.b ? tb : nullptr, tp, &dacc, a.part2 ? &dacc2 : nullptr);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_s2g(a.qout + (size_t)row0 * NX, stg, tbytes);
            bulk_commit();
            bulk_wait_all();   // the copy reads shared memory and must land before the CTA ends
        }
    } else {
        nrm_epilogue<NX, 2 * P, T, NXS>(a, row0, stg, &dacc, a.part2 ? &dacc2 : nullptr);
    }
    if (a.part) {
        float2 t, t2;
        block_pair_acc2(dacc, a.part2 ? &dacc2 : nullptr, reinterpret_cast<float*>(red), &t, &t2);
        if (a.part2) grid_sum_finalize2(t, t2, a.part, a.part2, blockIdx.x, gridDim.x, a.ticket, a.sum_out, a.sum_out2);
        else grid_sum_finalize(t, a.part, blockIdx.x, gridDim.x, a.ticket, a.sum_out);
    }
    if (a.count_iter) cg_count_iteration(a.cg);
    (void)MX;
}

template <class LF, int S, bool BULK = false, int PP = kP>
constexpr size_t xnrm_ct_smem()
{
    constexpr size_t nx = RInfo<LF>::n();
    return sizeof(float2) * (nx + 2 * nx * xnrm_ld<LF, PP>()) + (BULK ? sizeof(float) * 3 * 2 * PP * nx : 0);
}

// ---------------------------------------------------------------------------
// Fused T_z + drive-axis normal pass.  The normal operator's z and x steps
// act on different axes, so one y-slab (nz rows of nx) carries all the data
// both need.  A cluster of C CTAs (two or four) takes one slab:
//   phase 1: CTA c loads x-columns [c nx/C, (c+1) nx/C) of every z by one
//            TMA box and runs the z-axis convolution on them (the T pass's
//            stages, nx/2C column-pair pencils); the last inverse stage
//            stores each row z straight into the exchange buffer of the CTA
//            that owns it (rows [c' nz/C, (c'+1) nz/C) belong to CTA c'),
//            locally or through distributed shared memory;
//   cluster barrier;
//   phase 2: CTA c runs the drive-axis normal pass (alias blocks, then
//            q = b w + lambda p and the dot products) on its nz/C full rows.
// This removes the T_z launch and its round trip of the volume through L2.
// Every CTA of a cluster passes both cluster barriers or neither (the
// loop's done flag is the same for all), so no CTA waits on one that left.
// Host conditions: R = I, 16-byte aligned vectors, nx % 4C == 0,
// nz % 2C == 0.

// Stores of the z pass's last stage into the owners' exchange buffers:
// element e = z (row e - owner ROWS of CTA owner = e / ROWS), pencil p =
// columns x0 + 2p, x0 + 2p + 1.
template <int ROWS>
struct ZxExchangeSt {
    float* xb;           // this CTA's exchange buffer [ROWS][nxp]
    int x0, rank, nxp;
    __device__ __forceinline__ void operator()(int e, int p, float2 v) const
    {
        const int owner = e / ROWS;
        const int o = (e - owner * ROWS) * nxp + x0 + 2 * p;
        if (owner == rank) {
            xb[o] = v.x;
            xb[o + 1] = v.y;
        } else {
            const uint32_t peer = cluster_smem_addr(xb, (uint32_t)owner);
            st_cluster_f32(peer + 4u * (uint32_t)o, v.x);
            st_cluster_f32(peer + 4u * (uint32_t)(o + 1), v.y);
        }
    }
};
// Row pairs of the exchange buffer as the drive-axis pass's pencils.
struct XbPairLd {
    const float* xb;
    int nxp;
    __device__ __forceinline__ float2 operator()(int e, int p) const
    {
        return make_float2(xb[(2 * p) * nxp + e], xb[(2 * p + 1) * nxp + e]);
    }
};

template <class LZ, class LF, int C, int PZ, int PX>
struct ZxGeom {
    static constexpr int NZ = RInfo<LZ>::n(), NX = RInfo<LF>::n();
    static_assert(NX == 2 * C * PZ && NZ == 2 * C * PX, "pencil counts: nx/2C column pairs, nz/2C row pairs");
    static constexpr int NXP = NX + 1;                  // exchange rows: odd stride, conflict-free pencil reads
    static constexpr int LD = xnrm_ld<LF, PX>();        // drive-axis transform buffers
    static constexpr int NXS = xnrm_nxs<LF, false, PX>();
    static constexpr int TAB = 2 * NZ + NX;             // float2: W_nz, z multiplier, W_nx
    static constexpr int XB = (NZ / C) * NXP;           // floats
    static constexpr int OFF = (TAB + (XB + 1) / 2 + 15) / 16 * 16;   // float2 offset of the union, 128-byte aligned
    static constexpr int P1 = 2 * NZ * PZ;              // float2: tile + second buffer of the z pass
    static constexpr int P2 = 2 * NX * LD;              // float2: the drive-axis buffers
    static constexpr int UN = P1 > P2 ? P1 : P2;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(OFF + UN) + 128; }
};

// Phase 1 of the y-slab cluster passes: the z-axis convolution (multiplier
// mu) of this CTA's nx/C columns, every result row stored into its owner's
// exchange buffer.  Loads the phase-2 twiddles (W_nx) while the TMA box is
// in flight.  Returns whether the box landed; the caller takes the cluster
// barrier either way.
template <class LZ, int NX, int C, int PZ, int T>
__device__ __forceinline__ bool zx_zconv(const ZXArgs& a, const float2* __restrict__ mu_g, float2* twz, float2* muz,
                                         float2* twx, float* xb, float2* un, uint64_t* bar, int y, uint32_t rank)
{
    constexpr int NZ = RInfo<LZ>::n(), NSTZ = RInfo<LZ>::nst, RLZ = RInfo<LZ>::last(), ROWS = NZ / C, NXP = NX + 1;
    using LZI = Reverse<LZ>;
    float2* tile = un;
    float2* zb = un + NZ * PZ;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(NZ * PZ * sizeof(float2)));
        tma_load_3d(tile, &a.tz, (int)rank * (NX / C), y, 0, bar);
    }
    for (int i = threadIdx.x; i < NZ; i += T) {
        twz[i] = a.twz[i];
        muz[i] = mu_g[i];
    }
    for (int i = threadIdx.x; i < NX; i += T) twx[i] = a.x.twx[i];
    // a copy that never lands would be a hardware fault: the bounded wait
    // records MH3D_ERR_TIMEOUT
    const bool ok = __syncthreads_and(mbar_wait(bar, 0, a.x.status));
    if (ok) {
        constexpr int pf = result_parity<0, NSTZ - 1>();
        float2* fo = pf ? tile : zb;
        float2* fx = pf ? zb : tile;
        run_stages<LZ, 0, NSTZ - 1, PZ, T, 1, false, true, true>(BufLd{tile, PZ}, BufSt{fo, PZ}, zb, tile, PZ, twz);
        fused_conv_stage<NZ, RLZ, PZ, T>(BufLd{fo, PZ}, BufSt{fx, PZ}, muz, twz);
        __syncthreads();
        const ZxExchangeSt<ROWS> xs{xb, (int)rank * (NX / C), (int)rank, NXP};
        run_stages<LZI, 1, NSTZ, PZ, T, 1, true, true, true>(BufLd{fx, PZ}, xs, fo, fx, PZ, twz);
    }
    return ok;
}

template <class LZ, class LF, int S, int C, int PZ, int PX, int TT, bool EARLY = true>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(TT) k_zxnrm_ct(const __grid_constant__ ZXArgs a)
{
    using G = ZxGeom<LZ, LF, C, PZ, PX>;
    constexpr int NZ = G::NZ, NX = G::NX, T = TT;
    using IF = RInfo<LF>;
    using LI = Reverse<LF>;
    constexpr int NSTX = IF::nst, R = IF::last(), R2 = R / S;
    constexpr int NBL = NX / R, ITERL = (NBL * PX + T - 1) / T;
    constexpr int LD = G::LD, NXS = G::NXS, NXP = G::NXP, ROWS = NZ / C;
    static_assert(R % S == 0, "alias blocks must sit in one butterfly");
    static_assert(RInfo<LZ>::nst >= 2 && NSTX >= 2, "two stages at least on each axis");
    extern __shared__ __align__(128) float2 zx_raw[];
    __shared__ double red[34];
    __shared__ __align__(8) uint64_t bar;
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(zx_raw) + 127) & ~uintptr_t(127));
    float2* twz = sm;
    float2* muz = twz + NZ;
    float2* twx = muz + NZ;
    float* xb = reinterpret_cast<float*>(twx + NX);
    float2* un = sm + G::OFF;           // 128-byte aligned: the TMA box lands at its start
    const uint32_t rank = cluster_ctarank();
    const int y = (int)blockIdx.x / C;
    pdl_wait();   // a no-op unless launched with programmatic serialization
    // every CTA of the cluster is running before any of them stores remotely
    cluster_sync_all();
    float dummy;
    if (a.x.cg_active && !cg_enter(a.x.cg, false, &dummy, red)) return;

    // ---- phase 1: z-axis convolution of this CTA's columns
    const bool ok = zx_zconv<LZ, NX, C, PZ, T>(a, a.muz, twz, muz, twx, xb, un, &bar, y, rank);
    // every part of every owned row has landed (local and remote stores)
    cluster_sync_all();
    if (!ok) return;

    // ---- phase 2: drive-axis normal pass on rows z = rank nz/C + rr
    // The epilogue's b and p values (2 PX rows, volume row of staged row rr:
    // (rank nz/C + rr) ny + y).  With EARLY and a two-stage drive-axis
    // transform they are loaded into registers now, so that their latency
    // passes during the transform (64 -> 80 registers at n_x = 128).  Longer
    // schedules need those registers, and kernels that share the SMs with
    // other volumes' kernels (batched solves) keep the occupancy instead:
    // both load in the epilogue.
    constexpr int V = NX / 4, TOTAL = 2 * PX * V, ITER = (TOTAL + T - 1) / T;
    constexpr bool kEarly = EARLY && NSTX <= 2;
    const float* __restrict__ bp = a.x.b;
    const float* __restrict__ pp = a.x.pin;
    float4 B[ITER], Pv[ITER];
    auto load_bp = [&]() {
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int idx = (int)threadIdx.x + it * T;
            if ((TOTAL % T) != 0 && idx >= TOTAL) continue;
            const int rr = idx / V, c = idx - rr * V;
            const long long i = ((long long)((int)rank * ROWS + rr) * a.ny + y) * NX + 4 * c;
            B[it] = bp ? __ldg(reinterpret_cast<const float4*>(bp + i)) : make_float4(1.f, 1.f, 1.f, 1.f);
            Pv[it] = __ldg(reinterpret_cast<const float4*>(pp + i));
        }
    };
    if constexpr (kEarly) load_bp();
    float2* b0 = un;
    float2* b1 = b0 + NX * LD;
    constexpr int pfx = result_parity<0, NSTX - 1>();
    float2* fo = pfx ? b1 : b0;
    float2* fx = pfx ? b0 : b1;
    run_stages<LF, 0, NSTX - 1, PX, T, 1, false, false, true>(XbPairLd{xb, NXP}, BufSt{fo, LD}, b0, b1, LD, twx);
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % PX, j = idx / PX;
        if ((NBL * PX) % T != 0 && idx >= NBL * PX) break;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = fo[(j + r * NBL) * LD + p];
        if (NBL > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], twx[r * j]);
        }
        dft<R, false>(v);
        float2 g[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int al = r / R2, rr = r - al * R2;
            const int m = j + rr * NBL;
            const float2* __restrict__ q = a.x.Q + ((long long)m * S + al) * S;
            float2 sacc = c_mul(__ldg(q), v[rr]);
#pragma unroll
            for (int b = 1; b < S; ++b) sacc = c_add(sacc, c_mul(__ldg(q + b), v[rr + b * R2]));
            g[r] = sacc;
        }
        dft<R, true>(g);
#pragma unroll
        for (int r = 0; r < R; ++r) fx[(j * R + r) * LD + p] = g[r];
    }
    __syncthreads();
    float* stg = reinterpret_cast<float*>((NSTX % 2 == 0) ? fo : fx);
    run_stages<LI, 1, NSTX, PX, T, 1, true, true, false>(BufLd{fx, LD}, RowStageSt{stg, NXS}, fo, fx, LD, twx);

    // epilogue over the 2 PX staged rows
    if constexpr (!kEarly) load_bp();
    float* __restrict__ qp = a.x.qout;
    const float lam = a.x.reg.lambda;
    DotAcc dacc, dacc2;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        if ((TOTAL % T) != 0 && idx >= TOTAL) continue;
        const int rr = idx / V, c = idx - rr * V;
        const long long i = ((long long)((int)rank * ROWS + rr) * a.ny + y) * NX + 4 * c;
        const float4 w = *reinterpret_cast<const float4*>(stg + rr * NXS + 4 * c);
        float4 q;
        q.x = fmaf(B[it].x, w.x, lam * Pv[it].x);
        q.y = fmaf(B[it].y, w.y, lam * Pv[it].y);
        q.z = fmaf(B[it].z, w.z, lam * Pv[it].z);
        q.w = fmaf(B[it].w, w.w, lam * Pv[it].w);
        *reinterpret_cast<float4*>(qp + i) = q;
        dacc.add(Pv[it].x, q.x);
        dacc.add(Pv[it].y, q.y);
        dacc.add(Pv[it].z, q.z);
        dacc.add(Pv[it].w, q.w);
        if (a.x.part2) {
            dacc2.add(Pv[it].x, Pv[it].x);
            dacc2.add(Pv[it].y, Pv[it].y);
            dacc2.add(Pv[it].z, Pv[it].z);
            dacc2.add(Pv[it].w, Pv[it].w);
        }
    }
    if (a.x.part) {
        float2 t, t2;
        block_pair_acc2(dacc, a.x.part2 ? &dacc2 : nullptr, reinterpret_cast<float*>(red), &t, &t2);
        if (a.x.part2)
            grid_sum_finalize2(t, t2, a.x.part, a.x.part2, blockIdx.x, gridDim.x, a.x.ticket, a.x.sum_out,
                               a.x.sum_out2);
        else
            grid_sum_finalize(t, a.x.part, blockIdx.x, gridDim.x, a.x.ticket, a.x.sum_out);
    }
    if (a.x.count_iter) cg_count_iteration(a.x.cg);
}

// The forward operator's last two steps, T_z then the drive-axis forward
// (fold by s, phase, portrait store), for one y-slab per cluster of C
// CTAs: phase 1 as in k_zxnrm_ct (multiplier Zhat), phase 2 the forward
// pass on this CTA's nz/C rows, whose portrait rows are ny apart.
template <class LZ, class LF, class LI, int C, int PZ, int PX>
struct ZxFwdGeom {
    using B = ZxGeom<LZ, LF, C, PZ, PX>;
    static constexpr int NX = RInfo<LF>::n(), MX = RInfo<LI>::n();
    static constexpr int F2 = 2 * NX * PX > 2 * MX * xfwd_ldc<LI, PX>() ? 2 * NX * PX : 2 * MX * xfwd_ldc<LI, PX>();
    static constexpr int UN = B::P1 > F2 ? B::P1 : F2;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(B::OFF + UN) + 128; }
};

template <class LZ, class LF, class LI, int S, int C, int PZ, int PX, int TT>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(TT) k_zxfwd_ct(const __grid_constant__ ZXArgs a)
{
    using G = ZxGeom<LZ, LF, C, PZ, PX>;
    constexpr int NZ = G::NZ, NX = G::NX, MX = RInfo<LI>::n(), T = TT, ROWS = NZ / C;
    extern __shared__ __align__(128) float2 zf_raw[];
    __shared__ __align__(8) uint64_t bar;
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(zf_raw) + 127) & ~uintptr_t(127));
    float2* twz = sm;
    float2* muz = twz + NZ;
    float2* twx = muz + NZ;
    float* xb = reinterpret_cast<float*>(twx + NX);
    float2* un = sm + G::OFF;
    const uint32_t rank = cluster_ctarank();
    const int y = (int)blockIdx.x / C;
    cluster_sync_all();   // every CTA of the cluster runs before any remote store
    const bool ok = zx_zconv<LZ, NX, C, PZ, T>(a, a.muz, twz, muz, twx, xb, un, &bar, y, rank);
    cluster_sync_all();   // every part of every owned row has landed
    if (!ok) return;
    const PortraitStK pst{nullptr, nullptr, a.x.M, MX, ((int)rank * ROWS) * a.ny + y, a.x.rows, 0, PX, a.ny};
    xfwd_rows<LF, LI, S, PX, T>(XbPairLd{xb, G::NXP}, a.x, pst, 0, a.x.K, twx, un);
}

// The adjoint operator's first two steps, the drive-axis adjoint then the
// z-axis correlation (T_z^T), for one y-slab per cluster of C CTAs:
//   phase 1: CTA c runs the drive-axis adjoint of rows z in
//            [c nz/C, (c+1) nz/C) (portrait rows z ny + y, staged by per-row
//            bulk copies); its last inverse stage stores each row's x-columns
//            into the z-tile of the CTA that owns them (columns
//            [c' nx/C, (c'+1) nx/C) belong to CTA c'), locally or through
//            distributed shared memory;
//   cluster barrier;
//   phase 2: CTA c runs the z correlation on its nx/C columns of every z and
//            stores the result box with one TMA store.
// Every CTA passes the cluster barrier, whether or not its copies landed.
template <int QX>
struct XzExchangeSt {
    float* xt;           // this CTA's z-tile [nz][QX]; columns [c QX, (c+1) QX) belong to CTA c
    int z0, P, rank;
    __device__ __forceinline__ void operator()(int e, int p, float2 v) const
    {
        const int owner = e / QX;
        const int col = e - owner * QX;
        const int o1 = (z0 + p) * QX + col, o2 = (z0 + p + P) * QX + col;
        if (owner == rank) {
            xt[o1] = v.x;
            xt[o2] = v.y;
        } else {
            const uint32_t peer = cluster_smem_addr(xt, (uint32_t)owner);
            st_cluster_f32(peer + 4u * (uint32_t)o1, v.x);
            st_cluster_f32(peer + 4u * (uint32_t)o2, v.y);
        }
    }
};

template <class LF2, class LI, class LZ, int C, int PZ, int PX, int KB>
struct XzGeom {
    static constexpr int NX = RInfo<LI>::n(), NZ = RInfo<LZ>::n();
    static_assert(NX == 2 * C * PZ && NZ == 2 * C * PX, "pencil counts: nx/2C column pairs, nz/2C row pairs");
    static constexpr int TAB = NX + 2 * NZ;                       // float2: W_nx, W_nz, z multiplier
    static constexpr int TABR = (TAB + 15) / 16 * 16;             // 128-byte aligned z-tile
    static constexpr int XT = NZ * PZ;                            // float2: the z-tile
    static constexpr int A1 = 2 * xadj_buf<LF2, LI, PX, KB>() + xadj_pb<LF2, PX, KB>();   // phase-1 buffers
    static constexpr int UN = A1 > XT ? A1 : XT;                  // phase 2: the z pass's second buffer
    static constexpr size_t smem() { return sizeof(float2) * (size_t)(TABR + XT + UN) + 128; }
};

template <class LF2, class LI, class LZ, int S, int C, int PZ, int PX, int TT, int KB>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(TT) k_xzadj_ct(const __grid_constant__ ZXArgs a)
{
    using G = XzGeom<LF2, LI, LZ, C, PZ, PX, KB>;
    constexpr int NX = G::NX, NZ = G::NZ, T = TT, ROWS = NZ / C, QX = NX / C;
    constexpr int NSTZ = RInfo<LZ>::nst, RLZ = RInfo<LZ>::last();
    using LZI = Reverse<LZ>;
    constexpr int BUF = xadj_buf<LF2, LI, PX, KB>();
    static_assert(NSTZ >= 2, "two stages at least along z");
    extern __shared__ __align__(128) float2 xz_raw[];
    __shared__ __align__(8) uint64_t bars[2];
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(xz_raw) + 127) & ~uintptr_t(127));
    float2* tw = sm;
    float2* twz = tw + NX;
    float2* muz = twz + NZ;
    float2* xt = sm + G::TABR;          // the z-tile [NZ][PZ], written by both CTAs of the cluster
    float2* un = xt + G::XT;            // 128-byte aligned
    const uint32_t rank = cluster_ctarank();
    const int y = (int)blockIdx.x / C;
    for (int i = threadIdx.x; i < NZ; i += T) {
        twz[i] = a.twz[i];
        muz[i] = a.muz[i];
    }
    cluster_sync_all();   // every CTA of the cluster runs before any remote store
    // ---- phase 1: drive-axis adjoint of rows z = rank nz/C + r
    float2* b0 = un;
    float2* b1 = b0 + BUF;
    float2* pb = b1 + BUF;
    float* xtf = reinterpret_cast<float*>(xt);
    const XzExchangeSt<QX> st{xtf, (int)rank * ROWS, PX, (int)rank};
    const bool ok = xadj_rows<LF2, LI, S, true, PX, T, KB>(a.x, ((int)rank * ROWS) * a.ny + y, a.ny, ROWS, st, tw,
                                                           b0, b1, pb, bars);
    cluster_sync_all();   // every column of this CTA's z-tile has landed
    if (!ok) return;
    // ---- phase 2: z correlation of this CTA's columns, one TMA store
    float2* tile = xt;
    float2* zb = un;
    constexpr int pf = result_parity<0, NSTZ - 1>();
    float2* fo = pf ? tile : zb;
    float2* fx = pf ? zb : tile;
    run_stages<LZ, 0, NSTZ - 1, PZ, T, 1, false, true, true>(BufLd{tile, PZ}, BufSt{fo, PZ}, zb, tile, PZ, twz);
    fused_conv_stage<NZ, RLZ, PZ, T>(BufLd{fo, PZ}, BufSt{fx, PZ}, muz, twz);
    __syncthreads();
    float2* stg = (NSTZ % 2 == 0) ? fo : fx;   // the buffer the last stage does not read
    run_stages<LZI, 1, NSTZ, PZ, T, 1, true, true, true>(BufLd{fx, PZ}, BufSt{stg, PZ}, fo, fx, PZ, twz);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tma_store_3d(&a.tz, (int)rank * QX, y, 0, stg);
        bulk_commit();
        bulk_wait_all();   // the copy reads shared memory and must land before the CTA ends
    }
}

}  // namespace ct
}  // namespace mh3d
