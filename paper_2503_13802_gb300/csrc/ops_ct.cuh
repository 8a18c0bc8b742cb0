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

#include "fft_ct.cuh"
#include "ops_functors.cuh"

namespace mh3d {
namespace ct {

constexpr int kP = 16;    // pencils per CTA: 16 column pairs (T pass) or 16 row pairs (X pass)
constexpr int kT = 128;   // threads per CTA
constexpr int kKG = 2;    // harmonics per inverse batch in the X forward kernel

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

// T pass along y or z: TArgs as in ops.cu with cols = 2 kP.
template <class L>
__global__ void __launch_bounds__(kT) k_tpass_ct(const TArgs a)
{
    using I = RInfo<L>;
    constexpr int N = I::n(), NST = I::nst, RL = I::last();
    using LI = Reverse<L>;
    constexpr int P = kP, T = kT;
    extern __shared__ float2 sm[];
    __shared__ double red[34];
    float beta = 0.f;
    if (a.cg.flags && !cg_enter(a.cg, a.pupdate != 0, &beta, red)) return;
    float2* tw = sm;
    float2* mu = tw + N;
    float2* b0 = mu + N;
    float2* b1 = b0 + N * P;
    for (int i = threadIdx.x; i < N; i += T) {
        tw[i] = a.tw[i];
        mu[i] = a.mult[i];
    }
    __syncthreads();
    const int x0 = blockIdx.x * 2 * P;
    const long long base = (long long)blockIdx.y * a.os;
    DotAcc acc;
    const TLoad ld{&a, base, x0, beta};
    const TStore st{&a, base, x0, &acc};
    if constexpr (NST == 1) {
        fused_conv_stage<N, RL, P, T>(ld, st, mu, tw);
    } else {
        constexpr int pf = result_parity<0, NST - 1>();
        float2* fo = pf ? b1 : b0;   // output of forward stage NST-2
        float2* fx = pf ? b0 : b1;
        run_stages<L, 0, NST - 1, P, T, 1, false, true, true>(ld, BufSt{fo, P}, b0, b1, P, tw);
        fused_conv_stage<N, RL, P, T>(BufLd{fo, P}, BufSt{fx, P}, mu, tw);
        __syncthreads();
        run_stages<LI, 1, NST, P, T, 1, true, true, true>(BufLd{fx, P}, st, fo, fx, P, tw);
    }
    if (a.epilogue && a.part) {
        const double t = block_sum_f64(acc.value(), red);
        if (threadIdx.x == 0) a.part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

template <class L>
constexpr size_t tpass_ct_smem() { return sizeof(float2) * (size_t)(2 * RInfo<L>::n() + 2 * RInfo<L>::n() * kP); }

// Portrait store of one inverse batch (pencil q = kk * P + p), skipping
// harmonics beyond the last one of the batch.
struct PortraitStK {
    float2* d;
    const float2* __restrict__ phase;
    long long M;
    int mx, row0, rows, kn;
    __device__ __forceinline__ void operator()(int m, int q, float2 val) const
    {
        const int kk = q / kP, p = q - kk * kP;
        if (kk >= kn) return;
        const float2 ph = __ldg(phase + kk);
        const int r = row0 + 2 * p;
        float2* dk = d + (long long)kk * M;
        if (r < rows) dk[(long long)r * mx + m] = make_float2(ph.x * val.x, ph.y * val.x);
        if (r + 1 < rows) dk[(long long)(r + 1) * mx + m] = make_float2(ph.x * val.y, ph.y * val.y);
    }
};

// X forward: LF = radix schedule of length nx, LI = schedule of the length
// mx = nx / S inverse, whose first radix is LF's last divided by S.
template <class LF, class LI, int S>
__global__ void __launch_bounds__(kT) k_xfwd_ct(const XArgs a)
{
    using IF = RInfo<LF>;
    using II = RInfo<LI>;
    constexpr int NX = IF::n(), MX = II::n(), NSTF = IF::nst, NSTI = II::nst, RL = IF::last(), R2 = II::first();
    static_assert(NX == MX * S && RL == R2 * S, "inconsistent X forward schedules");
    constexpr int P = kP, T = kT, KG = kKG, PB = KG * P;
    constexpr int NBL = NX / RL;   // = MX / R2
    constexpr int ITERL = (NBL * P + T - 1) / T;
    constexpr int BREG = 2 * NX * P, CREG = 2 * MX * PB;
    extern __shared__ float2 sm[];
    float2* tw = sm;                 // W_NX^t; W_MX^t = tw[t S]
    float2* b0 = tw + NX;
    float2* b1 = b0 + NX * P;
    float2* c0 = tw + NX;            // reused after the forward transform
    float2* c1 = c0 + MX * PB;
    (void)BREG;
    (void)CREG;
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const RowPairLd ld{a.vin, NX, row0, a.rows};
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
    for (int k0 = 0; k0 < a.K; k0 += KG) {
        const int kn = min(KG, a.K - k0);
        const PortraitStK pst{a.dout + (long long)k0 * a.M, a.phase + k0, a.M, MX, row0, a.rows, kn};
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
                    if constexpr (NSTI > 1) c0[(j * R2 + r2) * PB + kk * P + p] = G[r2];
                    else pst(j * R2 + r2, kk * P + p, G[r2]);
                }
            }
        }
        __syncthreads();
        if constexpr (NSTI > 1) run_stages<LI, 1, NSTI, PB, T, S, true, true, false>(BufLd{c0, PB}, pst, c1, c0, PB, tw);
    }
}

template <class LF, class LI, int S>
constexpr size_t xfwd_ct_smem()
{
    constexpr size_t nx = RInfo<LF>::n(), mx = RInfo<LI>::n();
    constexpr size_t b = 2 * nx * kP, c = 2 * mx * kKG * kP;
    return sizeof(float2) * (nx + (b > c ? b : c));
}

// X adjoint: LF2 = schedule of the length-mx forward transforms (one per
// harmonic), LI = schedule of the length-nx inverse, first radix = LF2's
// last times S.
template <class LF2, class LI, int S>
__global__ void __launch_bounds__(kT) k_xadj_ct(const XArgs a)
{
    using IF = RInfo<LF2>;
    using II = RInfo<LI>;
    constexpr int MX = IF::n(), NX = II::n(), NST2 = IF::nst, NSTI = II::nst, R = IF::last(), RI = II::first();
    static_assert(NX == MX * S && RI == R * S, "inconsistent X adjoint schedules");
    constexpr int P = kP, T = kT;
    constexpr int NBL = MX / R;    // = NX / RI
    constexpr int ITERL = (NBL * P + T - 1) / T;
    extern __shared__ float2 sm[];
    float2* tw = sm;               // W_NX^t; W_MX^t = tw[t S]
    float2* b0 = tw + NX;
    float2* b1 = b0 + NX * P;
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    float2 acc[ITERL][RI];
#pragma unroll
    for (int it = 0; it < ITERL; ++it)
#pragma unroll
        for (int r = 0; r < RI; ++r) acc[it][r] = make_float2(0.f, 0.f);
    constexpr int pf = result_parity<0, NST2 - 1>();
    float2* fo = pf ? b1 : b0;
    for (int k = 0; k < a.K; ++k) {
        const PortraitLd ld{a.din + (long long)k * a.M, a.phase + k, a.M, MX, row0, a.rows, P};
        if constexpr (NST2 > 1) run_stages<LF2, 0, NST2 - 1, P, T, S, false, false, true>(ld, BufSt{fo, P}, b0, b1, P, tw);
        const float2* __restrict__ xk = a.Xhat + (long long)k * NX;
#pragma unroll
        for (int it = 0; it < ITERL; ++it) {
            const int idx = (int)threadIdx.x + it * T;
            const int p = idx % P, j = idx / P;
            if ((NBL * P) % T != 0 && idx >= NBL * P) break;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = (NST2 > 1) ? fo[(j + r * NBL) * P + p] : ld(j + r * NBL, p);
            if (NBL > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw[r * j * S]);
            }
            dft<R, false>(v);
#pragma unroll
            for (int r = 0; r < RI; ++r) acc[it][r] = c_add(acc[it][r], c_mulc(v[r % R], __ldg(xk + j + r * NBL)));
        }
        __syncthreads();
    }
    const RowPairSt st{a.vout, NX, row0, a.rows};
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % P, j = idx / P;
        if ((NBL * P) % T != 0 && idx >= NBL * P) break;
        dft<RI, true>(acc[it]);
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            if constexpr (NSTI > 1) b0[(j * RI + r) * P + p] = acc[it][r];
            else st(j * RI + r, p, acc[it][r]);
        }
    }
    __syncthreads();
    if constexpr (NSTI > 1) run_stages<LI, 1, NSTI, P, T, 1, true, true, false>(BufLd{b0, P}, st, b1, b0, P, tw);
}

template <class LF2, class LI, int S>
constexpr size_t xadj_ct_smem()
{
    constexpr size_t nx = RInfo<LI>::n();
    return sizeof(float2) * (nx + 2 * nx * kP);
}

// X normal: LF = schedule of length nx whose last radix is divisible by S;
// the inverse runs the reversed schedule.
template <class LF, int S>
__global__ void __launch_bounds__(kT) k_xnrm_ct(const XArgs a)
{
    using IF = RInfo<LF>;
    using LI = Reverse<LF>;
    constexpr int NX = IF::n(), NST = IF::nst, R = IF::last(), R2 = R / S, MX = NX / S;
    static_assert(R % S == 0, "alias blocks must sit in one butterfly");
    constexpr int P = kP, T = kT;
    constexpr int NBL = NX / R;
    constexpr int ITERL = (NBL * P + T - 1) / T;
    extern __shared__ float2 sm[];
    __shared__ double red[34];
    float dummy;
    if (a.cg_active && !cg_enter(a.cg, false, &dummy, red)) return;
    float2* tw = sm;
    float2* b0 = tw + NX;
    float2* b1 = b0 + NX * P;
    for (int i = threadIdx.x; i < NX; i += T) tw[i] = a.twx[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const RowPairLd ld{a.vin, NX, row0, a.rows};
    DotAcc dacc;
    const NrmEpiSt st{&a, row0, &dacc};
    constexpr int pf = result_parity<0, NST - 1>();
    float2* fo = pf ? b1 : b0;
    float2* fx = pf ? b0 : b1;
    if constexpr (NST > 1) run_stages<LF, 0, NST - 1, P, T, 1, false, false, true>(ld, BufSt{fo, P}, b0, b1, P, tw);
#pragma unroll
    for (int it = 0; it < ITERL; ++it) {
        const int idx = (int)threadIdx.x + it * T;
        const int p = idx % P, j = idx / P;
        if ((NBL * P) % T != 0 && idx >= NBL * P) break;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = (NST > 1) ? fo[(j + r * NBL) * P + p] : ld(j + r * NBL, p);
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
        for (int r = 0; r < R; ++r) {
            if constexpr (NST > 1) fx[(j * R + r) * P + p] = g[r];
            else st(j * R + r, p, g[r]);
        }
    }
    __syncthreads();
    if constexpr (NST > 1) run_stages<LI, 1, NST, P, T, 1, true, true, false>(BufLd{fx, P}, st, fo, fx, P, tw);
    if (a.part) {
        const double t = block_sum_f64(dacc.value(), red);
        if (threadIdx.x == 0) a.part[blockIdx.x] = t;
    }
    (void)MX;
}

template <class LF, int S>
constexpr size_t xnrm_ct_smem()
{
    constexpr size_t nx = RInfo<LF>::n();
    return sizeof(float2) * (nx + 2 * nx * kP);
}

}  // namespace ct
}  // namespace mh3d
