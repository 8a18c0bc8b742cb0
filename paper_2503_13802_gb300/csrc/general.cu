// The general MH3D model on the GPU: the three-component convolution model
// d_k = e^{i theta_k} S_s( sum_j h_kj * (b_j rho) )  (Sec. 3.2, Eq. MH3Dcont,
// Eq. matrixModel), with PSFs that need not be separable -- the harmonic
// PSFs of the tensor PSF (appendix, Eq. PSF, Eq. skMD) or simulated ones.
// The caller supplies the PSF samples (h_k)_j at the grid's minimal-image
// offsets; the plan keeps their spectra, DFT(h)/N, as K * 3 complex volumes.
//
// Forward: the weighted volumes b_j rho, packed in pairs b_0 rho + i b_1 rho
// and b_2 rho (real images, two per complex transform), go through complex
// pencil passes along x, y and z (no spectral step); one pointwise kernel
// separates the pairs' spectra by their symmetry and forms every harmonic's
// portrait-grid spectrum
//   D_k(w') = sum_{a < s} e^{2 pi i (w' + a m_x) r / n_x} sum_j H_kj W_j (w' + a m_x)
// (the row selector x = s i' + r is exactly this alias sum with the offset
// phase), packed in harmonic pairs D_{2c} + i D_{2c+1} (two real images per
// complex transform), and inverse passes along x (length m_x), y and z over
// the pairs return c_k[z][y][s i' + r]; d_k = e^{i theta_k} Re c for each of
// the pair.  Adjoint: the real parts u_k = Re(e^{-i theta_k} d_k), packed in
// pairs, are transformed on the portrait grid, the unfold kernel separates
// each pair's spectra by their symmetry and forms
// V_j(f) = e^{-2 pi i f r / n_x} sum_k conj(H_kj(f)) U_k(f mod m_x) (the
// spectrum of u_k inserted at x = s i' + r, periodic in m_x), and the
// inverse passes and sum_j b_j Re V_j finish.  Each pass covers every
// harmonic (or component) in one launch, whatever K: 9 launches a call, or,
// where the pencil passes run the compile-time kernel (lengths 64 and 128)
// and carry the weighting b_j rho, the phase and the unphasing in their
// loads and stores, 7 for the forward and 8 for the adjoint.  Unnormalised
// transforms throughout; the 1/N sits in the stored spectra.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "fft_ct.cuh"
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

// Fused pre- and post-steps of the compile-time pencil kernel (MODE):
//   0  in place;
//   1  load the component pair c: b_{2c} rho + i b_{2c+1} rho (rho real
//      [N], b [nc][N] or null: one component, b = 1; b_nc = 0) -- the x pass
//      of the forward's packed component volumes, written to v;
//   2  store the pair c of portraits: volume c holds z_c = c_{2c} + i c_{2c+1}
//      (two real images in one complex transform), so d_{2c} =
//      e^{i theta_2c} Re(z_c) and d_{2c+1} = e^{i theta_2c+1} Im(z_c) -- the
//      z pass of the forward's inverse, written to dst (K portraits);
//   3  load z_c = u_{2c} + i u_{2c+1}, u_k = Re(e^{-i theta_k} d_k) (src =
//      the K portraits) -- the x pass of the adjoint's portrait transform,
//      written to v.
// The volume of pencil p (a component or a harmonic pair) is p / per_vol.
struct GenIO {
    const float* rho = nullptr;
    const float* b = nullptr;
    const float2* src = nullptr;
    float2* dst = nullptr;
    const float2* ph = nullptr;
    int K = 0;              // harmonics (modes 2, 3)
    long long Q = 0;        // portrait samples per harmonic (modes 2, 3)
    int nc = 1;             // sensitivity components (mode 1)
};

// The same transform for the common lengths (64, 128) with a compile-time
// radix schedule L and kGPC pencils per CTA.  The pencils are staged through
// shared memory with the coalesced mapping of their axis (elements fastest
// along x, where a pencil is a contiguous row; pencils fastest along y and
// z, where the CTA's pencils are neighbours in memory), every stage runs
// pencil-fast from shared memory, and the result leaves the same way.  The
// pencil stride kGPC + 1 keeps the element-fast staging conflict-free.
constexpr int kGPC = 16;
template <class L, bool INV, bool X, int MODE>
__global__ void __launch_bounds__(kGT) k_gen_line_ct(float2* v, Pencils g, const float2* __restrict__ tw, GenIO io)
{
    constexpr int N = ct::RInfo<L>::n(), NST = ct::RInfo<L>::nst, P = kGPC, LD = P + 1;
    constexpr int IT = N * P / kGT;
    static_assert((N * P) % kGT == 0, "whole staging rounds");
    __shared__ __align__(16) float2 b0[N * LD];
    __shared__ __align__(16) float2 b1[N * LD];
    __shared__ long long sbase[P], svol[P];
    __shared__ float2 sph[P], sph2[P];   // modes 2, 3: the pair's phases (the second zero past K)
    const long long p0 = (long long)blockIdx.x * P, np = g.count();
    if (threadIdx.x < P) {
        const long long pg = p0 + threadIdx.x;
        const long long c = pg < np ? pg / g.per_vol() : 0;
        sbase[threadIdx.x] = pg < np ? g.base(pg) : -1;
        svol[threadIdx.x] = c;
        if (MODE == 2 || MODE == 3) {
            sph[threadIdx.x] = io.ph[2 * c];
            sph2[threadIdx.x] = 2 * c + 1 < io.K ? io.ph[2 * c + 1] : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    const long long sd = g.stride();
    float2 t[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int idx = (int)threadIdx.x + i * kGT;
        const int e = X ? idx % N : idx / P, p = X ? idx / N : idx % P;
        const long long b = sbase[p];
        if (b < 0) {
            t[i] = make_float2(0.f, 0.f);
        } else if (MODE == 1) {
            // unconditional loads (the lone last component reads its own b
            // twice and zeroes the second), so the loads of the unrolled
            // rounds issue together
            const long long c = svol[p], off = b + e * sd - c * g.vstride;
            const float x = io.rho[off];
            if (io.b) {
                const long long c1 = 2 * c + 1 < io.nc ? 2 * c + 1 : 2 * c;
                const float w1 = 2 * c + 1 < io.nc ? 1.f : 0.f;
                t[i] = make_float2(x * io.b[2 * c * g.vstride + off], w1 * x * io.b[c1 * g.vstride + off]);
            } else {
                t[i] = make_float2(x, 0.f);
            }
        } else if (MODE == 3) {
            // in-volume offset of the element, then the pair's two portraits
            const long long c = svol[p], o = b + e * sd - c * g.vstride;
            const float2 da = io.src[2 * c * io.Q + o], pa = sph[p], pb = sph2[p];
            const float2 db = 2 * c + 1 < io.K ? io.src[(2 * c + 1) * io.Q + o] : make_float2(0.f, 0.f);
            t[i] = make_float2(pa.x * da.x + pa.y * da.y, pb.x * db.x + pb.y * db.y);
        } else {
            t[i] = v[b + e * sd];
        }
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int idx = (int)threadIdx.x + i * kGT;
        const int e = X ? idx % N : idx / P, p = X ? idx / N : idx % P;
        b1[e * LD + p] = t[i];
    }
    __syncthreads();
    // stage 0 reads b1 and writes b0; the last stage writes the buffer it
    // does not read
    float2* out = ((NST - 1) & 1) ? b1 : b0;
    ct::run_stages<L, 0, NST, P, kGT, 1, INV, true, true>(BufLd{b1, LD}, BufSt{out, LD}, b0, b1, LD, tw);
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int idx = (int)threadIdx.x + i * kGT;
        const int e = X ? idx % N : idx / P, p = X ? idx / N : idx % P;
        const long long b = sbase[p];
        if (b >= 0) {
            const float2 o = out[e * LD + p];
            if (MODE == 2) {
                const long long c = svol[p], off = b + e * sd - c * g.vstride;
                const float2 pa = sph[p], pb = sph2[p];
                io.dst[2 * c * io.Q + off] = make_float2(pa.x * o.x, pa.y * o.x);
                if (2 * c + 1 < io.K) io.dst[(2 * c + 1) * io.Q + off] = make_float2(pb.x * o.y, pb.y * o.y);
            } else {
                v[b + e * sd] = o;
            }
        }
    }
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
    // the component pairs: W[c] = b_{2c} rho + i b_{2c+1} rho (b = 1 without bvec; b_nc = 0)
    const int nv = (nc + 1) / 2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N * nv;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = i / N, v = i - c * N;
        const float x = rho[v];
        const float re = bvec ? x * bvec[2 * c * N + v] : x;
        const float im = (bvec && 2 * c + 1 < nc) ? x * bvec[(2 * c + 1) * N + v] : 0.f;
        W[i] = make_float2(re, im);
    }
}

// Portrait-grid spectra of every harmonic, D_k(w) = sum_a e^{2 pi i f r / nx}
// sum_j H_kj(f) W_j(f), f = w + a mx (the row selector x = s i' + r as an
// alias sum), q over [nz][ny][mx], written in harmonic pairs: Z_c = D_{2c} +
// i D_{2c+1} (D_K = 0), the spectrum of the complex image c_{2c} + i c_{2c+1}
// of two real portrait images, so that one inverse transform serves two
// harmonics.  One thread per q walks the harmonics.  SR > 0 (s <= SR): the
// thread keeps W_j(f) and the offset phases of its s frequencies in
// registers; SR = 0: any s, re-read per k.
//
// Each D_k is the spectrum of a real image: D_k(-q) = conj(D_k(q)), so
// Z_c(-q) = conj(D_{2c}(q)) + i conj(D_{2c+1}(q)).  Threads cover the planes
// z <= nz / 2 and write the mirror of every q off the planes z = 0 and
// 2 z = nz (which hold their own mirrors and are computed in full): each
// spectrum sample is read for one of f and -f only.
template <int SR>
__global__ void k_gen_fold(const float2* __restrict__ H, const float2* __restrict__ W, float2* __restrict__ Z,
                           int nx, int ny, int nz, int mx, int s, int r, int nc, int K, long long N, long long Q,
                           const float2* __restrict__ twx)
{
    const long long Qh = (long long)(nz / 2 + 1) * ny * mx;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Qh; q += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(q % mx);
        const long long row = (q - w) / mx * nx;   // (z ny + y) nx
        const int yz = (int)((q - w) / mx), y = yz % ny, z = yz / ny;
        const bool mirror = z != 0 && 2 * z != nz;
        const long long qm = ((long long)(nz - z) * ny + (ny - y) % ny) * mx + (mx - w) % mx;
        auto put = [&](int c, float2 da, float2 db) {
            Z[(long long)c * Q + q] = make_float2(da.x - db.y, da.y + db.x);
            if (mirror) Z[(long long)c * Q + qm] = make_float2(da.x + db.y, db.x - da.y);
        };
        // W holds the component pairs b_{2c} rho + i b_{2c+1} rho transformed:
        // with A = P_c(f) and B = conj(P_c(-f)), W_{2c} = (A + B) / 2 and
        // W_{2c+1} = (A - B) / 2i; a lone last component is P_c(f) itself
        const int zm = (nz - z) % nz, ym = (ny - y) % ny;
        auto wcomp = [&](int f, float2* out) {
            const long long i = row + f, im = ((long long)zm * ny + ym) * nx + (nx - f) % nx;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (2 * c >= nc) break;
                const float2 A = W[(long long)c * N + i];
                if (2 * c + 1 < nc) {
                    const float2 Bm = W[(long long)c * N + im];
                    out[2 * c] = make_float2(0.5f * (A.x + Bm.x), 0.5f * (A.y - Bm.y));
                    out[2 * c + 1] = make_float2(0.5f * (A.y + Bm.y), -0.5f * (A.x - Bm.x));
                } else {
                    out[2 * c] = A;
                }
            }
        };
        if constexpr (SR > 0) {
            float2 wv[SR][3], ph[SR];
#pragma unroll
            for (int a = 0; a < SR; ++a) {
                const int f = w + a * mx;
                wv[a][0] = wv[a][1] = wv[a][2] = make_float2(0.f, 0.f);
                if (a < s) wcomp(f, wv[a]);
                // e^{+2 pi i f r / nx} = conj(W_nx^{f r mod nx})
                const float2 tw = a < s ? twx[(int)(((long long)f * r) % nx)] : make_float2(0.f, 0.f);
                ph[a] = make_float2(tw.x, -tw.y);
            }
            auto fold_k = [&](int k) {
                const float2* __restrict__ Hk = H + (long long)k * 3 * N + row + w;
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int a = 0; a < SR; ++a) {
                    if (a < s) {
                        float2 t = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (j < nc) t = c_add(t, c_mul(Hk[(long long)j * N + a * mx], wv[a][j]));
                        acc = c_add(acc, c_mul(t, ph[a]));
                    }
                }
                return acc;
            };
            for (int c = 0; 2 * c < K; ++c)
                put(c, fold_k(2 * c), 2 * c + 1 < K ? fold_k(2 * c + 1) : make_float2(0.f, 0.f));
        } else {
            auto fold_k = [&](int k) {
                const float2* __restrict__ Hk = H + (long long)k * 3 * N;
                float2 acc = make_float2(0.f, 0.f);
                for (int a = 0; a < s; ++a) {
                    const int f = w + a * mx;
                    const long long i = row + f;
                    float2 wj[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    wcomp(f, wj);
                    float2 t = make_float2(0.f, 0.f);
                    for (int j = 0; j < nc; ++j) t = c_add(t, c_mul(Hk[(long long)j * N + i], wj[j]));
                    const float2 tw = twx[(int)(((long long)f * r) % nx)];
                    acc = c_add(acc, c_mul(t, make_float2(tw.x, -tw.y)));
                }
                return acc;
            };
            for (int c = 0; 2 * c < K; ++c)
                put(c, fold_k(2 * c), 2 * c + 1 < K ? fold_k(2 * c + 1) : make_float2(0.f, 0.f));
        }
    }
}

// d_{2c} = e^{i theta_2c} Re(z_c), d_{2c+1} = e^{i theta_2c+1} Im(z_c): the
// harmonic pairs' images unpacked into the K portraits (ph[k] = e^{i theta_k})
__global__ void k_gen_phase(const float2* __restrict__ Zi, float2* __restrict__ d, long long Q, int K,
                            const float2* __restrict__ ph)
{
    const int Kh = (K + 1) / 2;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < Q * Kh;
         g += (long long)gridDim.x * blockDim.x) {
        const long long c = g / Q, o = g - c * Q;
        const float2 z = Zi[g], pa = ph[2 * c];
        d[2 * c * Q + o] = make_float2(pa.x * z.x, pa.y * z.x);
        if (2 * c + 1 < K) {
            const float2 pb = ph[2 * c + 1];
            d[(2 * c + 1) * Q + o] = make_float2(pb.x * z.y, pb.y * z.y);
        }
    }
}

// z_c = u_{2c} + i u_{2c+1}, u_k = Re(e^{-i theta_k} d_k): the harmonic
// pairs of real portrait images packed for one complex transform each
__global__ void k_gen_unphase(const float2* __restrict__ d, float2* __restrict__ U, long long Q, int K,
                              const float2* __restrict__ ph)
{
    const int Kh = (K + 1) / 2;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < Q * Kh;
         g += (long long)gridDim.x * blockDim.x) {
        const long long c = g / Q, o = g - c * Q;
        const float2 pa = ph[2 * c], va = d[2 * c * Q + o];
        float ub = 0.f;
        if (2 * c + 1 < K) {
            const float2 pb = ph[2 * c + 1], vb = d[(2 * c + 1) * Q + o];
            ub = pb.x * vb.x + pb.y * vb.y;
        }
        U[g] = make_float2(pa.x * va.x + pa.y * va.y, ub);
    }
}

// The adjoint of the fold.  u_k inserted at x = s i' + r (zero elsewhere)
// has the spectrum e^{-2 pi i f r / nx} U_k(f mod mx) along x, U_k the
// transform of u_k over the portrait grid (s / nx = 1 / mx), so
//   V_j(f) = e^{-2 pi i f r / nx} sum_k conj(H_kj(f)) U_k(f mod mx).
// One thread per frequency f walks the harmonics.  V_j is the spectrum of
// a real image (H, U real images' spectra): V_j(-f) = conj(V_j(f)), so the
// threads cover the planes z <= nz / 2 and write the mirrors off the planes
// z = 0 and 2 z = nz, as the fold does.
__global__ void k_gen_unfold(const float2* __restrict__ H, const float2* __restrict__ U, float2* __restrict__ V,
                             int nx, int ny, int nz, int mx, int r, int nc, int K, long long N, long long Q,
                             const float2* __restrict__ twx)
{
    const long long Nh = (long long)(nz / 2 + 1) * ny * nx;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nh; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i % nx);
        const int yz = (int)((i - f) / nx), y = yz % ny, z = yz / ny;
        const bool mirror = z != 0 && 2 * z != nz;
        const long long im = ((long long)(nz - z) * ny + (ny - y) % ny) * nx + (nx - f) % nx;
        const int w = f % mx;
        const long long qi = (long long)yz * mx + w;
        // the portrait-grid mirror -g of g = (w, y, z)
        const long long qim = ((long long)((nz - z) % nz) * ny + (ny - y) % ny) * mx + (mx - w) % mx;
        float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int c = 0; 2 * c < K; ++c) {
            // U holds z_c = u_{2c} + i u_{2c+1} transformed: with A = Z(g) and
            // B = conj(Z(-g)), U_{2c}(g) = (A + B) / 2, U_{2c+1}(g) = (A - B) / 2i
            const float2 A = U[(long long)c * Q + qi], Bm = U[(long long)c * Q + qim];
            const float2 B = make_float2(Bm.x, -Bm.y);
            const float2 ua = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
            const float2 ub = make_float2(0.5f * (A.y - B.y), -0.5f * (A.x - B.x));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * c + h;
                if (k >= K) break;
                const float2 u = h == 0 ? ua : ub;
                const float2* __restrict__ Hk = H + (long long)k * 3 * N + i;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j < nc) {
                        const float2 hv = Hk[(long long)j * N];
                        acc[j] = c_add(acc[j], c_mul(make_float2(hv.x, -hv.y), u));
                    }
                }
            }
        }
        const float2 tw = twx[(int)(((long long)f * r) % nx)];   // e^{-2 pi i f r / nx}
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (j < nc) {
                const float2 v = c_mul(acc[j], tw);
                V[(long long)j * N + i] = v;
                if (mirror) V[(long long)j * N + im] = make_float2(v.x, -v.y);
            }
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

// MH3D_GEN_RUNTIME=1 keeps every length on the runtime-schedule kernel.
bool gen_runtime_only()
{
    const char* e = std::getenv("MH3D_GEN_RUNTIME");
    return e && e[0] && e[0] != '0';
}

// Lengths served by the compile-time pencil kernel (and its fused modes).
bool gen_ct_length(int n) { return (n == 128 || n == 64) && !gen_runtime_only(); }

template <class L, bool INV, bool X>
void gen_line_ct_launch(int grid, float2* v, const Pencils& g, const float2* tw, int mode, const GenIO& io,
                        cudaStream_t st)
{
    if (mode == 1) k_gen_line_ct<L, INV, X, 1><<<grid, kGT, 0, st>>>(v, g, tw, io);
    else if (mode == 2) k_gen_line_ct<L, INV, X, 2><<<grid, kGT, 0, st>>>(v, g, tw, io);
    else if (mode == 3) k_gen_line_ct<L, INV, X, 3><<<grid, kGT, 0, st>>>(v, g, tw, io);
    else k_gen_line_ct<L, INV, X, 0><<<grid, kGT, 0, st>>>(v, g, tw, io);
}

template <class L>
void gen_line_ct(int grid, float2* v, const Pencils& g, const float2* tw, bool inv, int mode, const GenIO& io,
                 cudaStream_t st)
{
    const bool x = g.axis == 0;
    if (inv && x) gen_line_ct_launch<L, true, true>(grid, v, g, tw, mode, io, st);
    else if (inv) gen_line_ct_launch<L, true, false>(grid, v, g, tw, mode, io, st);
    else if (x) gen_line_ct_launch<L, false, true>(grid, v, g, tw, mode, io, st);
    else gen_line_ct_launch<L, false, false>(grid, v, g, tw, mode, io, st);
}

// Transform of every pencil of `vols` volumes (rows of width W, vstride
// float2 apart) along `axis`, in place, or with a fused step (mode, io: see
// GenIO; modes other than 0 need gen_ct_length(ap.n)).
cudaError_t gen_line(float2* v, int axis, int W, int ny, int nz, int vols, long long vstride, const AxisPlan& ap,
                     bool inv, cudaStream_t st, int mode = 0, const GenIO& io = GenIO{})
{
    Pencils g{axis, W, ny, nz};
    g.vols = vols;
    g.vstride = vstride;
    const long long np = g.count();
    if (gen_ct_length(ap.n)) {
        const int gc = (int)((np + kGPC - 1) / kGPC);
        if (ap.n == 128) gen_line_ct<ct::RList<16, 8>>(gc, v, g, ap.tw, inv, mode, io, st);
        else gen_line_ct<ct::RList<8, 8>>(gc, v, g, ap.tw, inv, mode, io, st);
        return cudaGetLastError();
    }
    if (mode != 0) return cudaErrorInvalidValue;
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
// of `axp`: three launches, each over every volume's pencils.  mode_x /
// io_x fuse a load step into the x pass, mode_z a store step into the z pass.
cudaError_t gen_fft3(const Plan& P, float2* v, int count, const AxisPlan& axp, bool inv, cudaStream_t st,
                     int mode_x = 0, int mode_z = 0, const GenIO& io = GenIO{})
{
    const long long vol = (long long)axp.n * P.ny * P.nz;
    cudaError_t e;
    if ((e = gen_line(v, 0, axp.n, P.ny, P.nz, count, vol, axp, inv, st, mode_x, io)) != cudaSuccess) return e;
    if ((e = gen_line(v, 1, axp.n, P.ny, P.nz, count, vol, P.ay, inv, st)) != cudaSuccess) return e;
    return gen_line(v, 2, axp.n, P.ny, P.nz, count, vol, P.az, inv, st, mode_z, io);
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
    if (P.gen_cg) cudaFree(P.gen_cg);
    P.gen_H = nullptr;
    P.gen_work = nullptr;
    P.gen_cg = nullptr;
    P.gen_cg_cap = 0;
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
    // work area: 3 component volumes + one portrait-grid volume per harmonic
    const long long Q = (long long)P.nz * P.ny * P.mx;
    if (!P.gen_work) GEN_CK(P, dev_malloc(&P.gen_work, sizeof(float2) * (size_t)(3 * N + P.K * Q)));
    // the real samples are staged in the work area (>= 3N float2 >= 3N floats per harmonic)
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
    float2* W = P.gen_work;           // the component pairs (nc + 1) / 2 volumes
    float2* Z = P.gen_work + 3 * N;   // the harmonic pairs' portrait-grid spectra, then images
    const int nv = (nc + 1) / 2;
    const int Kh = (P.K + 1) / 2;
    GenIO io;
    io.rho = rho;
    io.b = bvec;
    io.ph = P.phase;
    io.dst = (float2*)d;
    io.K = P.K;
    io.Q = Q;
    io.nc = nc;
    if (gen_ct_length(P.ax.n)) {   // the pairs b_j rho formed in the x pass's load
        GEN_CK(P, gen_fft3(P, W, nv, P.ax, false, st, 1, 0, io));
    } else {
        k_gen_weight<<<gen_blocks(N * nv), kGB, 0, st>>>(rho, bvec, W, N, nc);
        GEN_CK(P, cudaGetLastError());
        GEN_CK(P, gen_fft3(P, W, nv, P.ax, false, st));
    }
    const long long Qh = (long long)(P.nz / 2 + 1) * P.ny * P.mx;   // the planes the fold's threads cover
    if (P.s <= 2)
        k_gen_fold<2><<<gen_blocks(Qh), kGB, 0, st>>>(P.gen_H, W, Z, P.nx, P.ny, P.nz, P.mx, P.s, P.r, nc, P.K, N, Q,
                                                      P.ax.tw);
    else if (P.s <= 4)
        k_gen_fold<4><<<gen_blocks(Qh), kGB, 0, st>>>(P.gen_H, W, Z, P.nx, P.ny, P.nz, P.mx, P.s, P.r, nc, P.K, N, Q,
                                                      P.ax.tw);
    else
        k_gen_fold<0><<<gen_blocks(Qh), kGB, 0, st>>>(P.gen_H, W, Z, P.nx, P.ny, P.nz, P.mx, P.s, P.r, nc, P.K, N, Q,
                                                      P.ax.tw);
    GEN_CK(P, cudaGetLastError());
    if (gen_ct_length(P.az.n)) {   // the pairs unpacked and phased in the z pass's store
        GEN_CK(P, gen_fft3(P, Z, Kh, P.am, true, st, 0, 2, io));
    } else {
        GEN_CK(P, gen_fft3(P, Z, Kh, P.am, true, st));
        k_gen_phase<<<gen_blocks(Q * Kh), kGB, 0, st>>>(Z, (float2*)d, Q, P.K, P.phase);
        GEN_CK(P, cudaGetLastError());
    }
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
    float2* U = P.gen_work + 3 * N;  // the harmonic pairs of real portrait images, then their spectra
    const int Kh = (P.K + 1) / 2;
    if (gen_ct_length(P.am.n)) {   // the pairs formed in the x pass's load
        GenIO io;
        io.src = (const float2*)d;
        io.ph = P.phase;
        io.K = P.K;
        io.Q = Q;
        GEN_CK(P, gen_fft3(P, U, Kh, P.am, false, st, 3, 0, io));
    } else {
        k_gen_unphase<<<gen_blocks(Q * Kh), kGB, 0, st>>>((const float2*)d, U, Q, P.K, P.phase);
        GEN_CK(P, cudaGetLastError());
        GEN_CK(P, gen_fft3(P, U, Kh, P.am, false, st));
    }
    const long long Nh = (long long)(P.nz / 2 + 1) * P.ny * P.nx;   // the planes the unfold's threads cover
    k_gen_unfold<<<gen_blocks(Nh), kGB, 0, st>>>(P.gen_H, U, V, P.nx, P.ny, P.nz, P.mx, P.r, nc, P.K, N, Q, P.ax.tw);
    GEN_CK(P, cudaGetLastError());
    GEN_CK(P, gen_fft3(P, V, nc, P.ax, true, st));
    k_gen_out<<<gen_blocks(N), kGB, 0, st>>>(V, bvec, out, N, nc);
    GEN_CK(P, cudaGetLastError());
    return MH3D_OK;
}

}  // extern "C"
