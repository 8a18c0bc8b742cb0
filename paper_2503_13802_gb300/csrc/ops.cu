// Pencil kernels of the MH3D operator on sm_103a.
//
// The separable PSF h_k = c_k X_k (x) Y (x) Z (drive axis x) turns the 3D
// circular convolution of Eq. portz into one 1D circular convolution per
// axis; every axis is applied by a kernel that owns whole pencils of that
// axis in shared memory, transforms them (Stockham, fft_smem.cuh),
// multiplies in the Fourier domain and transforms back.  No 3D spectrum is
// ever stored.
//
//   T pass (y or z): tiles of `cols` consecutive x columns at one position of
//     the other transverse axis; column pairs are packed as one complex
//     pencil (both kernels are real, so real and imaginary parts convolve
//     independently).  Optional fusions: input or output times b (B of
//     Eq. dN), the CG direction update p = r + beta p in the loader, and the
//     CG epilogue q = b w + lambda R p with the partial p^T q in the storer.
//   X forward: row pairs packed as complex pencils; one forward FFT of
//     length nx, then per harmonic the product with the drive-axis spectrum
//     folded over the s aliases (the row selector P of Eq. dN is exactly a
//     spectral fold), an inverse FFT of length nx/s and the phase
//     e^{i theta_k} (Sec. 4.4) on the store.
//   X adjoint: per harmonic the projection Re(e^{-i theta_k} y_k), a forward
//     FFT of length nx/s, the periodised spectrum (zero insertion P^T) times
//     conj of the drive spectrum, summed over k on chip, one inverse FFT.
//   X normal: the drive-axis part of A^T A, sum_k X_k^T P^T P X_k, which in
//     the Fourier domain couples only the s aliases of each frequency:
//     an s x s block per alias class, precomputed in FP64.
#include <cstdio>

#include "ops_kernels.cuh"
#include "ops_functors.cuh"

namespace mh3d {

__global__ void __launch_bounds__(256) k_tpass(const TArgs a)
{
    extern __shared__ float2 sm[];
    __shared__ double red[34];
    __shared__ float cgs[3];
    float beta = 0.f, alpha = 0.f;
    if (a.cg.flags && !cg_enter_cta(a.cg, a.pupdate != 0, &beta, &alpha, cgs)) return;
    const int n = a.n, P = a.cols / 2, ld = P + 1;
    float2* tw = sm;
    float2* mu = tw + n;
    float2* s0 = mu + n;
    float2* s1 = s0 + n * ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tw[i] = a.tw[i];
        mu[i] = a.mult[i];
    }
    __syncthreads();
    const int x0 = blockIdx.x * a.cols;
    const long long base = (long long)blockIdx.y * a.os;
    const int res = fft_result_index(a.rp.nst);
    float2* sr = res ? s1 : s0;
    float2* so = res ? s0 : s1;
    DotAcc acc, acc2;
    fft_run<false, true, true>(a.rp, TLoad{&a, base, x0, beta, alpha}, BufSt{sr, ld}, s0, s1, ld, P, tw);
    fft_run<true, true, true>(a.rp, MulLd{sr, ld, mu}, TStore{&a, base, x0, &acc, a.part2 ? &acc2 : nullptr}, so,
                              sr, ld, P, tw);
    if (a.epilogue && a.part) {
        const int bid = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
        float2 t, t2;
        block_pair_acc2(acc, a.part2 ? &acc2 : nullptr, reinterpret_cast<float*>(red), &t, &t2);
        if (a.part2) grid_sum_finalize2(t, t2, a.part, a.part2, bid, nb, a.ticket, a.sum_out, a.sum_out2);
        else grid_sum_finalize(t, a.part, bid, nb, a.ticket, a.sum_out);
    }
    if (a.count_iter) cg_count_iteration(a.cg);
}

int tpass_blocks(int nx, int cols, int nouter) { return ((nx + cols - 1) / cols) * nouter; }

cudaError_t run_tpass(const TArgs& a, int nouter, cudaStream_t st)
{
    if (ct_tpass_available(a)) return run_tpass_ct(a, nouter, st);
    dim3 grid((a.nx + a.cols - 1) / a.cols, nouter);
    const size_t smem = tpass_smem_bytes(a.n, a.cols);
    k_tpass<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// X pass kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_xfwd(const XArgs a)
{
    extern __shared__ float2 sm[];
    const int nx = a.nx, mx = a.mx, P = a.pairs, ldA = P + 1;
    const int PB = a.kg * P, ldB = PB + 1;
    float2* twx = sm;
    float2* twm = twx + nx;
    float2* A0 = twm + mx;
    float2* A1 = A0 + nx * ldA;
    float2* B0 = A1 + nx * ldA;
    float2* B1 = B0 + mx * ldB;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) twx[i] = a.twx[i];
    for (int i = threadIdx.x; i < mx; i += blockDim.x) twm[i] = a.twm[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const int res = fft_result_index(a.rpx.nst);
    float2* Ar = res ? A1 : A0;
    fft_run<false, false, true>(a.rpx, RowPairLd{a.vin, nx, row0, a.rows}, BufSt{Ar, ldA}, A0, A1, ldA, P, twx);
    for (int k0 = 0; k0 < a.K; k0 += a.kg) {
        const int kn = min(a.kg, a.K - k0);
        fft_run<true, true, false>(a.rpm, FoldLd{Ar, ldA, a.Xhat + (long long)k0 * nx, nx, mx, a.s, P},
                                   PortraitSt{a.dout + (long long)k0 * a.M, a.phase + k0, a.M, mx, row0, a.rows, P},
                                   B0, B1, ldB, kn * P, twm);
    }
}

__global__ void __launch_bounds__(256) k_xadj(const XArgs a)
{
    extern __shared__ float2 sm[];
    const int nx = a.nx, mx = a.mx, P = a.pairs, ldA = P + 1;
    const int PB = a.kg * P, ldB = PB + 1;
    float2* twx = sm;
    float2* twm = twx + nx;
    float2* acc = twm + mx;            // [nx][ldA]
    float2* S0 = acc + nx * ldA;       // scratch region (max of both uses)
    float2* B1 = S0 + mx * ldB;
    float2* S1 = S0 + nx * ldA;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) twx[i] = a.twx[i];
    for (int i = threadIdx.x; i < mx; i += blockDim.x) twm[i] = a.twm[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const int resm = fft_result_index(a.rpm.nst);
    float2* Fr = resm ? B1 : S0;
    for (int k0 = 0; k0 < a.K; k0 += a.kg) {
        const int kn = min(a.kg, a.K - k0);
        fft_run<false, false, true>(a.rpm,
                                    PortraitLd{a.din + (long long)k0 * a.M, a.phase + k0, a.M, mx, row0, a.rows, P},
                                    BufSt{Fr, ldB}, S0, B1, ldB, kn * P, twm);
        // acc[w][p] (+)= sum_kk conj(Xhat_k[w]) F_kk[w mod mx][p]
        for (int idx = threadIdx.x; idx < nx * P; idx += blockDim.x) {
            const int p = idx % P, w = idx / P;
            const int m = w % mx;
            float2 v = (k0 == 0) ? make_float2(0.f, 0.f) : acc[w * ldA + p];
            for (int kk = 0; kk < kn; ++kk)
                v = c_add(v, c_mulc(Fr[m * ldB + kk * P + p], __ldg(a.Xhat + (long long)(k0 + kk) * nx + w)));
            acc[w * ldA + p] = v;
        }
        __syncthreads();
    }
    fft_run<true, true, false>(a.rpx, BufLd{acc, ldA}, RowPairSt{a.vout, nx, row0, a.rows}, S0, S1, ldA, P, twx);
}

__global__ void __launch_bounds__(256) k_xnrm(const XArgs a)
{
    extern __shared__ float2 sm[];
    __shared__ double red[34];
    float dummy;
    if (a.cg_active && !cg_enter(a.cg, false, &dummy, red)) return;
    const int nx = a.nx, P = a.pairs, ldA = P + 1;
    float2* twx = sm;
    float2* A0 = twx + nx;
    float2* A1 = A0 + nx * ldA;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) twx[i] = a.twx[i];
    __syncthreads();
    const int row0 = blockIdx.x * 2 * P;
    const int res = fft_result_index(a.rpx.nst);
    float2* Ar = res ? A1 : A0;
    float2* Ao = res ? A0 : A1;
    DotAcc dacc, dacc2;
    fft_run<false, false, true>(a.rpx, RowPairLd{a.vin, nx, row0, a.rows}, BufSt{Ar, ldA}, A0, A1, ldA, P, twx);
    fft_run<true, true, false>(a.rpx, QLd{Ar, ldA, a.Q, a.mx, a.s},
                               NrmEpiSt{&a, row0, &dacc, a.part2 ? &dacc2 : nullptr}, Ao, Ar, ldA, P, twx);
    if (a.part) {
        float2 t, t2;
        block_pair_acc2(dacc, a.part2 ? &dacc2 : nullptr, reinterpret_cast<float*>(red), &t, &t2);
        if (a.part2) grid_sum_finalize2(t, t2, a.part, a.part2, blockIdx.x, gridDim.x, a.ticket, a.sum_out, a.sum_out2);
        else grid_sum_finalize(t, a.part, blockIdx.x, gridDim.x, a.ticket, a.sum_out);
    }
    if (a.count_iter) cg_count_iteration(a.cg);
}

int xpass_blocks(int rows, int pairs) { return (rows + 2 * pairs - 1) / (2 * pairs); }

cudaError_t run_xfwd(const XArgs& a, cudaStream_t st)
{
    if (ct_xpass_available(a.nx, a.s, a.pairs)) return run_xfwd_ct(a, st);
    k_xfwd<<<xpass_blocks(a.rows, a.pairs), 256, xfwd_smem_bytes(a.nx, a.mx, a.pairs, a.kg), st>>>(a);
    return cudaGetLastError();
}
cudaError_t run_xadj(const XArgs& a, cudaStream_t st)
{
    if (ct_xpass_available(a.nx, a.s, a.pairs)) return run_xadj_ct(a, st);
    k_xadj<<<xpass_blocks(a.rows, a.pairs), 256, xadj_smem_bytes(a.nx, a.mx, a.pairs, a.kg), st>>>(a);
    return cudaGetLastError();
}
cudaError_t run_xnrm(const XArgs& a, cudaStream_t st)
{
    if (ct_xpass_available(a.nx, a.s, a.pairs)) return run_xnrm_ct(a, st);
    k_xnrm<<<xpass_blocks(a.rows, a.pairs), 256, xnrm_smem_bytes(a.nx, a.pairs), st>>>(a);
    return cudaGetLastError();
}

// Opt every pencil kernel into the device's full shared-memory carve-out
// (the opt-in limit minus the kernel's static shared memory).
template <class F>
static cudaError_t opt_in_smem(F* f, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

cudaError_t ops_set_attributes()
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if ((e = opt_in_smem(k_tpass, optin)) != cudaSuccess) return e;
    if ((e = opt_in_smem(k_xfwd, optin)) != cudaSuccess) return e;
    if ((e = opt_in_smem(k_xadj, optin)) != cudaSuccess) return e;
    if ((e = opt_in_smem(k_xnrm, optin)) != cudaSuccess) return e;
    if ((e = xw_set_attributes()) != cudaSuccess) return e;
    return ct_set_attributes(optin);
}

}  // namespace mh3d
