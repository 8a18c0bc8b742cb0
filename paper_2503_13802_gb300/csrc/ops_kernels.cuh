// Kernel argument blocks shared by ops.cu and solve.cu.
#pragma once

#include <cuda.h>

#include "fft_smem.cuh"

namespace mh3d {

// Control block of a device-resident CG loop.  Every kernel of an
// iteration reads only values written by earlier kernels; values that a
// kernel both reads and writes are double-buffered by iteration parity
// (`par`, baked into each captured graph node).
struct CgCtl {
    int* flags = nullptr;            // [0] done, [1] completed iterations, [2] status
    const double* rr_new = nullptr;  // r^T r after the previous update (scalar)
    const double* rr_old = nullptr;  // r^T r one update earlier (scalar)
    const double* bn = nullptr;      // ||A^T d||^2 (scalar)
    double* hist = nullptr;          // hist[it] = ||r_it|| / ||A^T d||
    int hist_cap = 0;
    int max_iter = 0;
    double tol2 = 0.0;               // rel_tol^2 (0 = fixed iterations)
    unsigned long long cond = 0;     // cudaGraphConditionalHandle of the loop
    int use_cond = 0;
    // single-reduction (Chronopoulos-Gear) form: delta = r^T A r of the
    // current residual, the previous step length, and where to store the new one
    int cgcg = 0;
    const double* delta = nullptr;
    const double* alpha_prev = nullptr;
    double* alpha_out = nullptr;
    // 1: beta and alpha are FP64 quotients (rounded to FP32 only where the
    // FP32 vectors are updated); 0: FP32 quotients of the split significands
    int fp64 = 1;
};

// Destination of a grid-wide FP64 reduction: per-CTA partials, the ticket
// counter of the last-CTA finalisation, and the scalar total.
struct RedSink {
    double* part = nullptr;
    unsigned int* ticket = nullptr;
    double* out = nullptr;
    double* part2 = nullptr;         // optional second total (input . input)
    double* out2 = nullptr;
};

// Regulariser applied in epilogues: out += lambda * R p.
struct RegArgs {
    int kind = 0;                    // 0: R = I; 1: T^T T + alpha P_a^T P_a
    float lambda = 0.f;
    float alpha = 0.f;
    int shell = 1;
    int nx = 1, ny = 1, nz = 1;
};

// Tensor maps of the T-pass tiles (one per vector), encoded on the host for
// the box (cols x n x 1) along y or (cols x 1 x n) along z.
enum { kTmIn = 0, kTmB, kTmR, kTmS, kTmP, kTmQ, kTmX, kTmOut, kTmPin, kTmCount };
struct TMaps {
    CUtensorMap m[kTmCount];
};

// T pass: 1D circular convolution along y or z of tiles of `cols` columns.
struct TArgs {
    TMaps tm;                        // filled by the bulk-copy launcher
    int axis = 1;                    // 1 = y, 2 = z
    const float* in = nullptr;
    float* out = nullptr;
    const float* bin = nullptr;      // input multiplied by b (or null)
    const float* bout = nullptr;     // output multiplied by b (or null)
    const float2* mult = nullptr;    // spectral multiplier [n]
    const float2* tw = nullptr;      // twiddles [n]
    RadixPlan rp{};
    int n = 1;
    long long es = 0;                // element stride along the axis (floats)
    long long os = 0;                // stride of blockIdx.y positions
    int nx = 1;
    int cols = 32;
    int vec2 = 1;                    // nx even: float2 global access
    int vec4 = 0;                    // nx % 4 == 0 and every vector 16-byte aligned: float4 access
    int* status = nullptr;           // device status word (bounded waits record timeouts here)
    unsigned debug_extra_tx = 0;     // fault test only: bytes the tile barrier waits for that never arrive
    int radix_alt = 0;               // 1: the alternative radix schedule (where instantiated)
    // CG fusions
    int pupdate = 0;                 // loader: 1 = p = r + beta p (written back), value = b p;
                                     //         2 = p = r + beta p, q = s + beta q, x += alpha p,
                                     //             r -= alpha q (all written back), value = b r
    float* pvec = nullptr;
    const float* rvec = nullptr;
    float* rvec_w = nullptr;         // r written back (mode 2)
    float* qdir = nullptr;           // q = A p recurrence (mode 2)
    const float* svec = nullptr;     // s = A r (mode 2)
    float* xvec = nullptr;           // iterate (mode 2)
    int epilogue = 0;                // storer: q = b w + lambda R p, partial p^T q
    float* qvec = nullptr;
    const float* pin = nullptr;      // p for the epilogue
    double* part = nullptr;          // per-CTA partials of p^T q (null: none)
    unsigned int* ticket = nullptr;  // grid reduction counter
    double* sum_out = nullptr;       // p^T q total
    double* part2 = nullptr;         // optional second total p^T p (same ticket)
    double* sum_out2 = nullptr;
    int count_iter = 0;              // last pass of a CG iteration: advance the counter
    RegArgs reg{};
    CgCtl cg{};
};

// X pass (drive axis, contiguous rows).
struct XArgs {
    const float* vin = nullptr;      // fwd / normal: input rows [rows][nx]
    float* vout = nullptr;           // adj: output rows
    float2* dout = nullptr;          // fwd: portraits [K][rows][mx]
    const float2* din = nullptr;     // adj: portraits
    const float2* Xhat = nullptr;    // [K][nx]
    const float2* phase = nullptr;   // [K]
    const float2* Q = nullptr;       // [mx][s][s]
    const float2* twx = nullptr;
    const float2* twm = nullptr;
    RadixPlan rpx{}, rpm{};
    int nx = 1, mx = 1, s = 1, K = 1;
    int rows = 1;
    long long M = 1;                 // rows * mx
    int pairs = 16;                  // row pairs per CTA
    int kg = 4;                      // harmonics per transform batch
    int kpc = 0;                     // specialised forward: harmonics per CTA (grid.y groups; 0: all)
    int vec4 = 0;                    // nx % 4 == 0 and every vector 16-byte aligned
    // normal-mode epilogue
    const float* b = nullptr;
    const float* pin = nullptr;
    float* qout = nullptr;
    double* part = nullptr;          // per-CTA partials of p^T q (null: none)
    unsigned int* ticket = nullptr;
    double* sum_out = nullptr;
    double* part2 = nullptr;         // optional second total p^T p (same ticket)
    double* sum_out2 = nullptr;
    int count_iter = 0;              // last pass of a CG iteration: advance the counter
    RegArgs reg{};
    CgCtl cg{};
    int cg_active = 0;
    int* status = nullptr;           // device status word for bounded-wait timeouts
    int ks = 0;                      // warp-centric passes: warps per row group (0: default)
};

// The y-slab cluster passes (ops_ct.cuh: k_zxnrm_ct, k_zxfwd_ct,
// k_xzadj_ct): one y-slab per cluster of C CTAs.
struct ZXArgs {
    CUtensorMap tz;                  // the z volume (input, or the adjoint's output), box (nx/C x 1 x nz)
    XArgs x;                         // the normal pass; x.vin unused (rows come through the cluster)
    const float2* twz = nullptr;     // W_nz^t
    const float2* muz = nullptr;     // z-axis normal multiplier [nz]
    int ny = 1, nz = 1;
    int C = 0;                       // CTAs per y-slab (2 or 4; 0: default)
};

// Shared-memory sizes in bytes.
__host__ __forceinline__ size_t tpass_smem_bytes(int n, int cols)
{
    const int P = cols / 2;
    return sizeof(float2) * (size_t)(2 * n + 2 * n * (P + 1));
}
__host__ __forceinline__ size_t xfwd_smem_bytes(int nx, int mx, int pairs, int kg)
{
    return sizeof(float2) * (size_t)(nx + mx + 2 * nx * (pairs + 1) + 2 * mx * (kg * pairs + 1));
}
__host__ __forceinline__ size_t xadj_smem_bytes(int nx, int mx, int pairs, int kg)
{
    size_t a = 2 * (size_t)mx * (kg * pairs + 1), b = 2 * (size_t)nx * (pairs + 1);
    return sizeof(float2) * (size_t)(nx + mx + (size_t)nx * (pairs + 1) + (a > b ? a : b));
}
__host__ __forceinline__ size_t xnrm_smem_bytes(int nx, int pairs)
{
    return sizeof(float2) * (size_t)(nx + 2 * nx * (pairs + 1));
}

// Launchers (ops.cu).
cudaError_t run_tpass(const TArgs& a, int nouter, cudaStream_t st);
cudaError_t run_xfwd(const XArgs& a, cudaStream_t st);
cudaError_t run_xadj(const XArgs& a, cudaStream_t st);
cudaError_t run_xnrm(const XArgs& a, cudaStream_t st);
int tpass_blocks(int nx, int cols, int nouter);

// Compile-time specialised kernels (ops_ct.cu) for the common lengths.
bool ct_tpass_available(const TArgs& a);
bool ct_xpass_available(int nx, int s, int pairs);
cudaError_t ct_set_attributes(int optin);
cudaError_t run_tpass_ct(const TArgs& a, int nouter, cudaStream_t st);
cudaError_t run_xfwd_ct(const XArgs& a, cudaStream_t st);
cudaError_t run_xadj_ct(const XArgs& a, cudaStream_t st);
// Fused T_z + normal pass where instantiated (false: use the two passes).
bool ct_zxnrm_available(int nx, int nz, int s);
// shared_sms: the pass runs beside other volumes' kernels (batched solves),
// so it keeps its occupancy rather than loading the epilogue's operands early.
cudaError_t run_zxnrm_ct(ZXArgs& a, const float* zin, cudaStream_t st, bool shared_sms = false);
// Fused T_z + drive-axis forward where instantiated.
bool ct_zxfwd_available(int nx, int nz, int s);
cudaError_t run_zxfwd_ct(ZXArgs& a, const float* zin, cudaStream_t st);
// Fused drive-axis adjoint + z correlation where instantiated (zout: its output).
bool ct_xzadj_available(int nx, int nz, int s);
cudaError_t run_xzadj_ct(ZXArgs& a, float* zout, cudaStream_t st);
cudaError_t run_xnrm_ct(const XArgs& a, cudaStream_t st);
int xpass_blocks(int rows, int pairs);
cudaError_t ops_set_attributes();
// Warp-centric drive-axis passes for n_x = 128, s = 2 (xwarp.cu).
// forward: the warp forward's opt-in (MH3D_XWARP_FWD=1 or a plan's tuned
// choice, `want`); the adjoint's is on by default.
bool xw_available(const XArgs& a, bool forward, bool want = false);
cudaError_t xw_set_attributes();
cudaError_t run_xfwd_w(const XArgs& a, cudaStream_t st);
cudaError_t run_xadj_w(const XArgs& a, cudaStream_t st);
// The warp adjoint with T_z^T fused (clusters of two CTAs per y-slab); zout:
// the z pass's output volume.
bool xzw_available(const XArgs& a, int nz);
cudaError_t run_xzadj_w(ZXArgs& a, float* zout, cudaStream_t st);
// The warp-centric cluster normal pass (T_z + drive-axis blocks + epilogue
// + dots; zin: the z pass's input); shared_sms as for run_zxnrm_ct.
bool zxnw_available(const XArgs& a, int nz);
cudaError_t run_zxnrm_w(ZXArgs& a, const float* zin, cudaStream_t st, bool shared_sms);
// The z volume's tensor map for the cluster passes (box box_x x 1 x nz).
bool ct_encode_z_map(CUtensorMap* m, const void* zvol, int nx, int ny, int nz, int box_x);

}  // namespace mh3d
