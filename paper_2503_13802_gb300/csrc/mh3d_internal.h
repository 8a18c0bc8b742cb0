// Internal declarations of the MH3D GB300 library (not part of the C ABI).
#pragma once

#include <atomic>
#include <cstdlib>
#include <complex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mh3d.h"

namespace mh3d {

using cplx = std::complex<double>;

constexpr int kMaxStages = 8;     // radix stages per 1D length (2^a 3^b <= 1024)
constexpr int kMaxLen = 1024;     // longest supported axis
constexpr int kMaxK = 31;         // harmonics per plan

// Radix schedule of one 1D length; passed to kernels by value.
struct RadixPlan {
    int n;
    int nst;
    int radix[kMaxStages];
};

// One axis of the plan: length, radix schedule, twiddle table (device).
struct AxisPlan {
    int n = 1;
    RadixPlan rp{};
    const float2* tw = nullptr;   // W_n^t, t in [0, n), FP32 from FP64
};

// Launch shape of the pencil kernels, chosen per plan (autotuner).
struct TileChoice {
    int tpass_cols = 16;          // x columns per T-pass CTA (pencils = cols / 2)
    int xpass_pairs = 16;         // row pairs per X-pass CTA
    int xpass_kgroup = 4;         // harmonics transformed together in the X pass
    int threads = 256;
    // chosen by mh3d_plan_autotune (0 = the library's default; environment
    // switches of the same name still take precedence for A/B checks)
    int tpass_radix = 0;          // T pass schedule: 0 the default, 1 the alternative (n = 64: 4x16, 128: 8x16)
    int zx_c = 0;                 // CTAs per y-slab of the cluster passes (2 or 4)
    int xw_ks = 0;                // warps per row group of the warp-centric adjoint (1, 2 or 4)
    int adj_path = 0;             // adjoint's drive-axis part: 1 warp + T_z^T fused, 2 warp then T_z^T, 3 CTA-level
    int fwd_path = 0;             // forward's drive-axis part: 1 cluster pass fusing T_z, 2 warp-centric
    int xw_ks_fwd = 0;            // warps per row group of the warp-centric forward
};

// Solver workspace (device), sized at plan time.
struct SolveWork {
    bool shared_sms = false;      // set while a batched solve captures this plan's kernels
    float* x = nullptr;           // iterate (copied to the caller's buffer at the end)
    float* r = nullptr;
    float* p = nullptr;
    float* q = nullptr;
    float* t1 = nullptr;
    float* t2 = nullptr;
    float* rhs = nullptr;
    float* s = nullptr;           // A r (single-reduction CG)
    float2* portrait = nullptr;   // explicit mode only (allocated on first use)
    float2* dstage = nullptr;     // padded plans: field-of-view portraits staged by mh3d_solve_host
    double* red = nullptr;        // reduction partials (see solve.cu)
    int* flags = nullptr;         // [done, iters, status, spare]
    double* hist = nullptr;       // per-iteration relative residual
    int hist_cap = 0;
    size_t red_cap = 0;
    int* flags_host = nullptr;    // pinned
    double* red_host = nullptr;   // pinned, red_cap doubles
    void* base = nullptr;         // one allocation backing the vectors
};

// Allocation hook for fault tests: with MH3D_DEBUG_FAIL_ALLOC=k the k-th
// device or pinned-host allocation after the counter was last reset (at the
// start of each plan creation, per thread) fails as out of memory, so every
// clean-up path of plan creation can be exercised on the host side.
inline int& alloc_counter()
{
    static thread_local int c = 0;
    return c;
}
inline bool alloc_should_fail()
{
    const char* e = std::getenv("MH3D_DEBUG_FAIL_ALLOC");
    if (!e) return false;
    const int k = std::atoi(e);
    return k > 0 && ++alloc_counter() == k;
}
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes)
{
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t host_malloc(T** p, size_t bytes)
{
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

inline unsigned long long next_plan_serial()
{
    static std::atomic<unsigned long long> n{0};
    return ++n;
}

struct Plan {
    // unique for the process's lifetime (caches key on it, never on addresses)
    unsigned long long serial = next_plan_serial();
    // geometry
    int nx = 1, ny = 1, nz = 1, s = 1, r = 0, K = 1, kmin = 2, kmax = 2;
    int mx = 1;
    long long N = 1, M = 1;       // voxels; portrait samples per harmonic
    // boundary padding (Sec. 3.x, boundary image padding): the model grid
    // above is the field of view (fnx, fny, fnz) extended by pad voxels on
    // each side; the portraits a caller passes cover the field of view only
    // (fmx samples per row, Mf per harmonic)
    int pad[3] = {0, 0, 0};
    int fnx = 1, fny = 1, fnz = 1, fmx = 1;
    long long Mf = 1;
    bool padded = false;
    double vox[3] = {1, 1, 1};
    double gamma = 1, gammaA = 1, tratio = 0.5;
    std::vector<double> theta;
    double opnorm2 = 1.0;         // ||A||_2^2 with b = 1 (FP64)
    const float* sens = nullptr;  // borrowed device pointer (may be null)

    AxisPlan ax, ay, az, am;      // x (drive), y, z, portrait length mx
    TileChoice tile;

    // device tables (FP32 complex)
    float2* Xhat = nullptr;       // [K][nx]  c_k DFT(X'_k) / nx
    float2* Yhat = nullptr;       // [ny]     DFT(Y)/ny
    float2* Zhat = nullptr;       // [nz]
    float2* Yhat_adj = nullptr;   // conj
    float2* Zhat_adj = nullptr;
    float2* Ynorm = nullptr;      // ny |DFT(Y)/ny|^2
    float2* Znorm = nullptr;
    float2* Qblk = nullptr;       // [mx][s][s]  x-normal blocks
    float2* phase = nullptr;      // [K] (cos theta, sin theta)
    void* table_mem = nullptr;    // one allocation backing all tables
    size_t table_bytes = 0;

    SolveWork w;
    size_t work_bytes = 0;
    std::string err;

    // MHAD native image (mhad.cu): filter tables cached per (lambda, upsample);
    // warm-start scratch portraits and scale partials, allocated on first use
    float2* mhad_tab = nullptr;
    double mhad_lambda = -1.0;
    int mhad_up = -1;
    float2* mhad_scratch = nullptr;
    double* mhad_red = nullptr;

    // general model (general.cu): PSF spectra DFT(h_kj)/N [K][3][N] and a
    // work area of 3 N + K n_z n_y m_x complex values, allocated by
    // mh3d_general_set_psf
    float2* gen_H = nullptr;
    float2* gen_work = nullptr;
    // the general CG's device scalars and residual history (solve.cu),
    // grown on demand: gen_cg_cap doubles
    double* gen_cg = nullptr;
    size_t gen_cg_cap = 0;

    // CUDA graph of the CG loop, cached per (mode, reg, fixed) key
    cudaGraphExec_t graph_exec = nullptr;
    unsigned long long graph_key = ~0ull;
    cudaStream_t graph_stream = nullptr;
};

// mhad.cu
void mhad_free(Plan& P);
// general.cu
void general_free(Plan& P);

// Padded plans (capi.cu): field-of-view portraits <-> the extended portrait
// mesh, and the mask of the explicit normal operator.
cudaError_t pad_portraits(const Plan& P, const float2* d_fov, float2* d_ext, cudaStream_t st);
cudaError_t crop_portraits(const Plan& P, const float2* d_ext, float2* d_fov, cudaStream_t st);
cudaError_t mask_portraits(const Plan& P, float2* d_ext, cudaStream_t st);
mh3d_status ensure_portrait(Plan& P);

// psf_host.cpp
double langevin_deriv_host(int k, double x);
std::vector<cplx> drive_spectrum(int n, double dx, int k, double gamma, double gammaA, int r);
std::vector<cplx> transverse_spectrum(int n, double d, double gt);
std::vector<cplx> twiddles(int n);
double hermitian_lambda_max(const std::vector<cplx>& H, int s);
bool radix_plan(int n, RadixPlan& pl, int variant);

// ops.cu: operator launches (all asynchronous on `st`)
struct OpCtx;
cudaError_t launch_forward(const Plan& P, const float* rho, float2* d, float* t1, float* t2, cudaStream_t st);
cudaError_t launch_adjoint(const Plan& P, const float2* d, float* rho, float* t1, float* t2, cudaStream_t st);
cudaError_t ops_configure(Plan& P);   // per-plan kernel attributes / smem sizes
size_t xpass_smem_fwd(const Plan& P, const TileChoice& t);
size_t xpass_smem_adj(const Plan& P, const TileChoice& t);
size_t xpass_smem_nrm(const Plan& P, const TileChoice& t);
size_t tpass_smem(const Plan& P, int n, const TileChoice& t);

}  // namespace mh3d
