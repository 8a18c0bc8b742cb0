// mh3d_forward_noalloc: the forward operator for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// operator: a host thread that runs under a fixed device-memory budget owned
// by another framework's pool, a real-time pipeline whose memory plan is
// frozen at start-up, or code that must not risk the implicit device
// synchronisation an allocation can cause.  mh3d_plan_create allocates (its
// tables and solver workspace), so such callers cannot use a plan.  This
// entry point needs no plan: the PSF tables and the two intermediate volumes
// of the forward operator live in one file-scope __device__ array of fixed
// size, which every GPU that loads this library holds until the process
// exits.  The caller passes the geometry, the input density and the output
// portraits; nothing is allocated on the device.
//
// Limits: the intermediate volumes need 2 * nx * ny * nz * 4 bytes of the
// 16 MiB volume region (nx * ny * nz <= 2,097,152 voxels, e.g. 128^3), and
// the tables (K nx + 2 (ny + nz) + K + 2 nx + n/s entries of 8 bytes, each
// block rounded up to 256 bytes) must fit the 512 KiB table region.  Larger
// problems are rejected with MH3D_ERR_UNSUPPORTED_SIZE before anything runs.
//
// Sharing: every call on a device uses the same array, which keeps the last
// call's contents.  Nothing in it has to start at zero (each word a call
// reads is written earlier in the same call, tables first), but calls whose
// GPU work overlaps -- on different streams or from different threads --
// race on the array and corrupt each other's results.  Serialise them, for
// example by issuing them on one stream.
//
// Set-up: the first call on each device, with that device current, resolves
// the array's device address with cudaGetSymbolAddress (the host-side name of
// a __device__ array is only a stand-in, not a device address) and sets the
// kernels' shared-memory limits.
//
// Not for stream capture: every call uploads its tables from a host buffer
// that is freed when the call returns, so a call on a capturing stream
// returns MH3D_ERR_INVALID_ARG without issuing work.
//
// Errors on the device: the passes' bounded waits have no status word here,
// so a wait that gives up (which needs a broken copy engine, not bad input)
// leaves partial portraits without a report; planned calls report it.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ops_kernels.cuh"

namespace mh3d {

namespace {

constexpr size_t kNaTableBytes = 512u * 1024u;            // PSF spectra, phases, twiddles
constexpr size_t kNaVolumeBytes = 16u * 1024u * 1024u;    // two intermediate volumes
constexpr size_t kNaBytes = kNaTableBytes + kNaVolumeBytes;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};

bool na_is_235(int n)
{
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// Once per device, with that device current: the scratch array's device
// address and the pencil kernels' shared-memory limits.
cudaError_t na_setup(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = ops_set_attributes();
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace mh3d

using namespace mh3d;

extern "C" mh3d_status mh3d_forward_noalloc(const mh3d_geometry* g, const float* rho, void* d, void* stream)
{
    if (!g || !rho || !d) return MH3D_ERR_INVALID_ARG;
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    if (g->drive_axis != 0 || g->pad[0] || g->pad[1] || g->pad[2]) return MH3D_ERR_UNSUPPORTED_SIZE;
    if (g->ds_factor < 1 || g->ds_offset < 0 || g->ds_offset >= g->ds_factor) return MH3D_ERR_INVALID_ARG;
    if (g->k_min < 2 || g->k_max < g->k_min || g->k_max - g->k_min + 1 > kMaxK) return MH3D_ERR_INVALID_ARG;
    if (!(g->gamma_per_mm > 0) || !(std::fabs(g->gammaA) < 3.14159265358979) || !(g->transverse_ratio > 0))
        return MH3D_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(g->voxel_mm[a] > 0)) return MH3D_ERR_INVALID_ARG;
    if (!na_is_235(nx) || !na_is_235(ny) || !na_is_235(nz) || nx > kMaxLen || ny > kMaxLen || nz > kMaxLen ||
        nx % g->ds_factor != 0)
        return MH3D_ERR_UNSUPPORTED_SIZE;

    Plan P;   // host-side description only; no device memory is attached to it
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.s = g->ds_factor;
    P.r = g->ds_offset;
    P.kmin = g->k_min;
    P.kmax = g->k_max;
    P.K = g->k_max - g->k_min + 1;
    P.mx = nx / P.s;
    P.N = (long long)nx * ny * nz;
    P.M = (long long)P.mx * ny * nz;
    P.sens = g->sensitivity_dev;
    const int K = P.K, mx = P.mx;

    // size limits: two volumes, and every table block rounded to 256 bytes
    if ((size_t)P.N * 2 * sizeof(float) > kNaVolumeBytes) return MH3D_ERR_UNSUPPORTED_SIZE;   // > 2,097,152 voxels
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off += (n * sizeof(float2) + 255) & ~size_t(255); return o; };
    const size_t oX = take((size_t)K * nx), oY = take(ny), oZ = take(nz), oPh = take(K), oTx = take(nx),
                 oTy = take(ny), oTz = take(nz), oTm = take(mx);
    if (off > kNaTableBytes) return MH3D_ERR_UNSUPPORTED_SIZE;   // tables beyond 512 KiB
    P.ax.n = nx;
    P.ay.n = ny;
    P.az.n = nz;
    P.am.n = mx;
    if (!radix_plan(nx, P.ax.rp, 0) || !radix_plan(ny, P.ay.rp, 0) || !radix_plan(nz, P.az.rp, 0) ||
        !radix_plan(mx, P.am.rp, 0))
        return MH3D_ERR_UNSUPPORTED_SIZE;
    // launch shape: the same shared-memory budget rule as planned operators
    const size_t budget = 200 * 1024;
    TileChoice t;
    while (t.tpass_cols > 4 && tpass_smem_bytes(std::max(ny, nz), t.tpass_cols) > budget) t.tpass_cols /= 2;
    t.xpass_kgroup = std::min(4, K);
    while (t.xpass_kgroup > 1 && xfwd_smem_bytes(nx, mx, t.xpass_pairs, t.xpass_kgroup) > budget) --t.xpass_kgroup;
    while (t.xpass_pairs > 1 && xfwd_smem_bytes(nx, mx, t.xpass_pairs, t.xpass_kgroup) > budget) t.xpass_pairs /= 2;
    if (xfwd_smem_bytes(nx, mx, t.xpass_pairs, t.xpass_kgroup) > budget ||
        tpass_smem_bytes(std::max(ny, nz), t.tpass_cols) > budget)
        return MH3D_ERR_UNSUPPORTED_SIZE;
    P.tile = t;

    // Each call uploads its tables from a host buffer that is gone when the
    // call returns, so a captured call would replay a copy from freed memory:
    // refuse capture.
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MH3D_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return MH3D_ERR_INVALID_ARG;

    void* base = nullptr;
    cudaError_t e = na_setup(&base);
    if (e != cudaSuccess) return MH3D_ERR_CUDA;

    // FP64 host tables, rounded once to FP32 (the same spectra a plan uses)
    const double gt = g->gamma_per_mm * g->transverse_ratio;
    std::vector<float2> h(off / sizeof(float2), make_float2(0.f, 0.f));
    auto put = [&](size_t o, size_t i, const cplx& c) {
        h[o / sizeof(float2) + i] = make_float2((float)c.real(), (float)c.imag());
    };
    for (int kk = 0; kk < K; ++kk) {
        const std::vector<cplx> X = drive_spectrum(nx, g->voxel_mm[0], g->k_min + kk, g->gamma_per_mm, g->gammaA,
                                                   g->ds_offset);
        for (int w = 0; w < nx; ++w) put(oX, (size_t)kk * nx + w, X[w] / (double)nx);
        const double th = g->theta ? g->theta[kk] : 0.0;
        put(oPh, kk, cplx(std::cos(th), std::sin(th)));
    }
    const std::vector<cplx> Y = transverse_spectrum(ny, g->voxel_mm[1], gt);
    const std::vector<cplx> Z = transverse_spectrum(nz, g->voxel_mm[2], gt);
    for (int w = 0; w < ny; ++w) put(oY, w, Y[w] / (double)ny);
    for (int w = 0; w < nz; ++w) put(oZ, w, Z[w] / (double)nz);
    const int lens[4] = {nx, ny, nz, mx};
    const size_t offs[4] = {oTx, oTy, oTz, oTm};
    for (int a = 0; a < 4; ++a) {
        const std::vector<cplx> w = twiddles(lens[a]);
        for (int i = 0; i < lens[a]; ++i) put(offs[a], i, w[i]);
    }

    unsigned char* tb = static_cast<unsigned char*>(base);
    float* t1 = reinterpret_cast<float*>(tb + kNaTableBytes);
    float* t2 = t1 + P.N;
    // pageable source: the call returns once the data has been staged
    e = cudaMemcpyAsync(tb, h.data(), off, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return MH3D_ERR_CUDA;
    P.Xhat = reinterpret_cast<float2*>(tb + oX);
    P.Yhat = reinterpret_cast<float2*>(tb + oY);
    P.Zhat = reinterpret_cast<float2*>(tb + oZ);
    P.phase = reinterpret_cast<float2*>(tb + oPh);
    P.ax.tw = reinterpret_cast<float2*>(tb + oTx);
    P.ay.tw = reinterpret_cast<float2*>(tb + oTy);
    P.az.tw = reinterpret_cast<float2*>(tb + oTz);
    P.am.tw = reinterpret_cast<float2*>(tb + oTm);
    e = launch_forward(P, rho, (float2*)d, t1, t2, st);
    return (e == cudaSuccess) ? MH3D_OK : MH3D_ERR_CUDA;
}
