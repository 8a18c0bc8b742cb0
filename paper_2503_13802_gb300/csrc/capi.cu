// Plan construction and operator entry points of the C ABI (include/mh3d.h).
#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "ops_kernels.cuh"
#include "solve_internal.h"

namespace mh3d {

namespace {

// Kernel attributes (dynamic shared-memory limits) belong to the current
// device, so they are set once per device, not once per process.
constexpr int kAttrMaxDevices = 64;
std::mutex g_attr_mu;
bool g_attr_done[kAttrMaxDevices] = {};
thread_local std::string g_create_err;   // message of the last failed mh3d_plan_create

bool is_235(int n)
{
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

}  // namespace

#define MH3D_TRY(P, call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (P)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                        \
            return MH3D_ERR_CUDA;                                                                 \
        }                                                                                         \
    } while (0)

// Shared-memory budget per CTA that the tile choice must respect.
constexpr size_t kSmemBudget = 200 * 1024;

static void choose_tiles(Plan& P)
{
    TileChoice t;
    const int nt = std::max(P.ny, P.nz);
    t.tpass_cols = 16;
    if (const char* e = std::getenv("MH3D_TPASS_COLS")) {   // A/B override: 8 or 16
        const int c = std::atoi(e);
        if (c == 8 || c == 16) t.tpass_cols = c;
    }
    while (t.tpass_cols > 4 && tpass_smem_bytes(nt, t.tpass_cols) > kSmemBudget) t.tpass_cols /= 2;
    t.xpass_pairs = 16;
    t.xpass_kgroup = std::min(4, P.K);
    while (t.xpass_kgroup > 1 &&
           (xfwd_smem_bytes(P.nx, P.mx, t.xpass_pairs, t.xpass_kgroup) > kSmemBudget ||
            xadj_smem_bytes(P.nx, P.mx, t.xpass_pairs, t.xpass_kgroup) > kSmemBudget))
        --t.xpass_kgroup;
    while (t.xpass_pairs > 1 && (xfwd_smem_bytes(P.nx, P.mx, t.xpass_pairs, t.xpass_kgroup) > kSmemBudget ||
                                 xadj_smem_bytes(P.nx, P.mx, t.xpass_pairs, t.xpass_kgroup) > kSmemBudget))
        t.xpass_pairs /= 2;
    P.tile = t;
}

// Builds all FP32 tables from FP64 host computations and uploads them.
static mh3d_status build_tables(Plan& P, cudaStream_t st)
{
    const int nx = P.nx, ny = P.ny, nz = P.nz, mx = P.mx, s = P.s, K = P.K;
    const double gt = P.gamma * P.tratio;
    std::vector<std::vector<cplx>> X(K);
    for (int kk = 0; kk < K; ++kk) {
        X[kk] = drive_spectrum(nx, P.vox[0], P.kmin + kk, P.gamma, P.gammaA, P.r);
        for (auto& v : X[kk]) v /= (double)nx;
    }
    std::vector<cplx> Y = transverse_spectrum(ny, P.vox[1], gt), Z = transverse_spectrum(nz, P.vox[2], gt);
    for (auto& v : Y) v /= (double)ny;
    for (auto& v : Z) v /= (double)nz;

    // layout (float2 units)
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off += (n + 31) & ~size_t(31); return o; };
    const size_t oX = take((size_t)K * nx), oY = take(ny), oZ = take(nz), oYa = take(ny), oZa = take(nz),
                 oYn = take(ny), oZn = take(nz), oQ = take((size_t)mx * s * s), oPh = take(K),
                 oTx = take(nx), oTy = take(ny), oTz = take(nz), oTm = take(mx);
    std::vector<float2> h(off, make_float2(0.f, 0.f));
    auto put = [&](size_t o, const cplx& c) { h[o] = make_float2((float)c.real(), (float)c.imag()); };
    for (int kk = 0; kk < K; ++kk)
        for (int w = 0; w < nx; ++w) put(oX + (size_t)kk * nx + w, X[kk][w]);
    for (int w = 0; w < ny; ++w) {
        put(oY + w, Y[w]);
        put(oYa + w, std::conj(Y[w]));
        put(oYn + w, cplx((double)ny * std::norm(Y[w]), 0.0));
    }
    for (int w = 0; w < nz; ++w) {
        put(oZ + w, Z[w]);
        put(oZa + w, std::conj(Z[w]));
        put(oZn + w, cplx((double)nz * std::norm(Z[w]), 0.0));
    }
    // Q[m][a][b] = mx sum_k conj(X_k[m + a mx]) X_k[m + b mx]
    for (int m = 0; m < mx; ++m)
        for (int a = 0; a < s; ++a)
            for (int b = 0; b < s; ++b) {
                cplx acc(0, 0);
                for (int kk = 0; kk < K; ++kk) acc += std::conj(X[kk][m + a * mx]) * X[kk][m + b * mx];
                put(oQ + ((size_t)m * s + a) * s + b, (double)mx * acc);
            }
    for (int kk = 0; kk < K; ++kk) put(oPh + kk, cplx(std::cos(P.theta[kk]), std::sin(P.theta[kk])));
    // ||A||_2^2 (b = 1) = max|DFT Y|^2 max|DFT Z|^2 max_m lambda_max(B_m), with
    // B_m[a][b] = (1/s) sum_k conj(x_k[m + a mx]) x_k[m + b mx] and x_k the
    // unnormalised drive spectra (X here holds x_k / nx).
    {
        double ym = 0, zm = 0, xm = 0;
        for (int w = 0; w < ny; ++w) ym = std::max(ym, std::norm(Y[w] * (double)ny));
        for (int w = 0; w < nz; ++w) zm = std::max(zm, std::norm(Z[w] * (double)nz));
        std::vector<cplx> B((size_t)s * s);
        for (int m = 0; m < mx; ++m) {
            for (int a = 0; a < s; ++a)
                for (int b = 0; b < s; ++b) {
                    cplx acc(0, 0);
                    for (int kk = 0; kk < K; ++kk)
                        acc += std::conj(X[kk][m + a * mx]) * X[kk][m + b * mx] * ((double)nx * nx);
                    B[(size_t)a * s + b] = acc / (double)s;
                }
            xm = std::max(xm, hermitian_lambda_max(B, s));
        }
        P.opnorm2 = xm * ym * zm;
    }
    auto put_tw = [&](size_t o, int n) {
        auto w = twiddles(n);
        for (int t = 0; t < n; ++t) put(o + t, w[t]);
    };
    put_tw(oTx, nx);
    put_tw(oTy, ny);
    put_tw(oTz, nz);
    put_tw(oTm, mx);

    void* mem = nullptr;
    P.table_bytes = off * sizeof(float2);
    if (dev_malloc(&mem, P.table_bytes) != cudaSuccess) {
        P.err = "cudaMalloc of tables failed";
        return MH3D_ERR_OOM;
    }
    P.table_mem = mem;
    MH3D_TRY(&P, cudaMemcpyAsync(mem, h.data(), P.table_bytes, cudaMemcpyHostToDevice, st));
    MH3D_TRY(&P, cudaStreamSynchronize(st));
    float2* b = (float2*)mem;
    P.Xhat = b + oX;
    P.Yhat = b + oY;
    P.Zhat = b + oZ;
    P.Yhat_adj = b + oYa;
    P.Zhat_adj = b + oZa;
    P.Ynorm = b + oYn;
    P.Znorm = b + oZn;
    P.Qblk = b + oQ;
    P.phase = b + oPh;
    P.ax.tw = b + oTx;
    P.ay.tw = b + oTy;
    P.az.tw = b + oTz;
    P.am.tw = b + oTm;
    return MH3D_OK;
}

// ---------------------------------------------------------------------------
// Padded plans: the portraits of the field of view sit inside the extended
// portrait mesh at rows z in [pz, pz + fnz), y in [py, py + fny) and samples
// i' in [px/s, px/s + fmx) of each row (Sec. 3.x: the padding is part of
// the model, not of the data).
// ---------------------------------------------------------------------------
struct PadGeom {
    int K, nz, ny, mx;          // extended mesh
    int fnz, fny, fmx;          // field of view
    int pz, py, pm;             // offsets (pm = px / s)
};
static PadGeom pad_geom(const Plan& P)
{
    return PadGeom{P.K, P.nz, P.ny, P.mx, P.fnz, P.fny, P.fmx, P.pad[2], P.pad[1], P.pad[0] / P.s};
}
// d_ext = the field-of-view portraits, zero elsewhere
__global__ void __launch_bounds__(256) k_pad_portraits(const float2* __restrict__ d, float2* __restrict__ e, PadGeom g)
{
    const long long n = (long long)g.K * g.nz * g.ny * g.mx;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long q = t;
        const int i = (int)(q % g.mx);
        q /= g.mx;
        const int y = (int)(q % g.ny);
        q /= g.ny;
        const int z = (int)(q % g.nz);
        const int k = (int)(q / g.nz);
        const int fi = i - g.pm, fy = y - g.py, fz = z - g.pz;
        float2 v = make_float2(0.f, 0.f);
        if (fi >= 0 && fi < g.fmx && fy >= 0 && fy < g.fny && fz >= 0 && fz < g.fnz)
            v = d[(((long long)k * g.fnz + fz) * g.fny + fy) * g.fmx + fi];
        e[t] = v;
    }
}
// d_fov = the field-of-view part of d_ext
__global__ void __launch_bounds__(256) k_crop_portraits(const float2* __restrict__ e, float2* __restrict__ d, PadGeom g)
{
    const long long n = (long long)g.K * g.fnz * g.fny * g.fmx;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long q = t;
        const int fi = (int)(q % g.fmx);
        q /= g.fmx;
        const int fy = (int)(q % g.fny);
        q /= g.fny;
        const int fz = (int)(q % g.fnz);
        const int k = (int)(q / g.fnz);
        d[t] = e[(((long long)k * g.nz + fz + g.pz) * g.ny + fy + g.py) * g.mx + fi + g.pm];
    }
}
// zero the extended portraits outside the field of view (in place)
__global__ void __launch_bounds__(256) k_mask_portraits(float2* __restrict__ e, PadGeom g)
{
    const long long n = (long long)g.K * g.nz * g.ny * g.mx;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long q = t;
        const int i = (int)(q % g.mx);
        q /= g.mx;
        const int y = (int)(q % g.ny);
        q /= g.ny;
        const int z = (int)(q % g.nz);
        const int fi = i - g.pm, fy = y - g.py, fz = z - g.pz;
        if (!(fi >= 0 && fi < g.fmx && fy >= 0 && fy < g.fny && fz >= 0 && fz < g.fnz)) e[t] = make_float2(0.f, 0.f);
    }
}
static int pad_blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }
cudaError_t pad_portraits(const Plan& P, const float2* d_fov, float2* d_ext, cudaStream_t st)
{
    k_pad_portraits<<<pad_blocks((long long)P.K * P.M), 256, 0, st>>>(d_fov, d_ext, pad_geom(P));
    return cudaGetLastError();
}
cudaError_t crop_portraits(const Plan& P, const float2* d_ext, float2* d_fov, cudaStream_t st)
{
    k_crop_portraits<<<pad_blocks((long long)P.K * P.Mf), 256, 0, st>>>(d_ext, d_fov, pad_geom(P));
    return cudaGetLastError();
}
cudaError_t mask_portraits(const Plan& P, float2* d_ext, cudaStream_t st)
{
    k_mask_portraits<<<pad_blocks((long long)P.K * P.M), 256, 0, st>>>(d_ext, pad_geom(P));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Argument builders
// ---------------------------------------------------------------------------
TArgs tpass_args(const Plan& P, int axis /*1 = y, 2 = z*/, const float* in, float* out, const float2* mult)
{
    TArgs a;
    a.in = in;
    a.out = out;
    a.mult = mult;
    a.nx = P.nx;
    a.cols = P.tile.tpass_cols;
    a.radix_alt = P.tile.tpass_radix;
    if (const char* e = std::getenv("MH3D_TPASS_RADIX")) a.radix_alt = (e[0] == '1') ? 1 : 0;   // A/B checks
    a.vec2 = (P.nx % 2 == 0) ? 1 : 0;
    a.vec4 = (P.nx % 4 == 0 && ((uintptr_t)P.sens % 16) == 0) ? 1 : 0;
    a.status = P.w.flags ? P.w.flags + 3 : nullptr;
    // Fault test (MH3D_DEBUG_WAIT_TIMEOUT=1): the tile barrier expects 16 bytes
    // that no copy delivers, so its bounded wait runs out and records
    // MH3D_ERR_TIMEOUT; every real copy has landed by then.
    if (const char* e = std::getenv("MH3D_DEBUG_WAIT_TIMEOUT"))
        if (e[0] == '1') a.debug_extra_tx = 16;
    a.axis = axis;
    if (axis == 1) {
        a.rp = P.ay.rp;
        a.tw = P.ay.tw;
        a.n = P.ny;
        a.es = P.nx;
        a.os = (long long)P.nx * P.ny;
    } else {
        a.rp = P.az.rp;
        a.tw = P.az.tw;
        a.n = P.nz;
        a.es = (long long)P.nx * P.ny;
        a.os = P.nx;
    }
    a.reg.nx = P.nx;
    a.reg.ny = P.ny;
    a.reg.nz = P.nz;
    return a;
}

int tpass_outer(const Plan& P, int axis) { return axis == 1 ? P.nz : P.ny; }

XArgs xpass_args(const Plan& P)
{
    XArgs a;
    a.Xhat = P.Xhat;
    a.phase = P.phase;
    a.Q = P.Qblk;
    a.twx = P.ax.tw;
    a.twm = P.am.tw;
    a.rpx = P.ax.rp;
    a.rpm = P.am.rp;
    a.nx = P.nx;
    a.mx = P.mx;
    a.s = P.s;
    a.K = P.K;
    a.rows = P.ny * P.nz;
    a.M = (long long)a.rows * P.mx;
    a.pairs = P.tile.xpass_pairs;
    a.kg = P.tile.xpass_kgroup;
    a.vec4 = (P.nx % 4 == 0 && ((uintptr_t)P.sens % 16) == 0) ? 1 : 0;
    a.reg.nx = P.nx;
    a.reg.ny = P.ny;
    a.reg.nz = P.nz;
    a.status = P.w.flags ? P.w.flags + 3 : nullptr;
    a.ks = P.tile.xw_ks;
    return a;
}

RegArgs reg_args(const Plan& P, const mh3d_solve_opts& o)
{
    RegArgs g;
    g.kind = o.reg_kind;
    g.lambda = (float)(o.lambda_relative ? o.lambda * P.opnorm2 : o.lambda);
    g.alpha = (float)o.alpha;
    g.shell = o.shell;
    g.nx = P.nx;
    g.ny = P.ny;
    g.nz = P.nz;
    return g;
}

cudaError_t launch_forward(const Plan& P, const float* rho, float2* d, float* t1, float* t2, cudaStream_t st)
{
    cudaError_t e;
    TArgs ty = tpass_args(P, 1, rho, t1, P.Yhat);
    ty.bin = P.sens;
    if ((e = run_tpass(ty, tpass_outer(P, 1), st)) != cudaSuccess) return e;
    XArgs xw = xpass_args(P);
    xw.vin = t2;
    xw.dout = d;
    xw.ks = P.tile.xw_ks_fwd;
    if (xw_available(xw, true, P.tile.fwd_path == 2)) {
        // T_z, then the warp-centric drive-axis forward
        TArgs tz = tpass_args(P, 2, t1, t2, P.Zhat);
        if ((e = run_tpass(tz, tpass_outer(P, 2), st)) != cudaSuccess) return e;
        return run_xfwd_w(xw, st);
    }
    if (ct_zxfwd_available(P.nx, P.nz, P.s) && ((uintptr_t)t1 & 15u) == 0) {
        // T_z and the drive-axis forward in one launch (a cluster of CTAs per y-slab)
        ZXArgs z;
        z.x = xpass_args(P);
        z.x.dout = d;
        z.twz = P.az.tw;
        z.muz = P.Zhat;
        z.ny = P.ny;
        z.nz = P.nz;
        z.C = P.tile.zx_c;
        return run_zxfwd_ct(z, t1, st);
    }
    TArgs tz = tpass_args(P, 2, t1, t2, P.Zhat);
    if ((e = run_tpass(tz, tpass_outer(P, 2), st)) != cudaSuccess) return e;
    XArgs x = xpass_args(P);
    x.vin = t2;
    x.dout = d;
    return run_xfwd(x, st);
}

cudaError_t launch_adjoint(const Plan& P, const float2* d, float* rho, float* t1, float* t2, cudaStream_t st)
{
    cudaError_t e;
    XArgs xw = xpass_args(P);
    xw.din = d;
    xw.vout = t1;
    // the plan's tuned path (adj_path: 1 warp fused, 2 warp then T_z^T, 3 CTA-level; 0 the default)
    const bool warp = P.tile.adj_path != 3 && xw_available(xw, false);
    const bool fused = !warp && ct_xzadj_available(P.nx, P.nz, P.s) && ((uintptr_t)d & 15u) == 0 &&
                       ((uintptr_t)t2 & 15u) == 0 && P.mx % 2 == 0 && P.M % 2 == 0;
    if (warp && P.tile.adj_path != 2 && xzw_available(xw, P.nz) && ((uintptr_t)t2 & 15u) == 0) {
        // the warp-centric drive-axis adjoint and T_z^T in one launch (a
        // cluster of two CTAs per y-slab)
        ZXArgs z;
        z.x = xw;
        z.twz = P.az.tw;
        z.muz = P.Zhat_adj;
        z.ny = P.ny;
        z.nz = P.nz;
        z.C = P.tile.zx_c;
        if ((e = run_xzadj_w(z, t2, st)) != cudaSuccess) return e;
    } else if (warp) {
        // the warp-centric drive-axis adjoint, then T_z^T
        if ((e = run_xadj_w(xw, st)) != cudaSuccess) return e;
        TArgs tz = tpass_args(P, 2, t1, t2, P.Zhat_adj);
        if ((e = run_tpass(tz, tpass_outer(P, 2), st)) != cudaSuccess) return e;
    } else if (fused) {
        // the drive-axis adjoint and T_z^T in one launch (a cluster of CTAs per y-slab)
        ZXArgs z;
        z.x = xpass_args(P);
        z.x.din = d;
        z.twz = P.az.tw;
        z.muz = P.Zhat_adj;
        z.ny = P.ny;
        z.nz = P.nz;
        z.C = P.tile.zx_c;
        if ((e = run_xzadj_ct(z, t2, st)) != cudaSuccess) return e;
    } else {
        XArgs x = xpass_args(P);
        x.din = d;
        x.vout = t1;
        if ((e = run_xadj(x, st)) != cudaSuccess) return e;
        TArgs tz = tpass_args(P, 2, t1, t2, P.Zhat_adj);
        if ((e = run_tpass(tz, tpass_outer(P, 2), st)) != cudaSuccess) return e;
    }
    TArgs ty = tpass_args(P, 1, t2, rho, P.Yhat_adj);
    ty.bout = P.sens;
    return run_tpass(ty, tpass_outer(P, 1), st);
}

// out = (A^T A + lambda R) in.  mode 0: fused Fourier-block normal operator;
// mode 1: explicit A then A^T through the portrait buffer.  `dots` (may be
// null) receives in^T out (and in^T in when dots->part2 is set) as grid
// totals; `cg` (may be null) is the loop control of a CG iteration; `upd`
// (may be null) fuses a CG vector update into the first pass's loader, in
// which case `in` is the vector that update produces.
cudaError_t launch_normal(const Plan& P, int mode, const RegArgs& reg, const float* in, float* out, float* t1,
                          float* t2, float2* portrait, const RedSink* dots, const CgCtl* cg, const LoaderUpdate* upd,
                          cudaStream_t st)
{
    cudaError_t e;
    TArgs ty = tpass_args(P, 1, in, t1, mode == 0 ? P.Ynorm : P.Yhat);
    ty.bin = P.sens;
    if (upd && upd->mode) {
        ty.pupdate = upd->mode;
        ty.pvec = upd->p;
        ty.rvec = upd->r;
        ty.rvec_w = upd->r_w;
        ty.qdir = upd->q;
        ty.svec = upd->s;
        ty.xvec = upd->x;
    }
    if (cg) ty.cg = *cg;
    if ((e = run_tpass(ty, tpass_outer(P, 1), st)) != cudaSuccess) return e;
    CgCtl cgp;
    if (cg) cgp = *cg;   // later kernels only check the done flag
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    XArgs xq = xpass_args(P);
    const bool zx_warp = mode == 0 && reg.kind == 0 && zxnw_available(xq, P.nz) && ct_zxnrm_available(P.nx, P.nz, P.s);
    if (mode == 0 && reg.kind == 0 && (ct_zxnrm_available(P.nx, P.nz, P.s) || zx_warp) && a16(t1) && a16(in) &&
        a16(out) && (!P.sens || a16(P.sens))) {
        // T_z and the drive-axis normal pass in one launch (a cluster of CTAs per y-slab)
        ZXArgs z;
        z.x = xpass_args(P);
        z.x.b = P.sens;
        z.x.pin = in;
        z.x.qout = out;
        if (dots) {
            z.x.part = dots->part;
            z.x.ticket = dots->ticket;
            z.x.sum_out = dots->out;
            z.x.part2 = dots->part2;
            z.x.sum_out2 = dots->out2;
        }
        z.x.reg = reg;
        if (cg) {
            z.x.cg = cgp;
            z.x.cg_active = 1;
            z.x.count_iter = cg->cgcg;
        }
        z.twz = P.az.tw;
        z.muz = P.Znorm;
        z.ny = P.ny;
        z.nz = P.nz;
        z.C = P.tile.zx_c;
        if (zx_warp) return run_zxnrm_w(z, t1, st, P.w.shared_sms);
        return run_zxnrm_ct(z, t1, st, P.w.shared_sms);
    }
    TArgs tz = tpass_args(P, 2, t1, t2, mode == 0 ? P.Znorm : P.Zhat);
    if (cg) tz.cg = cgp;
    if ((e = run_tpass(tz, tpass_outer(P, 2), st)) != cudaSuccess) return e;
    if (mode == 0) {
        XArgs x = xpass_args(P);
        x.vin = t2;
        x.b = P.sens;
        x.pin = in;
        x.qout = out;
        if (dots) {
            x.part = dots->part;
            x.ticket = dots->ticket;
            x.sum_out = dots->out;
            x.part2 = dots->part2;
            x.sum_out2 = dots->out2;
        }
        x.reg = reg;
        if (cg) {
            x.cg = cgp;
            x.cg_active = 1;
            x.count_iter = cg->cgcg;
        }
        return run_xnrm(x, st);
    }
    // Explicit mode.  The drive-axis kernels carry no loop control: once the
    // loop has finished, the first pass returns early and leaves t2 as it
    // was, so recomputing them is harmless (the epilogue pass checks the flag).
    XArgs xf = xpass_args(P);
    xf.vin = t2;
    xf.dout = portrait;
    if ((e = run_xfwd(xf, st)) != cudaSuccess) return e;
    // a padded plan's data cover the field of view only: A^T A becomes
    // A^T M A with M the field-of-view mask of the portraits
    if (P.padded && (e = mask_portraits(P, portrait, st)) != cudaSuccess) return e;
    XArgs xa = xpass_args(P);
    xa.din = portrait;
    xa.vout = t1;
    if ((e = xw_available(xa, false) ? run_xadj_w(xa, st) : run_xadj(xa, st)) != cudaSuccess) return e;
    TArgs tz2 = tpass_args(P, 2, t1, t2, P.Zhat_adj);
    if (cg) tz2.cg = cgp;
    if ((e = run_tpass(tz2, tpass_outer(P, 2), st)) != cudaSuccess) return e;
    TArgs ty2 = tpass_args(P, 1, t2, nullptr, P.Yhat_adj);
    ty2.bout = P.sens;
    ty2.epilogue = 1;
    ty2.qvec = out;
    ty2.pin = in;
    if (dots) {
        ty2.part = dots->part;
        ty2.ticket = dots->ticket;
        ty2.sum_out = dots->out;
        ty2.part2 = dots->part2;
        ty2.sum_out2 = dots->out2;
    }
    ty2.reg = reg;
    if (cg) {
        ty2.cg = cgp;
        ty2.count_iter = cg->cgcg;
    }
    return run_tpass(ty2, tpass_outer(P, 1), st);
}

int normal_part_count(const Plan& P, int mode)
{
    if (mode == 0) return xpass_blocks(P.ny * P.nz, P.tile.xpass_pairs);
    return tpass_blocks(P.nx, P.tile.tpass_cols, tpass_outer(P, 1));
}

mh3d_status ensure_portrait(Plan& P)
{
    if (P.w.portrait) return MH3D_OK;
    const size_t bytes = sizeof(float2) * (size_t)P.K * P.M;
    if (dev_malloc(&P.w.portrait, bytes) != cudaSuccess) {
        P.w.portrait = nullptr;
        P.err = "cudaMalloc of the portrait buffer failed";
        return MH3D_ERR_OOM;
    }
    P.work_bytes += bytes;
    return MH3D_OK;
}

}  // namespace mh3d

using namespace mh3d;

struct mh3d_plan_s : public Plan {};

extern "C" {

const char* mh3d_version(void) { return "mh3d-gb300 0.1 (sm_103a)"; }

mh3d_status mh3d_plan_create(const mh3d_geometry* g, void* stream, mh3d_plan* out)
{
    alloc_counter() = 0;   // fault-test hook: count this creation's allocations
    if (!out) return MH3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g) return MH3D_ERR_INVALID_ARG;
    if (g->drive_axis != 0) return MH3D_ERR_UNSUPPORTED_SIZE;
    if (g->ds_factor < 1 || g->ds_offset < 0 || g->ds_offset >= g->ds_factor) return MH3D_ERR_INVALID_ARG;
    // boundary padding: the model grid is the field of view extended by pad
    // voxels per side; along the drive axis a multiple of s keeps the field
    // of view's portrait mesh a sub-mesh of the extended one
    for (int a = 0; a < 3; ++a)
        if (g->pad[a] < 0 || g->n[a] < 1) return MH3D_ERR_INVALID_ARG;
    if (g->pad[0] % g->ds_factor != 0) return MH3D_ERR_INVALID_ARG;
    const int nx = g->n[0] + 2 * g->pad[0], ny = g->n[1] + 2 * g->pad[1], nz = g->n[2] + 2 * g->pad[2];
    if (g->k_min < 2 || g->k_max < g->k_min || g->k_max - g->k_min + 1 > kMaxK) return MH3D_ERR_INVALID_ARG;
    if (!(g->gamma_per_mm > 0) || !(std::fabs(g->gammaA) < 3.14159265358979) || !(g->transverse_ratio > 0))
        return MH3D_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(g->voxel_mm[a] > 0)) return MH3D_ERR_INVALID_ARG;
    if (!is_235(nx) || !is_235(ny) || !is_235(nz) || nx > kMaxLen || ny > kMaxLen || nz > kMaxLen)
        return MH3D_ERR_UNSUPPORTED_SIZE;
    if (nx % g->ds_factor != 0) return MH3D_ERR_UNSUPPORTED_SIZE;
    const int mx = nx / g->ds_factor;

    mh3d_plan_s* P = new (std::nothrow) mh3d_plan_s();
    if (!P) return MH3D_ERR_OOM;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->s = g->ds_factor;
    P->r = g->ds_offset;
    P->kmin = g->k_min;
    P->kmax = g->k_max;
    P->K = g->k_max - g->k_min + 1;
    P->mx = mx;
    P->N = (long long)nx * ny * nz;
    P->M = (long long)mx * ny * nz;
    for (int a = 0; a < 3; ++a) P->pad[a] = g->pad[a];
    P->padded = g->pad[0] || g->pad[1] || g->pad[2];
    P->fnx = g->n[0];
    P->fny = g->n[1];
    P->fnz = g->n[2];
    P->fmx = g->n[0] / g->ds_factor;
    P->Mf = (long long)P->fmx * P->fny * P->fnz;
    if (g->n[0] % g->ds_factor != 0) {
        delete P;
        return MH3D_ERR_UNSUPPORTED_SIZE;
    }
    for (int a = 0; a < 3; ++a) P->vox[a] = g->voxel_mm[a];
    P->gamma = g->gamma_per_mm;
    P->gammaA = g->gammaA;
    P->tratio = g->transverse_ratio;
    P->theta.assign(P->K, 0.0);
    if (g->theta)
        for (int k = 0; k < P->K; ++k) P->theta[k] = g->theta[k];
    P->sens = g->sensitivity_dev;
    P->ax.n = nx;
    P->ay.n = ny;
    P->az.n = nz;
    P->am.n = mx;
    if (!radix_plan(nx, P->ax.rp, 0) || !radix_plan(ny, P->ay.rp, 0) || !radix_plan(nz, P->az.rp, 0) ||
        !radix_plan(mx, P->am.rp, 0)) {
        delete P;
        return MH3D_ERR_UNSUPPORTED_SIZE;
    }
    choose_tiles(*P);
    if (xfwd_smem_bytes(nx, mx, P->tile.xpass_pairs, P->tile.xpass_kgroup) > kSmemBudget ||
        tpass_smem_bytes(std::max(ny, nz), P->tile.tpass_cols) > kSmemBudget) {
        delete P;
        return MH3D_ERR_UNSUPPORTED_SIZE;
    }
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess && (dev < 0 || dev >= kAttrMaxDevices)) e = cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(g_attr_mu);
        if (e == cudaSuccess && !g_attr_done[dev]) {
            e = ops_set_attributes();
            if (e == cudaSuccess) e = solve_set_attributes();
            if (e == cudaSuccess) g_attr_done[dev] = true;
        }
        if (e != cudaSuccess) {
            g_create_err = std::string("kernel attributes: ") + cudaGetErrorString(e);
            delete P;
            return MH3D_ERR_CUDA;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    mh3d_status s = build_tables(*P, st);
    if (s == MH3D_OK) s = solve_alloc(*P);
    if (s != MH3D_OK) {
        g_create_err = P->err;
        solve_free(*P);
        if (P->table_mem) cudaFree(P->table_mem);
        delete P;
        return s;
    }
    g_create_err.clear();
    *out = P;
    return MH3D_OK;
}

mh3d_status mh3d_plan_spectra(mh3d_plan P, void* X, void* Y, void* Z, void* phase, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    auto cp = [&](void* dst, const float2* src, size_t n) {
        return dst ? cudaMemcpyAsync(dst, src, sizeof(float2) * n, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
    };
    cudaError_t e = cp(X, P->Xhat, (size_t)P->K * P->nx);
    if (e == cudaSuccess) e = cp(Y, P->Yhat, (size_t)P->ny);
    if (e == cudaSuccess) e = cp(Z, P->Zhat, (size_t)P->nz);
    if (e == cudaSuccess) e = cp(phase, P->phase, (size_t)P->K);
    if (e != cudaSuccess) {
        P->err = std::string("mh3d_plan_spectra: ") + cudaGetErrorString(e);
        return MH3D_ERR_CUDA;
    }
    return MH3D_OK;
}

mh3d_status mh3d_plan_destroy(mh3d_plan P)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    batch_forget(*P);
    solve_free(*P);
    mhad_free(*P);
    general_free(*P);
    if (P->table_mem) cudaFree(P->table_mem);
    delete P;
    return MH3D_OK;
}

mh3d_status mh3d_operator_norm2(mh3d_plan P, double* out)
{
    if (!P || !out) return MH3D_ERR_INVALID_ARG;
    *out = P->opnorm2;
    return MH3D_OK;
}

const char* mh3d_last_error(mh3d_plan P) { return P ? P->err.c_str() : g_create_err.c_str(); }

unsigned long long mh3d_plan_workspace_bytes(mh3d_plan P)
{
    return P ? (unsigned long long)(P->table_bytes + P->work_bytes) : 0ull;
}

mh3d_status mh3d_forward(mh3d_plan P, const float* rho, void* d, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!rho || !d) {
        P->err = "mh3d_forward: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    P->err.clear();
    if (P->padded) {   // forward on the extended grid, then the field of view's portraits
        mh3d_status s = ensure_portrait(*P);
        if (s != MH3D_OK) return s;
        MH3D_TRY(P, launch_forward(*P, rho, P->w.portrait, P->w.t1, P->w.t2, (cudaStream_t)stream));
        MH3D_TRY(P, crop_portraits(*P, P->w.portrait, (float2*)d, (cudaStream_t)stream));
        return MH3D_OK;
    }
    MH3D_TRY(P, launch_forward(*P, rho, (float2*)d, P->w.t1, P->w.t2, (cudaStream_t)stream));
    return MH3D_OK;
}

mh3d_status mh3d_adjoint(mh3d_plan P, const void* d, float* rho, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!rho || !d) {
        P->err = "mh3d_adjoint: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    P->err.clear();
    if (P->padded) {   // the field of view's portraits zero-padded, then the adjoint on the extended grid
        mh3d_status s = ensure_portrait(*P);
        if (s != MH3D_OK) return s;
        MH3D_TRY(P, pad_portraits(*P, (const float2*)d, P->w.portrait, (cudaStream_t)stream));
        MH3D_TRY(P, launch_adjoint(*P, P->w.portrait, rho, P->w.t1, P->w.t2, (cudaStream_t)stream));
        return MH3D_OK;
    }
    MH3D_TRY(P, launch_adjoint(*P, (const float2*)d, rho, P->w.t1, P->w.t2, (cudaStream_t)stream));
    return MH3D_OK;
}

mh3d_status mh3d_normal(mh3d_plan P, const float* p, float* q, const mh3d_solve_opts* o, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!p || !q || !o) {
        P->err = "mh3d_normal: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    mh3d_status v = validate_opts(*P, *o);
    if (v != MH3D_OK) return v;
    P->err.clear();
    // a padded plan's normal operator is the masked explicit one (mode 1)
    const int mode = P->padded ? 1 : o->normal_mode;
    if (mode == 1) {
        mh3d_status s = ensure_portrait(*P);
        if (s != MH3D_OK) return s;
    }
    MH3D_TRY(P, launch_normal(*P, mode, reg_args(*P, *o), p, q, P->w.t1, P->w.t2, P->w.portrait, nullptr, nullptr,
                              nullptr, (cudaStream_t)stream));
    return MH3D_OK;
}

}  // extern "C"
