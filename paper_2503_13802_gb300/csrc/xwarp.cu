// Launchers of the warp-centric drive-axis passes (xwarp.cuh).
#include <cstdint>
#include <cstdlib>

#include "xwarp.cuh"

namespace mh3d {

namespace {

bool env_off(const char* name)
{
    const char* v = std::getenv(name);
    return v && v[0] == '0';
}
bool env_on(const char* name)
{
    const char* v = std::getenv(name);
    return v && v[0] && v[0] != '0';
}
bool al(const void* p, uintptr_t m) { return ((uintptr_t)p & (m - 1)) == 0; }

}  // namespace

// The warp passes serve n_x = 128 with s = 2 (any row count, K <= kMaxK).
// Measured at 128x128x64, K = 8 (A and A^T with L2 flushed, same box): the
// adjoint A^T = warp pass + T_z + T_y took 33.2 us against 43.7 us with the
// CTA-level cluster pass, so it is the default (MH3D_XWARP=0 keeps the
// CTA-level passes); the forward A = T_y + T_z + warp pass took 34.4 us
// against 30.2 us with the cluster pass that fuses T_z, so the warp
// forward is opt-in (MH3D_XWARP_FWD=1).  MH3D_GENERIC=1 turns both off.
bool xw_available(const XArgs& a, bool forward, bool want)
{
    if (env_on("MH3D_GENERIC") || env_off("MH3D_XWARP")) return false;
    if (forward && !(env_on("MH3D_XWARP_FWD") || (want && !env_off("MH3D_XWARP_FWD")))) return false;
    return a.nx == xw::kNX && a.s == 2 && a.mx == xw::kMX && a.K >= 1 && a.K <= kMaxK && a.rows >= 1;
}

// Warps per row group (harmonics split over them): MH3D_XWARP_KS = 1, 2 or
// 4.  Default 2 (same workload: A^T 35.4 us with 1, 33.2 us with 2,
// 36.3 us with 4).
int xw_ks(int plan_ks = 0)
{
    const char* v = std::getenv("MH3D_XWARP_KS");
    if (v && (v[0] == '1' || v[0] == '2' || v[0] == '4')) return v[0] - '0';
    return (plan_ks == 1 || plan_ks == 4) ? plan_ks : 2;
}

template <class F>
static cudaError_t smem_attr(F* f, size_t bytes)
{
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The cluster variant of the warp adjoint (T_z^T fused) for nz = 64;
// MH3D_XWARP_ZX=0 keeps the warp pass and T_z^T as two launches.
using LZ64 = ct::RList<8, 8>;
bool xzw_available(const XArgs& a, int nz)
{
    return xw_available(a, false) && !env_off("MH3D_XWARP_ZX") && nz == 64;
}

// The warp-centric cluster normal pass (n_x = 128, s = 2, n_z = 64),
// opt-in (MH3D_XWARP_NRM=1): in the CG loop at 128x128x64 it measured 25.8
// us per iteration against 23.1 us for the CTA-level cluster pass (same
// box).  Not for want of threads in its z part: with 256 threads per CTA
// (the drive-axis part on half of them) it measured 25.5 against 23.3 us.
bool zxnw_available(const XArgs& a, int nz)
{
    return !env_on("MH3D_GENERIC") && !env_off("MH3D_XWARP") && env_on("MH3D_XWARP_NRM") && a.nx == xw::kNX &&
           a.s == 2 && a.mx == xw::kMX && nz == 64;
}

cudaError_t xw_set_attributes()
{
    cudaError_t en = smem_attr(xw::k_zxnrm_w<LZ64, true>, xw::ZxwGeom<LZ64>::smem());
    if (en == cudaSuccess) en = smem_attr(xw::k_zxnrm_w<LZ64, false>, xw::ZxwGeom<LZ64>::smem());
    if (en != cudaSuccess) return en;
    cudaError_t e0 = smem_attr(xw::k_xzadj_w<LZ64, 1>, xw::XzwGeom<LZ64, 1>::smem(kMaxK));
    if (e0 == cudaSuccess) e0 = smem_attr(xw::k_xzadj_w<LZ64, 2>, xw::XzwGeom<LZ64, 2>::smem(kMaxK));
    if (e0 == cudaSuccess) e0 = smem_attr(xw::k_xzadj_w<LZ64, 4>, xw::XzwGeom<LZ64, 4>::smem(kMaxK));
    if (e0 != cudaSuccess) return e0;

    cudaError_t e = smem_attr(xw::k_xfwd_w128<1>, xw::fwd_smem(kMaxK));
    if (e == cudaSuccess) e = smem_attr(xw::k_xfwd_w128<2>, xw::fwd_smem(kMaxK));
    if (e == cudaSuccess) e = smem_attr(xw::k_xfwd_w128<4>, xw::fwd_smem(kMaxK));
    if (e == cudaSuccess) e = smem_attr(xw::k_xadj_w128<1>, xw::adj_smem(kMaxK));
    if (e == cudaSuccess) e = smem_attr(xw::k_xadj_w128<2>, xw::adj_smem(kMaxK));
    if (e == cudaSuccess) e = smem_attr(xw::k_xadj_w128<4>, xw::adj_smem(kMaxK));
    return e;
}

static int xw_grid(int rows, int ks)
{
    const int groups = (rows + xw::kRowsW - 1) / xw::kRowsW;
    const int per_cta = xw::kWarps / ks;
    return (groups + per_cta - 1) / per_cta;
}

cudaError_t run_xfwd_w(const XArgs& a, cudaStream_t st)
{
    if (!al(a.vin, 8) || !al(a.dout, 8)) return cudaErrorMisalignedAddress;
    const int ks = xw_ks(a.ks);
    const dim3 grid(xw_grid(a.rows, ks));
    const size_t smem = xw::fwd_smem(a.K);
    if (ks == 1) xw::k_xfwd_w128<1><<<grid, xw::kWarps * 32, smem, st>>>(a);
    else if (ks == 2) xw::k_xfwd_w128<2><<<grid, xw::kWarps * 32, smem, st>>>(a);
    else xw::k_xfwd_w128<4><<<grid, xw::kWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t run_xadj_w(const XArgs& a, cudaStream_t st)
{
    if (!al(a.din, 8) || !al(a.vout, 4)) return cudaErrorMisalignedAddress;
    const int ks = xw_ks(a.ks);
    const dim3 grid(xw_grid(a.rows, ks));
    const size_t smem = xw::adj_smem(a.K);
    if (ks == 1) xw::k_xadj_w128<1><<<grid, xw::kWarps * 32, smem, st>>>(a);
    else if (ks == 2) xw::k_xadj_w128<2><<<grid, xw::kWarps * 32, smem, st>>>(a);
    else xw::k_xadj_w128<4><<<grid, xw::kWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mh3d

namespace mh3d {

cudaError_t run_xzadj_w(ZXArgs& a, float* zout, cudaStream_t st)
{
    if (!al(a.x.din, 8) || !al(zout, 16) || a.nz != 64) return cudaErrorInvalidValue;
    if (!ct_encode_z_map(&a.tz, zout, a.x.nx, a.ny, a.nz, a.x.nx / 2)) return cudaErrorInvalidValue;
    const int ks = xw_ks(a.x.ks);
    const dim3 grid(2 * a.ny);
    if (ks == 1)
        xw::k_xzadj_w<LZ64, 1><<<grid, xw::XzwGeom<LZ64, 1>::T, xw::XzwGeom<LZ64, 1>::smem(a.x.K), st>>>(a);
    else if (ks == 2)
        xw::k_xzadj_w<LZ64, 2><<<grid, xw::XzwGeom<LZ64, 2>::T, xw::XzwGeom<LZ64, 2>::smem(a.x.K), st>>>(a);
    else
        xw::k_xzadj_w<LZ64, 4><<<grid, xw::XzwGeom<LZ64, 4>::T, xw::XzwGeom<LZ64, 4>::smem(a.x.K), st>>>(a);
    return cudaGetLastError();
}

}  // namespace mh3d

namespace mh3d {

cudaError_t run_zxnrm_w(ZXArgs& a, const float* zin, cudaStream_t st, bool shared_sms)
{
    using G = xw::ZxwGeom<LZ64>;
    if (a.nz != 64 || !al(zin, 16) || !al(a.x.pin, 16) || !al(a.x.qout, 16)) return cudaErrorInvalidValue;
    if (!ct_encode_z_map(&a.tz, zin, a.x.nx, a.ny, a.nz, a.x.nx / 2)) return cudaErrorInvalidValue;
    const dim3 grid(2 * a.ny);
    if (shared_sms) xw::k_zxnrm_w<LZ64, false><<<grid, G::T, G::smem(), st>>>(a);
    else xw::k_zxnrm_w<LZ64, true><<<grid, G::T, G::smem(), st>>>(a);
    return cudaGetLastError();
}

}  // namespace mh3d
