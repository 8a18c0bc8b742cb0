// Instantiations and dispatch of the compile-time specialised pencil kernels.
//
// Lengths covered: transverse passes n in {32, 64, 96, 128, 192, 256};
// drive-axis passes (nx, s) in {(32,1), (64,2), (96,2), (128,1), (128,2),
// (192,2), (256,1), (256,2)}.  Radix schedules are chosen so that a forward
// transform's last radix feeds the inverse's first one (see fft_ct.cuh).
// Every other size runs the runtime-general kernels of ops.cu; setting
// MH3D_GENERIC=1 forces those for every size (A/B checks).
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include <cudaTypedefs.h>

#include "ops_ct.cuh"

namespace mh3d {

using namespace ct;

namespace {

bool force_generic()
{
    const char* v = std::getenv("MH3D_GENERIC");
    return v && v[0] && v[0] != '0';
}

struct TDesc {
    void (*fn)(TArgs) = nullptr;
    size_t smem = 0;
    int threads = kT;
};
struct XDesc {
    void (*fn)(XArgs) = nullptr;
    size_t smem = 0;
    int threads = kT;
    int pairs = kP;
};

// P: column pairs (pencils) per CTA, 4 or 8 (tiles of 8 or 16 columns).
// (16-column tiles with 256 threads measured 41.8 us per CG iteration
// against 35.1 us with 128 threads at 128x128x64; not instantiated.)
template <class L>
TDesc tdesc(int P)
{
    if (P == 4) return TDesc{k_tpass_ct<L, 4, 64>, tpass_ct_smem<L, 4>(), 64};   // 8-column tiles, 64 threads
    if (P == 8) return TDesc{k_tpass_ct<L, 8>, tpass_ct_smem<L, 8>()};
    return TDesc{};
}

// alt = 1: the alternative schedule the autotuner may pick (n = 64, 128).
TDesc tpass_desc(int n, int P, int alt = 0)
{
    if (alt == 1 && n == 64) return tdesc<RList<4, 16>>(P);
    if (alt == 1 && n == 128) return tdesc<RList<8, 16>>(P);
    switch (n) {
        case 32: return tdesc<RList<4, 8>>(P);
        case 64: return tdesc<RList<8, 8>>(P);
        case 96: return tdesc<RList<3, 4, 8>>(P);
        case 128: return tdesc<RList<16, 8>>(P);
        case 192: return tdesc<RList<3, 8, 8>>(P);
        case 256: return tdesc<RList<16, 16>>(P);
        default: return TDesc{};
    }
}

// LFF/LIF: forward kernel's length-nx forward and length-nx/s inverse;
// LFA/LIA: adjoint kernel's length-nx/s forward and length-nx inverse;
// LFN: normal kernel's length-nx forward (inverse reversed).
template <int S, class LFF, class LIF, class LFA, class LIA, class LFN>
XDesc xdesc(int which)
{
    if (which == 0) return XDesc{k_xfwd_ct<LFF, LIF, S>, xfwd_ct_smem<LFF, LIF, S>()};
    if (which == 6) return XDesc{k_xfwd_ct<LFF, LIF, S, 8, 128>, xfwd_ct_smem<LFF, LIF, S, 8>(), 128, 8};
    if (which == 1) return XDesc{k_xadj_ct<LFA, LIA, S>, xadj_ct_smem<LFA, LIA, S>()};
    if (which == 5) return XDesc{k_xadj_ct<LFA, LIA, S, true>, xadj_ct_smem<LFA, LIA, S, true>()};
    if (which == 7)
        return XDesc{k_xadj_ct<LFA, LIA, S, true, 8, 128>, xadj_ct_smem<LFA, LIA, S, true, 8>(), 128, 8};
    if (which == 8)
        return XDesc{k_xadj_ct<LFA, LIA, S, true, 8, 128, 2>, xadj_ct_smem<LFA, LIA, S, true, 8, 2>(), 128, 8};
    if (which == 3) return XDesc{k_xnrm_ct<LFN, S, true>, xnrm_ct_smem<LFN, S, true>(), kTN, kP};
    if (which == 4) return XDesc{k_xnrm_ct<LFN, S, false, 8, 128>, xnrm_ct_smem<LFN, S, false, 8>(), 128, 8};
    return XDesc{k_xnrm_ct<LFN, S, false>, xnrm_ct_smem<LFN, S, false>(), kTN, kP};
}

XDesc xpass_desc(int nx, int s, int which /*0 forward, 1 adjoint, 2 normal, 3 normal with bulk copies*/)
{
    if (nx == 32 && s == 1)
        return xdesc<1, RList<4, 8>, RList<8, 4>, RList<4, 8>, RList<8, 4>, RList<4, 8>>(which);
    if (nx == 64 && s == 2)
        return xdesc<2, RList<8, 8>, RList<4, 8>, RList<4, 8>, RList<16, 4>, RList<8, 8>>(which);
    if (nx == 96 && s == 2)
        return xdesc<2, RList<3, 4, 8>, RList<4, 4, 3>, RList<3, 4, 4>, RList<8, 4, 3>, RList<3, 4, 8>>(which);
    if (nx == 128 && s == 1)
        return xdesc<1, RList<16, 8>, RList<8, 16>, RList<16, 8>, RList<8, 16>, RList<16, 8>>(which);
    if (nx == 128 && s == 2)
        return xdesc<2, RList<16, 8>, RList<4, 16>, RList<8, 8>, RList<16, 8>, RList<16, 8>>(which);
    if (nx == 192 && s == 2)
        return xdesc<2, RList<3, 8, 8>, RList<4, 8, 3>, RList<3, 4, 8>, RList<16, 4, 3>, RList<3, 8, 8>>(which);
    if (nx == 256 && s == 1)
        return xdesc<1, RList<16, 16>, RList<16, 16>, RList<16, 16>, RList<16, 16>, RList<16, 16>>(which);
    if (nx == 256 && s == 2)
        return xdesc<2, RList<16, 16>, RList<8, 16>, RList<16, 8>, RList<16, 16>, RList<16, 16>>(which);
    return XDesc{};
}

template <class F>
cudaError_t opt_in(F* f, size_t need, int optin)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if (need + fa.sharedSizeBytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
}

}  // namespace

static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// MH3D_PDL=1 (opt-in): launch the CG loop's kernels (T passes, drive-axis
// normal pass) with programmatic stream serialization, so each may be
// scheduled while its predecessor finishes; the kernels wait for it before
// reading its output.  Measured at 128x128x64 inside the CG graph: 40.9 us
// per iteration with it, 35.7 us without (the early-scheduled CTAs hold SM
// slots the running pass needs), hence off by default.
static bool pdl_enabled()
{
    const char* e = std::getenv("MH3D_PDL");
    return e && e[0] == '1';
}

// Programmatic dependent launch of the fused normal pass after the T pass
// (default; MH3D_PDL_ZX=0 turns it off): the T pass signals after its
// epilogue, so the cluster pass's CTAs take SM slots only as the T pass's
// CTAs drain, and they wait for its completion before reading anything.
// Measured in the CG graph at 128x128x64, K = 8 (same box, two pairs):
// 23.89-23.92 us per iteration against 24.15-24.20 us without.
static bool pdl_zx_enabled()
{
    const char* e = std::getenv("MH3D_PDL_ZX");
    return !(e && e[0] == '0');
}

template <class Args>
static cudaError_t launch_pdl(void (*fn)(Args), dim3 grid, int threads, size_t smem, cudaStream_t st, const Args& a)
{
    if (!pdl_enabled()) {
        fn<<<grid, threads, smem, st>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
// (no link-time dependency on libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Map of a float32 volume [nz][ny][nx] whose box is one T-pass tile:
// (box_x, n, 1) along y or (box_x, 1, n) along z.
static bool encode_tile_map(CUtensorMap* m, const void* base, int nx, int ny, int nz, int axis, int n, int box_x)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float), (cuuint64_t)nx * ny * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, axis == 1 ? (cuuint32_t)n : 1u, axis == 1 ? 1u : (cuuint32_t)n};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The bulk-copy T pass needs whole 16-float tiles and 16-byte aligned rows.
bool ct_tpass_available(const TArgs& a)
{
    if (force_generic() || (a.cols != 8 && a.cols != 16) || !tpass_desc(a.n, a.cols / 2).fn) return false;
    if (a.nx % a.cols != 0 || (a.es % 4) != 0 || (a.os % 4) != 0) return false;
    const void* ptrs[] = {a.in, a.out, a.bin, a.bout, a.pvec, a.rvec, a.rvec_w, a.qdir, a.svec, a.xvec, a.qvec, a.pin};
    for (const void* p : ptrs)
        if (p && !al16(p)) return false;
    if (a.epilogue && a.reg.kind != 0) return false;
    if (a.pupdate == 2 && a.rvec_w != a.rvec) return false;   // r is updated in place
    if (a.n > 256 || !tensor_map_encoder()) return false;     // TMA box limit
    return true;
}
bool ct_xpass_available(int nx, int s, int pairs) { return !force_generic() && pairs == kP && xpass_desc(nx, s, 0).fn; }

// The y-slab cluster passes (k_zxnrm_ct, k_zxfwd_ct, k_xzadj_ct), per
// (nx, nz, s) and cluster size C: C CTAs per y-slab, each with nz/C rows
// of the drive-axis part and nx/C columns of the z part; 256 threads per CTA
// for C = 2, 128 for C = 4.
struct ZXDesc {
    void (*fn)(ZXArgs) = nullptr;
    size_t smem = 0;
    int threads = 256;
    int C = 2;
};
constexpr int zx_threads(int C) { return C == 2 ? 256 : 128; }

// Harmonics per round of the pipelined adjoint: one by default.
// MH3D_XADJ_KB=2 runs pairs (one first-stage run and one barrier per pair;
// twice the staged rows): measured slower at 128x128x64, K = 8 -- the
// cluster adjoint 61.5 us against 43.9 us (one CTA per SM instead of two),
// the separate 16-row pass 47.0 us against 43.6-44.5 us for A^T.
static int xadj_kb()
{
    const char* e = std::getenv("MH3D_XADJ_KB");
    return (e && e[0] == '2') ? 2 : 1;
}

// MH3D_ZX_CLUSTER=4: clusters of four CTAs (A/B checks); default two.
static int zx_cluster()
{
    const char* e = std::getenv("MH3D_ZX_CLUSTER");
    return (e && e[0] == '4') ? 4 : 2;
}

template <class LZ, class LF, int S, int C, bool EARLY>
ZXDesc zxdesc_e()
{
    constexpr int PZ = RInfo<LF>::n() / (2 * C), PX = RInfo<LZ>::n() / (2 * C), T = zx_threads(C);
    return ZXDesc{k_zxnrm_ct<LZ, LF, S, C, PZ, PX, T, EARLY>, ZxGeom<LZ, LF, C, PZ, PX>::smem(), T, C};
}
// which 0: early epilogue loads (a solve on its own); 3: epilogue loads in
// the epilogue (kernels that run beside other volumes' kernels)
template <class LZ, class LF, int S, int C>
ZXDesc zxdesc(int which)
{
    return which == 3 ? zxdesc_e<LZ, LF, S, C, false>() : zxdesc_e<LZ, LF, S, C, true>();
}
template <class LZ, class LF, class LI, int S, int C>
ZXDesc zxfdesc()
{
    constexpr int PZ = RInfo<LF>::n() / (2 * C), PX = RInfo<LZ>::n() / (2 * C), T = zx_threads(C);
    return ZXDesc{k_zxfwd_ct<LZ, LF, LI, S, C, PZ, PX, T>, ZxFwdGeom<LZ, LF, LI, C, PZ, PX>::smem(), T, C};
}
template <class LF2, class LI, class LZ, int S, int C, int KB>
ZXDesc xzdesc_kb()
{
    constexpr int PZ = RInfo<LI>::n() / (2 * C), PX = RInfo<LZ>::n() / (2 * C), T = zx_threads(C);
    return ZXDesc{k_xzadj_ct<LF2, LI, LZ, S, C, PZ, PX, T, KB>, XzGeom<LF2, LI, LZ, C, PZ, PX, KB>::smem(), T, C};
}
// Clusters of two run the adjoint part in rounds of xadj_kb() harmonics
// where the two rounds of row blocks fit in 227 KB of shared memory;
// otherwise (and for clusters of four) in rounds of one.
constexpr size_t kSmemOptinMax = 227 * 1024;
template <class LF2, class LI, class LZ, int S, int C>
constexpr bool xz_kb2_fits()
{
    constexpr int PZ = RInfo<LI>::n() / (2 * C), PX = RInfo<LZ>::n() / (2 * C);
    return C == 2 && XzGeom<LF2, LI, LZ, C, PZ, PX, 2>::smem() <= kSmemOptinMax;
}
template <class LF2, class LI, class LZ, int S, int C>
ZXDesc xzdesc()
{
    if constexpr (xz_kb2_fits<LF2, LI, LZ, S, C>()) {
        if (xadj_kb() == 2) return xzdesc_kb<LF2, LI, LZ, S, C, 2>();
    }
    return xzdesc_kb<LF2, LI, LZ, S, C, 1>();
}

// which: 0 normal, 1 forward, 2 adjoint, 3 normal without early epilogue
// loads.  Schedules: the z one of the T
// pass; the normal kernel's length-nx forward; the forward kernel's
// length-nx forward and length-nx/s inverse; the adjoint kernel's
// length-nx/s forward and length-nx inverse.
template <int C>
ZXDesc zx_desc_c(int which, int nx, int nz)
{
    if (nx == 128 && nz == 64) {
        if (which == 0 || which == 3) return zxdesc<RList<8, 8>, RList<16, 8>, 2, C>(which);
        if (which == 1) return zxfdesc<RList<8, 8>, RList<16, 8>, RList<4, 16>, 2, C>();
        return xzdesc<RList<8, 8>, RList<16, 8>, RList<8, 8>, 2, C>();
    }
    if (nx == 64 && nz == 64) {
        if (which == 0 || which == 3) return zxdesc<RList<8, 8>, RList<8, 8>, 2, C>(which);
        if (which == 1) return zxfdesc<RList<8, 8>, RList<8, 8>, RList<4, 8>, 2, C>();
        return xzdesc<RList<4, 8>, RList<16, 4>, RList<8, 8>, 2, C>();
    }
    if (nx == 96 && nz == 64) {
        if (which == 0 || which == 3) return zxdesc<RList<8, 8>, RList<3, 4, 8>, 2, C>(which);
        if (which == 1) return zxfdesc<RList<8, 8>, RList<3, 4, 8>, RList<4, 4, 3>, 2, C>();
        return xzdesc<RList<3, 4, 4>, RList<8, 4, 3>, RList<8, 8>, 2, C>();
    }
    // (192, 96) is not instantiated: its cluster passes need 120-207
    // registers per thread, and the CG solve measured 110.5 us per iteration
    // against 91.4 us with the separate passes
    return ZXDesc{};
}
ZXDesc zx_desc(int which, int nx, int nz, int s, int C)
{
    if (s != 2) return ZXDesc{};
    return C == 4 ? zx_desc_c<4>(which, nx, nz) : zx_desc_c<2>(which, nx, nz);
}

cudaError_t ct_set_attributes(int optin)
{
    // resolve the driver's encoder now: a first call inside a stream capture
    // would query the driver while the capture is open
    tensor_map_encoder();
    static const int tn[] = {32, 64, 96, 128, 192, 256};
    for (int n : tn)
        for (int P : {4, 8})
            for (int alt : {0, 1}) {
                const TDesc d = tpass_desc(n, P, alt);
                cudaError_t e = opt_in(d.fn, d.smem, optin);
                if (e != cudaSuccess) return e;
            }
    static const int zx[][2] = {{128, 64}, {64, 64}, {96, 64}};
    for (const auto& p : zx)
        for (int which = 0; which < 4; ++which)
            for (int C : {2, 4}) {
                const ZXDesc d = zx_desc(which, p[0], p[1], 2, C);
                cudaError_t e = opt_in(d.fn, d.smem, optin);
                if (e != cudaSuccess) return e;
            }
    // both round sizes of the clusters-of-two adjoint (xzdesc picks by MH3D_XADJ_KB)
    {
        const ZXDesc d[] = {
            xzdesc_kb<RList<8, 8>, RList<16, 8>, RList<8, 8>, 2, 2, 1>(),
            xzdesc_kb<RList<4, 8>, RList<16, 4>, RList<8, 8>, 2, 2, 1>(),
            xzdesc_kb<RList<3, 4, 4>, RList<8, 4, 3>, RList<8, 8>, 2, 2, 1>(),
            xzdesc_kb<RList<8, 8>, RList<16, 8>, RList<8, 8>, 2, 2, 2>(),
            xzdesc_kb<RList<4, 8>, RList<16, 4>, RList<8, 8>, 2, 2, 2>(),
            xzdesc_kb<RList<3, 4, 4>, RList<8, 4, 3>, RList<8, 8>, 2, 2, 2>(),
        };
        for (const ZXDesc& x : d) {
            cudaError_t e = opt_in(x.fn, x.smem, optin);
            if (e != cudaSuccess) return e;
        }
    }
    static const int xs[][2] = {{32, 1}, {64, 2}, {96, 2}, {128, 1}, {128, 2}, {192, 2}, {256, 1}, {256, 2}};
    for (const auto& p : xs)
        for (int w = 0; w < 9; ++w) {
            const XDesc d = xpass_desc(p[0], p[1], w);
            cudaError_t e = opt_in(d.fn, d.smem, optin);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t run_tpass_ct(const TArgs& a0, int nouter, cudaStream_t st)
{
    TArgs a = a0;
    const int ny = (a.axis == 1) ? a.n : nouter, nz = (a.axis == 1) ? nouter : a.n;
    auto enc = [&](int slot, const void* ptr) {
        return !ptr || encode_tile_map(&a.tm.m[slot], ptr, a.nx, ny, nz, a.axis, a.n, a.cols);
    };
    const bool ok = enc(kTmIn, a.in) && enc(kTmB, a.bin ? a.bin : a.bout) && enc(kTmR, a.rvec) &&
                    enc(kTmS, a.svec) && enc(kTmP, a.pvec) && enc(kTmQ, a.qdir) && enc(kTmX, a.xvec) &&
                    enc(kTmOut, a.epilogue ? a.qvec : a.out) && enc(kTmPin, a.pin);
    if (!ok) return cudaErrorInvalidValue;
    const TDesc d = tpass_desc(a.n, a.cols / 2, a.radix_alt);
    dim3 grid((a.nx + a.cols - 1) / a.cols, nouter);
    return launch_pdl(d.fn, grid, d.threads, d.smem, st, a);
}

static cudaError_t run_x_ct(const XArgs& a, int which, cudaStream_t st)
{
    const XDesc d = xpass_desc(a.nx, a.s, which);
    if (which >= 2 && which <= 4)
        return launch_pdl(d.fn, dim3(xpass_blocks(a.rows, d.pairs)), d.threads, d.smem, st, a);
    d.fn<<<xpass_blocks(a.rows, d.pairs), d.threads, d.smem, st>>>(a);
    return cudaGetLastError();
}

// MH3D_XFWD_PAIRS=8: 16 rows per CTA for the forward pass (A/B).
static bool xfwd_small()
{
    const char* e = std::getenv("MH3D_XFWD_PAIRS");
    return e && e[0] == '8';
}

// Harmonics per CTA of the forward pass: all of them by default (13.5 us
// per launch at 128x128x64, K = 8, against 15.4 us in groups of 4 and
// 18.3 us in groups of 2 on grid.y); MH3D_XFWD_KPC=n sets groups of n.
static int xfwd_kpc(int K)
{
    int kpc = 0;
    if (const char* e = std::getenv("MH3D_XFWD_KPC")) kpc = std::atoi(e);
    return (kpc <= 0 || kpc >= K) ? K : kpc;
}

cudaError_t run_xfwd_ct(const XArgs& a0, cudaStream_t st)
{
    XArgs a = a0;
    a.kpc = xfwd_kpc(a.K);
    const XDesc d = xpass_desc(a.nx, a.s, xfwd_small() ? 6 : 0);
    const dim3 grid(xpass_blocks(a.rows, d.pairs), (a.K + a.kpc - 1) / a.kpc);
    d.fn<<<grid, d.threads, d.smem, st>>>(a);
    return cudaGetLastError();
}
// The pipelined adjoint needs 16-byte aligned portrait blocks: an aligned
// base, an even mx (rows of mx complex are then 16-byte multiples) and an
// even M; MH3D_XADJ_BULK=0 turns it off (A/B checks).
static bool xadj_bulk_ok(const XArgs& a)
{
    const char* e = std::getenv("MH3D_XADJ_BULK");
    if (e && e[0] == '0') return false;
    return al16(a.din) && (a.mx % 2) == 0 && (a.M % 2) == 0;
}

// 16 rows per CTA (512 CTAs of 128 threads at 128x128x64) for the
// pipelined adjoint by default: A^T 45.1 us against 51.2 us with 32 rows;
// MH3D_XADJ_PAIRS=16 selects the latter (A/B checks).
static bool xadj_small()
{
    const char* e = std::getenv("MH3D_XADJ_PAIRS");
    return !(e && e[0] == '1' && e[1] == '6');
}

cudaError_t run_xadj_ct(const XArgs& a, cudaStream_t st)
{
    if (!xadj_bulk_ok(a)) return run_x_ct(a, 1, st);
    if (!xadj_small()) return run_x_ct(a, 5, st);
    return run_x_ct(a, xadj_kb() == 2 ? 8 : 7, st);
}
// The bulk-copy normal pass (opt-in: MH3D_XNRM_BULK=1; measured 3 % slower
// per CG iteration than the register-loading pass at 128x128x64) needs
// 16-byte aligned vectors (rows of nx floats are then 16-byte aligned too,
// nx % 4 == 0) and R = I.
static bool xnrm_bulk_ok(const XArgs& a)
{
    const char* e = std::getenv("MH3D_XNRM_BULK");
    if (!e || e[0] != '1') return false;
    return a.vec4 && a.reg.kind == 0 && (a.nx % 4) == 0 && al16(a.vin) && al16(a.pin) && al16(a.qout) &&
           (!a.b || al16(a.b));
}

// 16 rows per CTA (512 CTAs at 128x128x64, 128 threads) by default: 35.3 us
// per CG iteration against 35.7 us with 32 rows and 256 threads;
// MH3D_XNRM_PAIRS=16 selects the latter (A/B checks).
static bool xnrm_small()
{
    const char* e = std::getenv("MH3D_XNRM_PAIRS");
    return !(e && e[0] == '1' && e[1] == '6');
}

// The cluster passes for the instantiated (nx, nz, s); MH3D_FUSE_ZX=0
// keeps the separate passes (A/B checks).
static bool zx_enabled(int which, int nx, int nz, int s)
{
    const char* e = std::getenv("MH3D_FUSE_ZX");
    if (e && e[0] == '0') return false;
    return !force_generic() && zx_desc(which, nx, nz, s, zx_cluster()).fn && tensor_map_encoder();
}
bool ct_zxnrm_available(int nx, int nz, int s) { return zx_enabled(0, nx, nz, s); }
bool ct_zxfwd_available(int nx, int nz, int s) { return zx_enabled(1, nx, nz, s); }
bool ct_xzadj_available(int nx, int nz, int s) { return zx_enabled(2, nx, nz, s); }

// C CTAs per y-slab; the z volume's tensor map (box nx/C x 1 x nz, x
// coordinates multiples of nx/C: 16-byte multiples for nx % 4C == 0) is
// encoded here.  zvol: the z pass's input (normal, forward) or output
// (adjoint).
static cudaError_t run_zx(ZXArgs& a, const void* zvol, int which, cudaStream_t st)
{
    const int nx = a.x.nx;
    const char* ev = std::getenv("MH3D_ZX_CLUSTER");
    const int C = (ev && ev[0]) ? zx_cluster() : (a.C == 4 ? 4 : 2);
    const ZXDesc d = zx_desc(which, nx, a.nz, a.x.s, C);
    if (!d.fn || nx % (4 * d.C) != 0 || a.nz % (2 * d.C) != 0 || !al16(zvol)) return cudaErrorInvalidValue;
    if (!encode_tile_map(&a.tz, zvol, nx, a.ny, a.nz, 2, a.nz, nx / d.C)) return cudaErrorInvalidValue;
    if ((which == 0 || which == 3) && pdl_zx_enabled()) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(d.C * a.ny);
        cfg.blockDim = dim3(d.threads);
        cfg.dynamicSmemBytes = d.smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, d.fn, a);
    }
    d.fn<<<d.C * a.ny, d.threads, d.smem, st>>>(a);
    return cudaGetLastError();
}
bool ct_encode_z_map(CUtensorMap* m, const void* zvol, int nx, int ny, int nz, int box_x)
{
    return al16(zvol) && encode_tile_map(m, zvol, nx, ny, nz, 2, nz, box_x);
}
cudaError_t run_zxnrm_ct(ZXArgs& a, const float* zin, cudaStream_t st, bool shared_sms)
{
    return run_zx(a, zin, shared_sms ? 3 : 0, st);
}
cudaError_t run_zxfwd_ct(ZXArgs& a, const float* zin, cudaStream_t st) { return run_zx(a, zin, 1, st); }
// The adjoint's cluster pass also needs the pipelined adjoint's conditions
// (16-byte aligned portraits, even mx and M).
cudaError_t run_xzadj_ct(ZXArgs& a, float* zout, cudaStream_t st)
{
    if (!al16(a.x.din) || (a.x.mx % 2) != 0 || (a.x.M % 2) != 0) return cudaErrorInvalidValue;
    return run_zx(a, zout, 2, st);
}

cudaError_t run_xnrm_ct(const XArgs& a, cudaStream_t st)
{
    return run_x_ct(a, xnrm_bulk_ok(a) ? 3 : (xnrm_small() ? 4 : 2), st);
}

}  // namespace mh3d
