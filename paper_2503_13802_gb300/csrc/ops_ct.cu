// Instantiations and dispatch of the compile-time specialised pencil kernels.
//
// Lengths covered: transverse passes n in {32, 64, 96, 128, 192, 256};
// drive-axis passes (nx, s) in {(32,1), (64,2), (96,2), (128,1), (128,2),
// (192,2), (256,1), (256,2)}.  Radix schedules are chosen so that a forward
// transform's last radix feeds the inverse's first one (see fft_ct.cuh).
// Every other size runs the runtime-general kernels of ops.cu; setting
// MH3D_GENERIC=1 forces those for every size (A/B checks).
#include <cstdlib>

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
};
struct XDesc {
    void (*fn)(XArgs) = nullptr;
    size_t smem = 0;
};

template <class L>
TDesc tdesc()
{
    return TDesc{k_tpass_ct<L>, tpass_ct_smem<L>()};
}

TDesc tpass_desc(int n)
{
    switch (n) {
        case 32: return tdesc<RList<4, 8>>();
        case 64: return tdesc<RList<8, 8>>();
        case 96: return tdesc<RList<3, 4, 8>>();
        case 128: return tdesc<RList<16, 8>>();
        case 192: return tdesc<RList<3, 8, 8>>();
        case 256: return tdesc<RList<16, 16>>();
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
    if (which == 1) return XDesc{k_xadj_ct<LFA, LIA, S>, xadj_ct_smem<LFA, LIA, S>()};
    return XDesc{k_xnrm_ct<LFN, S>, xnrm_ct_smem<LFN, S>()};
}

XDesc xpass_desc(int nx, int s, int which /*0 forward, 1 adjoint, 2 normal*/)
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

bool ct_tpass_available(int n, int cols) { return !force_generic() && cols == 2 * kP && tpass_desc(n).fn; }
bool ct_xpass_available(int nx, int s, int pairs) { return !force_generic() && pairs == kP && xpass_desc(nx, s, 0).fn; }

cudaError_t ct_set_attributes(int optin)
{
    static const int tn[] = {32, 64, 96, 128, 192, 256};
    for (int n : tn) {
        const TDesc d = tpass_desc(n);
        cudaError_t e = opt_in(d.fn, d.smem, optin);
        if (e != cudaSuccess) return e;
    }
    static const int xs[][2] = {{32, 1}, {64, 2}, {96, 2}, {128, 1}, {128, 2}, {192, 2}, {256, 1}, {256, 2}};
    for (const auto& p : xs)
        for (int w = 0; w < 3; ++w) {
            const XDesc d = xpass_desc(p[0], p[1], w);
            cudaError_t e = opt_in(d.fn, d.smem, optin);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t run_tpass_ct(const TArgs& a, int nouter, cudaStream_t st)
{
    const TDesc d = tpass_desc(a.n);
    dim3 grid((a.nx + 2 * kP - 1) / (2 * kP), nouter);
    d.fn<<<grid, kT, d.smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t run_x_ct(const XArgs& a, int which, cudaStream_t st)
{
    const XDesc d = xpass_desc(a.nx, a.s, which);
    d.fn<<<xpass_blocks(a.rows, kP), kT, d.smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t run_xfwd_ct(const XArgs& a, cudaStream_t st) { return run_x_ct(a, 0, st); }
cudaError_t run_xadj_ct(const XArgs& a, cudaStream_t st) { return run_x_ct(a, 1, st); }
cudaError_t run_xnrm_ct(const XArgs& a, cudaStream_t st) { return run_x_ct(a, 2, st); }

}  // namespace mh3d
