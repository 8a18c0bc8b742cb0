// The learned warm-start network behind the C ABI of include/mh3d_unet.h:
// parameters (FP32 master copy, Adam state), bfloat16 weight matrices laid
// out for the implicit-GEMM kernels, every stored activation of the last
// forward pass, and the gradient buffers of the backward pass.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../include/mh3d_unet.h"
#include "umma_conv.cuh"
#include "unet_kernels.cuh"

namespace mh3d {
namespace unet {

namespace {

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// MH3D_UNET_GATHER=1 forces the gather kernel for every convolution (A/B checks).
bool tiles_disabled()
{
    const char* e = std::getenv("MH3D_UNET_GATHER");
    return e && e[0] && e[0] != '0';
}
int tile_n(int n) { return n <= 16 ? 16 : (n <= 32 ? 32 : 64); }
unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Weights of one convolution in the tcgen05 kernel's B-operand layout
// ([27][c8p][np][8] bfloat16, umma_conv.cuh); w null: that kernel is not
// used for it.
struct UmmaW {
    __nv_bfloat16* w = nullptr;
    __nv_bfloat16* wp = nullptr;   // paired-tap layout (sources of at most 8 channels), or null
    int c8p = 0, np = 0;
    int sgn = 1;                   // -1: the input-gradient (flipped) operand
};

// FP32 workspace of the split-K partial sums of the gather kernel (owned
// by the network).
struct SplitWS {
    float* p = nullptr;
    size_t cap = 0;   // floats
};

struct Layer {
    int cin = 0, cout = 0;
    UmmaW uf, ub;                   // forward and input-gradient operands of the tcgen05 kernel
    long long woff = 0, boff = 0;   // offsets of W [cout][27][cin] and b [cout] in theta
    int Kf = 0, Nf = 0;             // forward matrix [Kf][Nf]
    int Kb = 0, Nb = 0;             // input-gradient matrix [Kb][Nb]
    __nv_bfloat16* Wf = nullptr;
    __nv_bfloat16* Wb = nullptr;
};

}  // namespace

constexpr int kMaxLevels = 5;
constexpr int kMaxChannels = 128;
constexpr int kMaxLayers = 4 * kMaxLevels - 1;

struct Net {
    int D = 0, H = 0, W = 0;
    int levels = 0;
    int ch[kMaxLevels] = {};          // channels per level
    long long V[kMaxLevels] = {};     // voxels per level (V[l] = V[0] / 8^l)
    int dims[kMaxLevels][3] = {};     // (D, H, W) per level
    int nlayers = 0;
    long long nparam = 0;
    int adam_t = 0;
    Layer L[kMaxLayers];
    std::vector<void*> allocs;
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    // forward activations (bfloat16, channels last) per level, and the FP32
    // output.  Encoder: ea, e (level l), p[l] = pool(e[l]) (level l + 1);
    // decoder (l < levels - 1): u, d; the bottleneck's d is its e.
    __nv_bfloat16 *ea[kMaxLevels] = {}, *e[kMaxLevels] = {}, *p[kMaxLevels] = {};
    __nv_bfloat16 *u[kMaxLevels] = {}, *d[kMaxLevels] = {};
    float* out = nullptr;
    const float* in = nullptr;       // the last forward's input (borrowed)
    const float* iscale = nullptr;   // the last forward's input scale (device scalar) or null
    float* scales = nullptr;         // {1 / r, r gain, 1 / (r gain)} of the scaled calls
    double* spart = nullptr;
    // gradients (w.r.t. the named activations): gd (d; the bottleneck's e),
    // gs (u + e), gup (up(d[l + 1]) at level l), ge (e), gea (ea), gp (p)
    __nv_bfloat16* gout = nullptr;
    __nv_bfloat16 *gd[kMaxLevels] = {}, *gs[kMaxLevels] = {}, *gup[kMaxLevels] = {};
    __nv_bfloat16 *ge[kMaxLevels] = {}, *gea[kMaxLevels] = {}, *gp[kMaxLevels] = {};
    __nv_bfloat16* scratch = nullptr;
    float *wpart = nullptr, *bpart = nullptr;
    int* status = nullptr;           // device word: MH3D_ERR_TIMEOUT from a bounded wait, else 0
    SplitWS skws;                    // split-K partial sums of the coarse gather convolutions
    double* lpart = nullptr;
    double* lhost = nullptr;
    size_t wpart_n = 0, bpart_n = 0;
    int lblocks = 0;
    bool weights_ready = false;
    std::string err;
};

namespace {

template <class T>
cudaError_t dalloc(Net& n, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        n.allocs.push_back(q);
        *p = (T*)q;
    }
    return e;
}

void free_net(Net& n)
{
    for (void* p : n.allocs) cudaFree(p);
    n.allocs.clear();
    if (n.lhost) cudaFreeHost(n.lhost);
    n.lhost = nullptr;
}

ConvSrc src_of(const __nv_bfloat16* a, int D, int H, int W, int C, const __nv_bfloat16* skip = nullptr, int up = 0)
{
    ConvSrc s;
    s.a = a;
    s.b = skip;
    s.D = D;
    s.H = H;
    s.W = W;
    s.C = C;
    s.up = up;
    return s;
}

int num_sms()
{
    static int v = -1;
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    }
    return v;
}

int smem_optin()
{
    static int v = -1;
    if (v < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 48 * 1024;
    }
    return v;
}

// The halo-tiled kernel when its shared memory fits; false otherwise.
template <int C, int BN, class OutT>
bool tile_conv(const ConvSrc& s, const __nv_bfloat16* Wt, int Kpad, int Npad, int N, const float* bias, int relu,
               const float* oscale, OutT* out, cudaStream_t st, cudaError_t* err)
{
    const size_t smem = tile_smem<C, BN>(Kpad);
    if (smem > (size_t)smem_optin()) return false;
    // the attribute belongs to the current device: set once per device
    static bool attr_dev[64] = {};
    int dev = 0;
    if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return true;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return true;
    }
    if (!attr_dev[dev] && smem > 48 * 1024) {
        if ((*err = cudaFuncSetAttribute(k_conv_tile<C, BN, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_optin())) != cudaSuccess)
            return true;
        attr_dev[dev] = true;
    }
    // persistent grid: resident CTAs per SM (cached per shared-memory size) x SMs
    static size_t occ_smem = 0;
    static int occ = 0;
    if (occ_smem != smem) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv_tile<C, BN, OutT>, kThreads, smem) !=
            cudaSuccess)
            occ = 1;
        occ = std::max(occ, 1);
        occ_smem = smem;
    }
    const int tiles = ((s.W + kTX - 1) / kTX) * ((s.H + kTY - 1) / kTY) * ((s.D + kTZ - 1) / kTZ);
    const int grid = std::min(tiles, num_sms() * occ);
    k_conv_tile<C, BN, OutT><<<dim3((unsigned)grid, (unsigned)(Npad / BN)), kThreads, smem, st>>>(
        s, Wt, Kpad, Npad, N, bias, relu, oscale, out, tiles);
    *err = cudaGetLastError();
    return true;
}

template <int C, class OutT>
bool tile_conv_n(const ConvSrc& s, const __nv_bfloat16* Wt, int Kpad, int Npad, int N, const float* bias, int relu,
                 const float* oscale, OutT* out, cudaStream_t st, cudaError_t* err)
{
    // output tiles of tile_n(N) columns; 32 outputs whose weights do not fit
    // in shared memory (64 input channels: 27 x 64 weight rows) take two
    // tiles of 16 (upsampled 64 -> 32 at 64x64x32: 228 us, 250 us on the
    // gather kernel).  For 64 outputs, narrower tiles lose to the split-K
    // gather kernel (64 -> 64 at 32x32x16: 79 against 62 us), which takes them.
    const int bn = tile_n(N);
    if (bn == 32 && tile_smem<C, 32>(Kpad) > (size_t)smem_optin())
        return tile_conv<C, 16>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, err);
    if (bn == 16) return tile_conv<C, 16>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, err);
    if (bn == 32) return tile_conv<C, 32>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, err);
    return tile_conv<C, 64>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, err);
}

// ---- the tcgen05 convolution (umma_conv.cuh) --------------------------------

// Chunk planes (8 channels each, padded to an even count) of a source the
// tcgen05 kernel takes: the FP32 single-channel input, or 8..32 bfloat16
// channels in multiples of 8; 0 otherwise.
int umma_c8p(int Cs, bool f32)
{
    if (f32) return Cs == 1 ? 2 : 0;
    if (Cs < 8 || Cs > 32 || Cs % 8 != 0) return 0;
    return (Cs / 8 + 1) / 2 * 2;
}
// Accumulator columns for N output channels (a multiple of 16), 0 past 64.
int umma_np(int N) { return N <= 16 ? 16 : (N <= 32 ? 32 : (N <= 64 ? 64 : 0)); }

// Which convolutions run on the tcgen05 kernel.  By default those whose
// rows fill most of a 128-voxel tile (W >= 96; the FP32 single-channel
// input only with paired taps): per launch at 128x128x64, channels
// (8, 16, 32), L2 flushed, it takes the full-resolution layers in 58 (FP32
// input 1 -> 8), 52 (8 -> 8), 68 (upsampled 16 -> 8), 71 (skip sum 8 -> 8)
// and 51 us (8 -> 1, FP32 out) against 62, 90, 158, 99 and 89 us on the
// mma.sync tiles, while the half- and quarter-resolution layers (rows of 64
// and 32 voxels in a 128-lane accumulator: 22-29 against 10-23 us) stay on
// mma.sync.
// MH3D_UNET_UMMA=1 sends every convolution it can take to the tcgen05
// kernel, 0 none.
int umma_mode()
{
    const char* e = std::getenv("MH3D_UNET_UMMA");
    if (e && e[0] == '0') return 0;
    if (e && e[0] == '1') return 2;
    return 1;
}
bool umma_enabled() { return umma_mode() != 0; }
bool umma_pair();
bool umma_prefers(const ConvSrc& s) { return umma_mode() == 2 || (s.W >= 96 && (!s.f32 || umma_pair())); }

template <int C8P, int NP, int NB, int R, class OutT>
cudaError_t launch_umma_t(const ConvSrc& s, const __nv_bfloat16* Wu, int N, const float* bias, int relu,
                          const float* oscale, OutT* out, int* status, cudaStream_t st,
                          const __nv_bfloat16* Wpair = nullptr)
{
    using G = umma::Geom<C8P, NP, NB, R>;
    auto* fn = umma::k_conv_umma<C8P, NP, NB, R, OutT>;
    const size_t smem = G::smem();
    if (smem > (size_t)smem_optin()) return cudaErrorInvalidValue;
    // resident CTAs per SM, with the attributes set, once per device (the
    // attributes belong to the current device)
    constexpr int kDevs = 64;
    static int occ_dev[kDevs] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
    int& occ = occ_dev[dev];
    if (occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // the whole carveout to shared memory, so that several CTAs fit
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the shared memory (each CTA also reserves
        // 1 KB), the registers and the threads; every resident CTA holds
        // G::kCols of the SM's 512 TMEM columns
        int smem_sm = 0, regs_sm = 0;
        cudaFuncAttributes fa{};
        if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, fn) != cudaSuccess)
            return cudaErrorInvalidValue;
        const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
        const int by_regs = regs_sm / std::max(1, fa.numRegs * umma::kT);
        occ = std::max(1, std::min(std::min(by_smem, by_regs), std::min(2048 / umma::kT, 512 / G::kCols)));
    }
    const long long tiles = (long long)((s.W + umma::kM - 1) / umma::kM) * ((s.H + R - 1) / R) * s.D;
    if (tiles > (1LL << 30)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(tiles, (long long)num_sms() * occ);
    fn<<<grid, umma::kT, smem, st>>>(s, Wu, N, bias, relu, oscale, out, (int)tiles, status, Wpair);
    return cudaGetLastError();
}

// The warp-specialised form (umma_conv.cuh: producer, MMA and epilogue
// warps, one persistent CTA per SM, NS halo slots): MH3D_UMMA_WS=1.
bool umma_ws()
{
    const char* e = std::getenv("MH3D_UMMA_WS");
    return e && e[0] == '1';
}

template <int C8P, int NP, int NS, class OutT>
cudaError_t launch_umma_ws_t(const ConvSrc& s, const __nv_bfloat16* Wu, int N, const float* bias, int relu,
                             const float* oscale, OutT* out, int* status, cudaStream_t st)
{
    using G = umma::GeomWs<C8P, NP, NS>;
    auto* fn = umma::k_conv_umma_ws<C8P, NP, NS, OutT>;
    const size_t smem = G::smem();
    constexpr int kDevs = 64;
    static bool attr_dev[kDevs] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
    if (!attr_dev[dev]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_dev[dev] = true;
    }
    const long long tiles = (long long)((s.W + umma::kM - 1) / umma::kM) * s.H * s.D;
    if (tiles > (1LL << 30)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(tiles, (long long)num_sms());   // one CTA per SM
    fn<<<grid, umma::kWsT, smem, st>>>(s, Wu, N, bias, relu, oscale, out, (int)tiles, status);
    return cudaGetLastError();
}

// The deepest halo ring that fits (4, 3 or 2 slots); false if none does.
template <int C8P, int NP, class OutT>
bool launch_umma_ws(const ConvSrc& s, const __nv_bfloat16* Wu, int N, const float* bias, int relu,
                    const float* oscale, OutT* out, int* status, cudaStream_t st, cudaError_t* err)
{
    const size_t lim = (size_t)smem_optin();
    if (umma::GeomWs<C8P, NP, 4>::smem() <= lim)
        *err = launch_umma_ws_t<C8P, NP, 4>(s, Wu, N, bias, relu, oscale, out, status, st);
    else if (umma::GeomWs<C8P, NP, 3>::smem() <= lim)
        *err = launch_umma_ws_t<C8P, NP, 3>(s, Wu, N, bias, relu, oscale, out, status, st);
    else if (umma::GeomWs<C8P, NP, 2>::smem() <= lim)
        *err = launch_umma_ws_t<C8P, NP, 2>(s, Wu, N, bias, relu, oscale, out, status, st);
    else
        return false;
    return true;
}

// Paired taps for sources of at most 8 channels (MH3D_UMMA_PAIR=0: off).
bool umma_pair()
{
    const char* e = std::getenv("MH3D_UMMA_PAIR");
    return !(e && e[0] == '0');
}

// Output rows per tile of the tcgen05 kernel (MH3D_UMMA_ROWS = 1, 2 or 4).
int umma_rows()
{
    const char* e = std::getenv("MH3D_UMMA_ROWS");
    if (e && (e[0] == '1' || e[0] == '2' || e[0] == '4')) return e[0] - '0';
    return 2;
}

// One halo buffer and accumulator per CTA, several CTAs per SM (the
// default), or two per CTA with the next tile staged during this tile's
// MMAs (MH3D_UMMA_NB=2, where it fits).  Measured at 128x128x64 (network
// forward, channels (8, 16, 32)): 0.576 ms with one, 0.847 ms with two
// (half the resident CTAs).
template <int C8P, int NP, class OutT>
cudaError_t launch_umma_nb(const ConvSrc& s, const UmmaW& u, int N, const float* bias, int relu, const float* oscale,
                           OutT* out, int* status, cudaStream_t st)
{
    if (umma_ws()) {
        cudaError_t err = cudaSuccess;
        if (launch_umma_ws<C8P, NP>(s, u.w, N, bias, relu, oscale, out, status, st, &err)) return err;
    }
    const char* e = std::getenv("MH3D_UMMA_NB");
    const bool two = e && e[0] == '2';
    if (two && umma::Geom<C8P, NP, 2>::smem() <= (size_t)smem_optin())
        return launch_umma_t<C8P, NP, 2, 1>(s, u.w, N, bias, relu, oscale, out, status, st);
    const int R = umma_rows();
    const __nv_bfloat16* wp = umma_pair() ? u.wp : nullptr;
    if (R == 4 && umma::Geom<C8P, NP, 1, 4>::smem() <= (size_t)smem_optin())
        return launch_umma_t<C8P, NP, 1, 4>(s, u.w, N, bias, relu, oscale, out, status, st, wp);
    if (R >= 2 && umma::Geom<C8P, NP, 1, 2>::smem() <= (size_t)smem_optin())
        return launch_umma_t<C8P, NP, 1, 2>(s, u.w, N, bias, relu, oscale, out, status, st, wp);
    return launch_umma_t<C8P, NP, 1, 1>(s, u.w, N, bias, relu, oscale, out, status, st, wp);
}

template <int C8P, class OutT>
cudaError_t launch_umma_np(const ConvSrc& s, const UmmaW& u, int N, const float* bias, int relu, const float* oscale,
                           OutT* out, int* status, cudaStream_t st)
{
    if (u.np == 16) return launch_umma_nb<C8P, 16>(s, u, N, bias, relu, oscale, out, status, st);
    if (u.np == 32) return launch_umma_nb<C8P, 32>(s, u, N, bias, relu, oscale, out, status, st);
    return launch_umma_nb<C8P, 64>(s, u, N, bias, relu, oscale, out, status, st);
}

// Whether the tcgen05 kernel runs this convolution (its operands prepared,
// the source of a form it stages, not switched off).
bool umma_takes(const ConvSrc& s, const UmmaW* u, int N)
{
    return u && u->w && umma_enabled() && umma_prefers(s) && u->c8p == umma_c8p(s.C, s.f32 != nullptr) &&
           u->np == umma_np(N) && u->np > 0 && !(s.b && s.up);
}

template <class OutT>
cudaError_t launch_umma(const ConvSrc& s, const UmmaW& u, int N, const float* bias, int relu, const float* oscale,
                        OutT* out, int* status, cudaStream_t st)
{
    if (u.c8p == 2) return launch_umma_np<2>(s, u, N, bias, relu, oscale, out, status, st);
    return launch_umma_np<4>(s, u, N, bias, relu, oscale, out, status, st);
}

// Builds the tcgen05 operand of a convolution from its implicit-GEMM
// matrix Wt [Kpad][Npad] (source channels Cs, N outputs); allocates u.w
// unless given.
cudaError_t prep_umma(const __nv_bfloat16* Wt, int Npad, int Cs, bool f32, int N, UmmaW& u, cudaStream_t st)
{
    u.c8p = umma_c8p(Cs, f32);
    u.np = umma_np(N);
    if (!u.c8p || !u.np || !u.w) return cudaSuccess;
    const int total = 27 * u.c8p * u.np * 8;
    umma::k_prep_umma<<<blocks_for(total, 256), 256, 0, st>>>(Wt, Npad, Cs, N, u.c8p, u.np, u.w);
    if (u.wp) {
        const int tp = 9 * 2 * 2 * u.np * 8;
        umma::k_prep_umma_pair<<<blocks_for(tp, 256), 256, 0, st>>>(Wt, Npad, Cs, N, u.np, u.sgn, u.wp);
    }
    return cudaGetLastError();
}
size_t umma_elems(int Cs, bool f32, int N)
{
    const int c = umma_c8p(Cs, f32), np = umma_np(N);
    return (c && np) ? (size_t)27 * c * np * 8 : 0;
}
// The paired-tap layout, for sources of at most 8 channels (one chunk).
size_t umma_pair_elems(int Cs, bool f32, int N)
{
    const int np = umma_np(N);
    return (umma_c8p(Cs, f32) && np && (f32 || Cs <= 8)) ? (size_t)9 * 2 * 2 * np * 8 : 0;
}

// ---- split K for the gather kernel ------------------------------------------

// Splits of the K loop that bring a gather launch of few CTAs (the coarse
// levels: a few thousand voxels, up to 128 channels) to about two per SM,
// each split at least two K steps; 1 when the launch fills the GPU.
// Measured at 128x128x64, channels (16, 32, 64, 128): the 128 -> 128
// bottleneck convolution (2048 voxels, 32 CTAs) took 215 us unsplit.
int splitk_parts(long long V, int Npad, int bn, int Kpad)
{
    const long long ctas = (long long)blocks_for(V, kBM) * (Npad / bn);
    const long long want = 2LL * num_sms();
    if (ctas >= want) return 1;
    const int steps = Kpad / kBK;
    const int S = (int)std::min<long long>((want + ctas - 1) / ctas, std::max(1, steps / 2));
    const int kl = (steps + S - 1) / S;   // K steps per split
    return (steps + kl - 1) / kl;
}
size_t splitk_floats(long long V, int Npad, int N, int Kpad)
{
    const int S = splitk_parts(V, Npad, tile_n(N), Kpad);
    return S > 1 ? (size_t)S * V * N : 0;
}

template <class OutT>
cudaError_t launch_conv(const ConvSrc& s, const __nv_bfloat16* Wt, int Kpad, int Npad, int N, const float* bias,
                        int relu, OutT* out, cudaStream_t st, const float* oscale = nullptr,
                        const UmmaW* uw = nullptr, int* status = nullptr, const SplitWS* ws = nullptr)
{
    cudaError_t e = cudaSuccess;
    if (umma_takes(s, uw, N)) return launch_umma(s, *uw, N, bias, relu, oscale, out, status, st);
    bool done = false;
    if (!tiles_disabled()) {
        if (s.C == 1)
            done = tile_conv_n<1>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, &e);
        else if (s.C == 8 && !s.f32)
            done = tile_conv_n<8>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, &e);
        else if (s.C == 16 && !s.f32)
            done = tile_conv_n<16>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, &e);
        else if (s.C == 32 && !s.f32)
            done = tile_conv_n<32>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, &e);
        else if (s.C == 64 && !s.f32)
            done = tile_conv_n<64>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, st, &e);
    }
    if (done) return e;
    const long long V = (long long)s.D * s.H * s.W;
    const int bn = tile_n(N);
    int S = ws ? splitk_parts(V, Npad, bn, Kpad) : 1;
    if (S > 1 && (size_t)S * V * N > ws->cap) S = 1;
    const int steps = Kpad / kBK, kl = (steps + S - 1) / S * kBK;
    float* part = S > 1 ? ws->p : nullptr;
    dim3 grid(blocks_for(V, kBM), (unsigned)(Npad / bn), (unsigned)S);
    if (bn == 16)
        k_conv<16, OutT><<<grid, kThreads, 0, st>>>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, kl, part);
    else if (bn == 32)
        k_conv<32, OutT><<<grid, kThreads, 0, st>>>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, kl, part);
    else
        k_conv<64, OutT><<<grid, kThreads, 0, st>>>(s, Wt, Kpad, Npad, N, bias, relu, oscale, out, kl, part);
    if (part)
        k_splitk_finish<OutT><<<blocks_for(V * N, 256), 256, 0, st>>>(part, S, V * N, N, bias, relu, oscale, out);
    return cudaGetLastError();
}

size_t wpart_floats(long long V, int Kpad, int N) { return (size_t)blocks_for(V, kWChunk) * Kpad * N; }

// gW [N][27 C] and gb [N] of a convolution with input s and output gradient
// g ([V][N] bfloat16), through the partial buffers.
cudaError_t launch_wgrad(const ConvSrc& s, const __nv_bfloat16* g, int N, float* wpart, float* bpart, float* gW,
                         float* gbias, cudaStream_t st)
{
    const long long V = (long long)s.D * s.H * s.W;
    const int Kpad = round_up(27 * s.C, kBK);
    const unsigned chunks = blocks_for(V, kWChunk);
    const int bn = tile_n(N);
    dim3 grid(blocks_for(Kpad, kBM), chunks, (unsigned)((N + bn - 1) / bn));
    if (bn == 16)
        k_conv_wgrad<16><<<grid, kThreads, 0, st>>>(s, g, N, Kpad, wpart);
    else if (bn == 32)
        k_conv_wgrad<32><<<grid, kThreads, 0, st>>>(s, g, N, Kpad, wpart);
    else
        k_conv_wgrad<64><<<grid, kThreads, 0, st>>>(s, g, N, Kpad, wpart);
    const int Kvalid = 27 * s.C;
    k_wgrad_reduce<<<blocks_for((long long)Kvalid * N, 256), 256, 0, st>>>(wpart, (int)chunks, Kpad, Kvalid, N, gW);
    k_bias_part<<<chunks, kThreads, 0, st>>>(g, V, N, bpart);
    k_bias_reduce<<<blocks_for(N, 64), 64, 0, st>>>(bpart, (int)chunks, N, gbias);
    return cudaGetLastError();
}

}  // namespace
}  // namespace unet
}  // namespace mh3d

namespace mh3d {
namespace unet {
namespace {

#define UN_CK(n, call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (n).err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
            return e_ == cudaErrorMemoryAllocation ? MH3D_ERR_OOM : MH3D_ERR_CUDA;                \
        }                                                                                         \
    } while (0)

mh3d_status prep_weights(Net& n, cudaStream_t st)
{
    for (int i = 0; i < n.nlayers; ++i) {
        Layer& l = n.L[i];
        k_prep_weights<<<blocks_for((long long)l.Kf * l.Nf, 256), 256, 0, st>>>(n.theta + l.woff, l.cin, l.cout,
                                                                                l.Kf, l.Nf, 0, l.Wf);
        k_prep_weights<<<blocks_for((long long)l.Kb * l.Nb, 256), 256, 0, st>>>(n.theta + l.woff, l.cin, l.cout,
                                                                                l.Kb, l.Nb, 1, l.Wb);
        const bool f32in = &l == &n.L[0];   // the network input: one FP32 channel
        UN_CK(n, prep_umma(l.Wf, l.Nf, l.cin, f32in, l.cout, l.uf, st));
        UN_CK(n, prep_umma(l.Wb, l.Nb, l.cout, false, l.cin, l.ub, st));
    }
    UN_CK(n, cudaGetLastError());
    n.weights_ready = true;
    return MH3D_OK;
}

template <class OutT>
cudaError_t fwd(const Net& n, int li, const ConvSrc& s, int relu, OutT* out, cudaStream_t st,
                const float* oscale = nullptr)
{
    const Layer& l = n.L[li];
    return launch_conv(s, l.Wf, l.Kf, l.Nf, l.cout, n.theta + l.boff, relu, out, st, oscale, &l.uf, n.status,
                       &n.skws);
}

// Layer indices: encoder level l: 2 l (a), 2 l + 1 (b); decoder level l
// (levels - 2 .. 0): 2 levels + 2 (levels - 2 - l) (a, on up(d[l + 1])) and
// the next (b, on u[l] + e[l]); the output convolution last.
inline int dec_layer(const Net& n, int l) { return 2 * n.levels + 2 * (n.levels - 2 - l); }

ConvSrc src_at(const Net& n, const __nv_bfloat16* a, int l, int C, const __nv_bfloat16* skip = nullptr, int up = 0)
{
    return src_of(a, n.dims[l][0], n.dims[l][1], n.dims[l][2], C, skip, up);
}

// iscale / oscale: device scalars multiplying the input and the output
// (null: 1).
mh3d_status forward_pass(Net& n, const float* in, cudaStream_t st, const float* iscale = nullptr,
                         const float* oscale = nullptr)
{
    const int Lv = n.levels;
    ConvSrc s0;
    s0.f32 = in;
    s0.D = n.D;
    s0.H = n.H;
    s0.W = n.W;
    s0.C = 1;
    s0.f32_scale = iscale;
    n.in = in;
    n.iscale = iscale;
    for (int l = 0; l < Lv; ++l) {
        const ConvSrc x = l == 0 ? s0 : src_at(n, n.p[l - 1], l, n.ch[l - 1]);
        UN_CK(n, fwd(n, 2 * l, x, 1, n.ea[l], st));
        UN_CK(n, fwd(n, 2 * l + 1, src_at(n, n.ea[l], l, n.ch[l]), 1, n.e[l], st));
        if (l + 1 < Lv)
            k_pool<<<blocks_for(n.V[l + 1] * n.ch[l], 256), 256, 0, st>>>(n.e[l], n.dims[l][0], n.dims[l][1],
                                                                          n.dims[l][2], n.ch[l], n.p[l]);
    }
    for (int l = Lv - 2; l >= 0; --l) {
        const __nv_bfloat16* below = l + 1 == Lv - 1 ? n.e[l + 1] : n.d[l + 1];
        const int li = dec_layer(n, l);
        UN_CK(n, fwd(n, li, src_at(n, below, l, n.ch[l + 1], nullptr, 1), 1, n.u[l], st));
        UN_CK(n, fwd(n, li + 1, src_at(n, n.u[l], l, n.ch[l], n.e[l]), 1, n.d[l], st));
    }
    UN_CK(n, fwd(n, n.nlayers - 1, src_at(n, n.d[0], 0, n.ch[0]), 0, n.out, st, oscale));
    return MH3D_OK;
}

// Backward through layer li: g is the gradient w.r.t. the layer's output
// (before the ReLU mask when y != null: masked into the scratch buffer);
// parameter gradients go to n.grad; the input gradient, when gin != null,
// is written at the convolution's resolution.
mh3d_status back_layer(Net& n, int li, const ConvSrc& s, const __nv_bfloat16* g, const __nv_bfloat16* y,
                       __nv_bfloat16* gin, cudaStream_t st)
{
    const Layer& l = n.L[li];
    const long long V = (long long)s.D * s.H * s.W;
    if (y) {
        k_relu_grad<<<blocks_for(V * l.cout, 256), 256, 0, st>>>(n.scratch, g, y, V * l.cout);
        g = n.scratch;
    }
    UN_CK(n, launch_wgrad(s, g, l.cout, n.wpart, n.bpart, n.grad + l.woff, n.grad + l.boff, st));
    if (gin) {
        ConvSrc sg = src_of(g, s.D, s.H, s.W, l.cout);
        sg.flip = 1;
        UN_CK(n, launch_conv(sg, l.Wb, l.Kb, l.Nb, l.cin, (const float*)nullptr, 0, gin, st, nullptr, &l.ub,
                             n.status, &n.skws));
    }
    return MH3D_OK;
}

mh3d_status backward_pass(Net& n, cudaStream_t st)
{
    const int Lv = n.levels;
    mh3d_status s;
#define UN_BACK(...)                                             \
    if ((s = back_layer(n, __VA_ARGS__, st)) != MH3D_OK) return s
    // output convolution: gradient w.r.t. d[0]
    UN_BACK(n.nlayers - 1, src_at(n, n.d[0], 0, n.ch[0]), n.gout, nullptr, n.gd[0]);
    for (int l = 0; l + 1 < Lv; ++l) {   // decoder, top to bottom
        const int li = dec_layer(n, l);
        const __nv_bfloat16* below = l + 1 == Lv - 1 ? n.e[l + 1] : n.d[l + 1];
        UN_BACK(li + 1, src_at(n, n.u[l], l, n.ch[l], n.e[l]), n.gd[l], n.d[l], n.gs[l]);
        UN_BACK(li, src_at(n, below, l, n.ch[l + 1], nullptr, 1), n.gs[l], n.u[l], n.gup[l]);
        const int* dn = n.dims[l + 1];
        k_up_grad<<<blocks_for(n.V[l + 1] * n.ch[l + 1], 256), 256, 0, st>>>(n.gup[l], dn[0], dn[1], dn[2],
                                                                              n.ch[l + 1], n.gd[l + 1]);
    }
    ConvSrc s0;
    s0.f32 = n.in;
    s0.f32_scale = n.iscale;
    s0.D = n.D;
    s0.H = n.H;
    s0.W = n.W;
    s0.C = 1;
    for (int l = Lv - 1; l >= 0; --l) {   // encoder, bottom to top
        const __nv_bfloat16* ge = l == Lv - 1 ? n.gd[l] : n.ge[l];   // the bottleneck's e is its d
        UN_BACK(2 * l + 1, src_at(n, n.ea[l], l, n.ch[l]), ge, n.e[l], n.gea[l]);
        const ConvSrc x = l == 0 ? s0 : src_at(n, n.p[l - 1], l, n.ch[l - 1]);
        UN_BACK(2 * l, x, n.gea[l], n.ea[l], l == 0 ? nullptr : n.gp[l - 1]);
        if (l > 0) {
            const int* dm = n.dims[l - 1];
            k_pool_grad_add<<<blocks_for(n.V[l - 1] * n.ch[l - 1], 256), 256, 0, st>>>(
                n.gs[l - 1], n.gp[l - 1], dm[0], dm[1], dm[2], n.ch[l - 1], n.ge[l - 1]);
        }
    }
#undef UN_BACK
    UN_CK(n, cudaGetLastError());
    return MH3D_OK;
}

constexpr int kScaleBlocks = 304;   // partial sums of the RMS (2 per SM)

// (cin, cout) of layer i of a network with channels ch[0 .. levels - 1].
void layer_io(int levels, const int* ch, int i, int* cin, int* cout)
{
    if (i < 2 * levels) {   // encoder
        const int l = i / 2;
        *cin = i % 2 == 0 ? (l == 0 ? 1 : ch[l - 1]) : ch[l];
        *cout = ch[l];
    } else if (i < 4 * levels - 2) {   // decoder level l = levels - 2 - (i - 2 levels) / 2
        const int l = levels - 2 - (i - 2 * levels) / 2;
        *cin = (i - 2 * levels) % 2 == 0 ? ch[l + 1] : ch[l];
        *cout = ch[l];
    } else {
        *cin = ch[0];
        *cout = 1;
    }
}

}  // namespace
}  // namespace unet
}  // namespace mh3d

using mh3d::unet::Net;
struct mh3d_unet_s : public Net {};

extern "C" {

long long mh3d_unet_param_count_levels(int levels, const int* channels)
{
    if (levels < 2 || levels > mh3d::unet::kMaxLevels || !channels) return -1;
    long long n = 0;
    for (int i = 0; i < 4 * levels - 1; ++i) {
        int ci = 0, co = 0;
        mh3d::unet::layer_io(levels, channels, i, &ci, &co);
        n += (long long)co * 27 * ci + co;
    }
    return n;
}

long long mh3d_unet_param_count(int c0, int c1, int c2)
{
    const int ch[3] = {c0, c1, c2};
    return mh3d_unet_param_count_levels(3, ch);
}

mh3d_status mh3d_unet_create_levels(int nx, int ny, int nz, int levels, const int* channels, mh3d_unet* out)
{
    using namespace mh3d::unet;
    if (!out) return MH3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (levels < 2 || levels > kMaxLevels || !channels) return MH3D_ERR_INVALID_ARG;
    const int q = 1 << (levels - 1);   // every level's grid halves the previous one
    if (nx < q || ny < q || nz < q || nx % q || ny % q || nz % q) return MH3D_ERR_INVALID_ARG;
    for (int l = 0; l < levels; ++l)
        if (channels[l] < 1 || channels[l] > kMaxChannels) return MH3D_ERR_INVALID_ARG;
    mh3d_unet n = new mh3d_unet_s();
    n->W = nx;
    n->H = ny;
    n->D = nz;
    n->levels = levels;
    n->nlayers = 4 * levels - 1;
    for (int l = 0; l < levels; ++l) {
        n->ch[l] = channels[l];
        n->dims[l][0] = nz >> l;
        n->dims[l][1] = ny >> l;
        n->dims[l][2] = nx >> l;
        n->V[l] = (long long)n->dims[l][0] * n->dims[l][1] * n->dims[l][2];
    }
    long long off = 0;
    size_t wp = 0, bp = 0, skn = 0;
    int cm = 1;
    for (int i = 0; i < n->nlayers; ++i) {
        Layer& l = n->L[i];
        layer_io(levels, channels, i, &l.cin, &l.cout);
        // the level the layer's output lives at
        const int lv = i < 2 * levels ? i / 2 : (i < 4 * levels - 2 ? levels - 2 - (i - 2 * levels) / 2 : 0);
        l.woff = off;
        off += (long long)l.cout * 27 * l.cin;
        l.boff = off;
        off += l.cout;
        l.Kf = round_up(27 * l.cin, kBK);
        l.Nf = round_up(l.cout, tile_n(l.cout));
        l.Kb = round_up(27 * l.cout, kBK);
        l.Nb = round_up(l.cin, tile_n(l.cin));
        wp = std::max(wp, wpart_floats(n->V[lv], l.Kf, l.cout));
        skn = std::max(skn, std::max(splitk_floats(n->V[lv], l.Nf, l.cout, l.Kf),
                                     splitk_floats(n->V[lv], l.Nb, l.cin, l.Kb)));
        bp = std::max(bp, (size_t)blocks_for(n->V[lv], kWChunk) * l.cout);
        cm = std::max(cm, std::max(l.cin, l.cout));
    }
    n->nparam = off;
    n->wpart_n = wp;
    n->bpart_n = bp;
    n->lblocks = (int)blocks_for(n->V[0], kThreads);
    bool ok = true;
    auto A = [&](auto** p, size_t count) { ok = ok && dalloc(*n, p, count) == cudaSuccess; };
    A(&n->theta, off);
    A(&n->grad, off);
    A(&n->am, off);
    A(&n->av, off);
    for (int i = 0; i < n->nlayers; ++i) {
        Layer& l = n->L[i];
        A(&l.Wf, (size_t)l.Kf * l.Nf);
        A(&l.Wb, (size_t)l.Kb * l.Nb);
        const size_t ef = umma_elems(l.cin, i == 0, l.cout), eb = umma_elems(l.cout, false, l.cin);
        if (ef) A(&l.uf.w, ef);
        if (eb) A(&l.ub.w, eb);
        const size_t pf = umma_pair_elems(l.cin, i == 0, l.cout), pb = umma_pair_elems(l.cout, false, l.cin);
        if (pf) A(&l.uf.wp, pf);
        if (pb) A(&l.ub.wp, pb);
        l.ub.sgn = -1;
    }
    A(&n->status, 1);
    if (ok && cudaMemset(n->status, 0, sizeof(int)) != cudaSuccess) ok = false;
    size_t smax = 0;   // the largest level volume x channels (the mask scratch)
    for (int l = 0; l < levels; ++l) {
        const size_t Vl = n->V[l], c = n->ch[l];
        A(&n->ea[l], Vl * c);
        A(&n->e[l], Vl * c);
        A(&n->gd[l], Vl * c);
        A(&n->ge[l], Vl * c);
        A(&n->gea[l], Vl * c);
        smax = std::max(smax, Vl * c);
        if (l + 1 < levels) {
            const size_t cn = n->ch[l + 1];
            A(&n->p[l], n->V[l + 1] * c);
            A(&n->gp[l], n->V[l + 1] * c);
            A(&n->u[l], Vl * c);
            A(&n->d[l], Vl * c);
            A(&n->gs[l], Vl * c);
            A(&n->gup[l], Vl * cn);
        }
    }
    A(&n->out, n->V[0]);
    A(&n->gout, n->V[0]);
    A(&n->scratch, std::max(smax, (size_t)n->V[0] * cm));
    A(&n->wpart, wp);
    A(&n->bpart, bp);
    if (skn) {
        A(&n->skws.p, skn);
        n->skws.cap = skn;
    }
    A(&n->lpart, (size_t)n->lblocks);
    A(&n->spart, (size_t)kScaleBlocks);
    A(&n->scales, 4);
    if (ok && cudaMallocHost(&n->lhost, sizeof(double) * n->lblocks) != cudaSuccess) {
        n->lhost = nullptr;
        ok = false;
    }
    if (!ok) {
        cudaGetLastError();
        free_net(*n);
        delete n;
        return MH3D_ERR_OOM;
    }
    *out = n;
    return MH3D_OK;
}

mh3d_status mh3d_unet_create(int nx, int ny, int nz, int c0, int c1, int c2, mh3d_unet* out)
{
    using namespace mh3d::unet;
    if (!out) return MH3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (c0 > 64 || c1 > 64 || c2 > 64) return MH3D_ERR_INVALID_ARG;
    const int ch[3] = {c0, c1, c2};
    return mh3d_unet_create_levels(nx, ny, nz, 3, ch, out);
}

mh3d_status mh3d_unet_destroy(mh3d_unet n)
{
    if (!n) return MH3D_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    mh3d::unet::free_net(*n);
    delete n;
    return MH3D_OK;
}

mh3d_status mh3d_unet_set_params(mh3d_unet n, const float* theta, void* stream)
{
    if (!n || !theta) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    UN_CK(*n, cudaMemcpyAsync(n->theta, theta, sizeof(float) * n->nparam, cudaMemcpyDeviceToDevice, st));
    UN_CK(*n, cudaMemsetAsync(n->am, 0, sizeof(float) * n->nparam, st));
    UN_CK(*n, cudaMemsetAsync(n->av, 0, sizeof(float) * n->nparam, st));
    n->adam_t = 0;
    return mh3d::unet::prep_weights(*n, st);
}

mh3d_status mh3d_unet_get_params(mh3d_unet n, float* theta, void* stream)
{
    if (!n || !theta) return MH3D_ERR_INVALID_ARG;
    UN_CK(*n, cudaMemcpyAsync(theta, n->theta, sizeof(float) * n->nparam, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
    return MH3D_OK;
}

mh3d_status mh3d_unet_forward(mh3d_unet n, const float* in, float* out, void* stream)
{
    if (!n || !in || !out) return MH3D_ERR_INVALID_ARG;
    if (!n->weights_ready) {
        n->err = "parameters not set";
        return MH3D_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    mh3d_status s = mh3d::unet::forward_pass(*n, in, st);
    if (s != MH3D_OK) return s;
    UN_CK(*n, cudaMemcpyAsync(out, n->out, sizeof(float) * n->V[0], cudaMemcpyDeviceToDevice, st));
    return MH3D_OK;
}

static mh3d_status loss_grad_impl(mh3d_unet n, const float* in, const float* target, float* grad, double* loss,
                                  const float* iscale, const float* tscale, cudaStream_t st)
{
    using namespace mh3d::unet;
    mh3d_status s = forward_pass(*n, in, st, iscale, nullptr);
    if (s != MH3D_OK) return s;
    k_mse<<<n->lblocks, kThreads, 0, st>>>(n->out, target, tscale, n->V[0], n->gout, n->lpart);
    if ((s = backward_pass(*n, st)) != MH3D_OK) return s;
    if (grad) UN_CK(*n, cudaMemcpyAsync(grad, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToDevice, st));
    if (loss) {
        UN_CK(*n, cudaMemcpyAsync(n->lhost, n->lpart, sizeof(double) * n->lblocks, cudaMemcpyDeviceToHost, st));
        UN_CK(*n, cudaStreamSynchronize(st));
        double L = 0.0;
        for (int i = 0; i < n->lblocks; ++i) L += n->lhost[i];
        *loss = L;
        int dst = 0;   // a bounded wait of the tcgen05 convolutions that ran out
        UN_CK(*n, cudaMemcpy(&dst, n->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (dst != 0) {
            n->err = "tensor-core convolution: bounded wait expired";
            return MH3D_ERR_TIMEOUT;
        }
    }
    return MH3D_OK;
}

static bool ready(mh3d_unet n)
{
    if (n->weights_ready) return true;
    n->err = "parameters not set";
    return false;
}

static void launch_scales(mh3d_unet n, const float* in, float gain, cudaStream_t st)
{
    using namespace mh3d::unet;
    k_sumsq_part<<<kScaleBlocks, kThreads, 0, st>>>(in, n->V[0], n->spart);
    k_scales<<<1, 32, 0, st>>>(n->spart, kScaleBlocks, n->V[0], gain, n->scales);
}

mh3d_status mh3d_unet_loss_grad(mh3d_unet n, const float* in, const float* target, float* grad, double* loss,
                                void* stream)
{
    if (!n || !in || !target) return MH3D_ERR_INVALID_ARG;
    if (!ready(n)) return MH3D_ERR_INVALID_ARG;
    return loss_grad_impl(n, in, target, grad, loss, nullptr, nullptr, (cudaStream_t)stream);
}

mh3d_status mh3d_unet_forward_scaled(mh3d_unet n, const float* in, float gain, float* out, void* stream)
{
    if (!n || !in || !out || !(gain > 0.f)) return MH3D_ERR_INVALID_ARG;
    if (!ready(n)) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    launch_scales(n, in, gain, st);
    mh3d_status s = mh3d::unet::forward_pass(*n, in, st, n->scales, n->scales + 1);
    if (s != MH3D_OK) return s;
    UN_CK(*n, cudaMemcpyAsync(out, n->out, sizeof(float) * n->V[0], cudaMemcpyDeviceToDevice, st));
    return MH3D_OK;
}

mh3d_status mh3d_unet_loss_grad_scaled(mh3d_unet n, const float* in, const float* target, float gain, float* grad,
                                       double* loss, void* stream)
{
    if (!n || !in || !target || !(gain > 0.f)) return MH3D_ERR_INVALID_ARG;
    if (!ready(n)) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    launch_scales(n, in, gain, st);
    return loss_grad_impl(n, in, target, grad, loss, n->scales, n->scales + 2, st);
}

mh3d_status mh3d_unet_adam_step(mh3d_unet n, float lr, void* stream)
{
    using namespace mh3d::unet;
    if (!n || !(lr > 0.f)) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    n->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow(0.9, n->adam_t), c2 = 1.f - (float)std::pow(0.999, n->adam_t);
    k_adam<<<blocks_for(n->nparam, 256), 256, 0, st>>>(n->theta, n->am, n->av, n->grad, n->nparam, lr, b1, b2, 1e-8f,
                                                       c1, c2);
    UN_CK(*n, cudaGetLastError());
    return prep_weights(*n, st);
}

const char* mh3d_unet_last_error(mh3d_unet n) { return n ? n->err.c_str() : ""; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Single-layer primitives (temporaries allocated per call)
// ---------------------------------------------------------------------------
namespace {

using namespace mh3d::unet;

bool desc_ok(const mh3d_unet_conv_desc* c)
{
    if (!c || c->nx < 1 || c->ny < 1 || c->nz < 1 || c->cin < 1 || c->cout < 1 || c->cin > 64 || c->cout > 64)
        return false;
    if (c->up && (c->nx % 2 || c->ny % 2 || c->nz % 2)) return false;
    if (c->src_f32) return c->cin == 1 && !c->up && !c->skip_bf16;
    return c->src_bf16 != nullptr;
}

ConvSrc src_from(const mh3d_unet_conv_desc* c)
{
    ConvSrc s;
    s.a = (const __nv_bfloat16*)c->src_bf16;
    s.b = (const __nv_bfloat16*)c->skip_bf16;
    s.f32 = c->src_f32;
    s.D = c->nz;
    s.H = c->ny;
    s.W = c->nx;
    s.C = c->cin;
    s.up = c->up;
    return s;
}

// RAII device buffer for the primitives.
struct Tmp {
    void* p = nullptr;
    explicit Tmp(size_t bytes) { if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr; }
    ~Tmp() { if (p) cudaFree(p); }
};

// Synchronises; with a device status word, reports a bounded wait that
// ran out (MH3D_ERR_TIMEOUT).
mh3d_status finish(cudaStream_t st, const int* status = nullptr)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return MH3D_ERR_CUDA;
    if (status) {
        int h = 0;
        if (cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MH3D_ERR_CUDA;
        if (h != 0) return MH3D_ERR_TIMEOUT;
    }
    return MH3D_OK;
}

}  // namespace

extern "C" {

mh3d_status mh3d_unet_conv_forward(const mh3d_unet_conv_desc* c, const float* W, const float* b, int relu,
                                   float* out, void* stream)
{
    if (!desc_ok(c) || !W || !out) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = round_up(27 * c->cin, kBK), Np = round_up(c->cout, tile_n(c->cout));
    Tmp wt(sizeof(__nv_bfloat16) * K * Np);
    if (!wt.p) return MH3D_ERR_OOM;
    k_prep_weights<<<blocks_for((long long)K * Np, 256), 256, 0, st>>>(W, c->cin, c->cout, K, Np, 0,
                                                                       (__nv_bfloat16*)wt.p);
    const ConvSrc s = src_from(c);
    const size_t ue = umma_elems(s.C, s.f32 != nullptr, c->cout);
    Tmp uw(sizeof(__nv_bfloat16) * std::max<size_t>(ue, 1)), stat(sizeof(int));
    if (!uw.p || !stat.p) return MH3D_ERR_OOM;
    const size_t pe = umma_pair_elems(s.C, s.f32 != nullptr, c->cout);
    Tmp pw(sizeof(__nv_bfloat16) * std::max<size_t>(pe, 1));
    if (!pw.p) return MH3D_ERR_OOM;
    UmmaW u;
    u.w = ue ? (__nv_bfloat16*)uw.p : nullptr;
    u.wp = pe ? (__nv_bfloat16*)pw.p : nullptr;
    if (prep_umma((const __nv_bfloat16*)wt.p, Np, s.C, s.f32 != nullptr, c->cout, u, st) != cudaSuccess ||
        cudaMemsetAsync(stat.p, 0, sizeof(int), st) != cudaSuccess)
        return MH3D_ERR_CUDA;
    if (launch_conv(s, (const __nv_bfloat16*)wt.p, K, Np, c->cout, b, relu, out, st, nullptr, &u, (int*)stat.p) !=
        cudaSuccess)
        return MH3D_ERR_CUDA;
    return finish(st, (int*)stat.p);
}

mh3d_status mh3d_unet_conv_input_grad(const mh3d_unet_conv_desc* c, const void* g, const float* W, float* gin,
                                      void* stream)
{
    if (!c || !g || !W || !gin || c->nx < 1 || c->ny < 1 || c->nz < 1 || c->cin < 1 || c->cout < 1 ||
        c->cin > 64 || c->cout > 64)
        return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = round_up(27 * c->cout, kBK), Np = round_up(c->cin, tile_n(c->cin));
    Tmp wt(sizeof(__nv_bfloat16) * K * Np);
    if (!wt.p) return MH3D_ERR_OOM;
    k_prep_weights<<<blocks_for((long long)K * Np, 256), 256, 0, st>>>(W, c->cin, c->cout, K, Np, 1,
                                                                       (__nv_bfloat16*)wt.p);
    ConvSrc s;
    s.a = (const __nv_bfloat16*)g;
    s.D = c->nz;
    s.H = c->ny;
    s.W = c->nx;
    s.C = c->cout;
    s.flip = 1;
    const size_t ue = umma_elems(s.C, false, c->cin);
    Tmp uw(sizeof(__nv_bfloat16) * std::max<size_t>(ue, 1)), stat(sizeof(int));
    if (!uw.p || !stat.p) return MH3D_ERR_OOM;
    const size_t pe = umma_pair_elems(s.C, false, c->cin);
    Tmp pw(sizeof(__nv_bfloat16) * std::max<size_t>(pe, 1));
    if (!pw.p) return MH3D_ERR_OOM;
    UmmaW u;
    u.w = ue ? (__nv_bfloat16*)uw.p : nullptr;
    u.wp = pe ? (__nv_bfloat16*)pw.p : nullptr;
    u.sgn = -1;
    if (prep_umma((const __nv_bfloat16*)wt.p, Np, s.C, false, c->cin, u, st) != cudaSuccess ||
        cudaMemsetAsync(stat.p, 0, sizeof(int), st) != cudaSuccess)
        return MH3D_ERR_CUDA;
    if (launch_conv(s, (const __nv_bfloat16*)wt.p, K, Np, c->cin, (const float*)nullptr, 0, gin, st, nullptr, &u,
                    (int*)stat.p) != cudaSuccess)
        return MH3D_ERR_CUDA;
    return finish(st, (int*)stat.p);
}

mh3d_status mh3d_unet_conv_weight_grad(const mh3d_unet_conv_desc* c, const void* g, float* gW, float* gb,
                                       void* stream)
{
    if (!desc_ok(c) || !g || !gW || !gb) return MH3D_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long V = (long long)c->nx * c->ny * c->nz;
    const int K = round_up(27 * c->cin, kBK);
    Tmp wp(sizeof(float) * wpart_floats(V, K, c->cout));
    Tmp bp(sizeof(float) * (size_t)blocks_for(V, kWChunk) * c->cout);
    if (!wp.p || !bp.p) return MH3D_ERR_OOM;
    if (launch_wgrad(src_from(c), (const __nv_bfloat16*)g, c->cout, (float*)wp.p, (float*)bp.p, gW, gb, st) !=
        cudaSuccess)
        return MH3D_ERR_CUDA;
    return finish(st);
}

}  // extern "C"
