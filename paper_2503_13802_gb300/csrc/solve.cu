// Regularised least-squares solvers of Sec. 4.3 on the GPU.
//
// CG on the normal equations (A^T A + lambda R) rho = A^T d runs entirely on
// the device: FP32 vectors, FP64 inner products (per-thread float pairs,
// FP64 across threads and CTAs, fixed summation order so every CTA derives
// the same scalars), step lengths computed where they are consumed, and a
// device-side stopping rule.  The iteration loop is one CUDA graph: a
// conditional WHILE node whose body holds two iterations (even and odd
// parity; partial-sum buffers are double-buffered by parity so no kernel
// reads a value that it also writes).  The first kernel of an iteration sets
// the graph condition to 0 when the loop is finished.
//
// The paper's own solver, accelerated projected gradient with rho >= 0
// (Sec. 4.3), runs the same normal operator with a fixed iteration count.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "solve_internal.h"

namespace mh3d {

int update_blocks(long long N)
{
    const long long b = (N + 1023) / 1024;
    return (int)std::max(1LL, std::min(b, 4LL * 152));
}

// Reduction memory (doubles): per-CTA partial arrays [RR | PQ | BN | RES],
// each red_cap long, then the scalars [RR0, RR1, PQ, BN, RES] written by the
// last CTA of each producer, then four ticket counters (unsigned int).
enum { kPartRR = 0, kPartPQ = 1, kPartBN = 2, kPartRES = 3, kNPart = 4 };
enum { kRR0 = 0, kRR1 = 1, kPQ = 2, kBN = 3, kRES = 4, kDL0 = 5, kDL1 = 6, kAL0 = 7, kAL1 = 8, kNScal = 9 };
enum { kTkRR = 0, kTkPQ = 1, kTkBN = 2, kTkRES = 3, kNTk = 4 };
// device flags: [0] loop decided, [1] iterations, [2] status, [3] timeout
// status, [4] warm start rejected
constexpr int kNFlags = 8;
static double* part_slot(const Plan& P, int s) { return P.w.red + (size_t)s * P.w.red_cap; }
static double* scal(const Plan& P, int s) { return P.w.red + (size_t)kNPart * P.w.red_cap + s; }
static unsigned int* ticket(const Plan& P, int s)
{
    return reinterpret_cast<unsigned int*>(P.w.red + (size_t)kNPart * P.w.red_cap + 16) + s;
}
static size_t red_bytes(size_t cap) { return sizeof(double) * (cap * kNPart + 16) + sizeof(unsigned int) * 8; }

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// r = rhs - q (q may be null: zero start), x = 0 on a zero start; the
// search direction starts as p = r (classic CG) or p = qd = 0 (single-
// reduction CG, whose first update forms p = r); totals r^T r, rhs^T rhs.
__global__ void __launch_bounds__(256) k_cg_init(const float* __restrict__ rhs, const float* __restrict__ q,
                                                 float* __restrict__ r, float* __restrict__ p, float* __restrict__ qd,
                                                 float* __restrict__ x, int zero_x, long long N, double* rr_part,
                                                 unsigned int* rr_tk, double* rr_out, double* bn_part,
                                                 unsigned int* bn_tk, double* bn_out)
{
    __shared__ double red[34];
    DotAcc ar, ab;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float b = rhs[i];
        const float rv = q ? b - q[i] : b;
        r[i] = rv;
        if (qd) {
            p[i] = 0.f;
            qd[i] = 0.f;
        } else {
            p[i] = rv;
        }
        if (zero_x) x[i] = 0.f;
        ar.add(rv, rv);
        ab.add(b, b);
    }
    float2 t, t2;
    block_pair_acc2(ar, &ab, reinterpret_cast<float*>(red), &t, &t2);
    grid_sum_finalize(t, rr_part, blockIdx.x, gridDim.x, rr_tk, rr_out);
    __syncthreads();   // every thread has read the first ticket's flag before thread 0 reuses it
    grid_sum_finalize(t2, bn_part, blockIdx.x, gridDim.x, bn_tk, bn_out);
}

// Warm-start fallback: if r0^T r0 >= rhs^T rhs the initial iterate is no
// better than zero, so restart from it: x = 0, r = rhs, the search state as
// k_cg_init leaves it for a zero start, r^T r = rhs^T rhs.  Every block
// reads the same two totals, so all take the same decision.
__global__ void __launch_bounds__(256) k_cg_fallback(const float* __restrict__ rhs, float* __restrict__ r,
                                                     float* __restrict__ p, float* __restrict__ qd,
                                                     float* __restrict__ x, long long N, double* rr, const double* bn,
                                                     int* flags)
{
    const double b = *bn;
    if (!(*rr >= b)) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float v = rhs[i];
        r[i] = v;
        x[i] = 0.f;
        if (qd) {
            p[i] = 0.f;
            qd[i] = 0.f;
        } else {
            p[i] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *rr = b;
        flags[4] = 1;
    }
}

// alpha = gamma / delta; x += alpha p; r -= alpha q; partials of r^T r.
__global__ void __launch_bounds__(256) k_cg_update(float* __restrict__ x, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   long long N, const CgCtl c, const double* pq, double* rr_part,
                                                   unsigned int* rr_tk, double* rr_out)
{
    __shared__ double red[34];
    if (*(volatile int*)&c.flags[0]) return;
    const bool lead = threadIdx.x == 0 && blockIdx.x == 0;
    const double g = __ldcg(c.rr_new);
    const double dl = __ldcg(pq);
    // every thread takes alpha: an FP64 quotient rounded to FP32, or (c.fp64
    // off) an FP32 division of the split significands
    const float a = c.fp64 ? (float)(g / dl) : ddiv_to_float(g, dl);
    const unsigned long long db = (unsigned long long)__double_as_longlong(dl);
    const bool dl_pos = (db >> 63) == 0 && (db << 1) != 0ull && !((db << 1) > 0xffe0000000000000ull);   // dl > 0
    if (!isfinite(a) || !dl_pos) {
        if (lead) {
            c.flags[2] = MH3D_ERR_NONFINITE;
            __threadfence();
            c.flags[0] = 1;
            if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
        }
        return;
    }
    DotAcc acc;
    // float4 body (vector buffers are 256-byte aligned), scalar tail
    const long long N4 = N >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N4; i += stride) {
        const float4 pv = reinterpret_cast<const float4*>(p)[i];
        const float4 qv = reinterpret_cast<const float4*>(q)[i];
        float4 xv = reinterpret_cast<float4*>(x)[i];
        float4 rv = reinterpret_cast<float4*>(r)[i];
        xv.x = fmaf(a, pv.x, xv.x); xv.y = fmaf(a, pv.y, xv.y); xv.z = fmaf(a, pv.z, xv.z); xv.w = fmaf(a, pv.w, xv.w);
        rv.x = fmaf(-a, qv.x, rv.x); rv.y = fmaf(-a, qv.y, rv.y); rv.z = fmaf(-a, qv.z, rv.z); rv.w = fmaf(-a, qv.w, rv.w);
        reinterpret_cast<float4*>(x)[i] = xv;
        reinterpret_cast<float4*>(r)[i] = rv;
        acc.add(rv.x, rv.x);
        acc.add(rv.y, rv.y);
        acc.add(rv.z, rv.z);
        acc.add(rv.w, rv.w);
    }
    for (long long i = 4 * N4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        x[i] = fmaf(a, p[i], x[i]);
        const float rv = fmaf(-a, q[i], r[i]);
        r[i] = rv;
        acc.add(rv, rv);
    }
    grid_sum_finalize(block_pair_acc(acc, red), rr_part, blockIdx.x, gridDim.x, rr_tk, rr_out);
    if (lead) {
        const int it = c.flags[1] + 1;
        c.flags[1] = it;
        // Hard bound: the first kernel of the next iteration stops the loop at
        // max_iter; this guard ends the graph loop even if that kernel never
        // ran.  It does not set the done flag (other CTAs of this kernel may
        // not have started yet); the host reports the missing decision.
        if (it > c.max_iter + 1) {
            c.flags[2] = MH3D_ERR_NOT_CONVERGED;
            if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
        }
    }
}

// Partials of ||a - b||^2.
__global__ void __launch_bounds__(256) k_diff_norm2(const float* __restrict__ a, const float* __restrict__ b,
                                                    long long N, double* part, unsigned int* tk, double* out)
{
    __shared__ double red[34];
    DotAcc acc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float d = a[i] - (b ? b[i] : 0.f);
        acc.add(d, d);
    }
    grid_sum_finalize(block_pair_acc(acc, red), part, blockIdx.x, gridDim.x, tk, out);
}

// Partials of a^T b (float-pair accumulation, as every solver dot product).
__global__ void __launch_bounds__(256) k_dot(const float* __restrict__ a, const float* __restrict__ b, long long N,
                                             double* part, unsigned int* tk, double* out)
{
    __shared__ double red[34];
    DotAcc acc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        acc.add(a[i], b[i]);
    grid_sum_finalize(block_pair_acc(acc, red), part, blockIdx.x, gridDim.x, tk, out);
}

// A fixed, index-hashed start vector in [-1, 1) for the power iteration
// (never orthogonal to a given eigenvector in practice, unlike A^T d, which
// vanishes for zero data).
__global__ void __launch_bounds__(256) k_fill_hash(float* __restrict__ v, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i + 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        v[i] = (float)((double)(z >> 40) * (1.0 / 8388608.0) - 1.0);
    }
}

// APG step (Sec. 4.3): given y and g = N y - rhs,
// x_prev <- x; x <- max(y - tau g, 0); y_next = x + mom (x - x_prev).
__global__ void __launch_bounds__(256) k_apg_step(float* __restrict__ x, float* __restrict__ xprev,
                                                  float* __restrict__ y, const float* __restrict__ ny,
                                                  const float* __restrict__ rhs, float tau, float mom_next, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float g = ny[i] - rhs[i];
        const float xn = fmaxf(fmaf(-tau, g, y[i]), 0.f);
        const float xo = x[i];
        xprev[i] = xo;
        x[i] = xn;
        y[i] = fmaf(mom_next, xn - xo, xn);
    }
}

__global__ void __launch_bounds__(256) k_scale(float* __restrict__ v, const float* __restrict__ u, float s, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        v[i] = s * u[i];
}

cudaError_t solve_set_attributes() { return cudaSuccess; }

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
mh3d_status solve_alloc(Plan& P)
{
    SolveWork& w = P.w;
    const size_t N = (size_t)P.N;
    const size_t vec = (N + 63) & ~size_t(63);
    // partial-sum slots for the widest grid any tile choice (8-column T pass) can launch
    const size_t cap = (size_t)std::max({update_blocks(P.N), normal_part_count(P, 0), normal_part_count(P, 1),
                                         tpass_blocks(P.nx, 8, tpass_outer(P, 1)),
                                         xpass_blocks(P.ny * P.nz, 8), 1});
    w.red_cap = cap;
    const size_t bytes = sizeof(float) * vec * 8 + red_bytes(cap) + 64;
    if (dev_malloc(&w.base, bytes) != cudaSuccess) {
        w.base = nullptr;
        P.err = "cudaMalloc of solver workspace failed";
        return MH3D_ERR_OOM;
    }
    float* f = (float*)w.base;
    w.x = f;
    w.r = f + vec;
    w.p = f + 2 * vec;
    w.q = f + 3 * vec;
    w.t1 = f + 4 * vec;
    w.t2 = f + 5 * vec;
    w.rhs = f + 6 * vec;
    w.s = f + 7 * vec;
    w.red = (double*)(f + 8 * vec);
    if (cudaMemset(w.red, 0, red_bytes(cap)) != cudaSuccess) return MH3D_ERR_CUDA;
    if (dev_malloc(&w.flags, kNFlags * sizeof(int)) != cudaSuccess ||
        host_malloc(&w.flags_host, kNFlags * sizeof(int)) != cudaSuccess ||
        host_malloc(&w.red_host, std::max(cap, (size_t)16) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        P.err = "allocation of the solver's flags or pinned scalars failed";
        return MH3D_ERR_OOM;
    }
    P.work_bytes = bytes + kNFlags * sizeof(int);
    return MH3D_OK;
}

void solve_free(Plan& P)
{
    SolveWork& w = P.w;
    if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
    P.graph_exec = nullptr;
    if (P.graph_stream) cudaStreamDestroy(P.graph_stream);
    P.graph_stream = nullptr;
    if (w.base) cudaFree(w.base);
    if (w.portrait) cudaFree(w.portrait);
    if (w.dstage) cudaFree(w.dstage);
    if (w.flags) cudaFree(w.flags);
    if (w.hist) cudaFree(w.hist);
    if (w.flags_host) cudaFreeHost(w.flags_host);
    if (w.red_host) cudaFreeHost(w.red_host);
    w = SolveWork();
}

static mh3d_status ensure_hist(Plan& P, int cap)
{
    if (P.w.hist_cap >= cap) return MH3D_OK;
    if (P.w.hist) cudaFree(P.w.hist);
    P.w.hist = nullptr;
    P.w.hist_cap = 0;
    const int c = std::max(cap, 1024);
    if (dev_malloc(&P.w.hist, sizeof(double) * c) != cudaSuccess) {
        P.err = "cudaMalloc of the residual history failed";
        return MH3D_ERR_OOM;
    }
    P.w.hist_cap = c;
    if (P.graph_exec) {   // the cached graph holds the old pointer
        cudaGraphExecDestroy(P.graph_exec);
        P.graph_exec = nullptr;
    }
    return MH3D_OK;
}

mh3d_status validate_opts(Plan& P, const mh3d_solve_opts& o)
{
    if (o.reg_kind < 0 || o.reg_kind > 1 || !(o.lambda > 0) || !(o.alpha >= 0) || o.shell < 1 || o.solver < 0 ||
        o.solver > 1 || o.max_iter < 1 || o.max_iter > 1000000 || o.normal_mode < 0 || o.normal_mode > 1 ||
        !(o.rel_tol >= 0) || o.cg_variant < 0 || o.cg_variant > 1) {
        P.err = "invalid solve options";
        return MH3D_ERR_INVALID_ARG;
    }
    return MH3D_OK;
}

// ---------------------------------------------------------------------------
// CG loop
// ---------------------------------------------------------------------------
static CgCtl base_ctl(const Plan& P, const mh3d_solve_opts& o)
{
    CgCtl c;
    c.flags = P.w.flags;
    c.bn = scal(P, kBN);
    c.hist = P.w.hist;
    c.hist_cap = P.w.hist_cap;
    c.max_iter = o.max_iter;
    c.tol2 = o.fixed_iters ? 0.0 : o.rel_tol * o.rel_tol;
    c.fp64 = o.fp32_scalar_div ? 0 : 1;
    return c;
}

static cudaError_t enqueue_iteration(Plan& P, const mh3d_solve_opts& o, int par, CgCtl c, cudaStream_t st)
{
    c.rr_new = scal(P, par ? kRR0 : kRR1);
    c.rr_old = scal(P, par ? kRR1 : kRR0);
    const int mode = o.normal_mode;
    SolveWork& w = P.w;
    if (o.cg_variant == 0) {
        // single-reduction CG: the first pass updates p, q, x, r and applies
        // the operator to the new r; the last pass produces s = A r with
        // delta = r^T s and gamma = r^T r (one grid reduction per iteration)
        c.cgcg = 1;
        c.delta = scal(P, par ? kDL0 : kDL1);
        c.alpha_prev = scal(P, par ? kAL0 : kAL1);
        c.alpha_out = scal(P, par ? kAL1 : kAL0);
        LoaderUpdate u;
        u.mode = 2;
        u.p = w.p;
        u.r = w.r;
        u.r_w = w.r;
        u.q = w.q;
        u.s = w.s;
        u.x = w.x;
        RedSink dots;
        dots.part = part_slot(P, kPartPQ);
        dots.ticket = ticket(P, kTkPQ);
        dots.out = scal(P, par ? kDL1 : kDL0);
        dots.part2 = part_slot(P, kPartRR);
        dots.out2 = scal(P, par ? kRR1 : kRR0);
        return launch_normal(P, mode, reg_args(P, o), w.r, w.s, w.t1, w.t2, w.portrait, &dots, &c, &u, st);
    }
    RedSink pq;
    pq.part = part_slot(P, kPartPQ);
    pq.ticket = ticket(P, kTkPQ);
    pq.out = scal(P, kPQ);
    LoaderUpdate u;
    u.mode = 1;
    u.p = w.p;
    u.r = w.r;
    cudaError_t e = launch_normal(P, mode, reg_args(P, o), w.p, w.q, w.t1, w.t2, w.portrait, &pq, &c, &u, st);
    if (e != cudaSuccess) return e;
    const int nU = update_blocks(P.N);
    k_cg_update<<<nU, 256, 0, st>>>(w.x, w.r, w.p, w.q, P.N, c, scal(P, kPQ), part_slot(P, kPartRR),
                                    ticket(P, kTkRR), scal(P, par ? kRR1 : kRR0));
    return cudaGetLastError();
}

static unsigned long long opts_key(const mh3d_solve_opts& o)
{
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    mix(&o.reg_kind, sizeof o.reg_kind);
    mix(&o.lambda, sizeof o.lambda);
    mix(&o.alpha, sizeof o.alpha);
    mix(&o.shell, sizeof o.shell);
    mix(&o.rel_tol, sizeof o.rel_tol);
    mix(&o.max_iter, sizeof o.max_iter);
    mix(&o.fixed_iters, sizeof o.fixed_iters);
    mix(&o.normal_mode, sizeof o.normal_mode);
    mix(&o.cg_variant, sizeof o.cg_variant);
    mix(&o.lambda_relative, sizeof o.lambda_relative);
    mix(&o.x0_fallback, sizeof o.x0_fallback);
    mix(&o.fp32_scalar_div, sizeof o.fp32_scalar_div);
    return h;
}

#define MH3D_CK(P, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (P).err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
            return MH3D_ERR_CUDA;                                                                 \
        }                                                                                         \
    } while (0)

// Adds to graph g, after deps, a conditional WHILE node whose body holds
// two CG iterations of plan P (captured on cap, which must not be
// capturing); the kernels set the condition from the device.
static cudaError_t add_cg_loop_node(Plan& P, const mh3d_solve_opts& o, cudaGraph_t g, const cudaGraphNode_t* deps,
                                    size_t ndeps, cudaStream_t cap, cudaGraphNode_t* node)
{
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    // cudaGraphNodeParams has no default constructor (union members): use
    // zeroed storage, as the runtime expects for unused fields.
    alignas(cudaGraphNodeParams) unsigned char np_storage[sizeof(cudaGraphNodeParams)];
    std::memset(np_storage, 0, sizeof np_storage);
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_storage);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(node, g, deps, nullptr, ndeps, &np);
    if (e != cudaSuccess) return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    CgCtl c = base_ctl(P, o);
    c.cond = h;
    c.use_cond = 1;
    cudaError_t e1 = enqueue_iteration(P, o, 0, c, cap);
    cudaError_t e2 = (e1 == cudaSuccess) ? enqueue_iteration(P, o, 1, c, cap) : e1;
    cudaGraph_t outg = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(cap, &outg);
    return (e2 != cudaSuccess) ? e2 : e3;
}

static mh3d_status build_graph(Plan& P, const mh3d_solve_opts& o)
{
    if (P.graph_exec) {
        cudaGraphExecDestroy(P.graph_exec);
        P.graph_exec = nullptr;
    }
    if (!P.graph_stream) MH3D_CK(P, cudaStreamCreateWithFlags(&P.graph_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    MH3D_CK(P, cudaGraphCreate(&g, 0));
    cudaGraphNode_t node;
    cudaError_t e = add_cg_loop_node(P, o, g, nullptr, 0, P.graph_stream, &node);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P.graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        P.graph_exec = nullptr;
        P.err = std::string("CUDA graph of the CG loop: ") + cudaGetErrorString(e);
        return MH3D_ERR_CUDA;
    }
    P.graph_key = opts_key(o);
    return MH3D_OK;
}

static bool graphs_disabled()
{
    const char* v = std::getenv("MH3D_NO_GRAPH");
    return v && v[0] && v[0] != '0';
}

static mh3d_status run_cg_loop(Plan& P, const mh3d_solve_opts& o, cudaStream_t st)
{
    if (!graphs_disabled()) {
        if (!P.graph_exec || P.graph_key != opts_key(o)) {
            mh3d_status s = build_graph(P, o);
            if (s != MH3D_OK) return s;
        }
        MH3D_CK(P, cudaGraphLaunch(P.graph_exec, st));
        return MH3D_OK;
    }
    // Host-driven loop: kernels exit early once the device flag is set; the
    // host polls the flag every 8 iterations.
    CgCtl c = base_ctl(P, o);
    for (int it = 0; it <= o.max_iter + 2; it += 2) {
        MH3D_CK(P, enqueue_iteration(P, o, 0, c, st));
        MH3D_CK(P, enqueue_iteration(P, o, 1, c, st));
        if ((it / 2) % 4 == 3) {
            MH3D_CK(P, cudaMemcpyAsync(P.w.flags_host, P.w.flags, kNFlags * sizeof(int), cudaMemcpyDeviceToHost, st));
            MH3D_CK(P, cudaStreamSynchronize(st));
            if (P.w.flags_host[0]) break;
        }
    }
    return MH3D_OK;
}


// What a CG solve enqueues before its loop: A^T d, zeroed flags and tickets,
// the initial residual and, for single-reduction CG, s0 = N r0 with its two
// dot products.
static mh3d_status cg_prefix(Plan& P, const float2* d, const mh3d_solve_opts& o, cudaStream_t st)
{
    SolveWork& w = P.w;
    const RegArgs reg = reg_args(P, o);
    const int nU = update_blocks(P.N);
    MH3D_CK(P, launch_adjoint(P, d, w.rhs, w.t1, w.t2, st));
    const float* qinit = nullptr;
    if (o.x0_dev) {
        // a batched warm start stages x0 in w.x before the graph runs
        if (o.x0_dev != w.x)
            MH3D_CK(P, cudaMemcpyAsync(w.x, o.x0_dev, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));
        MH3D_CK(P, launch_normal(P, o.normal_mode, reg, w.x, w.q, w.t1, w.t2, w.portrait, nullptr, nullptr, nullptr,
                                 st));
        qinit = w.q;
    }
    MH3D_CK(P, cudaMemsetAsync(w.flags, 0, kNFlags * sizeof(int), st));
    MH3D_CK(P, cudaMemsetAsync(ticket(P, 0), 0, kNTk * sizeof(unsigned int), st));
    const bool cgcg = (o.cg_variant == 0);
    k_cg_init<<<nU, 256, 0, st>>>(w.rhs, qinit, w.r, w.p, cgcg ? w.q : nullptr, w.x, o.x0_dev ? 0 : 1, P.N,
                                  part_slot(P, kPartRR), ticket(P, kTkRR), scal(P, kRR1), part_slot(P, kPartBN),
                                  ticket(P, kTkBN), scal(P, kBN));
    MH3D_CK(P, cudaGetLastError());
    if (o.x0_dev && o.x0_fallback) {
        k_cg_fallback<<<nU, 256, 0, st>>>(w.rhs, w.r, w.p, cgcg ? w.q : nullptr, w.x, P.N, scal(P, kRR1), scal(P, kBN),
                                          w.flags);
        MH3D_CK(P, cudaGetLastError());
    }
    if (cgcg) {   // s0 = A r0 with delta0 = r0^T s0 and gamma0 = r0^T r0 (parity-1 slots)
        RedSink dots;
        dots.part = part_slot(P, kPartPQ);
        dots.ticket = ticket(P, kTkPQ);
        dots.out = scal(P, kDL1);
        dots.part2 = part_slot(P, kPartRR);
        dots.out2 = scal(P, kRR1);
        MH3D_CK(P, launch_normal(P, o.normal_mode, reg, w.r, w.s, w.t1, w.t2, w.portrait, &dots, nullptr, nullptr,
                                 st));
    }
    return MH3D_OK;
}

// What a CG solve enqueues after its loop: the loop's flags to the host, the
// true residual ||rhs - N x||^2 and the scalars (||rhs||^2 among them).
static mh3d_status cg_suffix(Plan& P, const mh3d_solve_opts& o, cudaStream_t st)
{
    SolveWork& w = P.w;
    const int nU = update_blocks(P.N);
    MH3D_CK(P, cudaMemcpyAsync(w.flags_host, w.flags, kNFlags * sizeof(int), cudaMemcpyDeviceToHost, st));
    MH3D_CK(P, launch_normal(P, o.normal_mode, reg_args(P, o), w.x, w.q, w.t1, w.t2, w.portrait, nullptr, nullptr,
                             nullptr, st));
    k_diff_norm2<<<nU, 256, 0, st>>>(w.rhs, w.q, P.N, part_slot(P, kPartRES), ticket(P, kTkRES), scal(P, kRES));
    MH3D_CK(P, cudaGetLastError());
    MH3D_CK(P, cudaMemcpyAsync(w.red_host, scal(P, 0), kNScal * sizeof(double), cudaMemcpyDeviceToHost, st));
    return MH3D_OK;
}

// ||rhs - N x||^2 and ||rhs||^2 on the host (synchronises).
static mh3d_status true_residual(Plan& P, const mh3d_solve_opts& o, cudaStream_t st, double* res2, double* bn2)
{
    mh3d_status s = cg_suffix(P, o, st);
    if (s != MH3D_OK) return s;
    MH3D_CK(P, cudaStreamSynchronize(st));
    *res2 = P.w.red_host[kRES];
    *bn2 = P.w.red_host[kBN];
    return MH3D_OK;
}

constexpr int kRecSlot = 12;   // host slot of the final recurrence residual (after the scalars)

// Once the suffix's copies have landed: the recurrence residual of the last
// iteration, the image and the residual history.
static mh3d_status cg_tail(Plan& P, const mh3d_solve_opts& o, float* rho, mh3d_solve_info* info, cudaStream_t st)
{
    SolveWork& w = P.w;
    const int iters = w.flags_host[1];
    MH3D_CK(P, cudaMemcpyAsync(&w.red_host[kRecSlot], w.hist + std::min(iters, w.hist_cap - 1), sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    if (rho) MH3D_CK(P, cudaMemcpyAsync(rho, w.x, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));
    if (info && info->history)
        MH3D_CK(P, cudaMemcpyAsync(info->history, w.hist, sizeof(double) * (std::min(iters, o.max_iter) + 1),
                                   cudaMemcpyDeviceToHost, st));
    return MH3D_OK;
}

// Fills info from the host copies; returns the solve's status.
static mh3d_status cg_report(Plan& P, double res2, double bn2, mh3d_solve_info* info)
{
    SolveWork& w = P.w;
    const int status = w.flags_host[2];
    if (info) {
        info->iters = w.flags_host[1];
        info->rel_res_recurrence = w.red_host[kRecSlot];
        info->rel_res_true = bn2 > 0 ? std::sqrt(res2 / bn2) : 0.0;
        info->status = status;
        info->x0_rejected = w.flags_host[4];
        info->tau = 0.0;
    }
    if (w.flags_host[3] == MH3D_ERR_TIMEOUT) {
        P.err = "a bounded device wait (bulk copy) timed out";
        return MH3D_ERR_TIMEOUT;
    }
    if (!w.flags_host[0]) {
        P.err = "CG loop ended without a device decision";
        return MH3D_ERR_TIMEOUT;
    }
    if (status == MH3D_ERR_NOT_CONVERGED) P.err = "max_iter reached before rel_tol";
    if (status == MH3D_ERR_NONFINITE) P.err = "non-finite value in an FP64 reduction";
    return (mh3d_status)status;
}

static mh3d_status cg_solve(Plan& P, const float2* d, const mh3d_solve_opts& o, float* rho, mh3d_solve_info* info,
                            cudaStream_t st)
{
    mh3d_status s = ensure_hist(P, o.max_iter + 1);
    if (s != MH3D_OK) return s;
    if (o.normal_mode == 1 && (s = ensure_portrait(P)) != MH3D_OK) return s;
    if ((s = cg_prefix(P, d, o, st)) != MH3D_OK) return s;
    if ((s = run_cg_loop(P, o, st)) != MH3D_OK) return s;
    if ((s = cg_suffix(P, o, st)) != MH3D_OK) return s;
    MH3D_CK(P, cudaStreamSynchronize(st));
    const double res2 = P.w.red_host[kRES], bn2 = P.w.red_host[kBN];
    if ((s = cg_tail(P, o, rho, info, st)) != MH3D_OK) return s;
    MH3D_CK(P, cudaStreamSynchronize(st));
    return cg_report(P, res2, bn2, info);
}

// ---------------------------------------------------------------------------
// Batched CG: one CUDA graph, one independent branch per volume
// ---------------------------------------------------------------------------
// Each branch is a volume's whole solve: A^T d from the plan's staged
// portraits, the CG set-up, its own conditional WHILE loop driven by its own
// device flags, the true residual and the copies of its flags and scalars to
// pinned host memory.  Branches share nothing, so the GPU runs them
// concurrently and small volumes fill the SMs that one volume leaves idle.
// The graph is cached per (plans, options, plan buffers); portraits and
// images pass through plan-owned buffers, so a call with new pointers reuses
// it.
namespace {

struct BatchGraph {
    std::vector<unsigned long long> serials;
    unsigned long long key = 0;
    cudaGraphExec_t exec = nullptr;
};

std::mutex g_batch_mu;
std::vector<BatchGraph> g_batches;   // most recent last
constexpr size_t kMaxBatchGraphs = 4;

unsigned long long batch_key(const std::vector<Plan*>& ps, const mh3d_solve_opts& o)
{
    unsigned long long h = opts_key(o);
    auto mix = [&](unsigned long long v) {
        for (int i = 0; i < 8; ++i) h = (h ^ ((v >> (8 * i)) & 0xff)) * 1099511628211ull;
    };
    for (const Plan* P : ps) {
        mix(P->serial);
        mix((unsigned long long)(uintptr_t)P->w.hist);
        mix((unsigned long long)(uintptr_t)P->w.portrait);
    }
    return h;
}

}  // namespace

void batch_forget(const Plan& P)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
        const auto& v = g_batches[i].serials;
        if (std::find(v.begin(), v.end(), P.serial) != v.end()) {
            cudaGraphExecDestroy(g_batches[i].exec);
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}

static mh3d_status build_batch_graph(const std::vector<Plan*>& ps, const mh3d_solve_opts& o, bool warm,
                                     cudaGraphExec_t* out)
{
    Plan& P0 = *ps[0];
    cudaStream_t cs = nullptr, cb = nullptr;
    MH3D_CK(P0, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamCreateWithFlags(&cb, cudaStreamNonBlocking);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
    mh3d_status st = MH3D_OK;
    for (size_t v = 0; v < ps.size() && e == cudaSuccess && st == MH3D_OK; ++v) {
        Plan& P = *ps[v];
        e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        P.w.shared_sms = true;   // the volumes' branches share the SMs
        mh3d_solve_opts ov = o;
        ov.x0_dev = warm ? P.w.x : nullptr;   // warm starts are staged in each plan's iterate
        st = cg_prefix(P, P.w.portrait, ov, cs);
        if (st == MH3D_OK) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
            cudaGraphNode_t loop = nullptr;
            if (e == cudaSuccess) {
                std::vector<cudaGraphNode_t> dv(deps, deps + nd);
                e = add_cg_loop_node(P, o, g, dv.data(), dv.size(), cb, &loop);
            }
            if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &loop, nullptr, 1,
                                                                          cudaStreamSetCaptureDependencies);
            if (e == cudaSuccess) st = cg_suffix(P, ov, cs);
        }
        P.w.shared_sms = false;
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        if (e == cudaSuccess) e = e2;
        if (st != MH3D_OK && P0.err.empty()) P0.err = P.err;
    }
    if (e == cudaSuccess && st == MH3D_OK) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cb) cudaStreamDestroy(cb);
    cudaStreamDestroy(cs);
    if (st != MH3D_OK) return st;
    if (e != cudaSuccess) {
        cudaGetLastError();
        P0.err = std::string("CUDA graph of the batched solve: ") + cudaGetErrorString(e);
        return MH3D_ERR_CUDA;
    }
    return MH3D_OK;
}

static mh3d_status batch_graph(const std::vector<Plan*>& ps, const mh3d_solve_opts& o, bool warm,
                               cudaGraphExec_t* exec)
{
    std::vector<unsigned long long> serials;
    for (const Plan* P : ps) serials.push_back(P->serial);
    const unsigned long long key = batch_key(ps, o) ^ (warm ? 0x9e3779b97f4a7c15ull : 0ull);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size(); ++i)
        if (g_batches[i].key == key && g_batches[i].serials == serials) {
            BatchGraph b = g_batches[i];
            g_batches.erase(g_batches.begin() + i);
            g_batches.push_back(b);
            *exec = b.exec;
            return MH3D_OK;
        }
    BatchGraph b;
    b.serials = serials;
    b.key = key;
    mh3d_status s = build_batch_graph(ps, o, warm, &b.exec);
    if (s != MH3D_OK) return s;
    if (g_batches.size() >= kMaxBatchGraphs) {
        cudaGraphExecDestroy(g_batches.front().exec);
        g_batches.erase(g_batches.begin());
    }
    g_batches.push_back(b);
    *exec = b.exec;
    return MH3D_OK;
}

static mh3d_status cg_solve_batched(const std::vector<Plan*>& ps, const float2* const* d, const mh3d_solve_opts& o,
                                    const float* const* x0, float* const* rho, mh3d_solve_info* infos,
                                    cudaStream_t st)
{
    Plan& P0 = *ps[0];
    for (Plan* P : ps) {
        mh3d_status s = ensure_hist(*P, o.max_iter + 1);
        if (s == MH3D_OK) s = ensure_portrait(*P);
        if (s != MH3D_OK) {
            P0.err = P->err;
            return s;
        }
    }
    // stage the portraits (and warm starts) in the plans' own buffers (the
    // graph reads those)
    for (size_t v = 0; v < ps.size(); ++v) {
        MH3D_CK(P0, cudaMemcpyAsync(ps[v]->w.portrait, d[v], sizeof(float2) * (size_t)ps[v]->K * ps[v]->M,
                                    cudaMemcpyDeviceToDevice, st));
        if (x0)
            MH3D_CK(P0, cudaMemcpyAsync(ps[v]->w.x, x0[v], sizeof(float) * (size_t)ps[v]->N,
                                        cudaMemcpyDeviceToDevice, st));
    }
    cudaGraphExec_t exec = nullptr;
    mh3d_status s = batch_graph(ps, o, x0 != nullptr, &exec);
    if (s != MH3D_OK) return s;
    MH3D_CK(P0, cudaGraphLaunch(exec, st));
    MH3D_CK(P0, cudaStreamSynchronize(st));
    std::vector<double> res2(ps.size()), bn2(ps.size());
    for (size_t v = 0; v < ps.size(); ++v) {
        res2[v] = ps[v]->w.red_host[kRES];
        bn2[v] = ps[v]->w.red_host[kBN];
        if ((s = cg_tail(*ps[v], o, rho[v], infos ? &infos[v] : nullptr, st)) != MH3D_OK) {
            P0.err = ps[v]->err;
            return s;
        }
    }
    MH3D_CK(P0, cudaStreamSynchronize(st));
    mh3d_status worst = MH3D_OK;
    for (size_t v = 0; v < ps.size(); ++v) {
        const mh3d_status sv = cg_report(*ps[v], res2[v], bn2[v], infos ? &infos[v] : nullptr);
        if (sv != MH3D_OK && worst == MH3D_OK) {
            worst = sv;
            if (ps[v] != &P0) P0.err = "volume " + std::to_string(v) + ": " + ps[v]->err;
        }
    }
    return worst;
}

// ---------------------------------------------------------------------------
// Autotuning
// ---------------------------------------------------------------------------
// Times, on the plan's own workspace, the launch variants of the three
// operators and keeps the fastest of each, per size class (grid, s, K,
// weighted or not):
//   1. the normal operator (the CG loop's kernels): T-pass tile width (16 or
//      8 columns) x T-pass radix schedule (default or the alternative, where
//      instantiated) x CTAs per y-slab of the cluster pass (2 or 4);
//   2. the adjoint's drive-axis part: warp-centric fused with T_z^T, or then
//      T_z^T, with 1, 2 or 4 warps per row group, or the CTA-level pass;
//   3. the forward's drive-axis part: the cluster pass fusing T_z, or the
//      warp-centric pass with 1, 2 or 4 warps per row group.
// The choice is remembered for the process, and with MH3D_TUNE_CACHE set to
// a file path it is read from and written to that JSON file, so a later
// process takes it without timing.
namespace {
std::mutex g_tune_mu;
std::vector<std::pair<std::string, TileChoice>> g_tuned;
}  // namespace

static void drop_graphs(Plan& P)
{
    if (P.graph_exec) {
        cudaGraphExecDestroy(P.graph_exec);
        P.graph_exec = nullptr;
    }
    batch_forget(P);
}

static std::string tune_key(const Plan& P)
{
    char b[96];
    std::snprintf(b, sizeof b, "%dx%dx%d/s%d/K%d/b%d", P.nx, P.ny, P.nz, P.s, P.K, P.sens ? 1 : 0);
    return b;
}

static std::string tile_json(const TileChoice& t)
{
    char b[256];
    std::snprintf(b, sizeof b,
                  "{\"tpass_cols\": %d, \"tpass_radix\": %d, \"zx_c\": %d, \"adj_path\": %d, \"xw_ks\": %d, "
                  "\"fwd_path\": %d, \"xw_ks_fwd\": %d}",
                  t.tpass_cols, t.tpass_radix, t.zx_c, t.adj_path, t.xw_ks, t.fwd_path, t.xw_ks_fwd);
    return b;
}

// The integer after "name": in obj, or false.
static bool json_int(const std::string& obj, const char* name, int* v)
{
    const std::string k = std::string("\"") + name + "\":";
    const size_t i = obj.find(k);
    return i != std::string::npos && std::sscanf(obj.c_str() + i + k.size(), "%d", v) == 1;
}

// The cache file's entries: one line per key, "<key>": {<choices>}.
static std::vector<std::pair<std::string, TileChoice>> cache_read(const char* path)
{
    std::vector<std::pair<std::string, TileChoice>> out;
    FILE* f = std::fopen(path, "r");
    if (!f) return out;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        const std::string l(line);
        const size_t q0 = l.find('"'), q1 = (q0 == std::string::npos) ? q0 : l.find('"', q0 + 1);
        const size_t b0 = l.find('{', q1 == std::string::npos ? 0 : q1);
        if (q0 == std::string::npos || q1 == std::string::npos || b0 == std::string::npos) continue;
        const std::string key = l.substr(q0 + 1, q1 - q0 - 1), obj = l.substr(b0);
        TileChoice t;
        if (json_int(obj, "tpass_cols", &t.tpass_cols) && json_int(obj, "tpass_radix", &t.tpass_radix) &&
            json_int(obj, "zx_c", &t.zx_c) && json_int(obj, "adj_path", &t.adj_path) &&
            json_int(obj, "xw_ks", &t.xw_ks) && json_int(obj, "fwd_path", &t.fwd_path) &&
            json_int(obj, "xw_ks_fwd", &t.xw_ks_fwd) && (t.tpass_cols == 8 || t.tpass_cols == 16))
            out.push_back({key, t});
    }
    std::fclose(f);
    return out;
}

static void cache_write(const char* path, const std::vector<std::pair<std::string, TileChoice>>& e)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    for (size_t i = 0; i < e.size(); ++i)
        std::fprintf(f, "  \"%s\": %s%s\n", e[i].first.c_str(), tile_json(e[i].second).c_str(),
                     i + 1 < e.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

static void apply_choice(Plan& P, const TileChoice& c)
{
    TileChoice& t = P.tile;
    t.tpass_cols = c.tpass_cols;
    t.tpass_radix = c.tpass_radix;
    t.zx_c = c.zx_c;
    t.adj_path = c.adj_path;
    t.xw_ks = c.xw_ks;
    t.fwd_path = c.fwd_path;
    t.xw_ks_fwd = c.xw_ks_fwd;
    drop_graphs(P);
}

// Mean time (us) of one application of operator `which` (0 normal, 1
// adjoint, 2 forward) over 20 launches after 3 warm-ups.  The normal
// operator runs back to back, as in the CG loop, whose working set stays in
// L2; the adjoint and forward run once per solve on data that is not in L2,
// so with a flush buffer each of their launches is timed alone after the
// buffer has been written (10 launches).
static mh3d_status time_op(Plan& P, int which, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float* flush,
                           size_t flush_n, float* us)
{
    mh3d_solve_opts o{};
    o.lambda = 1e-3;
    o.lambda_relative = 1;
    const RegArgs reg = reg_args(P, o);
    SolveWork& w = P.w;
    auto one = [&]() -> cudaError_t {
        if (which == 0) return launch_normal(P, 0, reg, w.r, w.s, w.t1, w.t2, w.portrait, nullptr, nullptr, nullptr, st);
        if (which == 1) return launch_adjoint(P, w.portrait, w.x, w.t1, w.t2, st);
        return launch_forward(P, w.r, w.portrait, w.t1, w.t2, st);
    };
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = one();
    float total = 0.f;
    int reps = 20;
    if (which != 0 && flush) {
        reps = 10;
        for (int i = 0; i < reps && e == cudaSuccess; ++i) {
            e = cudaMemsetAsync(flush, i & 1, sizeof(float) * flush_n, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = one();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
    } else {
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int i = 0; i < reps && e == cudaSuccess; ++i) e = one();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&total, e0, e1);
    }
    if (e != cudaSuccess) {
        P.err = std::string("autotune: ") + cudaGetErrorString(e);
        return MH3D_ERR_CUDA;
    }
    *us = 1e3f * total / (float)reps;
    return MH3D_OK;
}

static mh3d_status tune_all(Plan& P, cudaStream_t st)
{
    mh3d_status s = ensure_portrait(P);
    if (s != MH3D_OK) return s;
    SolveWork& w = P.w;
    MH3D_CK(P, cudaMemsetAsync(w.r, 0, sizeof(float) * P.N, st));
    MH3D_CK(P, cudaMemsetAsync(w.portrait, 0, sizeof(float2) * (size_t)P.K * P.M, st));
    cudaEvent_t e0, e1;
    MH3D_CK(P, cudaEventCreate(&e0));
    MH3D_CK(P, cudaEventCreate(&e1));
    // a buffer twice the L2 size, written before each timed adjoint and
    // forward launch (freed at the end; without it those are timed warm)
    float* flush = nullptr;
    size_t flush_n = 0;
    {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
            l2 > 0) {
            flush_n = 2 * (size_t)l2 / sizeof(float);
            if (dev_malloc(&flush, sizeof(float) * flush_n) != cudaSuccess) {
                cudaGetLastError();
                flush = nullptr;
                flush_n = 0;
            }
        }
    }
    const TileChoice keep = P.tile;
    TileChoice best = P.tile;
    auto trial = [&](const TileChoice& c, int which, float* us) {
        apply_choice(P, c);
        return time_op(P, which, st, e0, e1, flush, flush_n, us);
    };
    // 1. the normal operator
    const bool alt = (P.ny == 64 || P.ny == 128 || P.nz == 64 || P.nz == 128);
    const bool zx = ct_zxnrm_available(P.nx, P.nz, P.s);
    float bt = 1e30f;
    for (int cols : {16, 8})
        for (int radix = 0; radix <= (alt ? 1 : 0); ++radix)
            for (int zc : {2, 4}) {
                if (!zx && zc == 4) continue;
                TileChoice c = best;
                c.tpass_cols = cols;
                c.tpass_radix = radix;
                c.zx_c = zx ? zc : 0;
                float us = 0.f;
                if ((s = trial(c, 0, &us)) != MH3D_OK) break;
                if (us < bt) {
                    bt = us;
                    best.tpass_cols = cols;
                    best.tpass_radix = radix;
                    best.zx_c = c.zx_c;
                }
            }
    // 2. the adjoint, 3. the forward
    XArgs xa = xpass_args(P);
    const bool warp = s == MH3D_OK && xw_available(xa, false);
    const bool wfused = warp && xzw_available(xa, P.nz);
    if (s == MH3D_OK) {
        std::vector<std::pair<int, int>> cand = {{3, 0}};
        if (warp)
            for (int ks : {1, 2, 4}) {
                if (wfused) cand.push_back({1, ks});
                cand.push_back({2, ks});
            }
        float ba = 1e30f;
        for (const auto& pk : cand) {
            TileChoice c = best;
            c.adj_path = pk.first;
            c.xw_ks = pk.second;
            float us = 0.f;
            if ((s = trial(c, 1, &us)) != MH3D_OK) break;
            if (us < ba) {
                ba = us;
                best.adj_path = pk.first;
                best.xw_ks = pk.second;
            }
        }
    }
    if (s == MH3D_OK) {
        std::vector<std::pair<int, int>> cand = {{1, 0}};
        if (xw_available(xa, true, true))
            for (int ks : {1, 2, 4}) cand.push_back({2, ks});
        float bf = 1e30f;
        for (const auto& pk : cand) {
            TileChoice c = best;
            c.fwd_path = pk.first;
            c.xw_ks_fwd = pk.second;
            float us = 0.f;
            if ((s = trial(c, 2, &us)) != MH3D_OK) break;
            if (us < bf) {
                bf = us;
                best.fwd_path = pk.first;
                best.xw_ks_fwd = pk.second;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) {
        cudaStreamSynchronize(st);
        cudaFree(flush);
    }
    apply_choice(P, s == MH3D_OK ? best : keep);
    return s;
}

static mh3d_status autotune(Plan& P, cudaStream_t st, int* chosen)
{
    const std::string key = tune_key(P);
    const char* path = std::getenv("MH3D_TUNE_CACHE");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& e : g_tuned)
        if (e.first == key) {
            apply_choice(P, e.second);
            *chosen = P.tile.tpass_cols;
            return MH3D_OK;
        }
    if (path && path[0])
        for (const auto& e : cache_read(path))
            if (e.first == key) {
                apply_choice(P, e.second);
                g_tuned.push_back(e);
                *chosen = P.tile.tpass_cols;
                return MH3D_OK;
            }
    mh3d_status s = tune_all(P, st);
    if (s != MH3D_OK) return s;
    g_tuned.push_back({key, P.tile});
    if (path && path[0]) {
        auto all = cache_read(path);
        bool found = false;
        for (auto& e : all)
            if (e.first == key) {
                e.second = P.tile;
                found = true;
            }
        if (!found) all.push_back({key, P.tile});
        cache_write(path, all);
    }
    *chosen = P.tile.tpass_cols;
    return MH3D_OK;
}

// APG (Sec. 4.3): y^k = rho^k + (k-1)/(k+2)(rho^k - rho^{k-1});
// rho^{k+1} = max(y^k - tau M^*(M y^k - b), 0), M^*(M y - b) = N y - A^T d.
static mh3d_status apg_solve(Plan& P, const float2* d, const mh3d_solve_opts& o, float* rho, mh3d_solve_info* info,
                             cudaStream_t st)
{
    SolveWork& w = P.w;
    mh3d_status s;
    if (o.normal_mode == 1 && (s = ensure_portrait(P)) != MH3D_OK) return s;
    const RegArgs reg = reg_args(P, o);
    const int nU = update_blocks(P.N);
    MH3D_CK(P, launch_adjoint(P, d, w.rhs, w.t1, w.t2, st));
    double tau = o.apg_tau;
    if (!(tau > 0)) {
        // tau = 1 / ||M||^2 (Sec. 4.3), ||M||^2 = lambda_max(N), N = A^T A + lambda R
        // with the plan's sensitivity: a power iteration on the device from a
        // fixed hashed vector, v <- N v / ||N v||, with the Rayleigh quotient
        // theta = v^T N v (v a unit vector) in FP64 after every step.  theta
        // rises towards lambda_max; it stops once theta has changed by less
        // than 1e-6 (relative) twice in a row, or after 2000 steps, and takes
        // tau = 0.99 / theta (the margin covers what theta still lacks).
        MH3D_CK(P, cudaMemsetAsync(ticket(P, 0), 0, kNTk * sizeof(unsigned int), st));
        k_fill_hash<<<nU, 256, 0, st>>>(w.p, P.N);
        k_diff_norm2<<<nU, 256, 0, st>>>(w.p, nullptr, P.N, part_slot(P, kPartRES), ticket(P, kTkRES),
                                         scal(P, kRES));
        MH3D_CK(P, cudaMemcpyAsync(w.red_host, scal(P, kRES), sizeof(double), cudaMemcpyDeviceToHost, st));
        MH3D_CK(P, cudaStreamSynchronize(st));
        double nrm = std::sqrt(w.red_host[0]);
        double theta = 0.0, prev = -1.0;
        int calm = 0;
        float* v = w.p;
        float* nv = w.q;
        for (int i = 0; i < 2000 && nrm > 0; ++i) {
            k_scale<<<nU, 256, 0, st>>>(v, v, (float)(1.0 / nrm), P.N);
            MH3D_CK(P, launch_normal(P, o.normal_mode, reg, v, nv, w.t1, w.t2, w.portrait, nullptr, nullptr,
                                     nullptr, st));
            k_dot<<<nU, 256, 0, st>>>(v, nv, P.N, part_slot(P, kPartRES), ticket(P, kTkRES), scal(P, kRES));
            k_diff_norm2<<<nU, 256, 0, st>>>(nv, nullptr, P.N, part_slot(P, kPartPQ), ticket(P, kTkPQ),
                                             scal(P, kPQ));
            MH3D_CK(P, cudaGetLastError());
            MH3D_CK(P, cudaMemcpyAsync(w.red_host, scal(P, 0), kNScal * sizeof(double), cudaMemcpyDeviceToHost, st));
            MH3D_CK(P, cudaStreamSynchronize(st));
            theta = w.red_host[kRES];
            nrm = std::sqrt(w.red_host[kPQ]);
            std::swap(v, nv);
            if (!std::isfinite(theta) || !std::isfinite(nrm)) break;
            calm = (std::fabs(theta - prev) < 1e-6 * std::fabs(theta)) ? calm + 1 : 0;
            prev = theta;
            if (calm >= 2) break;
        }
        if (!(theta > 0) || !std::isfinite(theta)) {
            P.err = "APG step: the power iteration for ||M||^2 failed (non-finite or zero)";
            return MH3D_ERR_NONFINITE;
        }
        tau = 0.99 / theta;
    }
    // x = x0 or 0, x_prev = x, y = x
    if (o.x0_dev) MH3D_CK(P, cudaMemcpyAsync(w.x, o.x0_dev, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));
    else MH3D_CK(P, cudaMemsetAsync(w.x, 0, sizeof(float) * P.N, st));
    MH3D_CK(P, cudaMemcpyAsync(w.r, w.x, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));   // x_prev
    MH3D_CK(P, cudaMemcpyAsync(w.p, w.x, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));   // y
    for (int k = 1; k <= o.max_iter; ++k) {
        MH3D_CK(P, launch_normal(P, o.normal_mode, reg, w.p, w.q, w.t1, w.t2, w.portrait, nullptr, nullptr, nullptr,
                                 st));
        const float mom_next = (float)k / (float)(k + 3);   // (k' - 1)/(k' + 2) with k' = k + 1
        k_apg_step<<<nU, 256, 0, st>>>(w.x, w.r, w.p, w.q, w.rhs, (float)tau, mom_next, P.N);
        MH3D_CK(P, cudaGetLastError());
    }
    double res2 = 0, bn2 = 0;
    // ||A^T d||^2 for the relative true residual
    k_diff_norm2<<<nU, 256, 0, st>>>(w.rhs, nullptr, P.N, part_slot(P, kPartBN), ticket(P, kTkBN), scal(P, kBN));
    MH3D_CK(P, cudaGetLastError());
    if ((s = true_residual(P, o, st, &res2, &bn2)) != MH3D_OK) return s;
    MH3D_CK(P, cudaMemcpyAsync(rho, w.x, sizeof(float) * P.N, cudaMemcpyDeviceToDevice, st));
    MH3D_CK(P, cudaStreamSynchronize(st));
    if (info) {
        info->iters = o.max_iter;
        info->rel_res_recurrence = 0.0;
        info->rel_res_true = bn2 > 0 ? std::sqrt(res2 / bn2) : 0.0;   // unconstrained gradient norm
        info->status = MH3D_OK;
        info->x0_rejected = 0;
        info->tau = tau;
    }
    return MH3D_OK;
}

// ---------------------------------------------------------------------------
// CG on the general three-component model (Sec. 3.2, Eq. matrixModel; the
// solver of Sec. 4.3 applies to any A): (A^T A + lambda I) x = A^T d with A
// the forward of mh3d_general_forward.  Classic CG (Hestenes-Stiefel) on the
// device: the normal operator goes through the plan's portrait buffer (A p,
// then A^T), the dot products are the solvers' float-pair sums into device
// FP64 scalars, the step lengths are formed from them per CTA (FP64), and a
// one-thread kernel keeps the count, the history and the stopping rule.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_axpy(float* __restrict__ y, const float* __restrict__ x, float a, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], y[i]);
}
// x += a p; r -= a q
__global__ void __launch_bounds__(256) k_cg_xr(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                                               const float* __restrict__ q, float a, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fmaf(a, p[i], x[i]);
        r[i] = fmaf(-a, q[i], r[i]);
    }
}
// p = r + beta p
__global__ void __launch_bounds__(256) k_xpby(float* __restrict__ p, const float* __restrict__ r, float beta,
                                              long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], r[i]);
}
// d = b - a (elementwise), for the residual
__global__ void __launch_bounds__(256) k_sub(float* __restrict__ d, const float* __restrict__ b,
                                             const float* __restrict__ a, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        d[i] = b[i] - a[i];
}

// The general CG's device state: g[kGB..] scalars, then the history.
enum GenCg { kGBn = 0, kGRr = 1, kGPq = 2, kGRn = 3, kGDone = 4, kGIt = 5, kGBad = 6, kGHist = 8 };

// x += alpha p, r -= alpha q with alpha = rr / pq (FP64, once per CTA), unless
// the loop is done or pq is not positive (recorded by k_gcg_step).
__global__ void __launch_bounds__(256) k_gcg_xr(float* __restrict__ x, float* __restrict__ r,
                                                const float* __restrict__ p, const float* __restrict__ q,
                                                const double* __restrict__ g, long long N)
{
    __shared__ float a_s;
    if (threadIdx.x == 0) {
        const double pq = g[kGPq];
        a_s = (g[kGDone] != 0.0 || !(pq > 0.0)) ? 0.f : (float)(g[kGRr] / pq);
    }
    __syncthreads();
    const float a = a_s;
    if (a == 0.f) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fmaf(a, p[i], x[i]);
        r[i] = fmaf(-a, q[i], r[i]);
    }
}

// p = r + beta p with beta = rr_new / rr, unless the loop is done.
__global__ void __launch_bounds__(256) k_gcg_p(float* __restrict__ p, const float* __restrict__ r,
                                               const double* __restrict__ g, long long N)
{
    __shared__ float b_s;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        const double pq = g[kGPq];
        skip = g[kGDone] != 0.0 || !(pq > 0.0);
        b_s = skip ? 0.f : (float)(g[kGRn] / g[kGRr]);
    }
    __syncthreads();
    if (skip) return;
    const float beta = b_s;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(beta, p[i], r[i]);
}

// The step's scalars (one thread): rr = rr_new, the iteration count, the
// history, and the stopping rule (converged, max_iter, or a non-finite or
// non-positive value: recorded in kGBad).
__global__ void k_gcg_step(double* __restrict__ g, double tol2, int max_iter)
{
    if (g[kGDone] != 0.0) return;
    const double pq = g[kGPq], rn = g[kGRn], bn = g[kGBn];
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rn)) {
        g[kGBad] = 1.0;
        g[kGDone] = 1.0;
        return;
    }
    const int it = (int)g[kGIt] + 1;
    g[kGRr] = rn;
    g[kGIt] = (double)it;
    g[kGHist + it] = bn > 0.0 ? sqrt(rn / bn) : 0.0;
    if (rn == 0.0 || (tol2 > 0.0 && rn <= tol2 * bn) || it >= max_iter) g[kGDone] = 1.0;
}

// The loop's initial state from bn and rr in g (one thread).
__global__ void k_gcg_init(double* __restrict__ g, double tol2, int max_iter)
{
    const double bn = g[kGBn], rr = g[kGRr];
    g[kGIt] = 0.0;
    g[kGBad] = (isfinite(bn) && isfinite(rr)) ? 0.0 : 1.0;
    g[kGHist] = bn > 0.0 ? sqrt(rr / bn) : 0.0;
    g[kGDone] = (g[kGBad] != 0.0 || rr == 0.0 || bn == 0.0 || (tol2 > 0.0 && rr <= tol2 * bn) || max_iter <= 0)
                    ? 1.0 : 0.0;
}

// a^T b on the device into *out (no host synchronisation).
static cudaError_t dot_dev(Plan& P, const float* a, const float* b, double* out, cudaStream_t st)
{
    const int nb = (int)std::min<long long>(update_blocks(P.N), (long long)P.w.red_cap);
    k_dot<<<nb, 256, 0, st>>>(a, b, P.N, part_slot(P, kPartRES), ticket(P, kTkRES), out);
    return cudaGetLastError();
}

// a^T b on the device, returned to the host (synchronises `st`).
static mh3d_status dot_host(Plan& P, const float* a, const float* b, cudaStream_t st, double* out)
{
    const int nb = (int)std::min<long long>(update_blocks(P.N), (long long)P.w.red_cap);
    k_dot<<<nb, 256, 0, st>>>(a, b, P.N, part_slot(P, kPartRES), ticket(P, kTkRES), scal(P, kRES));
    MH3D_CK(P, cudaGetLastError());
    MH3D_CK(P, cudaMemcpyAsync(P.w.red_host, scal(P, kRES), sizeof(double), cudaMemcpyDeviceToHost, st));
    MH3D_CK(P, cudaStreamSynchronize(st));
    *out = P.w.red_host[0];
    return MH3D_OK;
}

}  // namespace mh3d

using namespace mh3d;

struct mh3d_plan_s : public Plan {};

namespace mh3d {

// q = (A^T A + lambda I) p for the general model.
static mh3d_status general_normal(Plan& P, const float* p, const float* bvec, double lam, float* q, cudaStream_t st)
{
    mh3d_plan h = static_cast<mh3d_plan>(&P);
    mh3d_status s = mh3d_general_forward(h, p, bvec, P.w.portrait, st);
    if (s == MH3D_OK) s = mh3d_general_adjoint(h, P.w.portrait, bvec, q, st);
    if (s != MH3D_OK) return s;
    k_axpy<<<update_blocks(P.N), 256, 0, st>>>(q, p, (float)lam, P.N);
    MH3D_CK(P, cudaGetLastError());
    return MH3D_OK;
}

static mh3d_status general_cg(Plan& P, const void* d, const float* bvec, const mh3d_solve_opts& o, float* rho,
                              mh3d_solve_info* info, cudaStream_t st)
{
    SolveWork& w = P.w;
    mh3d_status s = ensure_portrait(P);
    if (s != MH3D_OK) return s;
    const int nU = update_blocks(P.N);
    const size_t vb = sizeof(float) * (size_t)P.N;
    mh3d_plan h = static_cast<mh3d_plan>(&P);
    MH3D_CK(P, cudaMemsetAsync(ticket(P, 0), 0, kNTk * sizeof(unsigned int), st));
    if ((s = mh3d_general_adjoint(h, d, bvec, w.rhs, st)) != MH3D_OK) return s;
    if (o.x0_dev) {
        MH3D_CK(P, cudaMemcpyAsync(w.x, o.x0_dev, vb, cudaMemcpyDeviceToDevice, st));
        if ((s = general_normal(P, w.x, bvec, o.lambda, w.q, st)) != MH3D_OK) return s;
        k_sub<<<nU, 256, 0, st>>>(w.r, w.rhs, w.q, P.N);
        MH3D_CK(P, cudaGetLastError());
    } else {
        MH3D_CK(P, cudaMemsetAsync(w.x, 0, vb, st));
        MH3D_CK(P, cudaMemcpyAsync(w.r, w.rhs, vb, cudaMemcpyDeviceToDevice, st));
    }
    MH3D_CK(P, cudaMemcpyAsync(w.p, w.r, vb, cudaMemcpyDeviceToDevice, st));
    // the scalars and the history live on the device; the host looks at the
    // done flag every kChunk iterations (kernels of iterations launched after
    // the stop return at once, so x and the count are exact)
    const size_t need = (size_t)kGHist + (size_t)std::max(o.max_iter, 0) + 1;
    if (P.gen_cg_cap < need) {
        if (P.gen_cg) cudaFree(P.gen_cg);
        P.gen_cg = nullptr;
        P.gen_cg_cap = 0;
        MH3D_CK(P, dev_malloc(&P.gen_cg, sizeof(double) * need));
        P.gen_cg_cap = need;
    }
    double* g = P.gen_cg;
    const double tol2 = o.fixed_iters ? 0.0 : o.rel_tol * o.rel_tol;
    MH3D_CK(P, dot_dev(P, w.rhs, w.rhs, g + kGBn, st));
    MH3D_CK(P, dot_dev(P, w.r, w.r, g + kGRr, st));
    k_gcg_init<<<1, 1, 0, st>>>(g, tol2, o.max_iter);
    MH3D_CK(P, cudaGetLastError());
    constexpr int kChunk = 8;
    int launched = 0;
    while (launched < o.max_iter) {
        MH3D_CK(P, cudaMemcpyAsync(P.w.red_host, g + kGDone, sizeof(double), cudaMemcpyDeviceToHost, st));
        MH3D_CK(P, cudaStreamSynchronize(st));
        if (P.w.red_host[0] != 0.0) break;
        for (int c = 0; c < kChunk && launched < o.max_iter; ++c, ++launched) {
            if ((s = general_normal(P, w.p, bvec, o.lambda, w.q, st)) != MH3D_OK) return s;
            MH3D_CK(P, dot_dev(P, w.p, w.q, g + kGPq, st));
            k_gcg_xr<<<nU, 256, 0, st>>>(w.x, w.r, w.p, w.q, g, P.N);
            MH3D_CK(P, cudaGetLastError());
            MH3D_CK(P, dot_dev(P, w.r, w.r, g + kGRn, st));
            k_gcg_p<<<nU, 256, 0, st>>>(w.p, w.r, g, P.N);
            k_gcg_step<<<1, 1, 0, st>>>(g, tol2, o.max_iter);
            MH3D_CK(P, cudaGetLastError());
        }
    }
    std::vector<double> gh(need);
    MH3D_CK(P, cudaMemcpyAsync(gh.data(), g, sizeof(double) * need, cudaMemcpyDeviceToHost, st));
    MH3D_CK(P, cudaStreamSynchronize(st));
    const double bn = gh[kGBn], rr = gh[kGRr];
    const int it = (int)gh[kGIt];
    std::vector<double> hist(gh.begin() + kGHist, gh.begin() + kGHist + it + 1);
    mh3d_status status = MH3D_OK;
    if (gh[kGBad] != 0.0 || !std::isfinite(rr) || !std::isfinite(bn))
        status = MH3D_ERR_NONFINITE;
    else if (tol2 > 0.0 && rr > tol2 * bn && bn > 0.0 && rr > 0.0)
        status = MH3D_ERR_NOT_CONVERGED;
    // true residual ||A^T d - (A^T A + lambda I) x|| / ||A^T d||
    if ((s = general_normal(P, w.x, bvec, o.lambda, w.q, st)) != MH3D_OK) return s;
    k_sub<<<nU, 256, 0, st>>>(w.q, w.rhs, w.q, P.N);
    MH3D_CK(P, cudaGetLastError());
    double res2 = 0.0;
    if ((s = dot_host(P, w.q, w.q, st, &res2)) != MH3D_OK) return s;
    MH3D_CK(P, cudaMemcpyAsync(rho, w.x, vb, cudaMemcpyDeviceToDevice, st));
    MH3D_CK(P, cudaStreamSynchronize(st));
    if (info) {
        info->iters = it;
        info->rel_res_recurrence = hist.back();
        info->rel_res_true = bn > 0 ? std::sqrt(res2 / bn) : 0.0;
        info->status = status;
        info->x0_rejected = 0;
        info->tau = 0.0;
        if (info->history)
            for (size_t i = 0; i < hist.size() && (int)i <= o.max_iter; ++i) info->history[i] = hist[i];
    }
    if (status == MH3D_ERR_NOT_CONVERGED) P.err = "max_iter reached before rel_tol";
    if (status == MH3D_ERR_NONFINITE) P.err = "non-finite value in a reduction of the general-model CG";
    return status;
}

}  // namespace mh3d

extern "C" {

mh3d_status mh3d_solve(mh3d_plan P, const void* d, const mh3d_solve_opts* o, float* rho, mh3d_solve_info* info,
                       void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d || !o || !rho) {
        P->err = "mh3d_solve: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    mh3d_status v = validate_opts(*P, *o);
    if (v != MH3D_OK) return v;
    P->err.clear();
    if (P->padded) {
        // the field of view's portraits zero-padded into the portrait buffer
        // (read once, by A^T d, before the explicit normal operator reuses
        // it); the masked explicit normal operator throughout
        mh3d_status s = ensure_portrait(*P);
        if (s != MH3D_OK) return s;
        MH3D_CK(*P, pad_portraits(*P, (const float2*)d, P->w.portrait, (cudaStream_t)stream));
        mh3d_solve_opts op = *o;
        op.normal_mode = 1;
        if (o->solver == 1) return apg_solve(*P, P->w.portrait, op, rho, info, (cudaStream_t)stream);
        return cg_solve(*P, P->w.portrait, op, rho, info, (cudaStream_t)stream);
    }
    if (o->solver == 1) return apg_solve(*P, (const float2*)d, *o, rho, info, (cudaStream_t)stream);
    return cg_solve(*P, (const float2*)d, *o, rho, info, (cudaStream_t)stream);
}

mh3d_status mh3d_general_solve(mh3d_plan P, const void* d, const float* bvec, const mh3d_solve_opts* o, float* rho,
                               mh3d_solve_info* info, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d || !o || !rho) {
        P->err = "mh3d_general_solve: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    if (!(o->lambda > 0) || !std::isfinite(o->lambda) || o->lambda_relative || o->solver != 0 || o->reg_kind != 0 ||
        o->max_iter < 1 || o->max_iter > 1000000 || !(o->rel_tol >= 0)) {
        P->err = "mh3d_general_solve: needs CG (solver 0), R = I (reg_kind 0), an absolute lambda > 0, "
                 "1 <= max_iter <= 1e6 and rel_tol >= 0";
        return MH3D_ERR_INVALID_ARG;
    }
    if (!P->gen_H) {
        P->err = "mh3d_general_solve: no PSF spectra (call mh3d_general_set_psf)";
        return MH3D_ERR_INVALID_ARG;
    }
    P->err.clear();
    return general_cg(*P, d, bvec, *o, rho, info, (cudaStream_t)stream);
}

mh3d_status mh3d_dot(mh3d_plan P, const float* a, const float* b, long long n, double* result, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!result || n < 0 || (n > 0 && (!a || !b))) {
        P->err = "mh3d_dot: null pointer or negative length";
        return MH3D_ERR_INVALID_ARG;
    }
    if (n == 0) {
        *result = 0.0;
        return MH3D_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)std::min<long long>(update_blocks(std::max(n, 1LL)), (long long)P->w.red_cap);
    MH3D_CK(*P, cudaMemsetAsync(ticket(*P, kTkRES), 0, sizeof(unsigned int), st));
    k_dot<<<nb, 256, 0, st>>>(a, b, n, part_slot(*P, kPartRES), ticket(*P, kTkRES), scal(*P, kRES));
    MH3D_CK(*P, cudaGetLastError());
    MH3D_CK(*P, cudaMemcpyAsync(P->w.red_host, scal(*P, kRES), sizeof(double), cudaMemcpyDeviceToHost, st));
    MH3D_CK(*P, cudaStreamSynchronize(st));
    *result = P->w.red_host[0];
    return MH3D_OK;
}

mh3d_status mh3d_plan_tuning(mh3d_plan P, char* buf, int buflen)
{
    if (!P || !buf || buflen < 1) return MH3D_ERR_INVALID_ARG;
    const std::string j = tile_json(P->tile);
    if ((int)j.size() + 1 > buflen) {
        P->err = "mh3d_plan_tuning: buffer too small";
        return MH3D_ERR_INVALID_ARG;
    }
    std::memcpy(buf, j.c_str(), j.size() + 1);
    return MH3D_OK;
}

mh3d_status mh3d_plan_autotune(mh3d_plan P, void* stream, int* tpass_cols)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    int c = 0;
    mh3d_status s = autotune(*P, (cudaStream_t)stream, &c);
    if (s == MH3D_OK && tpass_cols) *tpass_cols = c;
    return s;
}

mh3d_status mh3d_solve_host(mh3d_plan P, const void* d_host, const mh3d_solve_opts* o, float* rho_host,
                            mh3d_solve_info* info, void* stream)
{
    if (!P) return MH3D_ERR_INVALID_ARG;
    if (!d_host || !o || !rho_host) {
        P->err = "mh3d_solve_host: null pointer";
        return MH3D_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // device staging: the portrait buffer (allocated on demand) and the rhs slot
    mh3d_status s = ensure_portrait(*P);
    if (s != MH3D_OK) return s;
    // a padded plan stages the field of view's portraits in their own buffer
    // (the solve pads them into the portrait buffer)
    float2* stage = P->w.portrait;
    if (P->padded) {
        if (!P->w.dstage) {
            const size_t b = sizeof(float2) * (size_t)P->K * P->Mf;
            if (dev_malloc(&P->w.dstage, b) != cudaSuccess) {
                P->w.dstage = nullptr;
                P->err = "cudaMalloc of the portrait staging buffer failed";
                return MH3D_ERR_OOM;
            }
            P->work_bytes += b;
        }
        stage = P->w.dstage;
    }
    const size_t dbytes = sizeof(float2) * (size_t)P->K * P->Mf;
    MH3D_CK(*P, cudaMemcpyAsync(stage, d_host, dbytes, cudaMemcpyHostToDevice, st));
    // The staged portraits are read once (A^T d) before the explicit normal
    // mode reuses the buffer as scratch; the image is copied back from the
    // solver's iterate.
    s = mh3d_solve(P, stage, o, P->w.t2, info, stream);
    if (s != MH3D_OK && s != MH3D_ERR_NOT_CONVERGED) return s;
    MH3D_CK(*P, cudaMemcpyAsync(rho_host, P->w.x, sizeof(float) * P->N, cudaMemcpyDeviceToHost, st));
    MH3D_CK(*P, cudaStreamSynchronize(st));
    return s;
}

static mh3d_status solve_batched_impl(const mh3d_plan* plans, int nvol, const void* const* d,
                                      const mh3d_solve_opts* o, const float* const* x0, float* const* rho,
                                      mh3d_solve_info* infos, void* stream)
{
    if (nvol == 0) return MH3D_OK;   // nothing to do; the arrays may be NULL
    if (!plans || nvol < 0 || !d || !o || !rho) return MH3D_ERR_INVALID_ARG;
    std::vector<Plan*> ps(nvol);
    for (int v = 0; v < nvol; ++v) {
        if (!plans[v]) return MH3D_ERR_INVALID_ARG;
        ps[v] = plans[v];
    }
    Plan& P0 = *ps[0];
    P0.err.clear();
    for (int v = 0; v < nvol; ++v) {
        if (!d[v] || !rho[v]) {
            P0.err = "mh3d_solve_batched: null pointer for volume " + std::to_string(v);
            return MH3D_ERR_INVALID_ARG;
        }
        for (int u = 0; u < v; ++u)
            if (ps[u] == ps[v]) {
                P0.err = "mh3d_solve_batched: a plan appears twice (each volume needs its own plan)";
                return MH3D_ERR_INVALID_ARG;
            }
        mh3d_status s = validate_opts(*ps[v], *o);
        if (s != MH3D_OK) return s;
        if (ps[v]->padded) {
            P0.err = "mh3d_solve_batched: volume " + std::to_string(v) + " has a padded plan (solve it with mh3d_solve)";
            return MH3D_ERR_INVALID_ARG;
        }
    }
    if (o->x0_dev) {
        P0.err = "mh3d_solve_batched: opts->x0_dev must be NULL (per-volume warm starts go through "
                 "mh3d_solve_batched_warm)";
        return MH3D_ERR_INVALID_ARG;
    }
    if (x0)
        for (int v = 0; v < nvol; ++v)
            if (!x0[v]) {
                P0.err = "mh3d_solve_batched_warm: null x0 for volume " + std::to_string(v);
                return MH3D_ERR_INVALID_ARG;
            }
    cudaStream_t st = (cudaStream_t)stream;
    if (o->solver == 0 && !graphs_disabled()) {
        std::vector<const float2*> dv(nvol);
        for (int v = 0; v < nvol; ++v) dv[v] = (const float2*)d[v];
        return cg_solve_batched(ps, dv.data(), *o, x0, rho, infos, st);
    }
    // APG, or graphs switched off: one volume after another
    mh3d_status worst = MH3D_OK;
    for (int v = 0; v < nvol; ++v) {
        mh3d_solve_opts ov = *o;
        ov.x0_dev = x0 ? x0[v] : nullptr;
        mh3d_status s = mh3d_solve(plans[v], d[v], &ov, rho[v], infos ? &infos[v] : nullptr, stream);
        if (s != MH3D_OK && worst == MH3D_OK) worst = s;
    }
    return worst;
}

mh3d_status mh3d_solve_batched(const mh3d_plan* plans, int nvol, const void* const* d, const mh3d_solve_opts* o,
                               float* const* rho, mh3d_solve_info* infos, void* stream)
{
    return solve_batched_impl(plans, nvol, d, o, nullptr, rho, infos, stream);
}

mh3d_status mh3d_solve_batched_warm(const mh3d_plan* plans, int nvol, const void* const* d,
                                    const mh3d_solve_opts* o, const float* const* x0_dev, float* const* rho,
                                    mh3d_solve_info* infos, void* stream)
{
    if (nvol > 0 && !x0_dev) return MH3D_ERR_INVALID_ARG;
    return solve_batched_impl(plans, nvol, d, o, x0_dev, rho, infos, stream);
}

}  // extern "C"
