// Loader / storer functors and small device helpers shared by the runtime
// pencil kernels (ops.cu) and the compile-time specialised ones (ops_ct.cuh).
#pragma once

#include "ops_kernels.cuh"

namespace mh3d {

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ld2(const float* __restrict__ p, long long i, bool has2, int vec2)
{
    if (vec2 && has2) return *reinterpret_cast<const float2*>(p + i);
    return make_float2(p[i], has2 ? p[i + 1] : 0.f);
}
__device__ __forceinline__ void st2(float* __restrict__ p, long long i, bool has2, int vec2, float2 v)
{
    if (vec2 && has2) {
        *reinterpret_cast<float2*>(p + i) = v;
    } else {
        p[i] = v.x;
        if (has2) p[i + 1] = v.y;
    }
}

__device__ __forceinline__ int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

// lambda * (R p)[i] at voxel (x, y, z).
__device__ __forceinline__ float reg_term(const RegArgs& g, const float* __restrict__ p, long long i, int x, int y,
                                          int z)
{
    const float pc = p[i];
    if (g.kind == 0) return g.lambda * pc;
    // T^T T = sum_a D_a^2, D_a the periodic second difference: stencil
    // (1, -4, 6, -4, 1) along each axis.
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const long long base = i - x - (long long)y * sy - (long long)z * sz;
    float acc = 0.f;
    {
        const long long r = base + (long long)y * sy + (long long)z * sz;
        acc += p[r + wrap(x - 2, g.nx)] - 4.f * p[r + wrap(x - 1, g.nx)] + 6.f * pc
             - 4.f * p[r + wrap(x + 1, g.nx)] + p[r + wrap(x + 2, g.nx)];
    }
    {
        const long long r = base + x + (long long)z * sz;
        acc += p[r + wrap(y - 2, g.ny) * sy] - 4.f * p[r + wrap(y - 1, g.ny) * sy] + 6.f * pc
             - 4.f * p[r + wrap(y + 1, g.ny) * sy] + p[r + wrap(y + 2, g.ny) * sy];
    }
    {
        const long long r = base + x + (long long)y * sy;
        acc += p[r + wrap(z - 2, g.nz) * sz] - 4.f * p[r + wrap(z - 1, g.nz) * sz] + 6.f * pc
             - 4.f * p[r + wrap(z + 1, g.nz) * sz] + p[r + wrap(z + 2, g.nz) * sz];
    }
    const bool shell = x < g.shell || y < g.shell || z < g.shell || x >= g.nx - g.shell || y >= g.ny - g.shell ||
                       z >= g.nz - g.shell;
    if (shell) acc += g.alpha * pc;
    return g.lambda * acc;
}

// CG loop control at the start of an iteration's kernels.  Returns false
// when the loop is finished (every CTA of the kernel returns).  The first
// kernel of an iteration also evaluates the stopping rule and the CG beta
// (and, in the single-reduction form, alpha).  Every control word and scalar
// is read in one round of loads (values read before the done flag is tested
// are simply unused once the loop has ended).  The stopping test and
// alpha's cancellation-prone denominator are FP64.  With c.fp64 (the
// default) beta and alpha are FP64 quotients, rounded to FP32 only for the
// FP32 vector updates, and the recurrence keeps the FP64 alpha; otherwise
// the divisions run in FP32 on the split significands (ddiv_to_float,
// relative error below 3e-7), which keeps the narrow FP64 pipe of this part
// free of divides.  Every CTA computes them with the same operations, so all
// apply the same values.
__device__ __forceinline__ bool cg_enter(const CgCtl& c, bool first_kernel, float* beta, double* sh,
                                         float* alpha = nullptr)
{
    if (!first_kernel) return !*(volatile int*)&c.flags[0];
    const int done = *(volatile int*)&c.flags[0];
    const int it = *(volatile int*)&c.flags[1];
    const int gave_up = *(volatile int*)&c.flags[3];
    const double g_new = __ldcg(c.rr_new);
    const double bn = __ldcg(c.bn);
    const double ro = c.rr_old ? __ldcg(c.rr_old) : 0.0;
    const double dl = c.cgcg ? __ldcg(c.delta) : 0.0;
    const double ap = c.cgcg ? __ldcg(c.alpha_prev) : 0.0;
    if (done) return false;
    const bool lead = threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0;
    if (gave_up) {   // a bounded wait gave up earlier: stop the loop
        if (lead) {
            c.flags[2] = MH3D_ERR_TIMEOUT;
            __threadfence();
            c.flags[0] = 1;
            if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
        }
        return false;
    }
    int status = -1;
    if (!dbits_finite(g_new) || !dbits_finite(bn)) status = MH3D_ERR_NONFINITE;
    else if (dbits_zero(g_new) || dbits_zero(bn)) status = MH3D_OK;
    else if (c.tol2 > 0.0 && g_new <= c.tol2 * bn) status = MH3D_OK;   // ||r||^2 / ||A^T d||^2 <= tol^2
    else if (it >= c.max_iter) status = (c.tol2 > 0.0) ? MH3D_ERR_NOT_CONVERGED : MH3D_OK;
    if (lead && it < c.hist_cap) c.hist[it] = (bn > 0.0) ? sqrt(g_new / bn) : 0.0;
    if (status >= 0) {
        if (lead) {
            c.flags[2] = status;
            __threadfence();
            c.flags[0] = 1;
            if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
        }
        return false;
    }
    // beta_i = gamma_i / gamma_{i-1}
    *beta = (it > 0) ? (c.fp64 ? (float)(g_new / ro) : ddiv_to_float(g_new, ro)) : 0.f;
    if (c.cgcg) {
        // alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_{i-1})
        //         = gamma_i u / (delta_i u - gamma_i^2),  u = gamma_{i-1} alpha_{i-1}
        const double an = (it == 0) ? g_new : g_new * (ro * ap);
        const double ad = (it == 0) ? dl : fma(dl, ro * ap, -g_new * g_new);
        double a64 = 0.0;
        float a;
        if (c.fp64) {
            a64 = an / ad;
            a = (float)a64;
        } else {
            a = ddiv_to_float(an, ad);
            a64 = (double)a;
        }
        if (!isfinite(a) || !(a > 0.f)) {
            if (lead) {
                c.flags[2] = MH3D_ERR_NONFINITE;
                __threadfence();
                c.flags[0] = 1;
                if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
            }
            return false;
        }
        if (lead) *c.alpha_out = a64;
        if (alpha) *alpha = a;
    }
    return true;
}

// cg_enter for a whole CTA (every thread calls it; c.flags set): thread 0
// evaluates the loop control and shares beta, alpha and the decision through
// shared memory, so the FP64 divides run once per CTA instead of once per
// thread (the FP64 pipe is narrow on this part).
__device__ __forceinline__ bool cg_enter_cta(const CgCtl& c, bool first_kernel, float* beta, float* alpha,
                                             float* sh3)
{
    if (threadIdx.x == 0) {
        float b = 0.f, al = 0.f;
        const bool go = cg_enter(c, first_kernel, &b, nullptr, &al);
        sh3[0] = b;
        sh3[1] = al;
        sh3[2] = go ? 1.f : 0.f;
    }
    __syncthreads();
    *beta = sh3[0];
    *alpha = sh3[1];
    return sh3[2] != 0.f;
}

// End of a CG iteration whose last pass is this kernel: the lead thread
// advances the completed-iteration counter (read only by later kernels).
// The hard bound ends the graph loop even if the first kernel of the next
// iteration, which normally stops it at max_iter, never ran.
__device__ __forceinline__ void cg_count_iteration(const CgCtl& c)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
        const int it = c.flags[1] + 1;
        c.flags[1] = it;
        if (it > c.max_iter + 1) {
            c.flags[2] = MH3D_ERR_NOT_CONVERGED;
            if (c.use_cond) cudaGraphSetConditional(c.cond, 0);
        }
    }
}

// ---------------------------------------------------------------------------
// T pass
// ---------------------------------------------------------------------------
struct TLoad {
    const TArgs* a;
    long long base;
    int x0;
    float beta;
    float alpha = 0.f;
    __device__ __forceinline__ float2 operator()(int e, int p) const
    {
        const int x = x0 + 2 * p;
        if (x >= a->nx) return make_float2(0.f, 0.f);
        const long long i = base + (long long)e * a->es + x;
        const bool has2 = x + 1 < a->nx;
        float2 v;
        if (a->pupdate == 2) {
            const float2 rr = ld2(a->rvec, i, has2, a->vec2);
            const float2 ss = ld2(a->svec, i, has2, a->vec2);
            const float2 pp = ld2(a->pvec, i, has2, a->vec2);
            const float2 qq = ld2(a->qdir, i, has2, a->vec2);
            const float2 xx = ld2(a->xvec, i, has2, a->vec2);
            const float2 pn = make_float2(fmaf(beta, pp.x, rr.x), fmaf(beta, pp.y, rr.y));
            const float2 qn = make_float2(fmaf(beta, qq.x, ss.x), fmaf(beta, qq.y, ss.y));
            st2(a->pvec, i, has2, a->vec2, pn);
            st2(a->qdir, i, has2, a->vec2, qn);
            st2(a->xvec, i, has2, a->vec2, make_float2(fmaf(alpha, pn.x, xx.x), fmaf(alpha, pn.y, xx.y)));
            v = make_float2(fmaf(-alpha, qn.x, rr.x), fmaf(-alpha, qn.y, rr.y));
            st2(a->rvec_w, i, has2, a->vec2, v);
        } else if (a->pupdate) {
            const float2 rr = ld2(a->rvec, i, has2, a->vec2);
            const float2 pp = ld2(a->pvec, i, has2, a->vec2);
            v = make_float2(fmaf(beta, pp.x, rr.x), fmaf(beta, pp.y, rr.y));
            st2(a->pvec, i, has2, a->vec2, v);
        } else {
            v = ld2(a->in, i, has2, a->vec2);
        }
        if (a->bin) {
            const float2 bb = ld2(a->bin, i, has2, a->vec2);
            v.x *= bb.x;
            v.y *= bb.y;
        }
        return v;
    }
};

struct MulLd {
    const float2* b;
    int ld;
    const float2* mu;
    __device__ __forceinline__ float2 operator()(int e, int p) const { return c_mul(b[e * ld + p], mu[e]); }
};

struct TStore {
    const TArgs* a;
    long long base;
    int x0;
    DotAcc* acc;
    DotAcc* acc2 = nullptr;   // input . input (single-reduction CG)
    __device__ __forceinline__ void operator()(int e, int p, float2 v) const
    {
        const int x = x0 + 2 * p;
        if (x >= a->nx) return;
        const long long i = base + (long long)e * a->es + x;
        const bool has2 = x + 1 < a->nx;
        if (a->bout) {
            const float2 bb = ld2(a->bout, i, has2, a->vec2);
            v.x *= bb.x;
            v.y *= bb.y;
        }
        if (a->epilogue) {
            const RegArgs& g = a->reg;
            const long long sz = (long long)g.nx * g.ny;
            const int z = (int)(i / sz), y = (int)((i - (long long)z * sz) / g.nx);
            v.x += reg_term(g, a->pin, i, x, y, z);
            if (has2) v.y += reg_term(g, a->pin, i + 1, x + 1, y, z);
            st2(a->qvec, i, has2, a->vec2, v);
            const float p0 = a->pin[i];
            acc->add(p0, v.x);
            if (acc2) acc2->add(p0, p0);
            if (has2) {
                const float p1 = a->pin[i + 1];
                acc->add(p1, v.y);
                if (acc2) acc2->add(p1, p1);
            }
        } else {
            st2(a->out, i, has2, a->vec2, v);
        }
    }
};

// ---------------------------------------------------------------------------
// X pass: loaders and storers
// ---------------------------------------------------------------------------
// Pencil p of a row-pair batch = rows (row0 + 2p, row0 + 2p + 1) as re/im.
struct RowPairLd {
    const float* v;
    int nx, row0, rows;
    __device__ __forceinline__ float2 operator()(int e, int p) const
    {
        const int r = row0 + 2 * p;
        float2 o = make_float2(0.f, 0.f);
        if (r < rows) o.x = v[(long long)r * nx + e];
        if (r + 1 < rows) o.y = v[(long long)(r + 1) * nx + e];
        return o;
    }
};
struct RowPairSt {
    float* v;
    int nx, row0, rows;
    __device__ __forceinline__ void operator()(int e, int p, float2 val) const
    {
        const int r = row0 + 2 * p;
        if (r < rows) v[(long long)r * nx + e] = val.x;
        if (r + 1 < rows) v[(long long)(r + 1) * nx + e] = val.y;
    }
};

// Forward: portrait spectrum of harmonic k0 + q / P at bin m =
// sum_{j < s} A[m + j mx] Xhat_k[m + j mx]   (the fold that realises P).
struct FoldLd {
    const float2* A;
    int ldA;
    const float2* __restrict__ Xh;   // Xhat + k0 * nx
    int nx, mx, s, P;
    __device__ __forceinline__ float2 operator()(int m, int q) const
    {
        const int kk = q / P, p = q - kk * P;
        const float2* xk = Xh + (long long)kk * nx;
        float2 acc = c_mul(A[m * ldA + p], __ldg(xk + m));
        for (int j = 1; j < s; ++j) {
            const int w = m + j * mx;
            acc = c_add(acc, c_mul(A[w * ldA + p], __ldg(xk + w)));
        }
        return acc;
    }
};

struct PortraitSt {
    float2* d;
    const float2* __restrict__ phase;   // phase + k0
    long long M;
    int mx, row0, rows, P;
    __device__ __forceinline__ void operator()(int m, int q, float2 val) const
    {
        const int kk = q / P, p = q - kk * P;
        const float2 ph = __ldg(phase + kk);
        const int r = row0 + 2 * p;
        float2* dk = d + (long long)kk * M;
        if (r < rows) dk[(long long)r * mx + m] = make_float2(ph.x * val.x, ph.y * val.x);
        if (r + 1 < rows) dk[(long long)(r + 1) * mx + m] = make_float2(ph.x * val.y, ph.y * val.y);
    }
};

// Adjoint: (Re(e^{-i theta} y[row]), Re(e^{-i theta} y[row+1])) at sample m.
struct PortraitLd {
    const float2* __restrict__ d;
    const float2* __restrict__ phase;
    long long M;
    int mx, row0, rows, P;
    __device__ __forceinline__ float2 operator()(int m, int q) const
    {
        const int kk = q / P, p = q - kk * P;
        const float2 ph = __ldg(phase + kk);
        const int r = row0 + 2 * p;
        const float2* dk = d + (long long)kk * M;
        float2 o = make_float2(0.f, 0.f);
        if (r < rows) {
            const float2 y = dk[(long long)r * mx + m];
            o.x = fmaf(ph.x, y.x, ph.y * y.y);
        }
        if (r + 1 < rows) {
            const float2 y = dk[(long long)(r + 1) * mx + m];
            o.y = fmaf(ph.x, y.x, ph.y * y.y);
        }
        return o;
    }
};

// Normal: out[m + a mx] = sum_b Q[m][a][b] A[m + b mx].
struct QLd {
    const float2* A;
    int ldA;
    const float2* __restrict__ Q;
    int mx, s;
    __device__ __forceinline__ float2 operator()(int w, int p) const
    {
        const int a = w / mx, m = w - a * mx;
        const float2* qm = Q + ((long long)m * s + a) * s;
        float2 acc = make_float2(0.f, 0.f);
        for (int b = 0; b < s; ++b) acc = c_add(acc, c_mul(__ldg(qm + b), A[(m + b * mx) * ldA + p]));
        return acc;
    }
};

// Normal epilogue: q = b w + lambda R p, accumulating p^T q.
struct NrmEpiSt {
    const XArgs* a;
    int row0;
    DotAcc* acc;
    DotAcc* acc2 = nullptr;   // input . input (single-reduction CG)
    __device__ __forceinline__ void one(int r, int x, float w) const
    {
        const long long i = (long long)r * a->nx + x;
        float q = a->b ? a->b[i] * w : w;
        const RegArgs& g = a->reg;
        const int z = r / g.ny, y = r - z * g.ny;
        q += reg_term(g, a->pin, i, x, y, z);
        a->qout[i] = q;
        const float pv = a->pin[i];
        acc->add(pv, q);
        if (acc2) acc2->add(pv, pv);
    }
    __device__ __forceinline__ void operator()(int x, int p, float2 val) const
    {
        const int r = row0 + 2 * p;
        if (r < a->rows) one(r, x, val.x);
        if (r + 1 < a->rows) one(r + 1, x, val.y);
    }
};

}  // namespace mh3d
