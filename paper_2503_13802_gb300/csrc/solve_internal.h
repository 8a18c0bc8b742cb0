// Declarations shared between capi.cu and solve.cu.
#pragma once

#include "ops_kernels.cuh"

namespace mh3d {

TArgs tpass_args(const Plan& P, int axis, const float* in, float* out, const float2* mult);
int tpass_outer(const Plan& P, int axis);
XArgs xpass_args(const Plan& P);
RegArgs reg_args(const Plan& P, const mh3d_solve_opts& o);
// CG vector update fused into the first pass of the normal operator.
struct LoaderUpdate {
    int mode = 0;                 // 1: p = r + beta p; 2: single-reduction CG update (see TArgs)
    float* p = nullptr;
    const float* r = nullptr;
    float* r_w = nullptr;
    float* q = nullptr;
    const float* s = nullptr;
    float* x = nullptr;
};
cudaError_t launch_normal(const Plan& P, int mode, const RegArgs& reg, const float* in, float* out, float* t1,
                          float* t2, float2* portrait, const RedSink* dots, const CgCtl* cg, const LoaderUpdate* upd,
                          cudaStream_t st);
int normal_part_count(const Plan& P, int mode);
mh3d_status ensure_portrait(Plan& P);

mh3d_status solve_alloc(Plan& P);
// Drops every cached batch graph that holds this plan's buffers.
void batch_forget(const Plan& P);
void solve_free(Plan& P);
cudaError_t solve_set_attributes();
mh3d_status validate_opts(Plan& P, const mh3d_solve_opts& o);

// Number of CTAs of the elementwise solver kernels for N voxels.
int update_blocks(long long N);

}  // namespace mh3d
