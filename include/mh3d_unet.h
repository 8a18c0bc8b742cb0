/*
 * mh3d_unet.h -- C ABI of the learned warm start for the MH3D solver
 * (libmh3d.so).
 *
 * The paper reconstructs from a zero start (Sec. 4.3, accelerated projected
 * gradient; here also CG).  This adds a learned initial iterate: a small 3D
 * U-Net maps the normalised back-projection A^T d to a guess rho_0 from
 * which CG starts (mh3d_solve_opts.x0_dev).  The paper has no counterpart;
 * its architecture, loss and training recipe are this library's.
 *
 * Network (L levels, channels C_0 .. C_{L-1}; level l at 1 / 2^l of the
 * resolution).  For L = 3 (c0, c1, c2):
 *   e0a = relu(conv(in, W0a)); e0 = relu(conv(e0a, W0b))
 *   e1a = relu(conv(pool(e0), W1a)); e1 = relu(conv(e1a, W1b))
 *   ba = relu(conv(pool(e1), W2a)); b = relu(conv(ba, W2b))
 *   u1 = relu(conv(up(b), W3a)); d1 = relu(conv(u1 + e1, W3b))
 *   u0 = relu(conv(up(d1), W4a)); d0 = relu(conv(u0 + e0, W4b))
 *   out = conv(d0, W5)
 * In general: encoder levels l = 0 .. L-1 (W{l}a on the input, or on
 * pool(e_{l-1}); W{l}b), the last one the bottleneck; decoder levels
 * l = L-2 .. 0 (W{2L-2-l}a on up(d_{l+1}), W{2L-2-l}b on u_l + e_l; the
 * bottleneck's e is its d); out = conv(d0, W{2L-1}): 4 L - 1 convolutions.
 * conv: 3x3x3 cross-correlation, zero padding, bias; pool: 2x2x2 mean;
 * up: nearest x2.  Arithmetic: bfloat16 operands on the tensor cores with
 * FP32 accumulation; activations stored as bfloat16 (channels last); the
 * input and the output are FP32.
 *
 * Parameters: one flat FP32 vector; per layer in the order above
 * (L = 3: W0a, W0b, W1a, W1b, W2a, W2b, W3a, W3b, W4a, W4b, W5): W as
 * [cout][3][3][3][cin] (taps dz, dy, dx), then b [cout].
 * Loss of mh3d_unet_loss_grad: sum((out - target)^2) / (2 V).
 *
 * The convolutions run on the tcgen05 tensor cores (accumulators in tensor
 * memory) where the source is bfloat16 with 8..32 channels in multiples of
 * 8 or the FP32 input, at most 64 outputs, and rows of 96 voxels or more;
 * on mma.sync tiles otherwise.  MH3D_UNET_UMMA=0 / 1 sends none / every
 * convolution it can take to the tcgen05 kernel.
 *
 * Sizes: nx, ny, nz multiples of 2^(L-1) (4 for mh3d_unet_create); channels
 * in 1..64 (mh3d_unet_create) or 1..128 (mh3d_unet_create_levels).  Volumes are
 * C-order [nz][ny][nx].  All pointers are device pointers unless stated;
 * calls are asynchronous on `stream` unless stated.  Errors are status
 * codes (mh3d.h) with text from mh3d_unet_last_error.
 */
#ifndef MH3D_UNET_H
#define MH3D_UNET_H

#include "mh3d.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mh3d_unet_s* mh3d_unet;

/* Number of parameters of a network with channels c0, c1, c2 (three
 * levels), or with `levels` levels (2..5) of channels[0 .. levels-1]
 * (-1 for a bad level count or a null pointer). */
long long mh3d_unet_param_count(int c0, int c1, int c2);
long long mh3d_unet_param_count_levels(int levels, const int* channels);

/* Allocates a network for volumes of nx x ny x nz voxels: parameters (set
 * them with mh3d_unet_set_params before use), Adam state, activations and
 * gradient buffers.  MH3D_ERR_INVALID_ARG for bad sizes, MH3D_ERR_OOM. */
mh3d_status mh3d_unet_create(int nx, int ny, int nz, int c0, int c1, int c2, mh3d_unet* out);
/* The same for `levels` levels (2..5) with channels[0 .. levels-1] (host
 * array, 1..128 each); nx, ny, nz multiples of 2^(levels-1). */
mh3d_status mh3d_unet_create_levels(int nx, int ny, int nz, int levels, const int* channels, mh3d_unet* out);
mh3d_status mh3d_unet_destroy(mh3d_unet net);

/* Copies param_count floats in (and resets the Adam state) / out. */
mh3d_status mh3d_unet_set_params(mh3d_unet net, const float* theta, void* stream);
mh3d_status mh3d_unet_get_params(mh3d_unet net, float* theta, void* stream);

/* out = network(in): in and out are nz*ny*nx floats. */
mh3d_status mh3d_unet_forward(mh3d_unet net, const float* in, float* out, void* stream);

/* Forward pass on `in`, the loss against `target`, and the gradient of the
 * loss with respect to every parameter (kept for mh3d_unet_adam_step and,
 * when grad is not NULL, copied to grad: param_count floats).  When loss
 * (a HOST pointer) is not NULL the call synchronises the stream and stores
 * the loss there. */
mh3d_status mh3d_unet_loss_grad(mh3d_unet net, const float* in, const float* target, float* grad, double* loss,
                                void* stream);

/* Scale-free versions for back-projections of any magnitude.  With
 * r = RMS(in) (computed on the device, r = 1 for a zero input):
 *   forward_scaled:   out = (r gain) * network(in / r)
 *   loss_grad_scaled: the loss and gradient of network(in / r) against
 *                     target / (r gain)
 * gain > 0 (the warm start uses 1 / ||A||_2^2).  No host synchronisation
 * except for the loss, as above. */
mh3d_status mh3d_unet_forward_scaled(mh3d_unet net, const float* in, float gain, float* out, void* stream);
mh3d_status mh3d_unet_loss_grad_scaled(mh3d_unet net, const float* in, const float* target, float gain, float* grad,
                                       double* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the gradient of the last mh3d_unet_loss_grad. */
mh3d_status mh3d_unet_adam_step(mh3d_unet net, float lr, void* stream);

/* Single-layer primitives (the network's own kernels), for tests and for
 * callers that build other networks.  A source is a channels-last bfloat16
 * volume (src_bf16, cin channels; with skip_bf16 the elementwise sum of the
 * two, rounded to bfloat16; with up = 1 a half-resolution volume read by
 * nearest x2 upsampling), or, for cin == 1, a FP32 volume (src_f32).  These
 * allocate temporaries and synchronise the stream. */
typedef struct {
    int nx, ny, nz;           /* resolution of the convolution */
    int cin, cout;
    const void* src_bf16;     /* may be NULL when src_f32 is given */
    const void* skip_bf16;    /* NULL: no skip addend */
    const float* src_f32;     /* NULL: use src_bf16 */
    int up;
} mh3d_unet_conv_desc;

/* out[v][co] = b[co] + sum_{tap, ci} W[co][tap][ci] src[v + tap][ci] (FP32 out, ReLU when relu != 0). */
mh3d_status mh3d_unet_conv_forward(const mh3d_unet_conv_desc* c, const float* W, const float* b, int relu,
                                   float* out, void* stream);
/* gin[v][ci] = sum_{tap, co} W[co][tap][ci] g[v - tap][co]; g bfloat16 [V][cout], gin FP32 [V][cin]
 * (c->src_* and c->up are ignored: the gradient is at the convolution's resolution). */
mh3d_status mh3d_unet_conv_input_grad(const mh3d_unet_conv_desc* c, const void* g_bf16, const float* W, float* gin,
                                      void* stream);
/* gW[co][tap][ci] = sum_v g[v][co] src[v + tap][ci], gb[co] = sum_v g[v][co]. */
mh3d_status mh3d_unet_conv_weight_grad(const mh3d_unet_conv_desc* c, const void* g_bf16, float* gW, float* gb,
                                       void* stream);

const char* mh3d_unet_last_error(mh3d_unet net);

#ifdef __cplusplus
}
#endif

#endif /* MH3D_UNET_H */
