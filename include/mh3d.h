/*
 * mh3d.h -- C ABI of the GB300 MH3D operator and solver library (libmh3d.so).
 *
 * Multi-Harmonic Gridded 3D Deconvolution, arXiv 2503.13802.  The library
 * applies the drive-axis portrait model
 *
 *     d_k = e^{i theta_k} P ( h_k * (b . rho) ),   k = k_min .. k_max
 *
 * (Sec. 3.2, Eq. portz / matrixModelz; Sec. 4.1, Eq. dN: A = P H B; phase of
 * Sec. 4.4), its adjoint, and solves the regularised least-squares problem
 * of Sec. 4.3 (Eq. Amodel with R of Eq. finalR, stacked form M, b) on one
 * GPU.  The PSF is h_k(x) = c_k L^(k)(gamma x_d) phi(x_t1) phi(x_t2) with
 * c_k = (gamma A)^k / (k-1)! (Sec. 3.3, Eq. hkapprox; Theorem 1), L the
 * Langevin function, phi(t) = 3 L'(transverse_ratio * gamma * t); samples at
 * minimal-image offsets of the periodic grid (offset -n/2 at index n/2 for
 * even n), circular convolution (FFT-periodic model, Table ops).
 *
 * Conventions (every entry point):
 *   - Volumes are float32, C-order [nz][ny][nx]; x is the drive axis and is
 *     contiguous.  Portraits are complex64 (float2 = re, im), C-order
 *     [K][nz][ny][nx/s], K = k_max - k_min + 1; portrait row i' holds model
 *     row s*i' + ds_offset (the row selector P of Eq. dN).
 *   - Pointers named *_dev are device pointers owned by the caller; pointers
 *     named *_host are host pointers owned by the caller (pinned memory is
 *     faster but not required).  The plan owns its own tables and workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Operator calls are asynchronous on that stream; solver calls
 *     synchronise the stream once at the end to fill the info record.
 *   - Errors come back as an mh3d_status; no call aborts, throws or exits.
 *     mh3d_last_error(plan) returns a message for the last failing call on
 *     that plan (thread-compatible: one thread per plan at a time).
 *   - Grid lengths must factor into 2s and 3s (1 <= n <= 1024); nx must be a
 *     multiple of ds_factor; anything else is MH3D_ERR_UNSUPPORTED_SIZE at
 *     plan time.
 *   - All arithmetic on the operator path is FP32 (round to nearest, no fast
 *     math).  The solver's inner products and norms multiply FP32 values
 *     exactly and sum them in float pairs (hi + lo, compensated: about 48
 *     significand bits, error near FP64 summation's), each total becoming an
 *     FP64 scalar; the CG step lengths and the stopping test are FP64 on the
 *     GPU (see mh3d_solve_opts.fp32_scalar_div), rounded to FP32 only where
 *     they scale the FP32 vectors.
 */
#ifndef MH3D_H
#define MH3D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mh3d_plan_s* mh3d_plan;

typedef enum {
    MH3D_OK = 0,
    MH3D_ERR_INVALID_ARG = 1,      /* NULL pointer, bad enum, inconsistent sizes            */
    MH3D_ERR_UNSUPPORTED_SIZE = 2, /* a length with a prime factor > 3, or too large        */
    MH3D_ERR_OOM = 3,              /* device or host allocation failed                      */
    MH3D_ERR_CUDA = 4,             /* a CUDA runtime call failed (message has the detail)   */
    MH3D_ERR_NONFINITE = 5,        /* NaN/Inf met in an FP64 reduction of the solver        */
    MH3D_ERR_NOT_CONVERGED = 6,    /* max_iter reached before rel_tol (solution still kept) */
    MH3D_ERR_TIMEOUT = 7           /* a bounded device wait gave up                         */
} mh3d_status;

/* Scanner/model geometry (Sec. 2; Sec. 3.3; Sec. 4.1).  Copied at plan time
 * except sensitivity_dev, which the plan keeps as a borrowed pointer: the
 * caller keeps that buffer alive and unchanged for the plan's lifetime.
 * Boundary padding: n is the field of view; the model grid is n + 2 pad on
 * each axis (FFT-periodic there), and every image (rho, x0, the sensitivity)
 * of the plan lives on that grid, [nz+2pz][ny+2py][nx+2px], the field of
 * view at offsets (px, py, pz).  Portraits cover the field of view only:
 * K*nz*ny*(nx/s) samples, row i' of the field of view's mesh being row
 * px/s + i' of the padded one.  So A = C A_pad (C keeps the field of view's
 * samples), A^T = A_pad^T C^T (zero padding), and the normal operator is
 * A_pad^T C^T C A_pad, applied explicitly (normal_mode 1, whatever the
 * options say).  lambda_relative scales by ||A_pad||_2^2.  The caller crops
 * the field of view from the solution.  Padded plans are refused by
 * mh3d_solve_batched, mh3d_mhad and mh3d_forward_noalloc. */
typedef struct {
    int n[3];                    /* nx (drive axis), ny, nz                                 */
    double voxel_mm[3];          /* voxel size per axis, mm                                 */
    int drive_axis;              /* must be 0 (x, contiguous)                               */
    int ds_factor;               /* s >= 1: keep every s-th drive-axis row (Eq. dN, P)      */
    int ds_offset;               /* 0 <= r < s: kept rows are i = r (mod s)                 */
    int pad[3];                  /* boundary padding voxels per side per axis (Sec. 3.x,     */
                                 /* boundary image padding); pad[0] a multiple of ds_factor  */
    int k_min, k_max;            /* harmonics k_min..k_max, 2 <= k_min <= k_max <= 32       */
    double gamma_per_mm;         /* gamma = beta G along the drive axis, 1/mm (> 0)         */
    double gammaA;               /* gamma * drive excursion A, |gamma A| < pi (Theorem 1)   */
    double transverse_ratio;     /* transverse / drive gradient, 0.5 for G0 diag(1/2,1/2,1) */
    const double* theta;         /* host, K phases theta_k (Sec. 4.4); NULL = all zero      */
    const float* sensitivity_dev;/* device, N floats b (receive map, B of Eq. dN); NULL = 1 */
} mh3d_geometry;

/* Regularised least squares of Sec. 4.3:
 *   min ||A rho - d||^2 + lambda R(rho),
 *   R = ||rho||^2                                  (reg_kind 0)
 *   R = ||T rho||^2 + alpha ||P_a rho||^2          (reg_kind 1, Eq. finalR; T = periodic
 *       second differences on each axis, P_a = voxels within `shell` of a face).
 * solver 0 = conjugate gradients on the normal equations (unconstrained);
 * solver 1 = the paper's accelerated projected gradient with rho >= 0. */
typedef struct {
    int reg_kind;                /* 0 or 1                                                  */
    double lambda;               /* > 0                                                     */
    double alpha;                /* >= 0, used by reg_kind 1                                */
    int shell;                   /* >= 1, used by reg_kind 1                                */
    int solver;                  /* 0 = CG, 1 = APG                                         */
    double rel_tol;              /* CG: stop when ||r_k|| <= rel_tol ||A^T d|| (zero-start  */
                                 /*     norm, recurrence residual, FP64)                    */
    int max_iter;                /* >= 1                                                    */
    int fixed_iters;             /* nonzero: run exactly max_iter iterations, no tol check  */
    const float* x0_dev;         /* device, N floats initial iterate; NULL = zero start     */
    int normal_mode;             /* 0 = fused normal operator (exact A^T A, Fourier blocks) */
                                 /* 1 = explicit A then A^T through a portrait buffer       */
    double apg_tau;              /* APG step; <= 0: 0.99 / lambda_max(A^T A + lambda R) from */
                                 /*   a power iteration on the device (Rayleigh quotients,  */
                                 /*   FP64, until they change by < 1e-6); info.tau has it   */
    int lambda_relative;         /* nonzero: the weight of R is lambda * ||A||_2^2, the     */
                                 /* squared spectral norm of A with b = 1 (see              */
                                 /* mh3d_operator_norm2); zero: lambda is absolute          */
    int cg_variant;              /* 0 = single-reduction CG (Chronopoulos-Gear): the vector */
                                 /*     update runs inside the operator's first pass, one   */
                                 /*     grid reduction per iteration;                       */
                                 /* 1 = classic CG (Hestenes-Stiefel), two reductions and a */
                                 /*     separate update pass.  Same iterates in exact       */
                                 /*     arithmetic.                                         */
    int x0_fallback;             /* with x0_dev: if ||A^T d - N x0|| >= ||A^T d|| (the guess */
                                 /* is no better than zero) the solve restarts from x = 0;   */
                                 /* decided on the device, reported in info.x0_rejected      */
    int fp32_scalar_div;         /* 0 (default): CG's beta and alpha are FP64 quotients of  */
                                 /*   the FP64 scalars; nonzero: FP32 quotients of their    */
                                 /*   leading 24 significand bits (relative error < 3e-7,   */
                                 /*   no FP64 divide on the device)                         */
} mh3d_solve_opts;

typedef struct {
    int iters;                   /* iterations performed                                    */
    double rel_res_recurrence;   /* ||r_k|| / ||A^T d|| from the FP64 recurrence            */
    double rel_res_true;         /* ||A^T d - (A^T A + lambda R) x|| / ||A^T d||, recomputed */
    double* history;             /* host, caller-owned, >= max_iter+1 doubles, or NULL:     */
                                 /* receives ||r_k||/||A^T d|| for k = 0..iters             */
    int status;                  /* mh3d_status of the solve                                */
    int x0_rejected;             /* 1 if x0_fallback replaced x0 by the zero start          */
    double tau;                  /* APG: the step used (given or computed); CG: 0           */
} mh3d_solve_info;

/* Create a plan: validates the geometry, builds the PSF spectra in FP64 on
 * the host (rounded once to FP32), uploads tables, allocates workspace and
 * selects FFT radix/tile schedules for each axis.  `stream` is used for the
 * uploads.  On failure *out is NULL. */
mh3d_status mh3d_plan_create(const mh3d_geometry* geom, void* stream, mh3d_plan* out);

/* Release a plan and its device memory (synchronises the device first). */
mh3d_status mh3d_plan_destroy(mh3d_plan plan);

/* d_dev[K*nz*ny*(nx/s)] = A rho_dev[N]   (Eq. dN with the phase of Sec. 4.4). */
mh3d_status mh3d_forward(mh3d_plan plan, const float* rho_dev, void* d_dev, void* stream);

/* rho_dev[N] = A^T d_dev for the real inner product Re<.,.>:
 *   A^T y = b . sum_k h~_k * P^T Re(e^{-i theta_k} y_k), h~_k(x) = h_k(-x). */
mh3d_status mh3d_adjoint(mh3d_plan plan, const void* d_dev, float* rho_dev, void* stream);

/* q_dev = (A^T A + lambda R) p_dev with R from opts (reg_kind, lambda, alpha,
 * shell); opts->normal_mode picks the fused or the explicit evaluation.
 * p_dev and q_dev must not overlap. */
mh3d_status mh3d_normal(mh3d_plan plan, const float* p_dev, float* q_dev,
                        const mh3d_solve_opts* opts, void* stream);

/* Solve from device portraits d_dev into rho_dev (Sec. 4.3).  Synchronises
 * `stream` once at the end and fills *info (may be NULL).  Returns MH3D_OK,
 * MH3D_ERR_NOT_CONVERGED (rho_dev still holds the last iterate) or an error. */
mh3d_status mh3d_solve(mh3d_plan plan, const void* d_dev, const mh3d_solve_opts* opts,
                       float* rho_dev, mh3d_solve_info* info, void* stream);

/* mh3d_solve from HOST portraits to a HOST image: copies d_host to the
 * device, solves, copies the result back (all on `stream`). */
mh3d_status mh3d_solve_host(mh3d_plan plan, const void* d_host, const mh3d_solve_opts* opts,
                            float* rho_host, mh3d_solve_info* info, void* stream);

/* Solve nvol independent problems, each with its own plan (grid sizes may
 * differ) and data, in one launch: for CG (opts->solver == 0) the call
 * stages every volume's portraits into its plan, then launches ONE CUDA graph
 * that holds one independent branch per volume (A^T d, set-up, a
 * device-driven conditional while loop, true residual), so the GPU runs the
 * volumes concurrently; it synchronises twice and fills infos.  The graph
 * is cached for the same plans and options.  APG (solver 1), or
 * MH3D_NO_GRAPH=1, solves the volumes one after another.
 *   plans[v], d_dev[v] (K*M complex64 on the device), rho_dev[v] (N floats
 *   on the device) for v < nvol; each plan at most once (the branches use
 *   the plans' workspaces); opts applies to every volume and opts->x0_dev
 *   must be NULL (per-volume warm starts: mh3d_solve_batched_warm); infos
 *   (may be NULL) receives nvol records, and their
 *   history pointers (may be NULL) are honoured.
 *   Returns the first non-OK volume status (MH3D_ERR_NOT_CONVERGED keeps
 *   the iterates); mh3d_last_error(plans[0]) names the volume.  Plans must
 *   not be destroyed while a call that uses them runs. */
mh3d_status mh3d_solve_batched(const mh3d_plan* plans, int nvol, const void* const* d_dev,
                               const mh3d_solve_opts* opts, float* const* rho_dev,
                               mh3d_solve_info* infos, void* stream);

/* mh3d_solve_batched with a warm start per volume: x0_dev[v] (device, N_v
 * floats) is volume v's initial iterate, as opts->x0_dev is for mh3d_solve
 * (opts->x0_fallback applies to each volume; opts->x0_dev must be NULL).
 * The call copies each x0 into its plan's iterate before the graph runs, so
 * the cached graph serves any x0 pointers.  Each volume's result equals its
 * single warm-started solve bit for bit.  The learned warm start of the
 * batching pattern (a network's output per volume) goes through this call.
 * MH3D_ERR_INVALID_ARG for a NULL x0_dev or x0_dev[v]; otherwise as
 * mh3d_solve_batched. */
mh3d_status mh3d_solve_batched_warm(const mh3d_plan* plans, int nvol, const void* const* d_dev,
                                    const mh3d_solve_opts* opts, const float* const* x0_dev,
                                    float* const* rho_dev, mh3d_solve_info* infos, void* stream);

/* Copies the plan's FP32 spectral tables (device -> device, any pointer may
 * be NULL): X [K][nx] complex = c_k DFT_nx(L^(k)(gamma o dx) at o + ds_offset)
 * / nx (the drive-axis spectra, Eq. hkapprox and Theorem 1, shifted so that
 * portrait row i' is model row s i' + ds_offset), Y [ny] = DFT of the
 * transverse samples / ny, Z [nz] likewise, phase [K] = e^{i theta_k}.  With
 * these, d_k = e^{i theta_k} S_s IDFT(DFT(b rho) nx X_k ny Y nz Z) (the
 * forward model, Sec. 3.2 and 4.1).  Asynchronous on `stream`. */
mh3d_status mh3d_plan_spectra(mh3d_plan plan, void* X, void* Y, void* Z, void* phase, void* stream);

/* MHAD native image (App. D, Eq. mhadM), the paper's FFT-only closed-form
 * reconstruction along the drive axis, computed for every portrait row:
 *   rho_N = IDFT[ sum_k c_k^{-1} conj(DFT f^{k-1}) DFT(D_k) / (sum_k |DFT f^{k-1}|^2 + lambda) ]
 * over the plan's harmonics k, with D_k = Re(e^{-i theta_k} d_k) (the
 * portrait with its phase removed, Sec. 4.4), f the circular central
 * difference of the portrait mesh ((f * u)[j] = u[j+1] - u[j-1]),
 * c_k = (gamma A)^k / (k-1)! and DFTs of length mx = nx / ds_factor.
 *   d_dev: K*nz*ny*mx complex64 portraits (device, the layout of
 *   mh3d_forward).  lambda: the closed form's Tikhonov weight, finite and
 *   > 0 (absolute; f is zero at DC and at the mesh's Nyquist bin, where
 *   lambda alone keeps the quotient defined), else MH3D_ERR_INVALID_ARG.
 *   upsample = 0: out_dev receives the image on the portrait mesh,
 *   nz*ny*mx floats [nz][ny][mx].  upsample = 1: out_dev receives its
 *   band-limited interpolation onto the model grid, N floats [nz][ny][nx]:
 *   the drive-axis spectrum zero-padded from mx to nx bins (the mesh's
 *   Nyquist bin split between +mx/2 and -mx/2), portrait row i' on model
 *   row ds_factor i' + ds_offset, where it equals the upsample = 0 image.
 *   The filter tables are built in FP64 on the host and cached in the plan
 *   per (lambda, upsample); calls on one plan must be ordered on one stream.
 *   Asynchronous on `stream` (the first call allocates K*max(nx, mx)
 *   complex64 of tables). */
mh3d_status mh3d_mhad(mh3d_plan plan, const void* d_dev, double lambda, int upsample, float* out_dev, void* stream);

/* Warm start for mh3d_solve from the MHAD image: u = mh3d_mhad(upsample = 1)
 * divided by the sensitivity b where b > 0 (0 where b <= 0; no division for
 * a plan without b), then x0_dev = alpha u with alpha = Re<A u, d> /
 * ||A u||^2, the least-squares scale of u on the data (A applied by the
 * library, the two sums in FP64 on the device; alpha = 0 if A u = 0).
 * The paper uses MHAD as an image, not as a starting point; this is the
 * non-learned warm start compared with the learned one.
 *   d_dev, lambda: as for mh3d_mhad; x0_dev: N floats (device), written.
 *   alpha_dev: one double on the device receiving alpha, or NULL.
 *   The first call allocates K*M complex64 of scratch portraits and 16 KiB
 *   of partial sums, kept by the plan.  Uses the plan's workspace like
 *   mh3d_forward.  Asynchronous on `stream`. */
mh3d_status mh3d_mhad_warm_start(mh3d_plan plan, const void* d_dev, double lambda, float* x0_dev, double* alpha_dev,
                                 void* stream);

/* Portrait phase calibration (Sec. 4.4): estimates theta_k from portraits
 * measured as e^{i theta_k} times a real field.
 *   theta_k modulo pi: 1/2 arg of the sum of d_k^2 over the high-SNR samples
 *   (|d_k| >= frac max |d_k|).  The remaining pi, when ds_factor = 1: the
 *   single-harmonic back-projections A_k^T Re(e^{-i theta_k} d_k) correlate
 *   positively for the true signs (along the drive axis their product is
 *   non-negative at every frequency), which fixes every sign relative to
 *   the strongest one; the common sign is the one whose 30-iteration CG
 *   reconstruction (lambda 1e-2 relative) is positively skewed, as the
 *   image of a non-negative density is.  With ds_factor > 1 theta_k is
 *   returned modulo pi.
 *   d_dev: the caller's portraits (K*nz*ny*(nx/s) complex64, device);
 *   frac in (0, 1]; theta_out: K doubles (host) in (-pi, pi]; resolved_out:
 *   K ints (host, may be NULL), 1 where the pi was decided, 0 where theta_k
 *   is known modulo pi only.  Synchronises `stream`; allocates and frees its
 *   scratch (K + 1 images and one portrait set); uses the plan's workspace
 *   and runs a 30-iteration solve on it.
 *   The paper picks high-SNR regions by hand and decides the pi with a trial
 *   reconstruction; these rules are this library's automatic stand-ins. */
mh3d_status mh3d_estimate_phase(mh3d_plan plan, const void* d_dev, double frac, double* theta_out, int* resolved_out,
                                void* stream);

/* The general model (Sec. 3.2, Eq. MH3Dcont and Eq. matrixModel): three
 * receive components with PSFs that need not be separable -- the harmonic
 * PSFs of the tensor PSF (appendix, Eq. PSF, Eq. skMD) or simulated ones:
 *   d_k[z][y][i'] = e^{i theta_k} sum_j (h_kj * (b_j rho))[z][y][s i' + r],
 * * the 3D circular convolution on the plan's grid, theta_k, s and r the
 * plan's.  Not for padded plans.
 *
 * mh3d_general_set_psf: h_host (host, float32, K*3*N values, layout
 *   [k][j][z][y][x], component j = 0 drive axis, 1 y, 2 z) holds (h_k)_j at
 *   the minimal-image offsets of the grid (index i along an axis of length
 *   n is the offset i for 2i < n, else i - n, times the voxel size).  The
 *   plan keeps their spectra on the device: K*3*N + 4*N complex64 values,
 *   allocated on the first call and reused.  Synchronous.
 * mh3d_general_forward: rho (device, N floats) -> d (device, complex64
 *   K*nz*ny*(nx/s)).  bvec (device, 3*N floats [j][z][y][x]) or NULL for
 *   b = (1, 0, 0).  Asynchronous on `stream`; uses the plan's work area, so
 *   calls on one plan must not overlap.
 * mh3d_general_adjoint: the adjoint for the real inner product,
 *   Re<A x, d> = <x, A^T d>: d (device, complex64) -> out (device, N floats).
 * Errors: MH3D_ERR_INVALID_ARG for null pointers, a padded plan, or no PSF
 *   set; MH3D_ERR_CUDA with mh3d_last_error() text otherwise. */
mh3d_status mh3d_general_set_psf(mh3d_plan plan, const float* h_host);
mh3d_status mh3d_general_forward(mh3d_plan plan, const float* rho, const float* bvec, void* d, void* stream);
mh3d_status mh3d_general_adjoint(mh3d_plan plan, const void* d, const float* bvec, float* out, void* stream);

/* The regularised reconstruction of Sec. 4.3 on the general model:
 *   min ||A rho - d||^2 + lambda ||rho||^2,  A the forward of
 *   mh3d_general_forward with the plan's PSF spectra and bvec,
 * by conjugate gradients on (A^T A + lambda I) rho = A^T d (Hestenes-Stiefel).
 * Each iteration applies A (into the plan's portrait buffer, allocated on
 * first use) and A^T, two float-pair inner products (as mh3d_dot) and the
 * vector updates; the scalars are FP64 on the host, which synchronises
 * `stream` three times per iteration.
 *   d_dev: portraits (device, complex64 K*nz*ny*(nx/s)); bvec_dev: as for
 *   mh3d_general_forward (NULL = b = (1, 0, 0)); rho_dev: N floats (device,
 *   written).  opts: solver 0, reg_kind 0, lambda absolute and > 0
 *   (lambda_relative 0: the general model has no Fourier-block norm),
 *   rel_tol (stopping rule ||r_k|| <= rel_tol ||A^T d||, recurrence
 *   residual), max_iter, fixed_iters and x0_dev (device, or NULL) as for
 *   mh3d_solve; other fields ignored.  info (may be NULL): iterations,
 *   recurrence and recomputed true relative residuals, history (if its
 *   pointer is set, max_iter + 1 doubles), status.
 *   Errors: MH3D_ERR_INVALID_ARG (null pointers, unsupported options, no PSF
 *   set), MH3D_ERR_NOT_CONVERGED (rho_dev holds the last iterate),
 *   MH3D_ERR_NONFINITE, MH3D_ERR_CUDA. */
mh3d_status mh3d_general_solve(mh3d_plan plan, const void* d_dev, const float* bvec_dev,
                               const mh3d_solve_opts* opts, float* rho_dev, mh3d_solve_info* info, void* stream);

/* Autotuning (the batching pattern's per-size-class schedule choice; the
 * paper has no counterpart): times, on the plan's own workspace, the launch
 * variants of the three operators and keeps the fastest of each --
 *   the normal operator (the CG loop's kernels): transverse-pass tile width
 *   (16 or 8 columns) x its radix schedule (the default or the alternative
 *   one, e.g. 8 x 16 instead of 16 x 8 at length 128) x CTAs per y-slab of
 *   the fused cluster pass (2 or 4);
 *   the adjoint's drive-axis part: warp-centric fused with T_z^T, or
 *   followed by T_z^T, with 1, 2 or 4 warps per row group, or CTA-level;
 *   the forward's drive-axis part: the cluster pass fusing T_z or the
 *   warp-centric pass (1, 2 or 4 warps per row group).
 * The choice applies to this plan and is remembered for the process per
 * (grid, ds_factor, K, weighted or not), so later plans of a tuned size take
 * it without timing.  With the environment variable MH3D_TUNE_CACHE set to
 * a file path the choice is also read from and written to that JSON file
 * (a JSON object with one size class per line, the layout it writes), so a later
 * process takes it without timing.
 * The normal operator is timed back to back (in the CG loop its working
 * set stays in L2); the adjoint and forward, which a solve runs once on
 * data not in L2, are timed launch by launch after a write of a temporary
 * buffer twice the L2 size (allocated and freed by the call).
 * The radix and path choices change the FP32 rounding path (results agree
 * within the operators' tolerance, not bit for bit); the tile width alone
 * does not.  Synchronises `stream`; allocates the plan's portrait buffer
 * (K*M complex64) if it has none; drops the plan's cached graphs.
 * tpass_cols (may be NULL) receives the tile width. */
mh3d_status mh3d_plan_autotune(mh3d_plan plan, void* stream, int* tpass_cols);

/* The plan's current launch choices as a JSON object (the fields the
 * autotuner sets: tpass_cols, tpass_radix, zx_c, adj_path, xw_ks, fwd_path,
 * xw_ks_fwd; 0 = the library's default) written into buf (host, buflen
 * bytes, NUL-terminated).  MH3D_ERR_INVALID_ARG if buf is too small. */
mh3d_status mh3d_plan_tuning(mh3d_plan plan, char* buf, int buflen);

/* d_dev = A rho_dev like mh3d_forward, for callers that cannot allocate
 * device memory (a fixed device-memory budget owned by another framework's
 * pool, a frozen real-time memory plan, or code that must not risk the
 * implicit synchronisation of an allocation), and therefore cannot create a
 * plan.  No plan and no allocation: the PSF tables (built in FP64 on the host
 * from `geom`, rounded to FP32) and the two intermediate volumes live in one
 * fixed __device__ array that every GPU loading this library holds until
 * exit (512 KiB of tables + 16 MiB of volumes).  The paper has no
 * counterpart; this is a deployment variant of the forward operator.
 *   Limits: nx*ny*nz <= 2,097,152 voxels and tables within 512 KiB, else
 *   MH3D_ERR_UNSUPPORTED_SIZE before any work is issued; other arguments as
 *   for mh3d_plan_create / mh3d_forward.  rho_dev, d_dev and
 *   geom->sensitivity_dev must stay valid until the stream's work for this
 *   call has completed (the kernels read them asynchronously).
 *   Set-up: the first call on each device (with that device current)
 *   resolves the array's address.
 *   Capture: this entry point cannot be captured in a CUDA graph -- each call
 *   uploads its tables from a host buffer freed on return -- and a call on a
 *   capturing stream returns MH3D_ERR_INVALID_ARG without issuing work.
 *   Device-side timeouts (a bounded wait of the passes giving up) are not
 *   reported by this entry point, which has no status word; planned calls
 *   report them as MH3D_ERR_TIMEOUT.
 *   Sharing: all calls on a device share the array; calls whose GPU work
 *   overlaps (other streams, other threads) race and corrupt each other's
 *   results -- serialise them.  Nothing in the array needs to start at zero.
 *   The host table build makes this call far slower than mh3d_forward on a
 *   plan; it is for callers that have no other option. */
mh3d_status mh3d_forward_noalloc(const mh3d_geometry* geom, const float* rho_dev, void* d_dev, void* stream);

/* *norm2 = ||A||_2^2 for b = 1: the largest eigenvalue of A^T A, evaluated
 * in FP64 at plan time from the PSF spectra.  With the separable PSF it is
 * max|Y^|^2 max|Z^|^2 max_m lambda_max(B_m), B_m the s x s alias block
 * (1/s) sum_k conj(X^_k(m + a n/s)) X^_k(m + b n/s) of the drive axis.  The
 * PSF's overall scale is a free constant of the model (the paper drops
 * i 2 pi m f0 / Delta_t and the coil gain), so regularisation weights are
 * most meaningful relative to it. */
mh3d_status mh3d_operator_norm2(mh3d_plan plan, double* norm2);

/* *result = sum_i a_dev[i] b_dev[i] over n >= 0 FP32 device values, computed
 * as every inner product and norm of the solvers (Sec. 4.3; the precision
 * pattern of the CG reductions): each product split exactly into a float
 * pair by FMA, the pairs summed per thread by TwoSum with the rounding
 * errors carried in a low word, the per-thread pairs added as pairs through
 * fixed warp, block and grid trees, and the final pair converted to one FP64
 * value.  Deterministic (no atomics on values).  Uses the plan's reduction
 * workspace, so it must not overlap a solve on the same plan; synchronises
 * `stream`.  n = 0 gives 0 (the pointers may then be NULL);
 * MH3D_ERR_INVALID_ARG for null pointers with n > 0, or n < 0. */
mh3d_status mh3d_dot(mh3d_plan plan, const float* a_dev, const float* b_dev, long long n, double* result,
                     void* stream);

/* Message for the last failing call on `plan` ("" if none; never NULL).
 * With plan == NULL: the message of the calling thread's last failed
 * mh3d_plan_create. */
const char* mh3d_last_error(mh3d_plan plan);

/* Bytes of device workspace the plan holds (tables + solver scratch). */
unsigned long long mh3d_plan_workspace_bytes(mh3d_plan plan);

/* Library version string. */
const char* mh3d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MH3D_H */
