/*
 * skei.h - C ABI of the GB300 (sm_103a) operators inside one sketched
 * Equivariant Imaging (SkEI) step for parallel-beam CT.
 *
 * Paper: "Equivariant Test-Time Training with Operator Sketching for Imaging
 * Inverse Problems" (arXiv 2411.05771).  The operators are those of
 *   Sec. 2.1           y ~ A x; network input A^dagger y (FBP for CT)
 *   Eq. (e:eiloss)     MC term ||y - A F(A^dagger y)||^2 and EI term
 *                      ||T_g F(.) - F(A^dagger A T_g F(.))||^2
 *   Eq. (e:skeiloss), Eq. (e:skeilossttt)
 *                      the same with A_S = S A, y_S = S y, A_S^dagger
 *   Sec. 4.1.1, 4.1.3, 4.2.1
 *                      discrete Radon transform, rotations as the group,
 *                      interleaved angle subsets as the sketch.
 *
 * Discretisation (the paper leaves it open; these readings are fixed here):
 *   image x: N x N, row-major, row 0 at the top; pixel centre
 *     x_j = j - (N-1)/2, y_i = (N-1)/2 - i (pixel units, y up).
 *   detector: n_det unit bins, u_k = k - (n_det-1)/2; ray (theta, k) is the
 *     line x cos(theta) + y sin(theta) = u_k.
 *   A: Joseph's method - along rows when (theta mod 180) lies in [0,45] or
 *     (135,180), along columns otherwise; linear interpolation between the
 *     two nearest pixels of each row (column), zero outside the image,
 *     weighted by 1/|cos| (1/|sin|).
 *   H: Ram-Lak filter h(0)=1/4, h(odd n)=-1/(pi^2 n^2), h(even n)=0, linear
 *     convolution over the detector (zero outside).
 *   B: pixel-driven back-projection, linear interpolation on the bins at
 *     t = x_j cos + y_i sin + (n_det-1)/2.
 *   A_S^dagger = (pi/m) B_S H with m the number of angles in S (FBP).
 *   T_g: counter-clockwise rotation by g degrees about the image centre,
 *     bilinear, zero outside.
 *
 * Conventions for every entry point:
 *   - returns SKEI_OK (0) or a negative status; never throws, never aborts;
 *     skei_last_error() gives a message for the calling thread.
 *   - asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream); no entry point synchronises unless it says so.
 *   - every image / sinogram pointer is a DEVICE pointer owned by the caller,
 *     16-byte aligned, densely packed in the layout stated; `dtype` says how
 *     those buffers are stored (SKEI_F32 = float, SKEI_BF16 = bfloat16
 *     round-to-nearest-even).  Arithmetic is FP32 in every case; loss
 *     reductions are FP64.
 *   - angle index lists (`idx`) are DEVICE int32 arrays of m entries into the
 *     plan's angle list; idx == NULL means all angles in order (then m must
 *     equal n_angles).  Entries outside [0, n_angles) are not dereferenced:
 *     the kernel zeroes that row and records the fault in the plan's status
 *     word (skei_plan_status).
 *   - the library owns only plan objects (angle tables on the device) and
 *     batch objects (task lists, work queues, the batched FBP's workspace)
 *     and allocates nothing else; callers pass workspaces sized by the
 *     *_workspace_size queries.
 *   - results do not depend on the stream or on the launch order of
 *     independent calls; calls that write the same buffer concurrently race.
 *   - each call that does work opens an NVTX range named after it (visible
 *     to Nsight tools; a few nanoseconds when none is attached), except the
 *     allocation-free skei_fbp_noalloc.
 *   - environment: SKEI_AUTOTUNE_CACHE (skei_batch_tune's on-disk cache),
 *     SKEI_FAULT_ALLOC (tests: refuse the n-th device allocation).
 */
#ifndef SKEI_H
#define SKEI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKEI_OK        0
#define SKEI_EINVAL   (-1)  /* bad shape, pointer, alignment, dtype or size   */
#define SKEI_ENOMEM   (-2)  /* a device allocation failed (plans, batches);    */
                            /* SKEI_FAULT_ALLOC=n refuses the n-th one of the */
                            /* process, for tests of the failure paths        */
#define SKEI_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed     */

#define SKEI_F32  0
#define SKEI_BF16 1

/* Maximum image side and detector size accepted by a plan. */
#define SKEI_MAX_N     4096
#define SKEI_MAX_NDET  5800
#define SKEI_MAX_ANGLES 65535

typedef struct skei_plan_s *skei_plan;

/* Library version (major*10000 + minor*100 + patch). */
int skei_version(void);

/* Bounds-check build (no counterpart in the paper: a debugging aid in place
 * of a memory checker).  libskei_check.so is built with SKEI_CHECK = 1: the
 * operator kernels (band, tile and filter kernels) range-check their shared
 * and global indices; an index outside its buffer sets a bit of a device
 * check word and the access is skipped (a load reads 0), nothing traps.
 * skei_check_build returns 1 in that build, 0 otherwise.  skei_check_status
 * synchronises the device and returns the bits seen since the last reset
 * (band kernels: bits 0-7, tile kernels 8-15, filter 16-23; always 0 in the
 * normal build); reset != 0 clears them.  Errors: SKEI_EINVAL (NULL bits),
 * SKEI_ECUDA. */
int skei_check_build(void);
int skei_check_status(unsigned *bits, int reset);

/* Message describing the last failing call on this thread ("" if none).
 * The string stays valid until the next call on this thread. */
const char *skei_last_error(void);

/* ---------------------------------------------------------------- plans --
 * A plan fixes the geometry of A: image side N, detector bins n_det and the
 * full angle list (Sec. 4.1.1: n uniformly spaced views).
 *   N          1..SKEI_MAX_N
 *   n_det      0 selects the smallest odd integer >= N*sqrt(2); otherwise
 *              1..SKEI_MAX_NDET
 *   n_angles   1..SKEI_MAX_ANGLES
 *   angles_deg HOST array of n_angles degrees (any real values), or NULL for
 *              theta_a = 180 a / n_angles.
 * The plan copies the angles, derives its per-angle constants in FP64 and
 * uploads them to the CURRENT device; use it only with that device.
 * Errors: EINVAL for bad sizes or a NULL `out`; ENOMEM / ECUDA on device
 * allocation or copy failure (nothing is leaked). */
int skei_plan_create(int N, int n_det, int n_angles, const double *angles_deg,
                     skei_plan *out);
int skei_plan_destroy(skei_plan plan);
int skei_plan_geometry(skei_plan plan, int *N, int *n_det, int *n_angles);

/* Reads (and, if reset != 0, clears) the plan's device status word: bit 0 is
 * set when a kernel met an angle index outside [0, n_angles).  SYNCHRONISES
 * the device. */
int skei_plan_status(skei_plan plan, int reset, int *word);

/* --------------------------------------------------------------- A, A^T --
 * skei_proj_fwd: sinogram of x on the angle subset S (Sec. 2.3 and 3.1:
 * A_S = S A; Sec. 4.2.1: S selects interleaved angles).
 *   x    [B][N][N]                      (dtype)
 *   out  [B][m][n_det]                  (dtype)
 *        out[b][a][k] = (A x_b)[idx[a]][k]                     if y == NULL
 *        out[b][a][k] = y[b][idx[a]][k] - (A x_b)[idx[a]][k]   otherwise
 *   y    NULL or the FULL measurement [B][n_angles][n_det] (dtype): the
 *        measurement-consistency residual S y - A_S x of Eq. (e:skeiloss).
 * B >= 1, 1 <= m <= n_angles.  x and out must not overlap. */
int skei_proj_fwd(skei_plan plan, int dtype, const void *x, int B,
                  const int *idx, int m, const void *y, void *out, void *stream);

/* skei_proj_adj: x = alpha * A_S^T sino + beta * x, the exact transpose of
 * skei_proj_fwd (the same interpolation weights, gathered per pixel; needed
 * for the gradient of the MC and EI terms, Algorithm 2's update).
 *   sino [B][m][n_det] (dtype);  x [B][N][N] (dtype), read only if beta != 0. */
int skei_proj_adj(skei_plan plan, int dtype, const void *sino, int B,
                  const int *idx, int m, float alpha, float beta, void *x,
                  void *stream);

/* Batched forms: up to SKEI_MAX_JOBS image sets, each with its own
 * buffers, storage types and angle subset, in ONE kernel launch (e.g. the
 * MC-term projection of x1 and the EI-term projection of x2 of a SkEI step).
 * For skei_proj_fwd_multi a job computes out = A_S in, or aux_S - A_S in
 * when aux != NULL (aux = full measurement [B][n_angles][n_det]); alpha and
 * beta are ignored.  For skei_proj_adj_multi a job computes
 * out = alpha A_S^T in + beta aux (aux may alias out; read only if beta != 0).
 * Layouts as for skei_proj_fwd / skei_proj_adj.  The sum of the jobs' B
 * must not exceed 65535. */
#define SKEI_MAX_JOBS 2
typedef struct {
  int dtype_in, dtype_aux, dtype_out;   /* SKEI_F32 or SKEI_BF16 per buffer */
  const void *in;
  const void *aux;
  void *out;
  const int *idx;                       /* DEVICE angle list or NULL (all) */
  int m;                                /* angles in idx */
  int B;                                /* images */
  float alpha, beta;
} skei_job;

int skei_proj_fwd_multi(skei_plan plan, const skei_job *jobs, int njobs,
                        void *stream);
int skei_proj_adj_multi(skei_plan plan, const skei_job *jobs, int njobs,
                        void *stream);

/* Workspace forms of the line-summing operators A (skei_proj_fwd_multi_ws,
 * jobs as for skei_proj_fwd_multi) and B^T (skei_backproject_adj_multi_ws:
 * a job computes out = alpha B_S^T in, in [B][N][N], out [B][m][n_det];
 * aux and beta ignored).  Two launches: every CTA sums a thin band of image
 * lines for a block of angles into `work` (band sums [image][band][angle]
 * [bin], FP32), then the bands are added in a fixed order.  The image lines
 * are staged once per angle block instead of once per angle, which makes
 * these faster than the forms without workspace on large angle sets; the
 * results agree with them to FP32 rounding (different summation order).
 * `work` is a DEVICE buffer of at least skei_band_sums_workspace_size(plan,
 * jobs, njobs) bytes, 16-byte aligned, owned by the caller; calls sharing
 * it must not overlap. */
size_t skei_band_sums_workspace_size(skei_plan plan, const skei_job *jobs, int njobs);
int skei_proj_fwd_multi_ws(skei_plan plan, const skei_job *jobs, int njobs, void *work,
                           size_t work_bytes, void *stream);
int skei_backproject_adj_multi_ws(skei_plan plan, const skei_job *jobs, int njobs, void *work,
                                  size_t work_bytes, void *stream);

/* ---------------------------------------------------- H, B, B^T, FBP --
 * skei_filter: q = scale * H p for `rows` rows of n_det bins (dtype).
 * H is the Ram-Lak ramp of filtered back-projection (Sec. 2.1, 4.1.1); it is
 * symmetric, so it is also its own transpose. */
int skei_filter(skei_plan plan, int dtype, const void *p, int rows, float scale,
                void *q, void *stream);

/* skei_filter_fft: the same linear convolution through the FFT: two rows at a
 * time packed as one complex row, zero padded to the plan's power of two
 * L >= 2 n_det - 1, times the exact spectrum of the taps, inverse FFT.  Equal
 * to skei_filter up to FP32 rounding (not bitwise).  O(L log L) per row pair
 * instead of O(n_det^2) per row; at 725-bin rows the direct form is still
 * faster on GB300.  Plans with n_det < 64 or
 * L > 4096 run the direct form.  p and q must not alias. */
int skei_filter_fft(skei_plan plan, int dtype, const void *p, int rows, float scale,
                    void *q, void *stream);

/* skei_filter_tc: the same linear convolution as the matrix product
 * q = scale P H^T with the Toeplitz H[k][j] = h(|k - j|), on the tensor
 * cores: tiles of 16 rows x 32 outputs, warp-level TF32 MMAs with every FP32
 * operand split into a TF32 head and tail (x = hi + lo; the products
 * hi.hi + hi.lo + lo.hi keep FP32 accuracy).  Equal to skei_filter up to
 * FP32 rounding (not bitwise).  At 120 rows of 725 bins it measured 9.4 us
 * on GB300 against the direct form's 7.9 (staging the rows dominates), so
 * the EI loss keeps the direct form.  Rows of more than 2048 bins run the
 * direct form.  p and q must not alias. */
int skei_filter_tc(skei_plan plan, int dtype, const void *p, int rows, float scale,
                   void *q, void *stream);

/* skei_backproject: x = alpha * B_S q + beta * x (unscaled back-projection).
 *   q [B][m][n_det] (dtype);  x [B][N][N] (dtype). */
int skei_backproject(skei_plan plan, int dtype, const void *q, int B,
                     const int *idx, int m, float alpha, float beta, void *x,
                     void *stream);

/* skei_backproject_adj: q = alpha * B_S^T x, the exact transpose of
 * skei_backproject.  x [B][N][N];  q [B][m][n_det]. */
int skei_backproject_adj(skei_plan plan, int dtype, const void *x, int B,
                         const int *idx, int m, float alpha, void *q,
                         void *stream);

/* Workspace (bytes) for skei_fbp / skei_fbp_adj on B images and m angles. */
size_t skei_fbp_workspace_size(skei_plan plan, int dtype, int B, int m);

/* skei_fbp: x = A_S^dagger sino = (pi/m) B_S H sino - the FBP approximation
 * of the pseudo-inverse (Sec. 2.1; Sec. 3.1 uses it on the sketch).
 *   sino [B][m][n_det];  x [B][N][N];  work >= skei_fbp_workspace_size. */
int skei_fbp(skei_plan plan, int dtype, const void *sino, int B, const int *idx,
             int m, void *x, void *work, size_t work_bytes, void *stream);

/* skei_fbp_adj: sino = (A_S^dagger)^T x = (pi/m) H B_S^T x. */
int skei_fbp_adj(skei_plan plan, int dtype, const void *x, int B,
                 const int *idx, int m, void *sino, void *work,
                 size_t work_bytes, void *stream);

/* -------------------------------------------- FBP without allocation --
 * No counterpart in the paper.  skei_fbp_noalloc computes what skei_fbp
 * computes, but takes no workspace.  It is for callers that cannot call
 * cudaMalloc and so cannot hand skei_fbp its workspace: code whose device
 * memory is all owned by someone else's fixed pool, real-time loops that
 * forbid allocation once they are running, or plugin hosts that give a
 * plugin no allocator.
 *
 * Its scratch (the filtered sinogram, FP32) lives in one static device
 * array inside the library: SKEI_FBP_NOALLOC_MAX_FLOATS floats (4 MiB),
 * held by every GPU that loads the library until the process exits.
 *   - B * m * n_det must not exceed SKEI_FBP_NOALLOC_MAX_FLOATS; a larger
 *     call returns SKEI_EINVAL and launches nothing.
 *   - Every call looks the array's device address up on the current
 *     device (so a device reset between calls is safe); the first call on a
 *     device also loads the library's module there, so make that first call
 *     before any stream capture.
 *   - Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 *     routine runs in this call.
 *   - All calls share the one array and it keeps the last call's contents;
 *     each call writes the part it uses before reading it, so nothing needs
 *     clearing.  Calls that overlap on the GPU (other streams, other host
 *     threads) race on the array: serialise them.
 * Arguments, layouts and other errors are those of skei_fbp. */
#define SKEI_FBP_NOALLOC_MAX_FLOATS 1048576
int skei_fbp_noalloc(skei_plan plan, int dtype, const void *sino, int B,
                     const int *idx, int m, void *x, void *stream);

/* ----------------------------------------------- residual-network step --
 * skei_ttt_residual_step: one iteration of Algorithm 2 (test-time training
 * with the sketched EI loss, Eq. (e:skeilossttt); Eq. (e:skeiloss) over B
 * measurements) for the network F_theta(u) = u + theta, a learnable image
 * residual: the operator launches of skei_ei_loss_fwd, skei_ei_loss_finish
 * and skei_ei_loss_bwd, and Adam (Kingma and Ba; Algorithm 2's optimiser)
 * on theta, with the network folded into them:
 *   x1 = x0 + theta                 (written by the rotation launch)
 *   r, x2, z                        as skei_ei_loss_fwd (mc_idx, sk_idx)
 *   x3 = z + theta                  (the back-projection's second output)
 *   mc, ei, loss, g_x2, g_x3        as skei_ei_loss_finish (lambda, mc_scale)
 *   g_x1 = dL/dx1                   as skei_ei_loss_bwd (g_z = g_x3,
 *                                   mc_coef = mc_scale / B)
 *   theta, m, v                     one Adam step with dL/dtheta =
 *                                   sum_b g_x1[b] + sum_{b,g} g_x3[b][g]
 *                                   (lr, beta1, beta2, eps; *step >= 1, on
 *                                   the device, as skei_adam_step)
 * Every result is bitwise the one of that sequence of calls (with
 * skei_residual_add for F); one measurement (B = 1) takes 9 launches, more
 * measurements 11 (their gradients sum over the images).
 *   x0 [B][N][N], y [B][n_angles][n_det], x1 [B][N][N], r [B][mc_m][n_det],
 *   x2, z, x3, g_x2, g_x3 [B][G][N][N], g_x1 [B][N][N]: dtype; theta, m, v
 *   [N][N] FP32, updated in place; mc_out [B], ei_out [B][G], loss_out [1]
 *   device doubles (each may be NULL); g_deg DEVICE double [B][G];
 *   mc_idx / sk_idx DEVICE int angle lists (NULL: all angles).
 * work: DEVICE, skei_ttt_residual_workspace_size bytes.  Errors as
 * skei_ei_loss_fwd and skei_adam_step. */
size_t skei_ttt_residual_workspace_size(skei_plan plan, int dtype, int B, int G, int mc_m,
                                        int sk_m);
int skei_ttt_residual_step(skei_plan plan, int dtype, const void *x0, float *theta, float *m,
                           float *v, const int *step, const void *y, int B, const int *mc_idx,
                           int mc_m, const int *sk_idx, int sk_m, const double *g_deg, int G,
                           double lambda, double mc_scale, double lr, double beta1, double beta2,
                           double eps, void *x1, void *r, void *x2, void *z, void *x3, void *g_x2,
                           void *g_x3, void *g_x1, double *mc_out, double *ei_out,
                           double *loss_out, void *work, size_t work_bytes, void *stream);

/* ---------------------------------------------------------------- roofs --
 * skei_measure_roofs: measurement, no counterpart in the paper.  Times four
 * microbenchmarks on `stream` and returns the measured peaks that bound the
 * operator kernels (the projectors are bound by FP32 arithmetic and by
 * shared-memory taps, not by HBM or tensor cores):
 *   fp32_flops       FP32 FMA rate, flop/s (one FMA counts 2);
 *   smem_bytes       shared-memory load bandwidth (16-byte loads), bytes/s;
 *   l2_bytes         L2 read bandwidth (a 32 MiB buffer swept 16 times);
 *   dram_read_bytes  DRAM read bandwidth (the rest of `work`, swept once).
 * work: DEVICE scratch of at least SKEI_ROOFS_WORK_BYTES bytes (caller-owned;
 * its contents are read, never trusted).  Synchronises the stream (it waits
 * for its own CUDA events).  Errors: SKEI_EINVAL (NULL out, small or
 * non-device work), SKEI_ECUDA. */
typedef struct {
  double fp32_flops, smem_bytes, l2_bytes, dram_read_bytes;
  int sms;
} skei_roofs;
#define SKEI_ROOFS_L2_BYTES (32u << 20)
#define SKEI_ROOFS_WORK_BYTES (1u << 30)
int skei_measure_roofs(void *work, size_t work_bytes, skei_roofs *out, void *stream);

/* ------------------------------------------------------------ rotations --
 * skei_rotate: out[b][g] = T_{g_deg[b][g]} x[b] (Sec. 4.1.3: the transform
 * group of CT is rotations; Eq. (e:eiloss) applies T_i to F(A^dagger y)).
 *   x [B][N][N]; out [B][G][N][N] (dtype); g_deg DEVICE double [B][G]. */
int skei_rotate(int dtype, const void *x, int B, int N, const double *g_deg,
                int G, void *out, void *stream);

/* skei_rotate_adj: gx[b] = alpha * sum_g T_{g_deg[b][g]}^T gout[b][g]
 *                          + beta * gx[b]   (exact transpose, gathered). */
int skei_rotate_adj(int dtype, const void *gout, int B, int N,
                    const double *g_deg, int G, float alpha, float beta,
                    void *gx, void *stream);

/* The same for images of Ch channels rotated alike (e.g. the real and
 * imaginary planes of a complex MRI image): x [B][Ch][N][N] ->
 * out [B][G][Ch][N][N]; gout [B][G][Ch][N][N] -> gx [B][Ch][N][N].
 * B G Ch <= 65535. */
int skei_rotate_channels(int dtype, const void *x, int B, int Ch, int N,
                         const double *g_deg, int G, void *out, void *stream);
int skei_rotate_adj_channels(int dtype, const void *gout, int B, int Ch, int N,
                             const double *g_deg, int G, float alpha, float beta,
                             void *gx, void *stream);

/* ------------------------------------------------- fused EI / SkEI loss --
 * The loss of Eq. (e:skeiloss) / (e:skeilossttt), split around the caller's
 * network F, for B measurements and G rotations each:
 *   x1 = F(A^dagger y)                              (caller)
 *   skei_ei_loss_fwd:    r  = S_mc y - A_mc x1      [B][mc_m][n_det]
 *                        x2 = T_g x1                [B][G][N][N]
 *                        z  = A_S^dagger A_S x2     [B][G][N][N]
 *   x3 = F(z)                                       (caller)
 *   skei_ei_loss_finish: mc_b  = mc_scale ||r_b||^2
 *                        ei_bg = ||x2_bg - x3_bg||^2
 *                        loss  = (1/B) sum_b [mc_b + (lambda/G) sum_g ei_bg]
 *                        g_x2 = dloss/dx2 = 2 lambda/(B G) (x2 - x3) = -g_x3
 *   g_z = (dF/dz)^T g_x3                            (caller)
 *   skei_ei_loss_bwd:    g_x1 = -2 mc_coef A_mc^T r
 *                               + sum_g T_g^T [g_x2 + (pi/m) A_S^T H B_S^T g_z]
 * mc_idx/mc_m select the angles of the MC term (NULL = all), sk_idx/sk_m the
 * sketch S of the EI term (NULL = all: plain EI).  mc_scale multiplies a
 * sketched MC term (n/m makes it unbiased, Sec. 3.1's E(S^T S) = I).  With
 * loss as above, mc_coef = mc_scale / B.  All outputs are in `dtype` except
 * mc_out [B], ei_out [B][G] and loss_out [1], which are DEVICE doubles. */
size_t skei_ei_workspace_size(skei_plan plan, int dtype, int B, int G, int mc_m,
                              int sk_m);

/* Host-only query: the form skei_ei_loss_fwd (per_sample = 0) or
 * skei_ei_loss_fwd_per_sample (per_sample = 1) gives its fused A launch for
 * these arguments (the angle-list pointers are compared, not read):
 * 1 = per-band sums in the workspace, then their ordered reduction (two
 * launches, the kernels of skei_proj_fwd_multi_ws on the same two jobs);
 * 0 = the cluster form (one launch, those of skei_proj_fwd_multi).  The
 * band-sums form is taken for launches of many image-angles, and where the
 * MC and EI terms share one angle list with G = 4 (the MC image then rides
 * in the CTAs of the EI group's four images).  Returns SKEI_EINVAL on bad
 * arguments. */
int skei_ei_fwd_form(skei_plan plan, int B, int G, const int *mc_idx, int mc_m,
                     const int *sk_idx, int sk_m, int per_sample);

int skei_ei_loss_fwd(skei_plan plan, int dtype, const void *x1, const void *y,
                     int B, const int *mc_idx, int mc_m, const int *sk_idx,
                     int sk_m, const double *g_deg, int G, void *r, void *x2,
                     void *z, void *work, size_t work_bytes, void *stream);

/* Workspace (bytes) of skei_ei_loss_finish; skei_ei_workspace_size(...)
 * with the same B, G and sizes is never smaller. */
size_t skei_ei_finish_workspace_size(int B, int G, int N, int r_len);

int skei_ei_loss_finish(int dtype, const void *x2, const void *x3,
                        const void *r, int B, int G, int N, int r_len,
                        double lambda, double mc_scale, double *mc_out,
                        double *ei_out, double *loss_out, void *g_x2, void *g_x3,
                        void *work, size_t work_bytes, void *stream);

/* The same for transformed images of img_len values each (x2, x3
 * [B][G][img_len]; e.g. 2 N^2 for a planar complex image). */
size_t skei_ei_finish_len_workspace_size(int B, int G, int64_t img_len, int r_len);
int skei_ei_loss_finish_len(int dtype, const void *x2, const void *x3, const void *r, int B,
                            int G, int64_t img_len, int r_len, double lambda,
                            double mc_scale, double *mc_out, double *ei_out,
                            double *loss_out, void *g_x2, void *g_x3, void *work,
                            size_t work_bytes, void *stream);

/* g_x2 and g_z may be NULL (treated as zero). */
int skei_ei_loss_bwd(skei_plan plan, int dtype, const void *r, const void *g_x2,
                     const void *g_z, int B, const int *mc_idx, int mc_m,
                     const int *sk_idx, int sk_m, const double *g_deg, int G,
                     double mc_coef, void *g_x1, void *work, size_t work_bytes,
                     void *stream);

/* The same with an angle list per measurement (Algorithm 1: a sketch S_k
 * drawn for every sample y_j): mc_idx and sk_idx, where not NULL, are DEVICE
 * int32 [B][mc_m] and [B][sk_m]; measurement b uses row b for its MC term and
 * for the EI term of its G transformed images.  The loss is the mean of the
 * per-measurement losses, so skei_ei_loss_finish is unchanged; workspace,
 * layouts and errors are those of skei_ei_loss_fwd / skei_ei_loss_bwd.  The
 * kernels group each measurement's G images as with a shared sketch (groups
 * of 4 need G % 4 == 0; other G run single images). */
int skei_ei_loss_fwd_per_sample(skei_plan plan, int dtype, const void *x1, const void *y,
                                int B, const int *mc_idx, int mc_m, const int *sk_idx,
                                int sk_m, const double *g_deg, int G, void *r, void *x2,
                                void *z, void *work, size_t work_bytes, void *stream);
int skei_ei_loss_bwd_per_sample(skei_plan plan, int dtype, const void *r, const void *g_x2,
                                const void *g_z, int B, const int *mc_idx, int mc_m,
                                const int *sk_idx, int sk_m, const double *g_deg, int G,
                                double mc_coef, void *g_x1, void *work, size_t work_bytes,
                                void *stream);

/* ------------------------------------------ stand-in network utilities --
 * Not operators of the paper: the residual stand-in network
 * F_theta(u) = u + theta used by the benchmark's test-time-training loop,
 * and the Adam update of Algorithm 2 (Sec. 4.1.3: Adam, lr 5e-4).
 *
 * skei_residual_add: out[c][i] = u[c][i] + theta[i], c < count, i < n.
 *   u, out: dtype; theta: float. */
int skei_residual_add(int dtype, const void *u, const float *theta, int count,
                      int64_t n, void *out, void *stream);

/* skei_step_draws: the draws of one iteration from a resident table.
 * Algorithm 2 draws a sketch and G rotation angles every iteration; with
 * the draws of K iterations resident as rows of `table` [n_rows][row_bytes]
 * (DEVICE), this copies row *counter to dst (DEVICE, row_bytes) and
 * advances *counter (DEVICE int) by one, in stream order, so that a captured
 * step graph replays K iterations, each with its own draws, without a host
 * copy.  A counter outside [0, n_rows) copies nothing and is set to -1
 * (sticky: the caller reads it back after the run).  One CTA; 16-byte words
 * where row_bytes and both pointers allow.  Returns SKEI_EINVAL for NULL or
 * misaligned pointers, n_rows < 1 or row_bytes < 1. */
int skei_step_draws(const void *table, int n_rows, int64_t row_bytes, int *counter,
                    void *dst, void *stream);

/* skei_adam_step: g[i] = sum_{c<c1} g1[c][i] + sum_{c<c2} g2[c][i] (g1, g2 in
 * dtype; g2 may be NULL with c2 = 0), then one Adam update of theta, m, v
 * (float, n entries) with bias correction for the step number *step (DEVICE
 * int, >= 1; read, not modified). */
int skei_adam_step(float *theta, int64_t n, int dtype, const void *g1, int c1,
                   const void *g2, int c2, float *m, float *v, const int *step,
                   double lr, double beta1, double beta2, double eps,
                   void *stream);

/* ------------------------------------------ batch-norm layers (Sec. 3.3) --
 * The layers that BN-only test-time training adapts: normalisation with the
 * statistics of the current batch, then the learnable affine map (scale =
 * theta_1, shift = theta_2 of Sec. 3.3), then an optional ReLU.  For channel
 * c of v [B][C][HW] (B images of C channels of HW values, contiguous), over
 * its M = B HW values:
 *   mean_c = (1/M) sum v,  var_c = (1/M) sum (v - mean_c)^2 (biased),
 *   rstd_c = 1 / sqrt(var_c + eps),
 *   out = act(scale_c (v - mean_c) rstd_c + shift_c),  act = ReLU (relu != 0)
 *         or the identity.
 * skei_bn_act_fwd writes out (dtype, same layout as v) and the FP32 mean_c,
 * rstd_c it used (device [C], kept for the backward).
 * skei_bn_act_bwd takes the forward's v, mean, rstd and the gradient g_out of
 * out, and writes g_v (dtype, layout of v) and the FP32 per-channel
 * gradients g_scale = sum g_y (v - mean) rstd and g_shift = sum g_y, where
 * g_y = g_out where the activation passes (y > 0 for ReLU, y = the affine
 * map's output) and 0 elsewhere;
 *   g_v = scale rstd (g_y - g_shift / M - (v - mean) rstd g_scale / M).
 * Sums are reduced in a fixed order (FP32 within a warp, FP64 beyond), so
 * results are deterministic.  scale, shift, mean, rstd, g_scale, g_shift are
 * device float[C].  work: device workspace of at least
 * skei_bn_workspace_size(B, C, HW) bytes, 16-byte aligned, owned by the
 * caller.  Errors: SKEI_EINVAL for B, C or HW < 1, C > 65535, eps <= 0, a
 * NULL or host pointer, or too small a workspace. */
size_t skei_bn_workspace_size(int B, int C, int64_t HW);
int skei_bn_act_fwd(int dtype, const void *v, int B, int C, int64_t HW, const float *scale,
                    const float *shift, int relu, double eps, void *out, float *mean,
                    float *rstd, void *work, size_t work_bytes, void *stream);
int skei_bn_act_bwd(int dtype, const void *v, const void *g_out, int B, int C, int64_t HW,
                    const float *scale, const float *shift, const float *mean,
                    const float *rstd, int relu, void *g_v, float *g_scale, float *g_shift,
                    void *work, size_t work_bytes, void *stream);

/* ------------------------------------- multi-coil MRI (Sec. 3.4, Eq. (e:mri)) --
 * The forward model of the coil-sketched EI: k = M F (C x) for N_c coils,
 *   k_c[u][v] = M[u][v] (1/N) sum_{p,q} C_c[p][q] x[p][q] e^{-2 pi i (u p + v q) / N}
 * (unitary 2D DFT, frequency 0 at index 0, no shift; M a 0/1 mask shared by
 * the coils), its adjoint x = sum_c conj(C_c) F^H (M k_c), and the
 * coil-combined inverse A^dagger k = dinv * A^H k with dinv = 1 / sum_c |C_c|^2
 * (0 where that sum is 0).  A coil sketch (PCA virtual coils, then
 * S_c = [I_R 0; 0 S_low]) is a set of maps with fewer coils: the same calls
 * with the sketched maps (skei_coil_mix forms them, and the sketched data).
 *
 * All complex arrays are FP32 planar: image x [B][2][N][N] (real plane,
 * imaginary plane), k-space [B][N_c][2][N][N], maps [N_c][2][N][N]; mask and
 * dinv are real [N][N] (mask NULL = every sample taken).  N is a power of two
 * in [8, 256]; 1 <= N_c <= 64.  work: a device workspace of at least
 * skei_mri_workspace_size(N, Nc, B) bytes (16-byte aligned, owned by the
 * caller).  Errors: SKEI_EINVAL for bad sizes, NULL or host pointers or too
 * small a workspace.
 *
 * skei_mri_fwd: k = alpha (aux - M F (C (w x))) with aux (same layout as k;
 *   may be k itself), else alpha M F (C (w x)), w a real [N][N] weight on the
 *   image (xw; NULL = 1): the MC residual y - A x in one call, and A (dinv g)
 *   for the transpose of A^dagger A.
 * skei_mri_adj: x = alpha dinv sum_c conj(C_c) F^H (M k_c) + beta x (dinv NULL:
 *   the adjoint A^H; the per-coil images are summed in coil order).
 * skei_mri_dinv: dinv from the maps.
 * skei_coil_mix: out[b][j] = sum_i W[j][i] in[b][i] for complex weights W
 *   (device float [n_out][n_in][2]) and planar coil data in [B][n_in][2][plane],
 *   out [B][n_out][2][plane] (no aliasing); n_in, n_out <= 64. */
size_t skei_mri_workspace_size(int N, int Nc, int B);
int skei_mri_fwd(int N, int Nc, int B, const float *x, const float *maps, const float *mask,
                 const float *xw, const float *aux, float alpha, float *k, void *work,
                 size_t work_bytes, void *stream);
int skei_mri_adj(int N, int Nc, int B, const float *k, const float *maps, const float *mask,
                 const float *dinv, float alpha, float beta, float *x, void *work,
                 size_t work_bytes, void *stream);
int skei_mri_dinv(int N, int Nc, const float *maps, float *dinv, void *stream);
int skei_coil_mix(int plane, int B, int n_in, int n_out, const float *W, const float *in,
                  float *out, void *stream);

/* ------------------------------------------------ batched schedule --
 * One operator applied to many instances in one persistent launch per
 * kernel: images of different sizes (each item its own plan), each with its
 * own sketch S_k and its own storage type.  Eq. (e:skeiloss) and Algorithm 2
 * draw a sketch per sample and step; a batch runs all of them at once.
 *
 *   SKEI_BATCH_PROJ_FWD        out = scale A_S in      in [B][N][N], out [B][m][n_det]
 *   SKEI_BATCH_PROJ_ADJ        out = scale A_S^T in    in [B][m][n_det], out [B][N][N]
 *   SKEI_BATCH_BACKPROJECT     out = scale B_S in      in [B][m][n_det], out [B][N][N]
 *   SKEI_BATCH_BACKPROJECT_ADJ out = scale B_S^T in    in [B][N][N], out [B][m][n_det]
 *   SKEI_BATCH_FILTER          out = scale H in        in, out [B][m][n_det]
 *   SKEI_BATCH_FBP             out = scale (pi/m) B_S H in  (Sec. 2.1), two
 *                              persistent launches (filter, back-projection)
 *
 * Results are bitwise equal to the single-instance entry points on the same
 * item (each output element is computed by one task, in the same order).
 *
 * skei_batch_create validates every item (as the single-instance calls do)
 * and uploads the task list; it allocates the task list, a 2-int work queue
 * per launch and, for SKEI_BATCH_FBP, an FP32 workspace of sum(B m n_det)
 * floats.  It synchronises (host-to-device copies).  The item pointers are
 * baked into the batch: the buffers and plans must outlive it, and their
 * contents may change between runs.
 * skei_batch_run issues the launches on `stream` (asynchronous; it may be
 * captured in a CUDA graph and replayed).  Runs of one batch must not
 * overlap: each launch takes tasks from the batch's own work queue, which
 * its last worker resets for the next run.
 * skei_batch_tune(b, reps, stream) runs every candidate shape (angles per
 * task 1..8 for A and B^T; 1..max resident CTAs per SM for the others)
 * reps + 1 times on the items' own buffers (overwriting the outputs), times
 * them with events on `stream`, and keeps the fastest.  It synchronises and
 * returns SKEI_EINVAL inside a stream capture.  With the environment variable
 * SKEI_AUTOTUNE_CACHE naming a file, a launch phase whose signature (device
 * name and SM count, phase kernel, every item's N, n_det, n_angles, m, B and
 * storage types) the file records takes the recorded shape without timing,
 * and newly tuned phases are appended to it (text, one line per phase; a
 * file that cannot be read or written is skipped).
 * skei_batch_info(b, phase, ...) reports launch `phase` (0, or 1 for the
 * back-projection of SKEI_BATCH_FBP): the number of launches, tasks, workers
 * (CTAs, or 8-CTA clusters for A and B^T) and the block (angles per task for
 * A and B^T, CTAs per SM otherwise, 0 = all that fit).
 */
#define SKEI_BATCH_PROJ_FWD 0
#define SKEI_BATCH_PROJ_ADJ 1
#define SKEI_BATCH_BACKPROJECT 2
#define SKEI_BATCH_BACKPROJECT_ADJ 3
#define SKEI_BATCH_FILTER 4
#define SKEI_BATCH_FBP 5
#define SKEI_MAX_BATCH_ITEMS 65536

typedef struct {
  skei_plan plan;      /* geometry of this item; several items may share one */
  int dtype_in;        /* SKEI_F32 / SKEI_BF16 storage of in */
  int dtype_out;       /* ... of out */
  const void *in;      /* device, layout per operator above */
  void *out;           /* device, must not overlap another item's out */
  const int *idx;      /* device int32[m] rows of the plan's angles, or NULL */
  int m;               /* sketch size (n_angles when idx is NULL) */
  int B;               /* images in this item */
  float scale;         /* output scale (1 for the plain operator) */
} skei_batch_item;

typedef struct skei_batch_s *skei_batch;

int skei_batch_create(int op, const skei_batch_item *items, int n_items, skei_batch *out);
int skei_batch_run(skei_batch batch, void *stream);
int skei_batch_tune(skei_batch batch, int reps, void *stream);
int skei_batch_info(skei_batch batch, int phase, int *n_phases, int *n_tasks, int *workers,
                    int *block);
int skei_batch_destroy(skei_batch batch);

#ifdef __cplusplus
}
#endif
#endif /* SKEI_H */
