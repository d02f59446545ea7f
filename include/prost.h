/*
 * prost.h -- C ABI of the GB300 implementation of pROST's per-frame update
 * (Seidel, Hage, Kleinsteuber, arXiv:1302.2073).
 *
 * One handle tracks one video stream: a subspace U (m x k, orthonormal
 * columns, Eq. stiefeldef), the coefficients y of the last frame and the
 * labels of the last frame (which become the weights of the next, Eq.
 * pixelweighting).  prost_step() runs Steps 1-3 of Section 3.3 for one frame
 * on the GPU:
 *   Step 1  y = argmin_y h_{mu,w}(x - U y)            (Eq. onlinestep1)
 *           by n_cg nonlinear conjugate-gradient iterations (Polak-Ribiere+,
 *           majorise-minimise line step), warm-started at the previous y;
 *   Step 2  one geodesic step on the Grassmannian along the projected
 *           rank-one gradient pi(eta) y^T (Eqs. gproject, svd, geodesic) with
 *           t = max(exp(-tau i) t_init, t_min) (Section 3.4);
 *   Step 3  pixel labels  F_q = [max_c |x_{c,q} - u_{c,q}^T y| >= delta]
 *           (Section 3.4) and weights w_q = omega if F_q else 1 for the next
 *           frame (Eq. pixelweighting).
 * The cost is the weighted smoothed l_p norm of the residual,
 *   h_{mu,w}(x - U y) = sum_e w_e ((x_e - u_e^T y)^2 + mu)^(p/2)
 * (Eqs. smoothlpnorm, weightedLPnorm, spcacost).  After each frame the
 * representative U is re-orthonormalised by Cholesky-QR (U <- U R^{-1},
 * y <- R y); this is not in the paper and is the identity in exact arithmetic.
 * prost_step_many() runs the same steps for n consecutive frames of the
 * stream (in one launch where the kernel form allows, U staying on chip
 * between the frames) with the results of n prost_step() calls.
 *
 * Layouts.  A frame is channel-planar: channels planes of height x width
 * pixels, row-major, so entry e = c*P + q for pixel q of channel c (the colour
 * stacking x = [x_R; x_G; x_B] of Section 3.4), m = channels*P.  Frames are
 * uint8 or float32 (prost_params.frame_dtype); the entry used by the method is
 * x_e = in_scale * frame_e - in_offset.  Subspaces cross the ABI as float32
 * m x k row-major (row e is u_e^T); y as k doubles.  Labels/masks are P bytes,
 * 1 = foreground.
 *
 * Streams and memory.  prost_init() takes a cudaStream_t (as void*; NULL is
 * the legacy default stream) on which every later call is ordered.  The
 * library allocates and owns its device state (released by prost_destroy());
 * the caller owns every buffer it passes.  Calls with on_device = 0 take host
 * pointers, copy through the stream and return after the stream has
 * synchronised.  Calls with on_device = 1 take device pointers of the current
 * device and only enqueue work; errors found on the device (a frame with a
 * non-finite entry, a Gram matrix that is not positive definite) are then
 * reported by prost_sync() or prost_get_stats().  A handle is not thread safe.
 *
 * Errors.  Every int-returning call returns PROST_OK (0) or a negative code
 * below; prost_strerror() names it and prost_last_error() gives the detail of
 * the last failure on a handle.  A call that fails with PROST_EINVAL changes
 * nothing.
 */
#ifndef PROST_H
#define PROST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PROST_OK 0
#define PROST_EINVAL (-1)     /* bad argument or parameter; nothing changed */
#define PROST_ENOMEM (-2)     /* device or host allocation failed */
#define PROST_ECUDA (-3)      /* a CUDA call failed; see prost_last_error() */
#define PROST_EBADFRAME (-4)  /* frame had a non-finite entry; the frame was skipped,
                                 state (U, y, labels, frame counter) unchanged */
#define PROST_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define PROST_ENOTSPD (-6)    /* Gram matrix of the subspace not positive definite;
                                 the previous re-orthonormalisation is kept */

#define PROST_U8 0   /* frame entries uint8 */
#define PROST_F32 1  /* frame entries float32; subspace storage float32 */
#define PROST_BF16 2 /* subspace storage bfloat16 (u_dtype only): not in the paper.
                      * The stored rows are rounded stochastically at every
                      * update (unbiased, so that updates below half an ulp are
                      * not lost), all arithmetic stays FP32 with the k x k
                      * Cholesky-QR at FP64 accuracy, and the subspace streams
                      * at half the bytes.  The results differ from the FP32
                      * storage by the rounding; the error against the FP64
                      * reference is a measured quantity, not a bound. */

#define PROST_MASK_POST_UPDATE 0 /* Step 3 uses the subspace after Step 2 (default) */
#define PROST_MASK_PRE_UPDATE 1  /* Step 3 uses the subspace before Step 2 */

/* Kernel forms of a frame (not in the paper; the results agree within the
 * parity tolerances, the summation orders differ).  GRID: one cooperative
 * launch of one CTA per SM with bounded grid barriers in global memory.
 * CLUSTER: one thread-block cluster of up to 16 CTAs whose barriers are the
 * hardware cluster barrier, for small subspaces where the grid barriers of
 * many CTAs would cost more than the streaming.  AUTO picks CLUSTER when the
 * stored subspace takes at most PROST_CLUSTER_MAX_U_BYTES and a cluster fits
 * the device, else GRID.  PASSES: the frame as a sequence of ordinary
 * launches, one per pass over the rows (two per CG iteration: the gradient,
 * then the curvature sum_e c_e (u_e^T d)^2 of the line step), with k chosen at
 * run time; float32 storage only.  GRID and CLUSTER exist for
 * k <= PROST_MAX_K_SINGLE; PASSES for every k and the only form above it, which
 * AUTO then picks.  RESIDENT (k <= 10): the GRID form with each CTA owning
 * a range of pixels of every channel, whose rows, frame entries and labels it
 * keeps in shared memory after the first pass of a frame, so that the later
 * passes stream from there and only the rows that do not fit come from L2
 * again; AUTO picks it over GRID when at least half of the rows fit.
 * Failure injection (prost_inject_*) needs GRID or RESIDENT. */
#define PROST_FORM_AUTO 0
#define PROST_FORM_GRID 1
#define PROST_FORM_CLUSTER 2
#define PROST_FORM_PASSES 3
#define PROST_FORM_RESIDENT 4
#define PROST_CLUSTER_MAX_U_BYTES (1u << 20)

#define PROST_MAX_K 32        /* largest subspace dimension (PASSES form above PROST_MAX_K_SINGLE) */
#define PROST_MAX_K_SINGLE 16 /* largest k of the single-launch forms (GRID, CLUSTER) */
#define PROST_STATIC_MAX_K 16 /* largest k of prost_cost_grad_static() */
#define PROST_MAX_CG 32

typedef struct prost_handle prost_handle;

typedef struct prost_params {
    int32_t width, height, channels; /* frame size; m = channels*width*height, channels <= 4 */
    int32_t k;                       /* subspace dimension, 1 <= k <= min(m, PROST_MAX_K) */
    double p;                        /* l_p exponent, 0 < p <= 2 (Eq. smoothlpnorm; p >= 1 as in Section 5.3) */
    double mu;                       /* smoothing, mu > 0; 0 selects delta^2 (1 - p) (Eq. opt_mu2, needs p < 1) */
    double delta;                    /* label threshold, delta > 0 */
    double omega;                    /* weight of pixels labelled foreground, 0 <= omega <= 1 */
    double t_init, t_min;            /* step sizes, > 0 (Section 3.4) */
    int32_t i_init;                  /* frames of the initialisation phase, >= 1: tau = ln(t_init/t_min)/i_init */
    int32_t n_cg;                    /* CG iterations per frame, 0 <= n_cg <= PROST_MAX_CG (paper: 5) */
    double in_scale, in_offset;      /* x = in_scale * frame - in_offset */
    int32_t frame_dtype;             /* PROST_U8 or PROST_F32 */
    int32_t u_dtype;                 /* PROST_F32 or PROST_BF16 (subspace storage) */
    int32_t mask_from;               /* PROST_MASK_POST_UPDATE or PROST_MASK_PRE_UPDATE */
    int32_t form;                    /* kernel form: PROST_FORM_AUTO (0), PROST_FORM_GRID, PROST_FORM_CLUSTER,
                                        PROST_FORM_PASSES or PROST_FORM_RESIDENT */
    uint64_t seed;                   /* seed of the random initial subspace (Section 3.4) */
} prost_params;

typedef struct prost_stats {
    int64_t frames;                  /* frames processed (the step counter i of the next frame) */
    int64_t bad_frames;              /* frames skipped as PROST_EBADFRAME since init */
    int32_t n_cg;                    /* CG iterations of the last frame */
    int32_t status;                  /* status of the last frame (PROST_OK, PROST_EBADFRAME, ...) */
    double cost[PROST_MAX_CG + 1];   /* h_{mu,w}(x - U y_j) at each CG iterate j = 0..n_cg */
    double gnorm[PROST_MAX_CG + 1];  /* |grad_y h| at each CG iterate */
    double alpha[PROST_MAX_CG];      /* line step of CG iteration j */
    double beta[PROST_MAX_CG + 1];   /* PR+ coefficient at iterate j (beta[0] = 0; beta[n_cg] unused by Step 1) */
    double pi_norm;                  /* |pi(eta)| at the final y (Eq. gproject) */
    double y_norm;                   /* |y| */
    double sigma;                    /* sigma_1 = |pi(eta)| |y| (Eq. svd) */
    double t;                        /* step size of the frame */
    double theta;                    /* geodesic angle sigma_1 t; 0 when the step was skipped */
    int32_t updated;                 /* 0 when |y| = 0 or |pi(eta)| = 0 skipped Step 2 */
    int32_t pad0;
    int64_t n_foreground;            /* pixels labelled foreground in the last frame */
    double orth_err;                 /* max |U^T U - I| of the stored subspace before its
                                        re-orthonormalisation at the end of the last frame */
    double eta_norm;                 /* |eta| at the final y (Section 3.3) */
    int32_t pi_explicit;             /* 1 when |pi(eta)| was formed as sum_e (eta_e - u_e^T g)^2
                                        by an extra pass over U: the identity
                                        |pi(eta)|^2 = |eta|^2 - |U^T eta|^2 (Eq. gproject)
                                        loses its digits when |pi(eta)|^2 < |eta|^2 / 4 */
    int32_t form;                    /* PROST_FORM_GRID, PROST_FORM_CLUSTER, PROST_FORM_PASSES or
                                        PROST_FORM_RESIDENT: the handle's form */
} prost_stats;

/* Sizes of the device state of a handle with these parameters (bytes, device
 * memory).  Returns PROST_EINVAL for bad parameters. */
int prost_state_bytes(const prost_params *prm, size_t *bytes);

/* Create a stream tracker.  Validates prm, allocates the device state, draws
 * the initial subspace as the orthonormal factor of a seeded Gaussian m x k
 * matrix (Section 3.4, "Initialization"), sets y = 0, all labels background
 * and the frame counter to 0.  stream: cudaStream_t as void* (NULL = default
 * stream).  On success *out owns the state until prost_destroy(). */
int prost_init(const prost_params *prm, void *stream, prost_handle **out);

/* Process one frame (Steps 1-3).  frame: m entries of prm.frame_dtype,
 * channel-planar.  mask_out (nullable): P bytes, this frame's labels.
 * background_out (nullable): m floats, U y + in_offset with the subspace the
 * labels used (the reconstruction in the units of in_scale*frame).
 * on_device = 1: all three are device pointers and the call only enqueues the
 * work on the handle's stream (returns PROST_OK; device-detected errors are
 * reported by prost_sync()).  on_device = 0: all three are host pointers; the
 * frame is copied to the device and the call returns the frame's status after
 * the stream synchronised, with the outputs copied back only for a frame that
 * completed (PROST_OK, PROST_ENOTSPD).  A frame with a non-finite entry
 * (float32 frames only) leaves the state unchanged and, on the host path, its
 * outputs unwritten (PROST_EBADFRAME); so does a frame refused or aborted by a
 * bounded device-side wait (PROST_ETIMEOUT). */
int prost_step(prost_handle *h, const void *frame, int on_device, uint8_t *mask_out,
               float *background_out);

/* Process n consecutive frames of the stream (Steps 1-3 of Section 3.3 for
 * each in turn, the same results as n calls of prost_step()).  frames: n
 * frames of m entries each, one after another; masks_out (nullable): n * P
 * bytes, frame i's labels at i * P.  No background output.  In the resident
 * form the frames of each rebase period run in one launch, whose CTAs keep
 * their rows and labels in shared memory from one frame to the next, so only
 * the first frame of the launch reads the subspace from global memory; the
 * other forms make one launch per frame.  on_device = 1: device pointers,
 * enqueue only (PROST_OK; device-detected errors by prost_sync()); frames
 * whose planes do not start on 16-byte boundaries are first copied to a
 * staging buffer that the handle allocates on first use and keeps.
 * on_device = 0: host pointers, copied through that buffer; returns the last
 * frame's status after the stream synchronised, with the masks copied back
 * only when it completed (PROST_OK, PROST_ENOTSPD); a rejected frame before it
 * (PROST_EBADFRAME) is reported by prost_sync().  A wait that runs out aborts
 * the rest of the launch (PROST_ETIMEOUT, masks of the aborted frames
 * unwritten).  Errors: PROST_EINVAL (NULL handle or frames, n < 1, frames of
 * prost_step_async() in flight), PROST_ENOMEM, PROST_ECUDA. */
int prost_step_many(prost_handle *h, const void *frames, int32_t n, int on_device, uint8_t *masks_out);

/* Pipelined host frames (not in the paper).  prost_step_async() enqueues one
 * frame from host memory and returns without waiting: the frame is copied in
 * on a copy stream of the handle while the previous frame's kernel runs, the
 * frame's kernel runs on the handle's stream, and its labels (mask_out, P
 * bytes, nullable) and background (background_out, m floats, nullable) are
 * copied out on a second copy stream while the next frame's kernel runs.  All
 * three buffers are host memory that must stay valid, and frame unchanged,
 * until prost_wait() has returned this frame; page-locked memory lets the
 * copies overlap the kernels.  At most two frames are in flight: a third call
 * returns PROST_EINVAL.  prost_wait() waits for the oldest frame in flight and
 * returns its status (PROST_OK, PROST_EBADFRAME, PROST_ETIMEOUT or
 * PROST_ENOTSPD; PROST_EINVAL when none is in flight); the outputs of a frame
 * whose status is not PROST_OK or PROST_ENOTSPD hold no meaningful values.
 * prost_step() refuses (PROST_EINVAL) while such frames are in flight; the
 * other calls work on the handle's stream, ordered after the kernels. */
int prost_step_async(prost_handle *h, const void *frame, uint8_t *mask_out, float *background_out);
int prost_wait(prost_handle *h);

/* Pipelined host calls of n frames (not in the paper): prost_step_many() as a
 * prost_step_async() call.  frames: n * m host entries, one frame after
 * another; masks_out (nullable): n * P host bytes.  The frames are copied in
 * on the handle's copy stream while the previous call's kernels run, the
 * frames run as prost_step_many() runs them (one launch per rebase period in
 * the resident form), and the masks are copied out while the next call's
 * kernels run.  Each call takes one of the two slots that prost_step_async()
 * uses (at most two calls of either kind in flight), and prost_wait() returns
 * the status of its last frame; a rejected frame before it is reported by
 * prost_sync().  The handle keeps device room for the largest n seen per slot
 * (allocated on demand; growing a slot first waits for the call that used it
 * two calls before).  Buffers stay owned by the caller and must stay valid,
 * frames unchanged, until prost_wait() has returned the call; page-locked
 * memory lets the copies overlap the kernels.  Errors: PROST_EINVAL (NULL
 * handle or frames, n < 1, two calls in flight), PROST_ENOMEM, PROST_ECUDA. */
int prost_step_many_async(prost_handle *h, const void *frames, int32_t n, uint8_t *masks_out);

/* Synchronise the handle's stream.  Returns PROST_EBADFRAME if a frame was
 * skipped since the previous prost_sync(), PROST_ENOTSPD / PROST_ETIMEOUT if
 * one of those was raised, else PROST_OK, and clears these flags. */
int prost_sync(prost_handle *h);

/* Fault injection for failure-detection tests, on the host (not in the
 * paper).  Moves the handle's grid-barrier count by delta, as a frame launch
 * that gave up part-way leaves it.  The next frame launch finds the count
 * outside the range it expects and returns at once, leaving the state
 * untouched; on the host path prost_step() returns PROST_ETIMEOUT and leaves
 * its outputs unwritten.  Grid and resident forms only (PROST_EINVAL for the
 * cluster and passes forms, which have no software grid barrier).  The following prost_sync() reports PROST_ETIMEOUT
 * and resets the barrier, and later frames run normally (the refused frame
 * does not count towards the periodic rebase).  A launch can only detect a
 * backward skew (delta < 0) or a forward one of at least the frame kernel's
 * grid size: a smaller forward skew looks like CTAs that already arrived, so
 * 0 < delta < grid size returns PROST_EINVAL.  Synchronises the stream.
 * Errors: PROST_EINVAL (NULL handle, undetectable delta), PROST_ECUDA. */
int prost_inject_barrier_skew(prost_handle *h, int64_t delta);

/* Fault injection for failure-detection tests (not in the paper): the next
 * frame launch, at the grid barrier of residual pass `pass` (0..n_cg), waits
 * for one arrival more than any launch makes, and gives up after `cycles` SM
 * clock cycles (1..2e9; the default limit of every wait is 2e9, about one
 * second).  The bounded wait then runs out as it would on a stalled GPU: the
 * frame aborts with the state untouched (U, y, labels, frame counter), on the
 * host path prost_step() returns PROST_ETIMEOUT, and prost_sync() reports
 * PROST_ETIMEOUT and resets the barrier.  Applies to one launch.  Grid and
 * resident forms only.  Errors: PROST_EINVAL (NULL handle, pass or cycles out of range, the
 * cluster or passes form). */
int prost_inject_wait_timeout(prost_handle *h, int32_t pass, int64_t cycles);

/* Copy out the current subspace (the re-orthonormalised representative,
 * m x k row-major float32) and y (k doubles).  Either pointer may be NULL.
 * on_device selects device or host pointers; synchronises when on_device = 0. */
int prost_get_subspace(prost_handle *h, float *U_out, double *y_out, int on_device);

/* Replace the subspace and y (used to restart a stream or to hand the
 * tracker a known state).  U: m x k row-major float32 with linearly
 * independent columns (re-orthonormalised by Cholesky-QR on the device, y
 * transformed so that U y is kept); y: k doubles or NULL for y = 0. */
int prost_set_subspace(prost_handle *h, const float *U, const double *y, int on_device);

/* Replace the previous frame's labels (P bytes, nonzero = foreground); they
 * set the weights of the next frame.  NULL clears them (all weights 1). */
int prost_set_labels(prost_handle *h, const uint8_t *labels, int on_device);

/* Set the frame counter i used by the step-size rule of the next frame. */
int prost_set_frame_index(prost_handle *h, int64_t i);

/* Statistics of the last frame (the fields of prost_stats above: the cost and
 * gradient norm at every CG iterate of Step 1, the line steps and PR+
 * coefficients, sigma, t and theta of Step 2, the foreground count of Step 3,
 * the orthogonality error before the re-orthonormalisation) into *out (host).
 * Synchronises the stream.  PROST_EINVAL for NULL arguments. */
int prost_get_stats(prost_handle *h, prost_stats *out);

/* Checkpoint.  prost_get_state() with buf = NULL stores the needed size in
 * *len; otherwise writes the complete state (parameters, subspace, y,
 * re-orthonormalisation factors, labels, counters) into buf (host memory,
 * *len bytes available) and sets *len to the bytes written.  A handle
 * restored by prost_set_state() from that buffer continues bit-identically.
 * prost_set_state() fails with PROST_EINVAL when the buffer is malformed or
 * was made with other sizes, k, dtypes or step parameters. */
int prost_get_state(prost_handle *h, void *buf, size_t *len);
int prost_set_state(prost_handle *h, const void *buf, size_t len);

/* Tracing.  enable = 1 makes every later prost_step() record a CUDA event on
 * the handle's stream before and after its frame launch; the frame kernel
 * always stamps the device clock (%globaltimer) at the start of the frame, at
 * the end of each residual pass and at the end of the frame.  enable = 0
 * stops the events. */
int prost_set_timing(prost_handle *h, int enable);

/* Device time of each phase of the last traced prost_step(): ms[j] for
 * j < n_cg: CG pass j (residual, gradient, line-step sums and the CG step);
 * j = n_cg: the final pass (gradient at the final y, rank-one SVD, angle);
 * j = n_cg + 1: the update pass (geodesic update, labels, Cholesky-QR).  ms
 * holds at least n_cg + 2 floats; *n gets n_cg + 2.  Synchronises on the
 * frame's end event.  PROST_EINVAL if timing is off or no traced frame ran. */
int prost_get_timing(prost_handle *h, float *ms, int *n);

/* Cost and gradient of one frame without any device allocation.
 *
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: real-time loops that allow no allocation after
 * start-up (cudaMalloc can synchronise the whole device and has no latency
 * bound), plug-ins whose host application owns all device memory through its
 * own pool or arena and hands them only the buffers they work on, and
 * processes that reserve their memory once at start-up and run with what is
 * left.  Such callers cannot create a handle with prost_init(), which
 * allocates, so this call takes every buffer from the caller and keeps its
 * only scratch (the per-CTA partial sums and the arrival counter of the
 * reduction) in one file-scope static device array of about 74 KB, which
 * every GPU that loads the library holds until the process exits.
 *
 * Computes, for the caller's subspace U and coefficients y, the weighted
 * smoothed l_p cost h_{mu,w}(x - U y) (Eqs. weightedLPnorm, spcacost) and its
 * gradient with respect to y, U^T eta with eta_e = -p w_e r_e (r_e^2 + mu)^(p/2 - 1)
 * (Section 3.3), which is what the first residual pass of prost_step()
 * computes at the warm-start y.  Uses prm's width, height, channels, k, p, mu,
 * delta (for mu = 0), omega, in_scale, in_offset and frame_dtype.
 *   U          device, m x k float32 row-major (used as given, not
 *              re-orthonormalised)
 *   y          host, k doubles
 *   frame      device, m entries of prm->frame_dtype, channel-planar
 *   labels     device, P bytes (nonzero = foreground, weight omega) or NULL
 *              (all weights 1)
 *   out        device, k + 1 doubles: out[0] = cost, out[1 + j] = gradient j
 *   status_out device int32 or NULL: PROST_OK, or PROST_EBADFRAME when a
 *              float32 frame has a non-finite entry (out is then not finite)
 *   stream     cudaStream_t as void* (NULL = default stream)
 * The call only enqueues work on the stream; read out after synchronising it.
 * Limits: k <= PROST_STATIC_MAX_K (the width of the static partial rows),
 * m <= 2^30.
 * Larger k, bad parameters or NULL pointers return PROST_EINVAL; a failed CUDA
 * call returns PROST_ECUDA.  No detail string is recorded.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array, so calls that
 * overlap on the GPU (other streams, other host threads) race: serialise
 * them.  Each call clears the counter itself before its kernel runs. */
int prost_cost_grad_static(const prost_params *prm, const float *U, const double *y,
                           const void *frame, const uint8_t *labels, double *out,
                           int32_t *status_out, void *stream);

/* Raw device-clock stamps (%globaltimer, ns) of the last frame, for tracing
 * the inside of a phase.  ts receives PROST_TRACE_LEN values:
 *   ts[0 .. n_cg+2]      start of the frame, end of each residual pass, end of
 *                        the frame (as used by prost_get_timing);
 *   ts[PROST_MAX_CG+3 .. PROST_MAX_CG+12]  inside CG pass 1 (first CTA): rows
 *                        streamed, CTA partial row written, grid barrier passed,
 *                        all partial rows reduced, CG step done; inside the
 *                        update pass: rows streamed, partial row written,
 *                        arrival; (last CTA) partial rows reduced, Cholesky-QR
 *                        factors and state written.
 * Stamps of phases that did not run are stale.  The passes form writes no
 * stamps (its launches are timed by prost_set_timing's events).  Synchronises
 * the stream. */
#define PROST_TRACE_LEN (PROST_MAX_CG + 13)
int prost_get_trace(prost_handle *h, uint64_t *ts);

/* Release the device state (synchronises the stream first).  NULL is a no-op. */
void prost_destroy(prost_handle *h);

/* ---- many streams per tick (not in the paper) --------------------------------
 *
 * A batch tracks n independent streams (each its own prost_params: sizes, k,
 * storage and frame types may all differ) and advances all of them by one
 * frame per prost_batch_step().  The streams are grouped by kernel family (k,
 * storage type, frame type); each group is one cooperative launch in which the
 * CTAs are split between its streams, and with the CUDA graph on (the
 * default) a whole tick is one graph launch.  Each stream computes exactly what
 * a prost_handle with its parameters computes (Steps 1-3 of Section 3.3), up to
 * the summation order of its reductions.  Every stream must run a
 * single-launch form: k <= PROST_MAX_K_SINGLE and form AUTO, GRID or CLUSTER
 * (PROST_EINVAL otherwise).
 * The batch owns its handles; prost_batch_stream() lends one (for
 * prost_get_subspace, prost_get_stats, checkpoints...; frames must go through
 * prost_batch_step while the batch lives).  Work is ordered on the given stream.
 * Errors: PROST_EINVAL (bad parameters of a stream, NULL, unaligned frames),
 * PROST_ENOMEM, PROST_ECUDA; prost_batch_last_error() gives the detail. */
typedef struct prost_batch prost_batch;
int prost_batch_init(const prost_params *prms, int32_t n, void *stream, prost_batch **out);
/* One tick: frames[i] is stream i's frame, a device pointer whose channel
 * planes start on 16-byte boundaries (P * bytes per entry a multiple of 16);
 * masks[i] (device, P bytes) receives its labels, masks or masks[i] may be
 * NULL.  Only enqueues. */
int prost_batch_step(prost_batch *b, const void *const *frames, uint8_t *const *masks);
/* Wait for the stream and report the first device-side error of any stream. */
int prost_batch_sync(prost_batch *b);
int prost_batch_stream(prost_batch *b, int32_t i, prost_handle **h);
/* Capture ticks in a CUDA graph (1, the default) or launch them directly (0). */
int prost_batch_set_graph(prost_batch *b, int enable);
/* Run the kernel groups of a tick one after another (0, the default) or
 * concurrently (1): each group's launch on its own stream, forked from and
 * joined back into the batch stream (inside the graph too), on a share of
 * the SMs proportional to the bytes its streams move per tick, at least one
 * SM per stream.  The shares sum to at most the SM count, so every CTA of
 * every group is resident at once.  Synchronises the batch stream and
 * re-plans the CTA split.  PROST_EINVAL (the plan unchanged) when the groups'
 * streams outnumber the SMs. */
int prost_batch_set_concurrent(prost_batch *b, int enable);
int prost_batch_get_concurrent(prost_batch *b, int32_t *enabled);
/* Autotuner: times `ticks` ticks of each candidate plan (the split of each
 * group's CTAs between its streams in proportion to rows^alpha, alpha in
 * {0.5, 0.75, 1}; the groups in turn or concurrent, where they fit; graph on
 * or off) on the given frames and keeps the fastest.
 * The trackers' states are saved and restored around the trials.  best_ms:
 * the chosen plan's time per tick. */
int prost_batch_tune(prost_batch *b, const void *const *frames, int32_t ticks, float *best_ms);
/* The plan in use: CTAs per stream (n values), kernel groups, alpha, graph. */
int prost_batch_plan(prost_batch *b, int32_t *ctas_per_stream, int32_t *n_groups, float *alpha,
                     int32_t *graph);
/* The split of one kernel group's CTAs between its n streams that the batch
 * plans with (host only: no device call, no state).  weight[i] > 0 is stream
 * i's weight (the batch uses rows^alpha), cap[i] >= 1 the most CTAs it can use
 * (one per pixel tile).  Writes ctas[i] (n values, caller-owned) with
 *   ctas[i] = clamp(floor(budget * weight[i] / sum(weight)), 1, cap[i]),
 * then hands the CTAs left over one at a time to the stream with the largest
 * remaining fractional share that is under its cap (the lowest index on a
 * tie); where the minimum of one CTA each overshoots the budget, the stream
 * with the most CTAs (the lowest index on a tie) gives one back at a time.
 * So sum(ctas) = min(budget, sum(cap)).  Errors: PROST_EINVAL when
 * n < 1, budget < n, a pointer is NULL, a weight is not a positive finite
 * number or a cap is below 1 (ctas unwritten). */
int prost_batch_split(int32_t budget, int32_t n, const double *weight, const int32_t *cap, int32_t *ctas);
const char *prost_batch_last_error(const prost_batch *b);
void prost_batch_destroy(prost_batch *b);

/* ---- the cost over a window of frames and its gradients ------------------------
 *
 * Not in the paper as an interface: the cost of Eq. (spcacost) with the
 * weighted norm of Eq. (weightedLPnorm), summed over a window of n frames,
 *   F(U, Y, mu) = sum_t sum_e w_te ((x_te - u_e^T y_t)^2 + mu)^(p/2),
 * and its gradients dF/dU = H Y^T, dF/dY = U^T H, dF/dmu =
 * sum w (p/2)(r^2 + mu)^(p/2-1), with H_te = eta_te = -p w_te r_te
 * (r_te^2 + mu)^(p/2-1) the per-frame eta of Section 3.3.  Layouts (device,
 * float32): U m x k row-major, Y k x n row-major (column t is y_t), X n x m
 * (row t is frame t, channel-planar), labels n x P bytes (weight omega where
 * set, 1 elsewhere; NULL: all 1), mu one float.  m = channels * P.
 * prost_window_eval writes the cost (one float) and, when dU, dY and dmu are
 * all given, the gradients multiplied by *gscale (a device float, NULL: 1).
 * prost_window_ustep moves U along the window gradient dU: the projection
 * G = (I - U U^T) dU (Eq. gproject), V = U - t G and the Cholesky-QR
 * retraction U_out = V R^{-1} (V^T V = R^T R in FP64), one cooperative
 * launch with two bounded grid barriers; status_out (device int, or NULL)
 * receives 0, -1 if V^T V is not positive definite, or -2 if a grid barrier
 * gave up (about a second); U_out is unwritten in both error cases.
 * All calls only enqueue on the window's stream.  Errors: PROST_EINVAL (sizes:
 * 1 <= k <= 16, 1 <= n <= 128, 0 < p <= 2; NULL pointers), PROST_ENOMEM,
 * PROST_ECUDA. */
typedef struct prost_window prost_window;
int prost_window_init(int64_t m, int32_t channels, int32_t k, int32_t n, double p, double omega, void *stream,
                      prost_window **out);
int prost_window_eval(prost_window *w, const float *U, const float *Y, const float *X, const uint8_t *labels,
                      const float *mu, const float *gscale, float *cost, float *dU, float *dY, float *dmu);
int prost_window_ustep(prost_window *w, const float *U, const float *dU, float t, float *U_out,
                       int32_t *status_out);
/* Fault injection for failure-detection tests (not in the paper): the next
 * prost_window_ustep() waits at its grid barrier `barrier` (1: after U^T dU,
 * 2: after the Gram of V) for one arrival more than the launch makes and
 * gives up after `cycles` SM clock cycles (1..2e9).  That U-step then writes
 * status -2 (wait timed out) and leaves U_out unwritten; the next U-step runs
 * normally.  Errors: PROST_EINVAL (NULL, barrier or cycles out of range). */
int prost_window_inject_wait_timeout(prost_window *w, int32_t barrier, int64_t cycles);
const char *prost_window_last_error(const prost_window *w);
void prost_window_destroy(prost_window *w);

/* ---- pre- and post-processing (Section 3.4) -------------------------------
 *
 * Pre-processing: each frame (channels planes of h_in x w_in, uint8 or
 * float32 as frame_dtype, row-major) is resampled by area averaging to
 * h_out x w_out (160 x 120 in the paper); during the initialisation phase
 * (its first i_init frames) the running per-entry mean and the running sample
 * standard deviation of all entries are updated with every frame (the current
 * one included) and kept fixed afterwards; the output is (v - mean) / std,
 * float32, channels planes of h_out x w_out: the frame a prost_handle made with
 * frame_dtype = PROST_F32, in_scale = 1 and in_offset = 0 takes.
 * The handle owns its device state and orders its work on the given stream.
 * Errors: PROST_EINVAL for bad sizes (planes up to 2^30 pixels, 1..4
 * channels) or NULL pointers, PROST_ENOMEM, PROST_ECUDA. */
typedef struct prost_pre prost_pre;
int prost_pre_init(int32_t w_in, int32_t h_in, int32_t channels, int32_t w_out, int32_t h_out,
                   int32_t frame_dtype, int32_t i_init, void *stream, prost_pre **out);
/* One frame: frame and out are device pointers of the current device
 * (on_device = 1, only enqueued) or host pointers (on_device = 0, synchronous). */
int prost_pre_apply(prost_pre *p, const void *frame, int on_device, float *out);
/* The running statistics (synchronises): mean_out (host, channels*h_out*w_out
 * floats, or NULL), the standard deviation, the frames counted so far. */
int prost_pre_get_stats(prost_pre *p, float *mean_out, double *sigma_out, int32_t *frames_out);
/* Checkpoint of the running statistics (Section 3.4's initialisation phase).
 * prost_pre_get_state() with buf = NULL stores the needed size in *len;
 * otherwise writes the frames counted, the FP64 running sums of the entries
 * and of their squares, the deviation and the per-entry mean plane, behind a
 * header with the geometry, frame type and i_init, into buf (host, *len bytes
 * available) and sets *len to the bytes written.  prost_pre_set_state()
 * restores them into a pre-processor made with the same sizes, frame type and
 * i_init, which then continues bit-identically, inside the initialisation
 * phase or after it.  Both synchronise the stream.  PROST_EINVAL for NULL, a
 * short or malformed buffer, or one made with other parameters. */
int prost_pre_get_state(prost_pre *p, void *buf, size_t *len);
int prost_pre_set_state(prost_pre *p, const void *buf, size_t len);
const char *prost_pre_last_error(const prost_pre *p);
void prost_pre_destroy(prost_pre *p);

/* Post-processing (Section 3.4): the 3 x 3 median of a binary mask (height x
 * width bytes, row-major, nonzero = foreground) with border pixels replicated,
 * which is 1 exactly where at least 5 of the 9 neighbours are.  The paper runs
 * it on the CPU.  mask_in and mask_out are device pointers (on_device = 1,
 * distinct buffers, enqueued on stream) or host pointers (on_device = 0,
 * synchronous).  Errors: PROST_EINVAL (NULL, sizes, in-place on the device),
 * PROST_ENOMEM, PROST_ECUDA. */
int prost_median3x3(const uint8_t *mask_in, uint8_t *mask_out, int32_t width, int32_t height,
                    int on_device, void *stream);

/* Name of an error code (static string). */
const char *prost_strerror(int code);

/* Detail of the last error on this handle (static until the next call on
 * the handle); "" if none.  h = NULL gives the last error of prost_init(). */
const char *prost_last_error(const prost_handle *h);

/* ABI version: 100 * major + minor. */
int prost_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PROST_H */
