/*
 * fitspots.h -- C ABI of the GB300 (sm_103a) spot-fitting library.
 *
 * Batched least-squares fitting of 2-D Gaussian spots with implicit amplitudes
 * (Leutenegger & Weber, arXiv 2106.02045). For every spot the library minimises
 *     chi^2(p) = sum_i (alpha^(p) f_i(p) + beta^(p) - g_i)^2            (Eq. 2)
 * over the shaping parameters p only; the amplitude alpha^ and the background beta^
 * are the closed-form least-squares solution at each p (Eq. 5-6). The minimiser is the
 * scale-invariant damped Levenberg-Marquardt iteration of Eq. 12-14 with the damping
 * schedule and stop criteria of Sec. "Levenberg-Marquardt algorithm" and of the
 * Fit2DGaussian listing in Sec. "Implementation".
 *
 * Conventions shared by every entry point
 *   - Pointers named *images, *offsets, *roi_dims, *init_params, *model, out_* and
 *     *workspace are DEVICE pointers owned by the caller. The library never allocates,
 *     frees or retains them past the call's stream work.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *     default stream) and the call returns without synchronising. Outputs are valid
 *     once the stream has reached that point.
 *   - Spot s is a W x H row-major block of `images` starting at element offsets[s];
 *     pixel (x, y) is element offsets[s] + y*W + x, and its centre has coordinates
 *     (x, y) in the fitted parameters (the first pixel centre is the origin).
 *   - Parameters are 4 floats per spot: (x0, y0, sigma_x, sigma_y). The isotropic model
 *     (Eq. 10) reads sigma from slot 2 and writes the fitted sigma into slots 2 and 3.
 *   - Return value 0 (FS_OK) means the work was enqueued; a negative value means the
 *     call was rejected before anything was enqueued (see FS_ERR_*), except
 *     FS_ERR_CUDA, which reports a launch error after earlier work may have been
 *     enqueued. Per-spot problems never fail a call: they are reported in out_state.
 */
#ifndef FITSPOTS_H
#define FITSPOTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* spot models (one uint8 per spot) */
#define FS_MODEL_ISO 0      /* exp(-((x-x0)^2+(y-y0)^2)/(2 s^2)), Eq. 10 */
#define FS_MODEL_ELLIPTIC 1 /* exp(-(x-x0)^2/(2 sx^2) - (y-y0)^2/(2 sy^2)), axis-aligned */

/* pixel element types */
#define FS_U16 0
#define FS_F32 1

/* per-spot outcome in out_state (the Fit2DGaussian listing's stop conditions) */
#define FS_STATE_MAX_ITER 0        /* iteration budget used up, not converged          */
#define FS_STATE_MIN_DELTA 1       /* converged: chi^2 fell by less than min_delta      */
#define FS_STATE_MIN_STEP 2        /* converged: every |step_j| < min_step * |p_j|      */
#define FS_STATE_MAX_ERROR 3       /* converged: chi^2 < max_error                      */
#define FS_STATE_NO_DECREASE 4     /* converged: step below min_step without decrease   */
#define FS_STATE_NOT_CONVERGED (-1)/* NaN, singular system, or damping reached 10^4     */
#define FS_STATE_INVALID_ROI (-2)  /* W or H < 3, W*H > 1024 or <= P+2, bad model/offset */

/* error codes */
#define FS_OK 0
#define FS_ERR_NULL (-1)       /* a required pointer is NULL                        */
#define FS_ERR_SIZE (-2)       /* n < 0, n above the call's limit, image_elems < 0 */
#define FS_ERR_DTYPE (-3)      /* unknown pixel type                                */
#define FS_ERR_MAX_ITER (-4)   /* max_iter outside [1, 1000]                        */
#define FS_ERR_TOL (-5)        /* a tolerance is negative or not finite, or          */
                               /* min_delta >= 1                                     */
#define FS_ERR_WORKSPACE (-6)  /* workspace smaller than fit_spots_workspace(n)     */
#define FS_ERR_CUDA (-7)       /* a CUDA call failed; see fit_spots_last_cuda_error  */
#define FS_ERR_ARG (-8)        /* another argument is out of range                   */
#define FS_ERR_FULL (-9)       /* serving: the frame queue is full, frame rejected   */

/*
 * Largest spot count per call. The kernels hand out spots through 32-bit counters that
 * run past the count by up to a few hundred thousand before every warp sees the end, so n
 * stays 2^24 below 2^31. Every entry point that takes a spot count returns FS_ERR_SIZE
 * above it, before anything is enqueued.
 */
#define FS_MAX_SPOTS 2130706432LL   /* 2^31 - 2^24 */

/* Bytes of device workspace that fit_spots needs for n spots (0 for n <= 0):
 * 272 + 4 n. The workspace holds the spot schedule (counts, starts and cursors of the 17
 * size classes and a permutation of the spot indices); its contents on entry do not matter. */
size_t fit_spots_workspace(int64_t n);

/* Bytes of device workspace that fit_spots_uniform needs (272, independent of n). */
size_t fit_spots_uniform_workspace(void);

/*
 * Fit n spots.
 *   images       device, uint16 (FS_U16) or float32 (FS_F32) pixel buffer
 *   image_elems  number of elements in `images`; spots reaching past it are INVALID
 *   offsets      device int64[n], element offset of each spot
 *   roi_dims     device int32[n][2] = (W, H), each at least 3, W * H at most 1024 pixels
 *                (the bound of Sec. "Implementation"), so the longer side is at most 341;
 *                ROIs with a side above 32 form the elongated size class
 *   init_params  device float[n][4], start parameters; clamped by limit() first
 *   model        device uint8[n], FS_MODEL_*
 *   max_iter     iteration budget, 1..1000 (the paper's benchmark uses 20)
 *   max_error    absolute chi^2 below which a fit stops (0 disables; the paper's "A/3")
 *   min_delta    stop when chi^2 falls by less than min_delta * chi^2 (paper: 1e-6)
 *   min_step     stop when every |step_j| < min_step * |p_j| (paper: 1e-4)
 *   out_params   device float[n][4] fitted (x0, y0, sigma_x, sigma_y)
 *   out_alpha    device float[n], amplitude alpha^ at the fitted point (Eq. 6)
 *   out_beta     device float[n], background beta^ (Eq. 6)
 *   out_chi2     device float[n], normalised chi^2 = chi^2 / (W*H - P - 2)
 *   out_state    device int32[n], FS_STATE_*
 *   out_iters    device int32[n], LM iterations executed
 *   out_evals    device int32[n] or NULL: points at which the model was evaluated
 *   workspace    device scratch of at least fit_spots_workspace(n) bytes, 16-byte aligned
 * Invalid spots get their start parameters back, NaN amplitudes and chi^2, 0 iterations.
 * Results of a spot depend only on that spot's inputs and the size-class configuration
 * in force (fit_spots_set_config), never on the other spots of the batch.
 * Launches: a prepass (three small kernels) sorts the spots by size class, then one
 * persistent launch of the generic configuration fits every class of W, H <= 32 (each ROI
 * oriented with its longer side along the lanes, rows in a block of 8, 16, 24 or 32; the
 * classes with both sides at most 16 with a 16-lane geometry, two spots per warp, inside the
 * same launch), and a second launch the elongated class (a side above 32).
 * Arithmetic: FP32, with the 2x2 amplitude solve (Eq. 6) redone in FP64 where its determinant
 * cancels by a factor above 1024 and the damped solve (Eq. 14) redone in FP64 where the FP32
 * factorisation fails; a damped system that stays not positive definite gets tenfold more
 * damping, up to the 10^4 cap.
 */
int fit_spots(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
              const int32_t *roi_dims, const float *init_params, const uint8_t *model,
              int64_t n, int max_iter, double max_error, double min_delta, double min_step,
              float *out_params, float *out_alpha, float *out_beta, float *out_chi2,
              int32_t *out_state, int32_t *out_iters, int32_t *out_evals, void *workspace,
              size_t ws_bytes, void *stream);

/*
 * fit_spots with one persistent launch per size class in use (the prepass, then each class
 * alone, largest first, with the configuration fit_spots_set_config assigns to it) instead of
 * one launch of the generic configuration for all classes. Same arguments and workspace; the
 * results agree with fit_spots to FP32 rounding (bit for bit where the class's configuration
 * is the generic one). Assigning a class its per-spot configuration (fit_spots_config_batched
 * = 0) gives the plain form: every lane group runs its own spot's LM step.
 */
int fit_spots_per_class(const void *images, int dtype, int64_t image_elems,
                        const int64_t *offsets, const int32_t *roi_dims,
                        const float *init_params, const uint8_t *model, int64_t n, int max_iter,
                        double max_error, double min_delta, double min_step, float *out_params,
                        float *out_alpha, float *out_beta, float *out_chi2, int32_t *out_state,
                        int32_t *out_iters, int32_t *out_evals, void *workspace,
                        size_t ws_bytes, void *stream);

/*
 * Fit n spots of one size and model stored back to back, the layout of the paper's
 * Fit2DGaussian kernel (one width and pixel count per launch): spot s occupies elements
 * [s*W*H, (s+1)*W*H) of `images`. One kernel launch, no prepass.
 *   width, height  W and H, each at least 3 with W*H <= 1024 (FS_ERR_ARG otherwise, or if
 *                  W*H <= P + 2)
 *   model_id       FS_MODEL_ISO or FS_MODEL_ELLIPTIC for every spot
 *   workspace      device scratch of at least fit_spots_uniform_workspace() bytes,
 *                  16-byte aligned (the work cursor)
 * Other arguments and the results are as for fit_spots; a spot gives bit-identical
 * results through either entry point.
 */
int fit_spots_uniform(const void *images, int dtype, int width, int height, int model_id,
                      const float *init_params, int64_t n, int max_iter, double max_error,
                      double min_delta, double min_step, float *out_params, float *out_alpha,
                      float *out_beta, float *out_chi2, int32_t *out_state, int32_t *out_iters,
                      int32_t *out_evals, void *workspace, size_t ws_bytes, void *stream);

/*
 * fit_spots_uniform from and to HOST memory, with the transfers overlapped: the batch is cut
 * into chunks of `chunk` spots; while chunk k is fitted, chunk k+1's pixels and start values
 * go to the device and chunk k-1's results come back, on a copy stream the library keeps per
 * device. Even chunks are fitted on `stream`, odd chunks on a second fit stream the library
 * keeps per device (ordered after the work the caller queued on `stream` before the call),
 * so that the next chunk's fit fills the SMs while one launch finishes its last spots.
 * Host buffers should be pinned (cudaHostAlloc / page-locked):
 * from pageable memory the copies still work but do not overlap the fits.
 *   images, init_params   host arrays laid out as for fit_spots_uniform
 *   out_*                 host arrays (out_evals may be NULL)
 *   chunk                 spots per chunk, >= 1 (FS_ERR_ARG otherwise); larger chunks keep
 *                         more of the GPU busy, smaller ones start the first fit sooner
 *   workspace             device scratch of at least
 *                         fit_spots_uniform_host_workspace(chunk, width, height, dtype)
 *                         bytes, 256-byte aligned: two chunk buffers (images, start
 *                         values, outputs, schedule header)
 * Returns once everything is enqueued; when `stream` has completed, the host outputs hold
 * the results, identical to those of fit_spots_uniform on the same inputs. Calls from
 * several host threads on one device are serialised while they enqueue.
 */
size_t fit_spots_uniform_host_workspace(int64_t chunk, int width, int height, int dtype);
int fit_spots_uniform_host(const void *images, int dtype, int width, int height, int model_id,
                           const float *init_params, int64_t n, int max_iter, double max_error,
                           double min_delta, double min_step, float *out_params,
                           float *out_alpha, float *out_beta, float *out_chi2,
                           int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                           int64_t chunk, void *workspace, size_t ws_bytes, void *stream);

/*
 * fit_spots without a caller-provided workspace, for callers that cannot allocate device
 * memory: code that runs where cudaMalloc is unavailable or forbidden (inside a region
 * being captured into a CUDA graph, a real-time loop with a no-allocation rule, a plugin
 * whose host application owns every allocation) or that has no allocator of its own at
 * hand. The paper has no counterpart; this is a convenience of the library.
 * The schedule scratch is a fixed array compiled into the library, sized for
 * fit_spots_noalloc_max_spots() = 1,048,576 spots (4 MiB + 272 B), which every GPU that
 * loads the library holds until the process exits. n above that limit returns
 * FS_ERR_SIZE. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call before any
 * stream capture; later calls outside a capture look it up again (so a device reset does
 * not leave a stale address behind), calls inside one reuse the last address. The call
 * itself allocates nothing and frees nothing. Every call shares
 * the one array and leaves its schedule in it: calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. Each call
 * clears the parts that must start at zero, so results never depend on an earlier call.
 * Arguments and results are those of fit_spots, without workspace and ws_bytes.
 */
int fit_spots_noalloc(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
                      const int32_t *roi_dims, const float *init_params, const uint8_t *model,
                      int64_t n, int max_iter, double max_error, double min_delta,
                      double min_step, float *out_params, float *out_alpha, float *out_beta,
                      float *out_chi2, int32_t *out_state, int32_t *out_iters, int32_t *out_evals,
                      void *stream);

/* Largest n fit_spots_noalloc accepts. */
int64_t fit_spots_noalloc_max_spots(void);

/*
 * Backward pass: vector-Jacobian product of the fitted outputs with respect to the
 * pixels, by the implicit-function theorem at the minimum of Eq. 2 over (p, alpha,
 * beta). With K_i = (alpha df_i/dp, f_i, 1), r = g - h and
 *   M = sum_i K_i K_i^T - sum_i r_i d^2 h_i/d(p, alpha, beta)^2,
 * grad_images_i = (M^-1 u) . K_i + u_chi2 * 2 r_i / (W*H - P - 2), where u is the
 * upstream gradient of (params, alpha, beta) (for the isotropic model params[2] and
 * params[3] both carry sigma, so both upstream slots count) and u_chi2 that of out_chi2.
 * The start parameters do not move the minimum: their gradient is zero (not written).
 *   images, dtype, image_elems, offsets, roi_dims, model, n   as passed to fit_spots
 *   params, alpha, beta, state                                the fit_spots outputs
 *   grad_params [n][4], grad_alpha [n], grad_beta [n], grad_chi2 [n]   upstream (device;
 *                                                             any may be NULL = zero; with
 *                                                             grad_chi2 NULL the pixels are
 *                                                             read once instead of twice)
 *   grad_images  device float32 buffer of image_elems elements; the pixels of every valid
 *                spot are written (zeros for spots whose state is not a converged one
 *                or whose system M is singular); other elements are left untouched.
 * Not in the paper (the paper has no derivatives of the fit results); derived from Eq. 2.
 */
int fit_spots_backward(const void *images, int dtype, int64_t image_elems,
                       const int64_t *offsets, const int32_t *roi_dims, const uint8_t *model,
                       int64_t n, const float *params, const float *alpha, const float *beta,
                       const int32_t *state, const float *grad_params, const float *grad_alpha,
                       const float *grad_beta, const float *grad_chi2, float *grad_images,
                       void *stream);

/*
 * Serving (real-time fiducial tracking; the paper's motivation of stabilising a sample
 * at millisecond time scales by following sparse fiducial spots, Sec. "Introduction").
 * A batch covers up to max_batch frames of different sessions; desc (device int32
 * [1 + 2 * max_batch]) = count, then (frame slot, session) per batch entry.
 *
 * fs_serve_roi_cut: for every entry b < count and marker m, cut the roi x roi block of
 * frame slot desc[1+2b] (frames: device uint16 slots of frame_w x frame_h, slot s at
 * frames + s*frame_w*frame_h) at the rounded previous centre state[session][m] (device
 * float [sessions][markers][4] = x, y, sigma_x, sigma_y, frame coordinates), clamped into
 * the frame, into rois[(b*markers + m) * roi*roi] (uint16), the warm start
 * init[b*markers + m] (ROI coordinates) and origin[b*markers + m] = (x, y) of the block.
 * roi must be 3..32 and fit in the frame; markers and max_batch 1..65535 (else
 * FS_ERR_ARG, nothing launched; FS_ERR_NULL for a NULL pointer). Entries b >= count are
 * skipped. desc, state, rois, init and origin are caller-owned device memory.
 *
 * fs_serve_update: after fit_spots_uniform on the count*markers ROIs, move every marker
 * whose fit converged (state MIN_DELTA, MIN_STEP, MAX_ERROR or NO_DECREASE, finite
 * parameters) to origin + fitted centre (a lost marker keeps its last state), and write
 * results[b*markers + m][FS_SERVE_RESULT_FLOATS] = (x, y, sigma_x, sigma_y in frame
 * coordinates, alpha, beta, normalised chi^2, fit state, ROI origin x, y, the warm start
 * x0, y0, sigma_x, sigma_y in ROI coordinates, LM iterations, 0). fit_iters and init are the
 * fit's iteration counts and the start values fs_serve_roi_cut wrote.
 * The same argument rules. Both enqueue one kernel on stream and allocate nothing; a
 * serving step is cut -> fit -> update (the sessions below capture it in a CUDA graph).
 * Not in the paper (it names the use, not a serving design).
 */
#define FS_SERVE_RESULT_FLOATS 16
int fs_serve_roi_cut(const uint16_t *frames, int frame_w, int frame_h, int roi, int markers,
                     const int32_t *desc, int max_batch, const float *state, uint16_t *rois,
                     float *init, int32_t *origin, void *stream);
int fs_serve_update(const int32_t *desc, int max_batch, int markers, const float *params,
                    const float *alpha, const float *beta, const float *chi2,
                    const int32_t *fit_state, const int32_t *fit_iters, const float *init,
                    const int32_t *origin, float *state, float *results, void *stream);

/*
 * Serving sessions: real-time tracking of fiducial markers in camera streams with
 * continuous batching (the paper's motivation, Sec. "Introduction"; the serving design is
 * this library's). A session serves `streams` camera streams of one frame size, `markers`
 * markers each, on the device current at creation:
 *   - fs_session_submit_frame hands over a frame (host uint16 [frame_h][frame_w], pinned
 *     for the copy to overlap; the caller keeps it unchanged until the frame is retired).
 *     It waits in a queue of at most queue_limit frames for a device frame slot (frame_slots
 *     of them: the memory budget); beyond that it is rejected with FS_ERR_FULL and counted.
 *   - fs_session_poll makes progress without blocking: admitted frames are copied in on a
 *     copy stream; frames on the device form a batch (at most one per stream, at most
 *     max_batch, at most max_inflight batches on the device), run as one CUDA graph (ROI cut
 *     at the rounded previous centres, warm-started fit, marker-state update) while later
 *     frames are copied in; finished batches are retired, oldest first, into the caller's
 *     arrays: done[i] and results[i][markers][FS_SERVE_RESULT_FLOATS] (the fs_serve_update
 *     record) for up to max_frames frames; *n_done says how many.
 *   - Stamps: t_arrival is the caller's (use fs_session_clock), t_done is taken when the
 *     batch is seen complete in fs_session_poll; t_done - t_arrival is the frame latency.
 *   - A stream's results are the same whether its frames are batched alone or with other
 *     streams' frames (every marker's work depends on its own stream only).
 * Marker state (x, y, sigma_x, sigma_y in frame coordinates) stays on the device;
 * fs_session_add_markers sets a stream's start state, fs_session_get_markers reads it back
 * (checkpoint; add_markers with a saved state restores it). Both synchronise the session's
 * compute stream. The session allocates its buffers and streams at creation and frees them
 * in fs_session_destroy (which waits for its work); nothing is allocated while serving.
 * Not thread safe: one host thread drives a session.
 * Errors: FS_ERR_NULL, FS_ERR_ARG (a field of cfg or an argument out of range), FS_ERR_FULL,
 * FS_ERR_CUDA. Fit tolerances are as for fit_spots (max_error 0).
 */
typedef struct {
  int frame_w, frame_h;  /* frame size in pixels, each at least roi and at most 65536     */
  int roi;               /* ROI side, 3..32                                               */
  int markers;           /* markers per stream, 1..65535                                  */
  int streams;           /* camera streams, 1..65535                                      */
  int max_batch;         /* frames per batch, 1..64 and at most streams                   */
  int frame_slots;       /* device frame buffers, 1..4096                                 */
  int queue_limit;       /* frames waiting for a slot before new ones are rejected, >= 0  */
  int max_inflight;      /* batches on the device at once, 1..64                          */
  int max_iter;          /* LM iteration budget, 1..1000                                  */
  double min_delta, min_step; /* stop tolerances as for fit_spots                         */
} fs_session_config;

typedef struct {
  int32_t stream;        /* stream of the frame                                           */
  int32_t reserved;
  int64_t index;         /* the caller's frame index                                      */
  double t_arrival;      /* as submitted                                                  */
  double t_done;         /* fs_session_clock when the frame's batch was seen complete     */
} fs_frame_done;

typedef struct fs_session fs_session;

double fs_session_clock(void); /* seconds of a monotonic clock */
int fs_session_create(const fs_session_config *cfg, fs_session **out);
int fs_session_destroy(fs_session *s);
int fs_session_add_markers(fs_session *s, int stream, const float *host_state);
int fs_session_get_markers(fs_session *s, int stream, float *host_state);
int fs_session_submit_frame(fs_session *s, int stream, int64_t index, const uint16_t *host_frame,
                            double t_arrival);
int fs_session_poll(fs_session *s, fs_frame_done *done, float *results, int max_frames,
                    int *n_done);
int fs_session_pending(const fs_session *s); /* frames submitted and not yet retired */
/* frames rejected, frames retired and batches launched so far (any pointer may be NULL) */
int fs_session_stats(const fs_session *s, int64_t *dropped, int64_t *served, int64_t *batches);

/* Message for an FS_ERR_* / FS_OK code (static storage). */
const char *fit_spots_strerror(int code);

/* The cudaError_t value behind the last FS_ERR_CUDA returned on this thread (0 if none). */
int fit_spots_last_cuda_error(void);

/*
 * The comparison method for the paper's claim that implicit amplitudes need fewer
 * iterations: plain Levenberg-Marquardt over (x0, y0, sigma[, sigma_y], alpha, beta) with
 * h = alpha f + beta and the per-pixel Jacobian (alpha df/dp, f, 1), the same damping
 * schedule, limit() box on the shape parameters and stop tests as fit_spots (min_step on
 * the shape parameters), start amplitudes alpha0 = max g - min g, beta0 = min g. Arguments
 * and outputs as for fit_spots (iterations and evaluations counted the same way); no
 * workspace; one warp per spot, FP32.
 */
int fit_spots_explicit(const void *images, int dtype, int64_t image_elems,
                       const int64_t *offsets, const int32_t *roi_dims, const float *init_params,
                       const uint8_t *model, int64_t n, int max_iter, double max_error,
                       double min_delta, double min_step, float *out_params, float *out_alpha,
                       float *out_beta, float *out_chi2, int32_t *out_state, int32_t *out_iters,
                       int32_t *out_evals, void *stream);

/*
 * Variance-weighted implicit-amplitude fit: minimises sum w_i (g_i - alpha f_i - beta)^2 with
 * w_i = 1 / max(g_i, 1) (Poisson variance from the data), alpha and beta from the weighted
 * Eq. 5-6 at every evaluated point, the same damping schedule, box and stop tests as
 * fit_spots; out_chi2 is the weighted chi^2 / (N - P - 2). Arguments and outputs as for
 * fit_spots; no workspace; one warp per spot, FP32.
 */
int fit_spots_weighted(const void *images, int dtype, int64_t image_elems,
                       const int64_t *offsets, const int32_t *roi_dims, const float *init_params,
                       const uint8_t *model, int64_t n, int max_iter, double max_error,
                       double min_delta, double min_step, float *out_params, float *out_alpha,
                       float *out_beta, float *out_chi2, int32_t *out_state, int32_t *out_iters,
                       int32_t *out_evals, void *stream);

/*
 * Poisson-likelihood implicit-amplitude fit: minimises the deviance
 * D = 2 sum [h - g + g ln(g / h)] of h = alpha f + beta (pixel values below 0 count as 0),
 * alpha and beta at their Poisson maximum likelihood for the profile at every evaluated point
 * (the implicit amplitudes of Eq. 5-6 with the likelihood in place of chi^2, found by
 * reweighted least squares), the LM step from the deviance's gradient and Fisher information
 * with the amplitudes regressed out, and the same damping schedule, box and stop tests as
 * fit_spots applied to D; out_chi2 is D / (N - P - 2). ROIs of 3..32 pixels a side. Arguments
 * and outputs as for fit_spots (dtype FS_U16 or FS_F32); no workspace; one warp per spot,
 * FP32.
 */
int fit_spots_poisson(const void *images, int dtype, int64_t image_elems,
                      const int64_t *offsets, const int32_t *roi_dims, const float *init_params,
                      const uint8_t *model, int64_t n, int max_iter, double max_error,
                      double min_delta, double min_step, float *out_params, float *out_alpha,
                      float *out_beta, float *out_chi2, int32_t *out_state, int32_t *out_iters,
                      int32_t *out_evals, void *stream);

/*
 * Local background pre-subtraction. The fit assumes a uniform background in each ROI; where
 * the background varies, the paper allows it to be estimated and subtracted beforehand (Sec.
 * "Implicit-amplitudes least-squares fitting"). This call fits the plane
 * c0 + cx (x - xc) + cy (y - yc), xc = (W - 1) / 2, yc = (H - 1) / 2, by least squares to each
 * ROI's border ring (the pixels within `border` of an edge) and writes the ROI minus the
 * plane's tilt cx (x - xc) + cy (y - yc) to out_images as float32; the level c0 is left for
 * the fit's beta. Fit the result with dtype FS_F32 and the same offsets and dims.
 *   images, dtype, image_elems, offsets, roi_dims, n: as for fit_spots (FS_U16 or FS_F32;
 *                  ROIs of 3..341 pixels a side and at most 1024 pixels)
 *   border         ring width, 1..8 (FS_ERR_ARG otherwise)
 *   out_images     device float32[image_elems]: each valid ROI's pixels are written at the
 *                  same element positions; everything else is left untouched. It may be
 *                  `images` itself for FS_F32 when no two ROIs overlap.
 *   out_plane      device float32[n, 3] (c0, cx, cy per ROI) or NULL; NaN for an invalid
 *                  ROI (bad size or offset), whose pixels are not written
 * Sums are exact integers for uint16 pixels and FP32 within a warp lane, FP64 across lanes,
 * for float32 pixels. Asynchronous on `stream`; no workspace.
 */
int fit_spots_subtract_background(const void *images, int dtype, int64_t image_elems,
                                  const int64_t *offsets, const int32_t *roi_dims, int64_t n,
                                  int border, float *out_images, float *out_plane, void *stream);

/*
 * Start values (x0, y0, s0, s0) for the fit, estimated on the device from each ROI's pixels
 * (the paper estimates start values from the image before fitting, Results section).
 *   rule FS_START_CENTROID  centre = centroid of max(g - min g, 0), the ROI centre
 *                           ((W-1)/2, (H-1)/2) if that weight is zero everywhere
 *   rule FS_START_PAPER     centre = the pixel whose in-ROI 3x3 neighbourhood has the
 *                           largest mean, ties to the lowest row-major index
 *   both                    s0 = sqrt(max(M, 1) / pi), M = #{g > (max g - min g) e^(-1/2) + min g}
 * FP32 throughout; the decisions (the threshold test and the comparison of two means
 * S_i / c_i > S_j / c_j as S_i c_j > S_j c_i, S summed row by row: each row's neighbours left
 * to right, then the rows top to bottom) are exact for integer-valued pixels below 2^21.
 * images/offsets/roi_dims as for fit_spots (W, H in 1..32); out_init device float[n][4]; an
 * invalid ROI gets four NaNs. Asynchronous on `stream`. Errors, before anything is
 * enqueued: FS_ERR_SIZE (n < 0 or above FS_MAX_SPOTS, image_elems < 0), FS_ERR_DTYPE,
 * FS_ERR_ARG (unknown rule), FS_ERR_NULL; n = 0 returns FS_OK without work.
 */
#define FS_START_CENTROID 0
#define FS_START_PAPER 1
int fit_spots_start(const void *images, int dtype, int64_t image_elems, const int64_t *offsets,
                    const int32_t *roi_dims, int64_t n, int rule, float *out_init, void *stream);

/*
 * Size classes and their kernel configurations.
 * A spot with W, H <= 32 has size class (ceil(W/8)-1)*4 + (ceil(H/8)-1) (classes 0..15);
 * a spot with a side above 32 (W*H <= 1024) is in class 16, the elongated class. Each class
 * runs one kernel configuration: `lanes` threads per spot (4, 8, 16 or 32), `cols` ROI
 * columns held by each thread (lanes*cols covers the class's width bound), and the class's
 * row bound (8, 16, 24 or 32) as the per-thread row count. A configuration is per-spot (each
 * lane group fits one spot from start to stop, every lane running the LM step) or batched
 * (fit_spots_config_batched = 1): a warp keeps 16 spots in flight, its lane groups evaluate
 * them with that geometry, re-reading the pixels at each evaluation, and lane j runs the LM
 * step of spot j; per-spot and batched results of the same geometry agree to FP32 rounding.
 * The generic configuration (32 lanes, 1 column, 32 rows, up to 11 row blocks) takes any ROI
 * of at most 1024 pixels: each ROI is oriented with its longer side along the lanes when that
 * side is at most 32, else with its shorter side there, and its rows are walked in blocks of
 * 32 (an oriented ROI may be the caller's transpose; the parameters come back in the caller's
 * orientation). It is the only configuration of the elongated class and the one fit_spots
 * launches once for a whole mixed batch.
 * fit_spots_num_configs / fit_spots_config_info
 * enumerate the compiled configurations; fit_spots_set_config assigns one to a class
 * (the autotuner's output) and fails with FS_ERR_ARG if it cannot hold the class.
 */
int fit_spots_num_classes(void);
int fit_spots_num_configs(void);
int fit_spots_config_info(int config, int *lanes, int *cols, int *rows);
int fit_spots_config_batched(int config); /* 1 batched, 0 per-spot, FS_ERR_ARG if unknown */
int fit_spots_config_fits(int size_class, int config); /* 1 if usable, else 0 */
/* 1 if `config` is the generic configuration (the one fit_spots launches once for all size
 * classes, and the only one that serves the elongated class), 0 otherwise, FS_ERR_ARG if
 * unknown */
int fit_spots_config_generic(int config);
int fit_spots_get_config(int size_class);
int fit_spots_default_config(int size_class); /* the built-in choice the library starts with */
int fit_spots_set_config(int size_class, int config);

/*
 * Throughput probes for the roofline of the fits (not in the paper; measurement support).
 * fit_spots_probe_rates runs dependency chains of FP32 FMA, MUFU exp2 and FP64 FMA on `sms`
 * x 8 blocks of 256 threads, times each with CUDA events on `stream` (one warm-up launch
 * first) and writes lane-operations per second to *ffma, *ex2 and *dfma. It synchronises
 * on its events. scratch: device memory of at least fit_spots_probe_scratch_bytes(sms)
 * bytes (the chains' results are written there). Returns FS_OK, FS_ERR_NULL, FS_ERR_ARG
 * (sms outside 1..4096), FS_ERR_WORKSPACE or FS_ERR_CUDA.
 */
size_t fit_spots_probe_scratch_bytes(int sms);
int fit_spots_probe_rates(int sms, void *scratch, size_t scratch_bytes, double *ffma, double *ex2,
                          double *dfma, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FITSPOTS_H */
