/*
 * fgbd.h - C ABI of the GB300 (sm_103a) implementation of FGBD, the fast
 * graph-based colour denoiser of Watanabe, Nonaka, Pavez, Kobayashi and Ortega,
 * "Fast Graph-Based Denoising for Point Cloud Color Information", ICASSP 2024.
 *
 * The per-frame path has four steps (Section 2.1):
 *   fgbd_build_graph     scan-line graph, Section 2.2 (Eq. 1-4)
 *   fgbd_estimate_noise  NE-GBP noise level, Section 2.3
 *   fgbd_select_filter   FSLR choice of the filter power q, Section 2.4 (Eq. 6)
 *   fgbd_denoise         graph low-pass filter, Section 2.4 (Eq. 5)
 * and fgbd_run chains all four.
 *
 * Conventions
 *  - Every array argument is DEVICE memory on the context's device, owned by
 *    the caller, unless its name ends in _host.  Point arrays are row-major:
 *    xyz is int32 [n][3] as (x, y, z); colours are [n][3] as (R, G, B), either
 *    uint8 (FGBD_U8) or float32 (FGBD_F32) on the 0..255 scale.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    only enqueue work and return; nothing synchronises unless stated.
 *  - Errors are returned as fgbd_status, never thrown or trapped.  Errors
 *    found on the device (a coordinate out of range, a bounded device wait
 *    that gave up) are latched in the context and returned by the next call
 *    that synchronises (fgbd_sync, fgbd_get_stats, fgbd_graph_export, a call
 *    given a _host output).
 *  - The four steps act on the context's working graph, the one built by its
 *    last fgbd_build_graph (one frame at a time, as in Section 2.1); it is
 *    kept in the scan orders' own form, not as CSR.  fgbd_graph_export makes
 *    a standalone CSR copy of it (an fgbd_graph) for callers that want the
 *    graph itself.
 *  - A context is not thread-safe; use one per stream.  The context owns all
 *    scratch memory, allocated once by fgbd_ctx_create for `capacity` points;
 *    the per-frame calls allocate nothing.
 */
#ifndef FGBD_H
#define FGBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FGBD_ABI_VERSION 3
#define FGBD_PATCH_DIM 21   /* D = 3 colour channels x (1 point + 6 neighbours), Section 2.3, window 1 */
#define FGBD_MAX_WINDOW 3   /* largest window implemented */
#define FGBD_PATCH_DIM_MAX 57  /* D = 3 (6 w + 1) at window FGBD_MAX_WINDOW */
#define FGBD_Q_CAP 256      /* largest accepted q_max */

typedef enum fgbd_status {
  FGBD_OK = 0,
  FGBD_EINVAL = 1,    /* invalid argument: null pointer, n or a parameter out of range */
  FGBD_ERANGE = 2,    /* a coordinate outside [0, 2^bits) was found on the device */
  FGBD_ENOMEM = 3,    /* device allocation failed */
  FGBD_ECUDA = 4,     /* a CUDA runtime call failed; see fgbd_last_error */
  FGBD_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  FGBD_ESTATE = 6,    /* calls out of order (e.g. select before estimate) */
  FGBD_ENOTIMPL = 7   /* parameter combination not implemented */
} fgbd_status;

typedef enum fgbd_dtype { FGBD_U8 = 0, FGBD_F32 = 1 } fgbd_dtype;

typedef struct fgbd_params {
  int32_t bits;         /* b, coordinate bits (Section 2.2); 1..10 so a code fits 32 bits */
  int32_t window;       /* w: points linked on each side along a scan line, 1..FGBD_MAX_WINDOW (paper: 1) */
  double fslr_factor;   /* FSLR skips points whose mean patch std exceeds factor * sigma_est (paper: 2) */
  int32_t q_max;        /* largest filter power searched, 0..FGBD_Q_CAP (the paper states none; default 64) */
  int32_t variant;      /* OR of FGBD_VARIANT_* ablation switches; 0 is the method as published */
  int32_t flags;        /* OR of FGBD_FLAG_* execution choices (same results); 0 is the default */
  int32_t reserved[5];  /* must be zero */
} fgbd_params;

/* Execution choices that do not change any result.
 *   FGBD_FLAG_FUSED_SELECT: fgbd_run takes the FSLR selection and the filter
 *     inside the noise-estimate launch (the blocks that take the speculative
 *     filter steps continue once sigma_est is published) instead of a second
 *     cooperative launch.  It pays off only while sigma_est arrives before the
 *     speculative steps end; on the 1M-point frame it is 4 us slower, so it is
 *     off by default. */
#define FGBD_FLAG_FUSED_SELECT 1

/* Ablation switches of Section 3 (Tables 4 and 5), for comparison runs only.
 *   FGBD_VARIANT_NO_FSLR: "FGBD w/o FSLR" (Table 5): Eq. 6 is evaluated over
 *     every point; the limited region of Section 2.4 is not applied.
 *   FGBD_VARIANT_UNSORTED_PATCH: "NE-GBP w/o sort" (Table 4): the neighbours of
 *     a patch are not ordered by distance (Section 2.3) but taken in the order
 *     the scan-line graph links them: previous and next along C1, then along C2,
 *     then along C3. */
#define FGBD_VARIANT_NO_FSLR 1
#define FGBD_VARIANT_UNSORTED_PATCH 2
/*   FGBD_VARIANT_SAME_LINE: links only join points of the same scan line of a
 *     code (equal in its two major coordinates).  The method as published links
 *     consecutive points of the global sorted order, so the last point of one
 *     scan line is also linked to the first of the next (Section 2.2); this
 *     switch drops those links, to measure what they contribute. */
#define FGBD_VARIANT_SAME_LINE 4
/* Alternative readings where the paper leaves a choice open (for comparison
 * runs; the method as read here is 0):
 *   FGBD_VARIANT_SIGMA_NODE: sigma_g of Eq. 4 is the mean over the points of
 *     each point's mean edge length (Section 2.2 speaks of the average distance
 *     between points and their neighbours) instead of the mean edge length.
 *   FGBD_VARIANT_SIGMA_PAIR: a bandwidth per point, sigma_i = its mean edge
 *     length, and w_ij = exp(-d_ij^2 / (sigma_i sigma_j)) (window 1; not with
 *     the differentiable filter, whose bandwidth is one scalar).
 *   FGBD_VARIANT_POOLED_PATCH: NE-GBP with patches of D = 6 w + 1 entries per
 *     colour channel, the three channels pooled in one covariance (Section 2.3
 *     defines patches of a point and its neighbours; window 1), instead of
 *     D = 3 (6 w + 1) RGB patches.
 *   FGBD_VARIANT_GLOBAL_Q: q* is the argmin of Eq. 6 over q = 0..q_max (the
 *     smaller q among equal values) instead of the first q whose objective does
 *     not fall; every J(q) up to q_max is evaluated (Section 2.4). */
#define FGBD_VARIANT_SIGMA_NODE 8
#define FGBD_VARIANT_SIGMA_PAIR 16
#define FGBD_VARIANT_POOLED_PATCH 32
#define FGBD_VARIANT_GLOBAL_Q 64

typedef struct fgbd_stats {
  int64_t n;                                /* points of the last graph */
  int64_t n_edges;                          /* distinct undirected SLG edges */
  double sigma_g;                           /* mean edge length, Eq. 4's bandwidth */
  int64_t n_patches;                        /* points with exactly 6 w neighbours (Section 2.3) */
  int32_t patch_dim;                        /* D = 3 (6 w + 1): valid entries of eigenvalues[] */
  double eigenvalues[FGBD_PATCH_DIM_MAX];   /* of the patch covariance, descending */
  int32_t m;                                /* leading eigenvalues dropped by the tail rule */
  int32_t q;                                /* selected (or last applied) filter power */
  double tau;                               /* mean of the noise eigenvalues */
  double sigma_est;                         /* sqrt(tau) */
  int64_t n_keep;                           /* points kept by FSLR (0: none, so all were used) */
  int32_t n_objective;                      /* number of valid entries of objective[] */
  int32_t valid;                            /* bit 0 graph, bit 1 noise estimate, bit 2 selection */
  double objective[FGBD_Q_CAP + 1];         /* Eq. 6 over the kept points, J(0..n_objective-1) */
  int64_t launches;                         /* kernels this context has launched since creation */
} fgbd_stats;

typedef struct fgbd_ctx fgbd_ctx;

/* ABI version compiled into the library (FGBD_ABI_VERSION). */
int32_t fgbd_abi_version(void);

/* Human-readable name of a status code (static string). */
const char* fgbd_status_str(fgbd_status s);

/* Fill `p` with the paper's settings: bits 10, window 1, fslr_factor 2, q_max 64.
 * Returns FGBD_EINVAL if p is NULL. */
fgbd_status fgbd_params_default(fgbd_params* p);

/* Create a context on the current CUDA device for frames of up to `capacity`
 * points (1 <= capacity < 2^30) and allocate all its device memory (about
 * 205 bytes per point), zeroed once.  `params` may be NULL for the defaults.
 * On success *out owns the context; release it with fgbd_ctx_destroy.  A
 * window w > 1 adds 24 (w - 1) bytes per point (less the 24 of the stored
 * window-1 filter weights) and a few MB of noise-estimate scratch.
 * Errors: FGBD_EINVAL (bad capacity or parameters), FGBD_ENOTIMPL (window
 * above FGBD_MAX_WINDOW, or FGBD_VARIANT_UNSORTED_PATCH with window > 1),
 * FGBD_ENOMEM, FGBD_ECUDA. */
fgbd_status fgbd_ctx_create(int64_t capacity, const fgbd_params* params, fgbd_ctx** out);

/* Free a context and its device memory (waits for its work to finish). NULL is ignored. */
void fgbd_ctx_destroy(fgbd_ctx* ctx);

/* Message of the last FGBD_ECUDA error of this context ("" if none). */
const char* fgbd_last_error(const fgbd_ctx* ctx);

/* Section 2.2, Eq. 1-4: scan-line graph of n points.  Computes the three
 * raster codes, radix-sorts the points along each (ties by input index),
 * links consecutive points of each order (with window w, each point to the w
 * before and the w after it), merges the three link sets into
 * one symmetric graph (a pair linked twice is one edge) and sigma_g, the mean
 * edge length used by the Gaussian weights of Eq. 4.
 *   xyz: int32 [n][3] device, each coordinate in [0, 2^bits).
 *   n:   0 <= n <= capacity.
 * A coordinate out of range is reported as FGBD_ERANGE by the next
 * synchronising call.  Errors: FGBD_EINVAL, FGBD_ECUDA. */
fgbd_status fgbd_build_graph(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, void* stream);

/* Section 2.3 (NE-GBP): noise level of colours on the graph of the last build.
 * Patches of the points with exactly 6 w neighbours (the point then its
 * neighbours by increasing distance; D = 3 (6 w + 1) entries), their
 * covariance, its eigenvalues, and
 * sigma_est = sqrt(tau) with tau the mean of the eigenvalues left by the tail
 * rule.  Also computes each point's patch colour spread for FSLR.
 *   rgb:             colours [n][3] device, dtype FGBD_U8 or FGBD_F32.
 *   sigma_est:       optional device double receiving sigma_est (may be NULL).
 *   sigma_est_host:  optional host double receiving sigma_est (may be NULL);
 *                    if given, the call synchronises `stream` and returns a
 *                    latched device error like fgbd_sync.
 * With no complete patch sigma_est is 0.  Errors: FGBD_EINVAL, FGBD_ESTATE
 * (no graph), FGBD_ECUDA. */
fgbd_status fgbd_estimate_noise(fgbd_ctx* ctx, const void* rgb, int32_t dtype, double* sigma_est,
                                double* sigma_est_host, void* stream);

/* Section 2.4 (FSLR, Eq. 5-6): the integer filter power q minimising
 * |sigma_est^2 - (sum y^2 - sum x_q^2)/N| over the points whose mean patch
 * colour std is at most fslr_factor * sigma_est (all points if none is), with
 * N = 3 x (points used).  q is searched upward from 0 and the first q whose
 * objective is not below the previous one ends the search (q* = q - 1), or
 * q_max.  The filtered colours x_{q*} are kept in the context for
 * fgbd_denoise with q < 0.
 *   rgb:        the colours given to fgbd_estimate_noise (same pointer and dtype,
 *               unchanged contents).
 *   sigma_est:  device double to use as sigma_est, or NULL for this context's estimate.
 *   q_out:      optional device int32 receiving q* (may be NULL).
 *   q_host:     optional host int32 receiving q* (may be NULL); if given, the
 *               call synchronises `stream` and returns a latched device error
 *               like fgbd_sync.
 * Errors: FGBD_EINVAL, FGBD_ESTATE (no estimate, or other colours), FGBD_ECUDA. */
fgbd_status fgbd_select_filter(fgbd_ctx* ctx, const void* rgb, int32_t dtype, const double* sigma_est,
                               int32_t* q_out, int32_t* q_host, void* stream);

/* Eq. 5: f_out = (D_g^{-1} W_g)^q f_in with W_g = D + W, D_g = 2D, i.e. q steps
 * of x <- x/2 + D^{-1} W x / 2 with W the Gaussian weights of Eq. 4.
 *   q >= 0:  filter rgb_in (dtype in_dtype) q times (q <= FGBD_Q_CAP).
 *   q <  0:  write the colours x_{q*} kept by the last fgbd_select_filter;
 *            rgb_in and in_dtype are ignored (FGBD_ESTATE if there is none).
 *   rgb_out: [n][3] device, out_dtype FGBD_F32 (exact filter output) or FGBD_U8
 *            (rounded half to even and clipped to 0..255).
 * Errors: FGBD_EINVAL, FGBD_ESTATE, FGBD_ECUDA. */
fgbd_status fgbd_denoise(fgbd_ctx* ctx, const void* rgb_in, int32_t in_dtype, int32_t q, void* rgb_out,
                         int32_t out_dtype, void* stream);

/* All four steps on one frame (Section 2.1): build, estimate, select, and the
 * selected filter written to rgb_out.  Same arguments and errors as the four
 * calls it replaces; rgb_in and rgb_out must not overlap.
 * Repeated calls with the same arguments (buffers, n, dtypes) replay a CUDA
 * graph of the whole run: the second such call records the kernels into a
 * graph on the context's own stream, later ones only launch it on `stream`
 * (the contents of the buffers may change between calls).  Up to 8 argument
 * sets are kept per context.  Per-kernel timing (fgbd_set_timing) and a
 * `stream` that is being captured by the caller use the kernels directly. */
fgbd_status fgbd_run(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                     void* rgb_out, int32_t out_dtype, void* stream);

/* fgbd_run on HOST buffers (no counterpart in the paper): the coordinates and
 * colours are copied into one of two device staging slots owned by the
 * context, the run takes place on `stream` exactly as fgbd_run, and the result
 * is copied back into rgb_out.  The copies run on two copy streams of the
 * context, so consecutive calls pipeline: a call's input copy overlaps the
 * previous call's device work, and its output copy overlaps the next call's.
 *   xyz [n][3], rgb_in [n][3], rgb_out [n][3]: host memory, page-locked
 *     (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous;
 *     pageable memory also works, with synchronous copies.
 * Ownership: the host buffers of a call are read / written asynchronously.
 * They are free again (inputs no longer read, output complete) once
 * fgbd_sync(ctx, stream) has returned, or once the call after the next one on
 * this context has returned (it waits for this call's output copy before it
 * reuses its staging slot).  The first call allocates the staging memory
 * (about 72 bytes per point of capacity) and synchronises the device once.
 * Errors: as fgbd_run; FGBD_ENOMEM if the staging memory cannot be had. */
fgbd_status fgbd_run_host(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                          void* rgb_out, int32_t out_dtype, void* stream);

/* Streaming mode of Section 3 (2): the noise estimate and the selection run
 * on some frames only, and the other frames reuse the q of the previous one.
 * This call builds the graph of the new frame (Section 2.2) and filters it
 * (Eq. 5) with the q this context selected last (fgbd_select_filter or
 * fgbd_run), read on the device: no host synchronisation.  The estimate,
 * FSLR and the q search are skipped; stats keep the last estimate's values.
 * Arguments as fgbd_run.  Errors: FGBD_ESTATE (this context has never
 * selected a q), FGBD_EINVAL, FGBD_ECUDA. */
fgbd_status fgbd_run_reuse(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                           void* rgb_out, int32_t out_dtype, void* stream);

/* Batched path (no counterpart in the paper, which processes one frame at a
 * time): fgbd_run on `count` frames of any sizes, frame f with its own context
 * ctxs[f], all enqueued in one call.  A single 1M-point frame leaves most of
 * the GPU idle in its short, latency-bound kernels; frames run side by side
 * fill it.
 *   ctxs, xyz, n, rgb_in, in_dtype, rgb_out, out_dtype: host arrays of
 *     `count` entries, the fgbd_run arguments of each frame (device buffers).
 *   count: 0..FGBD_BATCH_MAX; the contexts must be distinct and on one device.
 * Segmented batches: when every frame has at least one point, window 1, the
 * same ablation switches and the same input colour type, each stage may run as
 * one launch over up to 16 frames (the sort passes, the link, the colour
 * gather, the moments: every frame's blocks in one grid; the noise estimate:
 * one eigen block per frame while the other SMs, shared out by frame size,
 * take the frames' speculative filter steps; the selection and filter: one
 * cooperative launch in which each frame's blocks, shared out by frame size,
 * synchronise among themselves).  Whether a batch that can be segmented is,
 * how many frames a launch takes and the block shapes of the sort scatter and
 * of the selection/filter are those fgbd_tune_batch chose for this device and
 * frame size (or fgbd_set_batch_shape set; by default segmented below 2^18
 * points a frame); they do not change any result.  Other batches run every
 * frame on a stream of its own, forked from `stream` and joined back into it,
 * the cooperative selection/filter launches one frame after another.
 * Either way results, stats and errors are per context, exactly as after
 * fgbd_run (the outputs are bit-identical), everything earlier on `stream`
 * finishes first and later work on `stream` waits for every frame.  The call
 * contains no host synchronisation, so it can be captured into a CUDA graph
 * once the contexts have run a frame (the first launches set kernel
 * attributes).  Like fgbd_run, the second call with the same contexts, buffers
 * and block shapes records a CUDA graph of the whole batch (kept by ctxs[0],
 * up to 4 of them) and later calls launch it.  In a segmented batch the
 * launches are counted in the stats of ctxs[0] (kernel timing too).
 * Errors: FGBD_EINVAL (any argument), checked before anything is enqueued;
 * FGBD_ECUDA. */
#define FGBD_BATCH_MAX 64
fgbd_status fgbd_run_batch(fgbd_ctx* const* ctxs, const int32_t* const* xyz, const int64_t* n,
                           const void* const* rgb_in, const int32_t* in_dtype, void* const* rgb_out,
                           const int32_t* out_dtype, int32_t count, void* stream);

/* How a batch runs (no counterpart in the paper). */
typedef struct fgbd_batch_shape {
  int32_t seg_frames;            /* frames per segmented launch, 1..16; 0: per-frame streams.  Default: 16
                                    below 2^18 points a frame, 0 above (fgbd_tune_batch: -1 when the batch
                                    cannot be segmented, and nothing was tuned) */
  int32_t scatter_threads;       /* threads ranking one 4096-key sort tile: 256, 512 (default) or 1024 */
  int32_t filter_threads;        /* threads per block of the selection/filter: 256 or 512 (default) */
  int32_t filter_blocks_per_sm;  /* its blocks per SM (default 2; capped by what fits) */
  float ms;                      /* fgbd_tune_batch: device time of one batch with the chosen shape */
  int32_t reserved[3];
} fgbd_batch_shape;

/* Autotuner of batches: runs the batch (the arguments of fgbd_run_batch) with
 * candidate shapes - per-frame streams against segmented launches of 16, 8, 4
 * and 2 frames, then, if segmented won, the sort scatter at 256, 512 and 1024
 * threads a tile, then the selection/filter at 512 threads x 1 or 2 blocks per
 * SM and 256 threads x 2 or 4 - timing each (median of three after one untimed
 * run, CUDA events on `stream`), one coordinate at a time, and keeps the
 * fastest for this device and frame-size class (floor(log2(mean points per
 * frame))); later fgbd_run_batch calls use it.  Synchronises; the frames'
 * outputs and stats are those of the batch (every candidate gives the same).
 * *chosen (optional, host) receives the shape and its time.  A batch that
 * cannot be segmented is not run (seg_frames = -1).  Errors: as
 * fgbd_run_batch. */
fgbd_status fgbd_tune_batch(fgbd_ctx* const* ctxs, const int32_t* const* xyz, const int64_t* n,
                            const void* const* rgb_in, const int32_t* in_dtype, void* const* rgb_out,
                            const int32_t* out_dtype, int32_t count, void* stream, fgbd_batch_shape* chosen);

/* The shapes a segmented batch of frames of about `mean_points` points on CUDA
 * device `device` uses, into *out (host); set them (or, with shape NULL, go
 * back to the defaults) with fgbd_set_batch_shape.  Errors: FGBD_EINVAL. */
fgbd_status fgbd_get_batch_shape(int32_t device, int64_t mean_points, fgbd_batch_shape* out);
fgbd_status fgbd_set_batch_shape(int32_t device, int64_t mean_points, const fgbd_batch_shape* shape);

/* Differentiable filter (no counterpart in the paper; a training extension
 * of Eq. 5).  With R = D^-1 W, W_ij = exp(-d_ij^2 / sigma^2) on the graph of
 * the last fgbd_build_graph (Eq. 4), the filter
 *   x_0 = rgb_in,  x_{t+1} = (1 - alpha) x_t + alpha R x_t,  rgb_out = x_q
 * is Eq. 5 for alpha = 1/2 and sigma = sigma_g (W_g = D + W, D_g = 2D).
 *   rgb_in, rgb_out: float32 [n][3] device, input order, 0..255 scale.
 *   q:          0..FGBD_Q_CAP filter steps.
 *   alpha:      filter strength (any finite value; 1/2 in the paper).
 *   sigma:      weight bandwidth; 0 means sigma_g of the graph.
 *   checkpoint: keep every checkpoint-th iterate for the backward call and
 *               recompute the others there (0 or 1: keep all); memory about
 *               (100 + 16 (q / checkpoint + checkpoint + 1)) bytes per point,
 *               allocated on the first call that needs more (that call
 *               synchronises the device).
 * The call records q, alpha, sigma for fgbd_filter_backward.
 * Errors: FGBD_EINVAL, FGBD_ESTATE (no graph), FGBD_ENOTIMPL (window != 1),
 * FGBD_ENOMEM, FGBD_ECUDA. */
fgbd_status fgbd_filter_forward(fgbd_ctx* ctx, const float* rgb_in, int32_t q, double alpha, double sigma,
                                int32_t checkpoint, float* rgb_out, void* stream);

/* Adjoint of the last fgbd_filter_forward of this context: given
 * grad_out = dL/d rgb_out (float32 [n][3], input order) it writes
 *   grad_in        = dL/d rgb_in = ((1 - alpha) I + alpha W D^-1)^q grad_out,
 *   grad_params[0] = dL/d alpha,  grad_params[1] = dL/d sigma
 * (grad_params: device double[2]), summing over the q steps with the stored
 * or recomputed iterates.  The reductions are float64 in a fixed order.
 * Errors: FGBD_EINVAL, FGBD_ESTATE (no forward call since the last graph
 * build), FGBD_ECUDA. */
fgbd_status fgbd_filter_backward(fgbd_ctx* ctx, const float* grad_out, float* grad_in, double* grad_params,
                                 void* stream);

/* Testing / fault injection: the time in nanoseconds after which every
 * device-side wait of this context (the grid barriers of the filter and of the
 * speculative steps, the fused selection's wait for sigma_est) gives up,
 * latches FGBD_ETIMEOUT and lets its kernel return; 2 s by default.  With 0 a
 * barrier gives up as soon as it is not already complete, which tests use to
 * check that a timeout is reported by the next synchronising call and that the
 * context then works again.  Waits for the context's earlier work first.
 * Errors: FGBD_EINVAL (ns < 0), FGBD_ECUDA. */
fgbd_status fgbd_debug_set_wait_limit(fgbd_ctx* ctx, int64_t ns);

/* Testing (not part of the method): q_newton[i] = a[i] / b[i] by the float64
 * quotient the eigen step of the noise estimate uses (a float32 reciprocal
 * refined by Newton steps, Section 2.3's tail mean and Rayleigh quotients),
 * and q_div[i] by CUDA's own division, for n pairs (device arrays of double,
 * on the current device).  Enqueues on `stream`.  Errors: FGBD_EINVAL,
 * FGBD_ECUDA. */
fgbd_status fgbd_debug_div(const double* a, const double* b, double* q_newton, double* q_div, int64_t n,
                           void* stream);

/* Testing (not part of the method): the patch moments of the context's last
 * noise estimate with uint8 colours (Section 2.3), as exact integers over the
 * patches' entries centred on 128: s2[r * D + c] = sum_i a_ir a_ic for
 * r <= c (entries below the diagonal are 0), s1[r] = sum_i a_ir, *n_patches =
 * the number of patches; D = fgbd_stats.patch_dim (host arrays of D * D and D
 * int64).  Synchronises the device.  Errors: FGBD_EINVAL (a null pointer),
 * FGBD_ESTATE (no estimate with uint8 colours yet), FGBD_ECUDA. */
fgbd_status fgbd_debug_moments(fgbd_ctx* ctx, int64_t* s2, int64_t* s1, int64_t* n_patches);

/* Wait for the context's work on `stream` (and for the output copies of
 * fgbd_run_host) and return any latched device error (FGBD_ERANGE,
 * FGBD_ETIMEOUT), clearing it. */
fgbd_status fgbd_sync(fgbd_ctx* ctx, void* stream);

/* Synchronise `stream`, then copy the scalars of the last build, estimate and
 * selection into *out_host.  Returns latched device errors like fgbd_sync. */
fgbd_status fgbd_get_stats(fgbd_ctx* ctx, fgbd_stats* out_host, void* stream);

/* The graph of the last build as CSR in input order, rows sorted by column,
 * with the Eq. 4 weights w_ij = exp(-|g_i - g_j|^2 / sigma_g^2) (float32; long
 * edges may underflow to 0), copied into caller buffers.  Synchronises `stream`.
 *   row_ptr:   int64 [n+1] device, or NULL to only query *nnz_host.
 *   col:       int32 [col_capacity] device (ignored if row_ptr is NULL).
 *   w:         float32 [col_capacity] device, or NULL.
 *   nnz_host:  receives the number of stored entries (2 x edges).
 * Errors: FGBD_EINVAL (col_capacity too small), FGBD_ESTATE, FGBD_ECUDA. */
fgbd_status fgbd_graph_csr_copy(fgbd_ctx* ctx, int64_t* row_ptr, int32_t* col, float* w, int64_t col_capacity,
                                int64_t* nnz_host, void* stream);

/* A standalone copy of a context's graph (Section 2.2) as symmetric CSR in
 * input order: row_ptr int64 [n+1], col int32 [nnz] (rows sorted by column),
 * the Eq. 4 weights w float32 [nnz], and sigma_g.  It owns its device memory
 * (on the context's device) and outlives the context. */
typedef struct fgbd_graph fgbd_graph;

/* Export the graph of the context's last build as a new fgbd_graph (device
 * memory allocated here, about 12 bytes per stored entry plus 8 per point).
 * Synchronises `stream`; returns a latched device error like fgbd_sync.
 * Release it with fgbd_graph_free.  Errors: FGBD_EINVAL, FGBD_ESTATE (no
 * graph), FGBD_ENOMEM, FGBD_ECUDA. */
fgbd_status fgbd_graph_export(fgbd_ctx* ctx, fgbd_graph** out, void* stream);

/* Borrowed views of an exported graph: device pointers that stay valid until
 * fgbd_graph_free(g), and host scalars.  Any output pointer may be NULL.
 *   row_ptr, col, w: device arrays as described at fgbd_graph (NULL when the
 *                    graph has no points / no entries).
 *   n_host, nnz_host, sigma_g_host: points, stored entries (2 x edges), the
 *                    mean edge length sigma_g of Eq. 4.
 * Errors: FGBD_EINVAL (g is NULL). */
fgbd_status fgbd_graph_csr(const fgbd_graph* g, const int64_t** row_ptr, const int32_t** col, const float** w,
                           int64_t* n_host, int64_t* nnz_host, double* sigma_g_host);

/* Free an exported graph and its device memory.  NULL is ignored. */
void fgbd_graph_free(fgbd_graph* g);

/* The three scan orders of the last build: orders[l][k] is the input index of
 * the k-th point along code l+1 (Eq. 1-3).  orders: int32 [3][n] device. */
fgbd_status fgbd_get_orders(fgbd_ctx* ctx, int32_t* orders, void* stream);

/* FSLR data in input order (Section 2.4): spread[i] = mean over channels of
 * the population colour std over point i and its neighbours (float32, from
 * the last estimate) and keep[i] = 1 if point i entered the objective of the
 * last selection.  Either pointer may be NULL.  FGBD_ESTATE if the context
 * holds no selection. */
fgbd_status fgbd_get_fslr(fgbd_ctx* ctx, float* spread, uint8_t* keep, void* stream);

/* Instrumentation (not part of the method).  With timing enabled, every
 * kernel the context launches is bracketed by two CUDA events recorded on the
 * launching stream.  fgbd_get_timings synchronises those events, writes up to
 * `max` entries (kernel name, NUL-padded to FGBD_NAME_LEN bytes, into
 * names_host; duration in milliseconds into ms_host), sets *count_host to the
 * number written and clears the list.  Launches beyond FGBD_TIMING_CAP per
 * list are not timed.  Errors: FGBD_EINVAL, FGBD_ECUDA. */
#define FGBD_NAME_LEN 32
#define FGBD_TIMING_CAP 256
fgbd_status fgbd_set_timing(fgbd_ctx* ctx, int32_t enable);
fgbd_status fgbd_get_timings(fgbd_ctx* ctx, int32_t max, int32_t* count_host, char* names_host, float* ms_host);

/* Allocation-free scan orders.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * the result: a real-time frame loop where a cudaMalloc would stall the frame
 * (it can synchronise the device), a plug-in whose host application owns all
 * device memory, or a service held to a fixed memory budget.  It computes the
 * same three scan orders as fgbd_build_graph (the codes of the three scan
 * directions, each sorted stably, ties broken by input index) without a
 * context.
 *   xyz:    int32 [n][3] device, coordinates in [0, 2^bits).
 *   n:      0 <= n <= FGBD_STATIC_MAX_POINTS; larger n returns FGBD_EINVAL.
 *   bits:   1..10.
 *   orders: int32 [3][n] device; orders[l][k] is the input index of the k-th
 *           point along code l+1.
 *   status: optional device uint32 receiving 0, or 1 if a coordinate was out
 *           of range (the orders are then unspecified); NULL to skip.
 * Scratch: one file-scope device array of about 1.3 MiB (FGBD_STATIC_MAX_POINTS
 * points) reserved on every GPU that loads the library until the process
 * exits.  The call allocates and frees nothing.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call
 * shares the array and it keeps the previous call's contents; each call clears
 * what must start at zero, but calls that overlap on the GPU (different
 * streams or threads without ordering between them) race on it and give wrong
 * results.  Enqueues on `stream` and returns without synchronising.
 * Errors: FGBD_EINVAL, FGBD_ECUDA. */
#define FGBD_STATIC_MAX_POINTS 32768
fgbd_status fgbd_scan_orders_static(const int32_t* xyz, int64_t n, int32_t bits, int32_t* orders, uint32_t* status,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FGBD_H */
