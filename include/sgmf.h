/*
 * sgmf.h -- C ABI of the GB300 stereo-LiDAR semi-global matching library.
 *
 * The library computes, on one GPU, the pipeline of "Stereo-LiDAR Fusion by
 * Semi-Global Matching with Discrete Disparity-Matching Cost and
 * Semidensification" (Yao, Ishikawa, Oishi, RA-L 2025), Fig. 1:
 *
 *   sparse LiDAR disparity d-bar  (Sec. IV: integer, aligned with the left view)
 *   census / Hamming cost H       (Sec. IV-A)
 *   semidensification d-hat       (Sec. IV-B, Eq. 5)
 *   joint cost C-bar with DDC     (Sec. IV-A, Eq. 4)
 *   8-path SGM aggregation        (Sec. III, Eq. 2)
 *   winner-takes-all d*, d'       (Sec. III, Eq. 3; Sec. IV-C)
 *   three-view consistency        (Sec. IV-C, Eq. 6)
 *
 * Inputs are a rectified stereo pair and a sparse disparity map aligned with
 * the left (base) image (Sec. II-A, Sec. IV); the output is the consistent
 * dense disparity map D^{c*} with invalid pixels (Eq. 6).
 *
 * Conventions for every entry point:
 *   - images and maps are row-major, y outermost, pitch = width elements;
 *   - an invalid disparity is -1 (int16);
 *   - no C++ exception crosses this ABI; every call returns an sgmf_status
 *     and, on error, leaves a message for sgmf_last_error();
 *   - a context is used by one host thread at a time.
 */
#ifndef SGMF_H_
#define SGMF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgmf_ctx sgmf_ctx;

typedef enum {
    SGMF_OK = 0,
    SGMF_ERR_ARG = 1,      /* NULL pointer, bad stage id, buffer too small */
    SGMF_ERR_PARAM = 2,    /* parameter outside the supported range */
    SGMF_ERR_SHAPE = 3,    /* width/height/disparity range outside the supported range */
    SGMF_ERR_OOM = 4,      /* device or pinned-host allocation failed */
    SGMF_ERR_CUDA = 5,     /* a CUDA runtime call or kernel failed */
    SGMF_ERR_TIMEOUT = 6   /* a bounded device-side wait gave up (kernel returned early) */
} sgmf_status;

/* Census kinds.  The paper uses the Hamming distance of census-transformed
 * images after Spangenberg et al. (Sec. IV-A) without giving the window.
 * Offsets o = (dx, dy), dx in [-4, 4], dy in [-3, 3], are enumerated in
 * raster order (dy outer, dx inner) without the centre; the k-th offset sets
 * bit k.  A bit whose compared samples are not all inside the image is 0. */
enum {
    SGMF_CENSUS_CS9X7 = 0, /* 31 bits: bit = I(p+o) > I(p-o), the offsets before the centre */
    SGMF_CENSUS_9X7 = 1    /* 62 bits: bit = I(p+o) > I(p), every offset */
};

/* Consistency-check variants of Table V. */
enum {
    SGMF_CHECK_STEREO_LIDAR = 0, /* Eq. 6: stereo term OR LiDAR term (the method) */
    SGMF_CHECK_STEREO = 1,       /* stereo term only (left-right check) */
    SGMF_CHECK_LIDAR = 2,        /* LiDAR term only (camera-LiDAR check) */
    SGMF_CHECK_NONE = 3          /* no check: D^{c*} = D* */
};

/* Parameters; sgmf_default_params() fills Table II of the paper. */
typedef struct {
    int32_t p1, p2;               /* SGM penalties, Eq. 1/2 (10, 120); 0 <= p1 <= p2 <= 2048 */
    int32_t q1, q2;               /* DDC penalties, Eq. 4 (5, 160); 0 <= q1 <= q2 */
    int32_t alpha_num, alpha_den; /* alpha = num/den of Eq. 4 (7/10); 0 <= num <= den, den >= 1 */
    int32_t ts, rs;               /* semidensification threshold / window radius, Eq. 5 (2, 6); ts <= 65535, rs <= 255 */
    int32_t tc, rc;               /* consistency threshold / window radius, Eq. 6 (2, 20); tc <= 65535, rc <= 255 */
    int32_t lr_max_diff;          /* stereo term of Eq. 6: |d* - d'| <= lr_max_diff (1); <= 65535 */
    int32_t census;               /* SGMF_CENSUS_* (SGMF_CENSUS_CS9X7) */
    int32_t semidense;            /* 1 = SDSGM, 0 = DSGM (Table I) */
    int32_t consistency;          /* SGMF_CHECK_* (SGMF_CHECK_STEREO_LIDAR) */
    int32_t num_paths;            /* 8 (Sec. III) or 4 (horizontal + vertical) */
    int32_t subpixel;             /* 0 (default): out_disp holds integer d*; 1: pixels that pass the
                                     check hold the parabola-fit disparity of Sec. III (after Eq. 3)
                                     in 1/16 px, i.e. 16 d* + round-half-up(16 (S(d*-1) - S(d*+1)) /
                                     (2 (S(d*-1) - 2 S(d*) + S(d*+1)))), and 16 d* where d* = 0 or
                                     D - 1; invalid stays -1 */
} sgmf_params;

/* Intermediate maps that sgmf_debug_stage() can copy out (test use). */
enum {
    SGMF_STAGE_DBAR = 0,     /* int16 H x W: sparse map d-bar (Sec. IV) */
    SGMF_STAGE_CENSUS_L = 1, /* uint64 H x W: census of the left image */
    SGMF_STAGE_CENSUS_R = 2, /* uint64 H x W: census of the right image */
    SGMF_STAGE_DHAT = 3,     /* int16 H x W: prior used by the DDC (d-hat, or d-bar for DSGM) */
    SGMF_STAGE_COST = 4,     /* uint8 H x W x D: joint cost C-bar of Eq. 4 */
    SGMF_STAGE_SUM = 5,      /* uint16 H x W x D: S = sum_r L_r; only after sgmf_set_debug(c, 1) */
    SGMF_STAGE_DSTAR = 6,    /* int16 H x W: d* of Eq. 3 */
    SGMF_STAGE_DPRIME = 7,   /* int16 H x W: d' of the right view (diagonal search) */
    SGMF_STAGE_DSUB = 8,     /* int16 H x W: sub-pixel disparity in 1/16 px; only with subpixel = 1 */
    SGMF_STAGE_BOX_S = 9,    /* uint32 MW x H x W (MW = 2, 4, 6, 8 for D <= 64, 128, 192, 256):
                                bit d % 32 of word plane d / 32 set when a pixel of the
                                (2 rs + 1)^2 window (Eq. 5) has d-bar = d; only with semidense */
    SGMF_STAGE_BOX_C = 10    /* the same with radius rc (Eq. 6); only with a LiDAR check */
};

/* Fill *p with Table II of the paper (and the documented readings). */
void sgmf_default_params(sgmf_params *p);

/* Create a context for width x height images and max_disp disparities
 * (d in [0, max_disp - 1]) on the CURRENT CUDA device.  Allocates all device
 * scratch (census, masks, cost volume, partial sums) once; nothing is
 * allocated per frame.  Limits: 1 <= width, height <= 8192,
 * 1 <= max_disp <= 256.  *out receives the context (NULL on error).
 * Errors: SGMF_ERR_ARG (out NULL), SGMF_ERR_SHAPE, SGMF_ERR_OOM,
 * SGMF_ERR_CUDA. */
sgmf_status sgmf_create(int width, int height, int max_disp, sgmf_ctx **out);

/* As sgmf_create, for batches: the context holds device buffers for up to
 * max_batch frames (1 <= max_batch <= 4096) of the same shape, which
 * sgmf_compute_batch processes in one pass of every kernel (each launch
 * covers all frames).  Device memory grows linearly with max_batch. */
sgmf_status sgmf_create_batched(int width, int height, int max_disp, int max_batch, sgmf_ctx **out);

/* Number of frames the context's buffers hold (its max_batch). */
int sgmf_batch_capacity(const sgmf_ctx *c);

/* Validate *p and copy it into the context.  On SGMF_ERR_PARAM the previous
 * parameters stay in force.  Besides the ranges listed in sgmf_params, the
 * largest joint cost C-bar (over H <= census bits and q in {0, q1, q2}) must
 * not exceed 255 (costs are stored as uint8). */
sgmf_status sgmf_set_params(sgmf_ctx *c, const sgmf_params *p);

/* Copy the context's parameters into *p. */
sgmf_status sgmf_get_params(const sgmf_ctx *c, sgmf_params *p);

/* Run every later call on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream).  The stream stays owned by the caller. */
sgmf_status sgmf_set_stream(sgmf_ctx *c, void *cuda_stream);

/* The whole pipeline on DEVICE pointers, enqueued on the context's stream;
 * returns without waiting.  left, right: uint8 H x W rectified images.
 * sparse_lidar_disp: float32 H x W LiDAR disparity aligned with the left
 * image, 0 (or any value <= 0, or non-finite) = no return; NULL = no LiDAR.
 * out_disp: int16 H x W, receives D^{c*} (-1 invalid).  The caller owns all
 * four buffers and must keep them alive until the stream reaches this work.
 * Errors: SGMF_ERR_ARG for NULL images/output; SGMF_ERR_CUDA if a launch
 * fails; asynchronous device errors surface in sgmf_sync(). */
sgmf_status sgmf_compute(sgmf_ctx *c, const uint8_t *left, const uint8_t *right,
                         const float *sparse_lidar_disp, int16_t *out_disp);

/* The pipeline on n frames at once (1 <= n <= the batch capacity), DEVICE
 * pointers: left, right, out hold n contiguous H x W frames ([n][H][W]);
 * sparse_lidar_disp is [n][H][W] float32 or NULL (no LiDAR for any frame).
 * Same ownership, stream and error behaviour as sgmf_compute; the frames are
 * independent (sgmf_compute is this call with n = 1). */
sgmf_status sgmf_compute_batch(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                               const float *sparse_lidar_disp, int16_t *out_disp);

/* The same pipeline on HOST pointers: copies the inputs to device staging
 * buffers owned by the context, runs sgmf_compute, copies the result back
 * and waits for the stream.  Pinned host memory gives asynchronous copies;
 * pageable memory works too.  Same arguments and errors as sgmf_compute,
 * plus everything sgmf_sync reports. */
sgmf_status sgmf_compute_host(sgmf_ctx *c, const uint8_t *left, const uint8_t *right,
                              const float *sparse_lidar_disp, int16_t *out_disp);

/* sgmf_compute_host for n frames ([n][H][W] host buffers), with the
 * copies of all n frames in and out around one sgmf_compute_batch. */
sgmf_status sgmf_compute_host_batch(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                    const float *sparse_lidar_disp, int16_t *out_disp);

/* sgmf_compute_host_batch without the wait: copies in, pipeline and copy out
 * are enqueued on the context's stream and the call returns; the host
 * buffers must stay untouched (and `out` unread) until sgmf_sync(c).  With
 * PINNED host buffers the copies run asynchronously, so two contexts on two
 * streams overlap one batch's copies with the other's kernels. */
sgmf_status sgmf_compute_host_batch_async(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                          const float *lidar, int16_t *out);

/* Wait for the context's stream and report the first asynchronous error:
 * SGMF_ERR_TIMEOUT if a bounded device wait gave up, SGMF_ERR_CUDA for a
 * CUDA error.  The timeout flag is cleared by this call. */
sgmf_status sgmf_sync(sgmf_ctx *c);

/* Free the context and everything it allocated.  NULL is allowed. */
void sgmf_destroy(sgmf_ctx *c);

/* Message of the last failed call on c (never NULL; "" when none).  With
 * c == NULL, the message of the last failed sgmf_create on this thread. */
const char *sgmf_last_error(const sgmf_ctx *c);

/* Static name of a status code. */
const char *sgmf_status_string(sgmf_status s);

/* Keep the aggregate S of frame 0 of the next sgmf_compute calls for
 * SGMF_STAGE_SUM (allocates H x W x D uint16 once; enable = 0 frees it). */
sgmf_status sgmf_set_debug(sgmf_ctx *c, int enable);

/* Copy an intermediate of frame 0 of the last sgmf_compute or
 * sgmf_compute_batch (see SGMF_STAGE_*) into host memory host_dst of `bytes`
 * bytes; waits for the stream first.
 * Errors: SGMF_ERR_ARG for an unknown stage, a NULL destination, too few
 * bytes, or SGMF_STAGE_SUM without sgmf_set_debug(c, 1). */
sgmf_status sgmf_debug_stage(sgmf_ctx *c, int stage, void *host_dst, size_t bytes);

/* Number of kernel launches one sgmf_compute enqueues with the current
 * parameters (for launch accounting). */
int sgmf_launches_per_compute(const sgmf_ctx *c);

/* Record CUDA events around every kernel of the following sgmf_compute
 * calls (enable = 1) or stop (0). */
sgmf_status sgmf_set_profiling(sgmf_ctx *c, int enable);

/* After sgmf_sync: per-kernel durations (ms) of the last profiled
 * sgmf_compute.  names[i] (static strings) and ms[i] for i < *n on input
 * (capacity); *n receives the number of kernels recorded. */
sgmf_status sgmf_kernel_times(sgmf_ctx *c, const char **names, float *ms, int *n);

/* Bytes of device memory the context holds. */
size_t sgmf_device_bytes(const sgmf_ctx *c);

/* ---- Failure handling (no counterpart in the paper) ---------------------
 * Every device wait of the library (TMA and bulk copies into shared memory,
 * the cluster sweep's messages) polls a bounded number of times.  A wait
 * that gives up records SGMF_ERR_TIMEOUT in the context's error word, waits
 * again (with the default limit) for the copies its CTA issued, and returns:
 * nothing faults, the context stays usable, and sgmf_sync reports
 * SGMF_ERR_TIMEOUT (the outputs of that call are then undefined). */
#define SGMF_WAIT_CENSUS 0   /* the census kernel's wait for its TMA image tiles */

/* Poll limit of one kind of device wait of c (which = SGMF_WAIT_CENSUS):
 * polls >= 0 sets it (0 gives up before the first poll, so every census CTA
 * takes the timeout path: this is how the tests reach it), polls < 0
 * restores the default 2^22.  Applies to the following computes.
 * Errors: SGMF_ERR_ARG (NULL c, unknown wait). */
sgmf_status sgmf_set_wait_limit(sgmf_ctx *c, int which, long long polls);

/* ---- Instruction rates (no counterpart in the paper) ----------------------
 * The integer path's roofline needs the rates at which the device issues the
 * instructions the method is made of.  Lanes per clock per SM of each kind,
 * measured on the current device by one CTA of 1024 threads per SM, eight
 * independent chains a thread, iters x 16 steps a chain, timed by the CTA's
 * clock64 span (the median CTA); independent of the SM clock. */
typedef struct {
  int sms;               /* SMs of the device                              */
  double min3_u16x2;     /* __vimin3_u16x2: 3-input min of two u16 halves  */
  double addmin_u16x2;   /* __viaddmin_u16x2: min(a + b, c) per u16 half   */
  double iadd;           /* 32-bit add                                     */
  double popc;           /* __popc (population count)                      */
  double prmt;           /* __byte_perm                                    */
} sgmf_rates;

/* Run the probes (synchronises the device; a few ms at iters = 256).
 * Errors: SGMF_ERR_ARG (out NULL, iters outside [1, 2^20]), SGMF_ERR_CUDA. */
sgmf_status sgmf_measure_rates(int iters, sgmf_rates *out);

/* Test hook for allocation failure: on the calling thread, the n-th device
 * allocation that a context makes from now on (n >= 1) fails as if the
 * device were out of memory, without calling cudaMalloc; n <= 0 clears it.
 * The failing call (sgmf_create*, or the first sgmf_compute_host* or
 * sgmf_set_debug that allocates) returns SGMF_ERR_OOM and keeps nothing it
 * allocated: a failed sgmf_create frees every buffer it had obtained. */
void sgmf_debug_fail_alloc(int n);

/* ---- Banded mode (no counterpart in the paper) ---------------------------
 * The method restricted to a disparity band per pixel: pixel p keeps the
 * disparities [lo_p, lo_p + band); lo_p is constant on 8 x 8 pixel tiles.
 * Eq. 2 runs on the bands (a term whose disparity is outside the previous
 * pixel's band is left out; m is the min over that band), d* is the argmin
 * over the pixel's band, d'(x') the argmin over the cells (x' + d, d) that
 * lie inside the bands (-1 where there is none, and the stereo term of Eq. 6
 * then fails); census, semidensification, Eq. 4 and the check are unchanged.
 * With band starts 0 and band = max_disp this is the plain method.  Cost,
 * path costs and S take band / Dp of the plain volumes' memory and work. */

/* A banded context: band = 64 or 128, band <= max_disp.  sgmf_compute on it
 * fails; use sgmf_compute_banded.  Errors as sgmf_create_batched. */
sgmf_status sgmf_create_banded(int width, int height, int max_disp, int band, int max_batch, sgmf_ctx **out);

/* sgmf_compute_batch with band starts: band_lo is a DEVICE int16 array
 * [n][ceil(H / 8)][ceil(W / 8)] (tile rows, then tile columns); values are
 * clamped to [0, max_disp - band].  subpixel must be 0. */
sgmf_status sgmf_compute_banded(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                const float *lidar, const int16_t *band_lo, int16_t *out);

/* The two halves of sgmf_compute_banded, for callers that choose the bands
 * from the semidensified map: sgmf_compute_front runs ingest, census and
 * semidensification of n frames; the prior of Eq. 4 (d-hat, or d-bar for
 * DSGM) is then in the DEVICE buffer sgmf_prior_device(c), int16
 * [frame][H][W] (stream-ordered: read it on the context's stream);
 * sgmf_compute_banded_back(c, n, band_lo, out) finishes the same n frames. */
sgmf_status sgmf_compute_front(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                               const float *lidar);
const int16_t *sgmf_prior_device(const sgmf_ctx *c);
sgmf_status sgmf_compute_banded_back(sgmf_ctx *c, int n, const int16_t *band_lo, int16_t *out);

/* ---- Band-proposal network (no counterpart in the paper) -------------------
 * A six-layer 3x3 CNN with 32 channels at quarter resolution (H4 =
 * ceil(H/4), W4 = ceil(W/4)) proposes a band per pixel from the left image
 * and d-hat.  Its convolutions run on the tensor cores (BF16 operands, FP32
 * accumulation).  All pointers are DEVICE pointers; every call is
 * asynchronous on `stream` (NULL = legacy default stream) and returns
 * SGMF_ERR_ARG for bad sizes or NULL buffers, SGMF_ERR_CUDA when a launch
 * (or the device query that sizes its grid) fails.  Tensors are channel-last:
 * activations bf16 [n][h][w][32]; weights bf16 [co][ky][kx][ci] (32 x 3 x 3 x
 * 32); bias f32 [32].  `err` is a device int that a bounded wait sets to
 * SGMF_ERR_TIMEOUT (6). */

/* Pack weights into the tensor-core operand images (18432 bytes each):
 * packed_fwd for sgmf_bn_conv forward, packed_dgrad (the kernel rotated by
 * 180 degrees, in and out channels swapped) for the data gradient.  Either
 * output may be NULL. */
sgmf_status sgmf_bn_pack(const uint16_t *w, uint16_t *packed_fwd, uint16_t *packed_dgrad, void *stream);

/* y = conv3x3(x) with zero padding: + bias (or NULL), ReLU if relu, then
 * zeroed where mask (bf16 activations, or NULL) is not > 0; written as bf16
 * to y and / or f32 to yf (either may be NULL, not both).  With packed_dgrad
 * weights, no bias, no ReLU and the layer input as mask this is the data
 * gradient through conv + ReLU. */
sgmf_status sgmf_bn_conv(int n, int h, int w, const uint16_t *x, const uint16_t *packed, const float *bias,
                         int relu, const uint16_t *mask, uint16_t *y, float *yf, int *err, void *stream);

/* Weight gradient: dw[co][ky][kx][ci] += sum_p dy[p][co] x[p + (ky-1, kx-1)][ci]
 * and db[co] += sum_p dy[p][co] (f32, accumulated: zero them first).  The
 * sums are deterministic (per-CTA partials added in a fixed order); the
 * partials live in one library-wide device array, so calls must not overlap
 * on the GPU. */
sgmf_status sgmf_bn_wgrad(int n, int h, int w, const uint16_t *x, const uint16_t *dy, float *dw, float *db,
                          int *err, void *stream);

/* Network input from left uint8 [n][H][W] and d-hat int16 [n][H][W]: per 4 x 4
 * block (clipped at the border) channel 0 = mean(left) / 255 - 0.5, 1 = mean
 * of the valid d-hat / max_disp (0 without one), 2 = valid d-hat / 16; the
 * other channels 0.  x: bf16 [n][H4][W4][32]. */
sgmf_status sgmf_bn_input(int n, int width, int height, int max_disp, const uint8_t *left, const int16_t *dhat,
                          uint16_t *x, void *stream);

/* Training labels from disparity maps disp int16 [n][H][W] (-1 invalid): per
 * quarter pixel lohi[2i] / lohi[2i+1] = min / max of the valid disparities
 * of its 4 x 4 block (-1 / -1 without one); *count += labelled pixels. */
sgmf_status sgmf_bn_labels(int n, int width, int height, const int16_t *disp, int16_t *lohi, int *count,
                           void *stream);

/* Band loss over npix quarter pixels (out: f32 [npix][32], the last layer):
 * centre c = D o0, half-width w = 8 + 40 sigmoid(o1), confidence q =
 * sigmoid(o2); per labelled pixel lam_c |c - c_t| / D + lam_w |w - w_t| / D +
 * BCE(q, y) with c_t = (lo + hi) / 2, w_t = clamp((hi - lo) / 2 + 2, 8, 48),
 * y = [c - w, c + w] covers [lo, hi]; mean over *count.  grad: bf16
 * [npix][32] (channels 0..2); *loss += the loss. */
sgmf_status sgmf_bn_loss(long long npix, int max_disp, const float *out, const int16_t *lohi, const int *count,
                         uint16_t *grad, float *loss, float lam_c, float lam_w, void *stream);

/* Adam on count f32 parameters (bias-corrected, step >= 1); w_bf16 (or NULL)
 * receives the bf16 copy. */
sgmf_status sgmf_bn_adam(int count, float *w, float *m, float *v, const float *g, float lr, float b1, float b2,
                         float eps, int step, uint16_t *w_bf16, void *stream);

/* Training batch: dst row i = src row idx[i] for i < n <= 65535 (rows of
 * row_bytes bytes, a multiple of 4; src and dst 4-byte aligned; idx device
 * int32; src holds `rows` rows, and an entry outside [0, rows) leaves its
 * destination row untouched).  Errors: SGMF_ERR_ARG. */
sgmf_status sgmf_bn_gather(int n, const int *idx, long long rows, long long row_bytes, const void *src, void *dst,
                           void *stream);

/* bf16 copy (round to nearest, ties to even) of count f32 weights. */
sgmf_status sgmf_bn_to_bf16(int count, const float *w, uint16_t *w_bf16, void *stream);

/* Band starts from the network output out (f32 [n][H4][W4][32]) for a
 * banded context of width `band`: per 8 x 8 tile the union [lo, hi] of the
 * pixels' bands [c - w, c + w], start round((lo + hi) / 2) - band / 2 clamped
 * to [0, max_disp - band] into lo_tiles int16 [n][ceil(H/8)][ceil(W/8)];
 * uncertain[f] (n device ints, zeroed by the caller) += the tiles of frame f
 * whose smallest confidence is below conf_min or whose union is wider than
 * the band. */
sgmf_status sgmf_bn_tiles(int n, int width, int height, int max_disp, int band, float conf_min, const float *out,
                          int16_t *lo_tiles, int *uncertain, void *stream);

/* sgmf_debug_stage on a banded context returns COST as uint8 and SUM as
 * uint16 H x W x band (cell j = disparity lo_p + j; SUM needs no
 * sgmf_set_debug there).  The context's band width (0 for a plain context): */
int sgmf_band_width(const sgmf_ctx *c);

/* The per-frame choice among band widths and the plain method, made on the
 * device (no host round trip): gate[f] = value when frame f has at most
 * max_frac * tiles uncertain tiles (uncertain: the counts of sgmf_bn_tiles
 * for one band width), else `otherwise` (otherwise < 0 keeps gate[f]).
 * Called once per band width, widest first with otherwise = the plain
 * method's value, then narrower ones with otherwise = -1, the narrowest
 * acceptable width wins.  Each context then runs only its frames
 * (sgmf_set_gate).  Errors: SGMF_ERR_ARG. */
sgmf_status sgmf_bn_decide(int n, int tiles, float max_frac, const int *uncertain, int value, int otherwise,
                           int *gate, void *stream);

/* Per-frame gating of a context's kernels (no counterpart in the paper):
 * with gate (device int array, one word per frame of a compute call, frame i
 * at gate[i]) non-NULL, every kernel the context launches does nothing for
 * frame i unless gate[i] == run; NULL runs every frame (the default).  The
 * launches still happen (a skipped frame costs only its CTAs' start), so
 * several contexts can share one batch's frames by a decision that a kernel
 * wrote, without the host waiting for it.  The gate memory must stay valid
 * while launches that read it are in flight.  Errors: SGMF_ERR_ARG. */
sgmf_status sgmf_set_gate(sgmf_ctx *c, const int *gate, int run);

/* ---- Launch tuning (no counterpart in the paper) -----------------------
 * Launch shapes only: every choice gives bit-identical results. */
typedef struct {
    int32_t line_warps;   /* warps per CTA of the vertical/diagonal line kernels
                             (each warp walks two lines): 1, 2, 4 (default) or 8 */
    int32_t cost_px;      /* the cost kernel takes row segments of at most
                             8 x cost_px pixels per CTA: 32, 64 or 128 (default;
                             segments of up to 1024 pixels) */
    int32_t sweep;        /* 1: the six vertical and diagonal directions run as two
                             row-synchronous sweeps of a thread-block cluster per
                             frame (one launch) instead of the three line kernels
                             (line_warps is then unused).  0 (default) or 1; 1 needs
                             a row of at most 16 CTAs x 128 pixels (Dp <= 128; banded:
                             x 160) or 16 x 80 pixels (Dp > 128) and
                             a device that can place such a cluster (the context
                             picks the cluster size that keeps the most CTAs
                             resident), and is refused otherwise; it takes effect
                             with 8 paths. */
    int32_t parts;        /* with the sweep: 1 (default) runs a batch in parts of one
                             sweep wave, each part's row kernel on a second stream
                             beside the next part's sweep; 0 runs the whole batch
                             through each kernel in one launch.  0 or 1. */
} sgmf_tuning;

/* Set / read the context's tuning.  SGMF_ERR_ARG for other values. */
sgmf_status sgmf_set_tuning(sgmf_ctx *c, const sgmf_tuning *t);
sgmf_status sgmf_get_tuning(const sgmf_ctx *c, sgmf_tuning *t);

/* Autotuner.  Runs sgmf_compute_batch(c, n, left, right, lidar, out) on the
 * caller's DEVICE frames once per candidate (the 4 x 3 line-kernel tunings,
 * and the sweep with each of the 3 cost shapes where it fits) as a
 * warm-up, then `reps` timed runs, each after overwriting up to 256 MiB of
 * the context's scratch so that it starts with a cold L2 (CUDA events on the
 * context's stream, 1 <= reps <= 100); keeps the candidate with the smallest median time in
 * the context and returns it in *best and its median in *best_ms (either may
 * be NULL).  Synchronises the stream; out receives the (identical) output. */
sgmf_status sgmf_autotune(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right, const float *lidar,
                          int16_t *out, int reps, sgmf_tuning *best, float *best_ms);

/* ---- Mixed-size batches in one CUDA-graph launch (no counterpart in the paper)
 * A multi-batch holds n frames whose shapes may differ.  Frames of equal
 * (width, height, max_disp) form a class; each class owns one batched context
 * (all of a class's frames go through each kernel in one launch), one stream
 * and RESIDENT device buffers for its frames' inputs and outputs, so that the
 * whole batch can be captured once as a CUDA graph (the classes as parallel
 * branches) and replayed with one cudaGraphLaunch per call.  Errors of these
 * calls are reported in sgmf_last_error(NULL). */
typedef struct {
    int32_t width, height, max_disp;
} sgmf_shape;
typedef struct sgmf_multi sgmf_multi;

/* Creates the batch on the current device; p = NULL selects Table II.
 * Errors: SGMF_ERR_ARG, SGMF_ERR_SHAPE (1 <= n <= 4096, shapes as in
 * sgmf_create), SGMF_ERR_PARAM, SGMF_ERR_OOM / SGMF_ERR_CUDA. */
sgmf_status sgmf_multi_create(const sgmf_shape *shapes, int n, const sgmf_params *p, sgmf_multi **out);

/* Device buffers of frame i (any pointer may be NULL): left / right uint8
 * H x W, lidar float32 H x W (0 = no return; zero-filled at creation), out
 * int16 H x W.  They stay valid and fixed until sgmf_multi_destroy: fill the
 * inputs (on any stream, ordered before sgmf_multi_launch) and read out_disp
 * after it. */
sgmf_status sgmf_multi_frame(sgmf_multi *m, int i, uint8_t **left, uint8_t **right, float **lidar,
                             int16_t **out);

/* Number of classes; shape, frame count and tuning of class `cls`. */
int sgmf_multi_classes(const sgmf_multi *m);
sgmf_status sgmf_multi_class_info(const sgmf_multi *m, int cls, sgmf_shape *shape, int *frames,
                                  sgmf_tuning *t);

/* sgmf_autotune for every class on its resident frames (`reps` timed runs
 * per candidate); drops a captured graph so that the next launch recaptures
 * with the chosen tunings.  Synchronous. */
sgmf_status sgmf_multi_autotune(sgmf_multi *m, int reps);

/* Runs the whole batch on `stream` (NULL = the batch's own stream) as one
 * CUDA graph launch.  The first call (and the first after autotuning) runs
 * every class once outside capture, then captures the batch into a graph;
 * later calls only launch the graph.  Asynchronous: sgmf_multi_sync waits and
 * surfaces device errors (including SGMF_ERR_TIMEOUT). */
sgmf_status sgmf_multi_launch(sgmf_multi *m, void *stream);
sgmf_status sgmf_multi_sync(sgmf_multi *m);

/* Kernel launches one sgmf_multi_launch replays (summed over classes). */
int sgmf_multi_launches(const sgmf_multi *m);

/* Device bytes held (contexts and resident buffers). */
size_t sgmf_multi_device_bytes(const sgmf_multi *m);

/* Frees everything (NULL-safe); waits for the batch's work first. */
void sgmf_multi_destroy(sgmf_multi *m);

/* ---- Serving: a request loop for several cameras (no counterpart in the paper)
 * Requests (one pair + LiDAR map in HOST memory, pinned memory recommended)
 * are submitted from any thread and come back through sgmf_server_poll.
 * Cameras of equal shape share one queue.  One worker thread owns the GPU
 * work: whenever a batched context ("slot", max_batch frames with resident
 * device buffers and its own stream) of a shape is idle it takes every
 * waiting request of that shape, up to max_batch, and runs copy-in, the
 * pipeline (one sgmf_compute_batch) and copy-out on the slot's stream.
 * Requests that arrive meanwhile wait for the next idle slot: batches form
 * continuously while earlier ones are on the GPU, and the slots of
 * different shapes (and up to max_slots_per_shape of one shape) overlap on
 * the device.  Slots are created while their device bytes fit the budget
 * (admission by device memory).  A frame's result does not depend on which
 * batch or slot it ran in.  Errors of these calls are reported in
 * sgmf_last_error(NULL). */
typedef struct sgmf_server sgmf_server;
typedef struct {
    uint64_t submitted, completed;  /* requests */
    uint64_t batches, batched_frames;
    int32_t largest_batch;          /* frames in the largest batch so far */
    int32_t max_concurrent_batches; /* most batches in flight at once */
    int32_t slots;                  /* slots created */
    size_t device_bytes, peak_device_bytes, budget_bytes;
} sgmf_server_counters;

/* Starts the worker on the current device.  p = NULL selects Table II.
 * 1 <= max_batch <= 256, 1 <= max_slots_per_shape <= 16.  Errors:
 * SGMF_ERR_ARG, SGMF_ERR_PARAM, SGMF_ERR_OOM. */
sgmf_status sgmf_server_create(const sgmf_params *p, size_t device_budget_bytes, int max_batch,
                               int max_slots_per_shape, sgmf_server **out);

/* Registers a camera; returns its id (>= 0) or minus an sgmf_status.  The
 * first camera of a shape creates that shape's first slot and is refused
 * with -SGMF_ERR_OOM if it does not fit the remaining budget.  Call from one
 * thread (cameras may be added while requests run). */
int sgmf_server_add_camera(sgmf_server *s, int width, int height, int max_disp);

/* Queues one request.  left / right uint8 H x W, lidar float32 H x W or NULL
 * (no LiDAR), out int16 H x W: host buffers that must stay valid until the
 * request is returned by sgmf_server_poll.  Returns at once. */
sgmf_status sgmf_server_submit(sgmf_server *s, int camera, const uint8_t *left, const uint8_t *right,
                               const float *lidar, int16_t *out, uint64_t tag);

/* Returns 1 and one finished request (tag, camera, status, latency from
 * submit to the output landing in host memory, in ms), or 0 if none finished
 * within wait_ms; -SGMF_ERR_ARG for a NULL server.  Any pointer may be NULL. */
int sgmf_server_poll(sgmf_server *s, int wait_ms, uint64_t *tag, int *camera, int *status, double *latency_ms);

sgmf_status sgmf_server_stats(sgmf_server *s, sgmf_server_counters *out);

/* Finishes every queued and running request, stops the worker, frees all
 * slots (NULL-safe).  Requests finished but not polled are dropped. */
void sgmf_server_destroy(sgmf_server *s);

/* The three-view consistency stage alone, without a context and without
 * allocating anything.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory where they call it
 * (a pool they do not own, a real-time loop that forbids cudaMalloc after
 * start-up, a plugin host that only hands out input and output buffers).
 *
 * Gives the same output as sgmf_compute's consistency stage for the same
 * d*, d' and LiDAR map, for one width x height frame, from caller-owned
 * DEVICE buffers: dstar and
 * dprime (int16 H x W, d* and d' of the frame, e.g. SGMF_STAGE_DSTAR /
 * SGMF_STAGE_DPRIME), sparse_lidar_disp (float32 H x W, the same LiDAR map
 * given to sgmf_compute, or NULL) and out_disp (int16 H x W).  p supplies
 * tc, rc, lr_max_diff and consistency (validated like sgmf_set_params;
 * subpixel must be 0: the output is the integer d* or -1).
 * Enqueued on cuda_stream (NULL = legacy default stream); returns without
 * waiting.
 *
 * Working memory is one file-scope device array of 32 MiB (8 Mi 32-bit
 * words) that every GPU loading this library holds until the process exits;
 * a frame needs 3 * W * H * ceil(max_disp / 64) * 2 words (for max_disp <= 128
 * about 700 000 pixels fit).  Larger frames are rejected with SGMF_ERR_SHAPE
 * before anything is launched.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * (and again if the device's context was made anew, e.g. after
 * cudaDeviceReset); make that first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU race.  No cudaMalloc, cudaFree or
 * allocating library call is made.  Errors: SGMF_ERR_ARG, SGMF_ERR_SHAPE,
 * SGMF_ERR_PARAM, SGMF_ERR_CUDA; the message is in sgmf_last_error(NULL). */
sgmf_status sgmf_check_static(int width, int height, int max_disp, const sgmf_params *p,
                              const int16_t *dstar, const int16_t *dprime,
                              const float *sparse_lidar_disp, int16_t *out_disp, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SGMF_H_ */
