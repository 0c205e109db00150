/*
 * bfm.h -- C ABI of the GB300 BFAST Monitor library (libbfm.so).
 *
 * BFAST Monitor (von Mehren et al., "Massively-Parallel Break Detection for
 * Satellite Data", 2018) fits, for every pixel of an image time series, the
 * season-trend model of Section 2.1 (Eq. 1-2) by least squares on a stable
 * history period (Eq. 5-6), then tests the residual MOSUM process of the
 * monitoring period (Eq. 3) against the boundary lambda*sqrt(log+(t/n))
 * (Eq. 4); Algorithm 1 lists the steps for one series, Algorithm 2 the
 * many-series form this library implements on the GPU.
 *
 * Conventions common to all calls
 *  - No exceptions and no aborts cross this ABI.  Every call returns a
 *    bfm_status; on failure bfm_last_error() gives a message (per thread).
 *  - Device pointers are CUDA device addresses on the current device; the
 *    caller owns them and keeps them alive until the work on `stream` ends.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device calls only enqueue work and return; nothing
 *    synchronises unless stated.
 *  - Y is time-major: Y[t*m + p] is date t of pixel p (the matrix Y of
 *    Section 3, Eq. 7).  BFM_F32: float, NaN marks a missing observation.
 *    BFM_I16: int16 (e.g. NDVI*1e4), -32768 marks a missing observation; the
 *    stored integers are the series values (outputs are in those units).
 *  - mask_bits (nullable) adds an explicit validity mask [N][ceil(m/32)]
 *    uint32 words, bit (p % 32) of word p/32 of row t, 1 = valid; it is
 *    ANDed with the missing marker.
 *  - Missing data (a reading; the paper assumes complete series, Section 3):
 *    each pixel keeps its valid observations in date order; history size
 *    n_p counts valid observations among the first n_hist dates; MOSUM
 *    positions, n and h count valid observations; regressors use the actual
 *    date values (Section 4.3).  For complete series this is exactly
 *    Algorithm 1 with h terms per window (Eq. 3, Algorithm 3).
 */
#ifndef BFM_H
#define BFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFM_OK = 0,
    BFM_EINVAL = 1,      /* an argument is out of range (message says which) */
    BFM_ENOMEM = 2,      /* a host or device allocation failed */
    BFM_ECUDA = 3,       /* a CUDA runtime/driver call failed */
    BFM_ETIMEOUT = 4,    /* a bounded wait gave up (device error word set) */
    BFM_EBUSY = 5,       /* admission refused: over the memory budget */
    BFM_EUNSUPPORTED = 6 /* valid request this build cannot run (e.g. N too long) */
} bfm_status;

typedef enum { BFM_F32 = 0, BFM_I16 = 1 } bfm_dtype;

/* Per-pixel status codes written to the `status` output (not errors). */
enum {
    BFM_PX_OK = 0,
    BFM_PX_INSUFFICIENT_HISTORY = 1, /* n_p <= K: no fit; beta, sigma, mean NaN */
    BFM_PX_SINGULAR = 2,             /* rank test failed (see bfm_monitor); NaN outputs */
    BFM_PX_DEGENERATE = 3,           /* sigma-hat <= 1e-6 max|y_hist|: MO = 0, mean 0 */
    BFM_PX_NO_MONITOR = 4,           /* no valid monitoring observation: mean NaN */
    BFM_PX_INCOMPLETE = 5,           /* BFM_ALGO_COMPLETE only: a missing value; NaN outputs */
    BFM_PX_TIMEOUT = 255             /* the tile's load wait gave up (device error) */
};

/* Algorithm variants for bfm_monitor_ex.  BFM_ALGO_AUTO takes the hybrid
 * form (BFM_ALGO_HYBRID, below) where it applies, else the streaming form
 * (BFM_ALGO_STREAM) where it applies, else the tensor-core form where it
 * applies -- its shared memory (basis tables over the N dates, a MOSUM ring
 * of floor(h_frac * n_hist) + 17 prefix sums per pixel, the Y stages) fits
 * one SM, and Y can be described by a tensor map (16-byte aligned base,
 * m >= 128, rows a multiple of 16 bytes) -- else the CUDA-core form
 * (bfm_algo_auto tells which).
 * BFM_ALGO_COMPLETE is never chosen by AUTO: it is the fast path for series
 * without missing values (Section 3, Eq. 8-11), where every pixel shares the
 * history design X_h and beta = M y_h with one M = (X_h'X_h)^-1 X_h' built in
 * FP64 on the host on first use per (design, n_hist) (a synchronous upload
 * of (n_hist + N) * K floats, kept with the design).  One thread per pixel
 * streams its column: beta = M y_h (FP32, 32-date blocks added with TwoSum
 * compensation), the history residuals and sigma-hat (history re-read from
 * L2), then the monitoring dates with a running window sum whose leaving
 * term is recomputed from y (Algorithm 3).  The same outputs as the other
 * forms, with h = clamp(floor(h_frac * n_hist), 1, n_hist) for every pixel;
 * when the shared design fails the rank test every pixel is SINGULAR
 * (n_hist <= K: INSUFFICIENT_HISTORY).  A pixel with any missing value
 * (NaN, -32768 or a 0 mask bit) gets BFM_PX_INCOMPLETE, break -1 and NaN
 * outputs; run the general forms on such pixels.
 * BFM_ALGO_STREAM: the general definition (missing values allowed) with one
 * CUDA-core thread per pixel.  Each pixel's column is streamed four times
 * (masked basis sums and X'My; refinement sums; the first window; the
 * monitoring dates) through shared-memory stages filled by 2-D TMA boxes of
 * 256 pixels, the history kept in L2 between its passes; FP32 normal
 * equations with one refinement step as in the CUDA-core form, the MOSUM
 * window from a per-thread ring of the last h_p residuals.  Needs Y with a
 * 16-byte aligned base and rows of a multiple of 16 bytes, and the basis
 * tables plus floor(h_frac * n_hist) ring slots per pixel within 112 KB of
 * shared memory (else BFM_EUNSUPPORTED).
 * BFM_ALGO_HYBRID: the streaming scan with every contraction over dates on
 * the tensor cores (tcgen05, accumulators and A operands in tensor memory):
 * the masked basis sums (fp16 basis hi + lo) and X'My (tf32) per 16-date
 * chunk, the fitted values of beta0 and of beta0 + delta (fp16 hi + lo
 * coefficients and regressors) per 32-date piece, and the refinement sums
 * X'M r0 (fp16 hi + lo residuals).  512 pixels per CTA, one CTA per SM, three
 * passes over each pixel's column (history twice, then the dates from the
 * earliest first-window observation of the tile on).  Same outputs and
 * conventions as BFM_ALGO_STREAM.  Needs Y with a 16-byte aligned base and
 * rows of a multiple of 16 bytes, and the tables, three 16 KB stages and a
 * ring of floor(h_frac * n_hist) residuals for 512 pixels within one SM's
 * shared memory (else BFM_EUNSUPPORTED). */
typedef enum {
    BFM_ALGO_AUTO = 0,
    BFM_ALGO_SIMT = 1, /* FP32 CUDA-core path ("plain form") */
    BFM_ALGO_MMA = 2,  /* tensor-core normal equations, fitted values and refinement */
    BFM_ALGO_COMPLETE = 3, /* series without missing values: one shared pseudo-inverse */
    BFM_ALGO_STREAM = 4,   /* one CUDA-core thread per pixel, Y streamed through TMA stages */
    BFM_ALGO_HYBRID = 5    /* as STREAM, with every contraction over dates on the tensor cores */
} bfm_algo;

typedef struct bfm_design_s *bfm_design_t;

/* Library version string, e.g. "bfm 0.1.0 sm_103a". */
const char *bfm_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *bfm_last_error(void);

/*
 * bfm_design_create -- season-trend design for one set of acquisition dates
 * (Algorithm 1, step 1; regressors of Eq. 2).
 *   dates  host, N doubles, strictly increasing date values in a unit in
 *          which f dates make one seasonal period (t = index for regular
 *          series; day numbers with f = 365 for irregular ones, Section 4.3).
 *   N      number of dates, 2 <= N <= bfm_max_dates().
 *   k_harm number of harmonic terms k, 1 <= k <= 3 (K = 2 + 2k regressors).
 *   f      season length (frequency), f > 0.
 *   out    receives a handle.  Identical (dates, k, f) share one cached
 *          handle (reference counted).  The library owns the handle and its
 *          device tables (allocated on the current device).
 * Internally the trend column is centred and scaled, t' = (t - c)/s with c,
 * s the midpoint and half-range of the dates; results are mapped back to the
 * raw parameterisation of Eq. 2.
 * Errors: BFM_EINVAL (bad argument), BFM_ENOMEM, BFM_ECUDA.
 */
bfm_status bfm_design_create(const double *dates, int N, int k_harm, double f, bfm_design_t *out);

/* Drop one reference; the design is freed with its last reference.  Device
 * work that uses it must have finished. */
bfm_status bfm_design_destroy(bfm_design_t d);

/* K = 2 + 2k of the design (0 for a NULL handle). */
int bfm_design_K(bfm_design_t d);

/* N of the design (0 for a NULL handle). */
int bfm_design_N(bfm_design_t d);

/* Longest date set this build processes in one pass (tile held on chip). */
int bfm_max_dates(void);

/*
 * bfm_monitor -- the per-pixel hot path for m pixels on `stream`.
 * For each pixel p (Algorithm 1 steps 2-12 with the missing-data reading):
 *   beta    OLS fit on the valid history observations (Eq. 5-6);
 *   sigma   sqrt(sum of squared history residuals / (n_p - K)) (Alg. 1 step 5);
 *   MO_j    sum of the h_p residuals y - x'beta ending at valid position j,
 *           divided by sigma*sqrt(n_p), for j = n_p+1 .. N_p (Eq. 3), with
 *           h_p = clamp(floor(h_frac * n_p), 1, n_p);
 *   break   original date index of the first j with |MO_j| >
 *           lambda*sqrt(log+(j/n_p)) (Eq. 4, strict), else -1;
 *   mean    mean of MO_j over the monitoring positions.
 * Arguments:
 *   d          design (its N is the number of rows of Y).
 *   Y          device, [N][m] of `dtype` (any alignment of the element type;
 *              in the CUDA-core form a 16-byte aligned base and m a multiple
 *              of 4 (f32) / 8 (i16) take the TMA tile loader, other layouts a
 *              plain-load loader with the same results).
 *   mask_bits  device, nullable, [N][ceil(m/32)] uint32 (see above).
 *   m          number of pixels, m >= 0 (m = 0 enqueues nothing).
 *   n_hist     history dates, 1 <= n_hist < N (Algorithm 1 Require list).
 *   h_frac     bandwidth as a fraction of n_p, 0 < h_frac <= 1.
 *   lambda     critical value, lambda > 0 (depends on alpha, h and N/n).
 * Outputs (device, caller-owned, each written for every pixel):
 *   break_idx  int32 [m]; mean_mosum float [m]; sigma float [m];
 *   beta       float [K][m] (coefficient i of pixel p at beta[i*m + p], Eq. 2
 *              order: intercept, slope, then sin/cos pairs per harmonic);
 *   status     uint8 [m] (BFM_PX_*).
 * Rank test: with the trend column (t-c)/s, the pixel is SINGULAR when some
 * Cholesky pivot of its history Gram matrix, relative to the matching
 * diagonal entry, is below 1e-5.
 * Arithmetic: float arithmetic with one step of iterative refinement of the
 * least-squares solution, in the form BFM_ALGO_AUTO picks: the hybrid form
 * (the masked sums, X'My, fitted values and the refinement's X'r on tensor
 * cores, fp16 operands split hi/lo or three ways with exact power-of-two
 * scales per pixel, tf32 y, FP32 accumulation; the scans on CUDA cores), the
 * streaming or CUDA-core forms (float sums) or the tensor-core form.  Against
 * an FP64 reference on well-conditioned pixels every form stays within 1e-5
 * on float series (the tensor-core form within 1e-4 on int16 series); the
 * forms differ in the last bits.
 * Errors: BFM_EINVAL, BFM_EUNSUPPORTED (N > bfm_max_dates()), BFM_ECUDA.
 */
bfm_status bfm_monitor(bfm_design_t d, const void *Y, int dtype, const uint32_t *mask_bits, int64_t m,
                       int n_hist, double h_frac, double lambda, int32_t *break_idx, float *mean_mosum,
                       float *sigma, float *beta, uint8_t *status, void *stream);

/* As bfm_monitor_ex with one more output: max_mosum (device, nullable,
 * float [m]) receives for each pixel the MO_j of largest magnitude over its
 * monitoring positions (signed; the first of equal magnitudes) -- the map of
 * maximum absolute MOSUM values of Section 4.3 (Chile scene).  0 for
 * BFM_PX_DEGENERATE, NaN for the other statuses without a fit or without
 * monitoring data. */
bfm_status bfm_monitor_ext(bfm_design_t d, const void *Y, int dtype, const uint32_t *mask_bits, int64_t m,
                           int n_hist, double h_frac, double lambda, int32_t *break_idx, float *mean_mosum,
                           float *sigma, float *beta, uint8_t *status, float *max_mosum, int algo, void *stream);

/*
 * bfm_lambda -- the critical value lambda(alpha, h, N/n) of the boundary
 * lambda*sqrt(log+(t)) (Eq. 4), found by simulation of the limiting process
 * as the paper prescribes (Section 2.3; Section 4.3 prints 2.39 for
 * alpha = 0.05, h = 0.5, N/n = 2).  `reps` Brownian paths on a grid of G
 * steps per unit time up to T = N/n (T * G steps, rounded), one per GPU
 * thread, each from its own SplitMix64 stream (path r: state
 * seed * 0xA0761D6478BD642F + r * 0xE7037ED1A0B428DB + 1, one draw
 * discarded) with Box-Muller normals; the statistic of a path is
 * sup over t = i/G in [1, T] of |W(t) - W(t-h) - h W(1)| / sqrt(log+ t),
 * with h rounded to whole steps.  *lambda_out receives the
 * ceil((1 - alpha) * reps)-th smallest statistic; stats_host (nullable,
 * host, reps doubles) receives all of them.  Runs on `stream` and returns
 * when done (synchronising it).  FP64 arithmetic.
 * Errors: BFM_EINVAL (0 < alpha < 1, 0 < h <= 1, T > 1, G >= 1, reps >= 1
 * and round(h * G) >= 1 are required), BFM_ECUDA.
 */
bfm_status bfm_lambda(double alpha, double h, double T, int G, int reps, uint64_t seed, double *lambda_out,
                      double *stats_host, void *stream);

/*
 * bfm_trace -- residuals and MOSUM process of selected pixels, for the
 * examination of individual series once the breaks are known (Section 3.2,
 * after Algorithm 2: the device path returns only the breaks, the
 * intermediate results of chosen series are looked at afterwards).
 * One warp per selected pixel redoes the pixel's fit in FP64 (Eq. 5-6 by
 * Cholesky on the normal equations of the Eq. 2 regressors, trend centred
 * and scaled), then writes, indexed by the ORIGINAL date t:
 *   resid[i*N + t]  y_t - x_t'beta (Eq. 3 sign) where date t is valid, NaN
 *                   where it is missing;
 *   mo[i*N + t]     MO_j of Eq. 3 where date t is the valid monitoring
 *                   observation at position j (j > n_p), NaN elsewhere
 *                   (history and missing dates); sigma-hat with n_p - K
 *                   degrees of freedom, h_p = clamp(floor(h_frac * n_p), 1,
 *                   n_p) as in bfm_monitor.
 * Arguments: d, Y, dtype, mask_bits, m, n_hist, h_frac as for bfm_monitor
 * (the same values the statuses came from); pixels (device, nullable)
 * int64 [count] pixel indices in 0..m-1 (NULL: pixels 0..count-1);
 * status (device) uint8 [m], the status array bfm_monitor wrote for these
 * data -- only pixels with status OK, DEGENERATE or NO_MONITOR have a fit,
 * the rows of the others (and of an index outside 0..m-1) are all NaN, and
 * DEGENERATE pixels get MO = 0 at their monitoring dates; mo and resid
 * (device, each nullable but not both) float [count][N], caller-owned.
 * Asynchronous on `stream`; no workspace.  Each selected pixel's column of
 * Y is read with one gather per date, so this is meant for the pixels of
 * interest, not for whole scenes.
 * Errors: BFM_EINVAL (arguments as listed), BFM_EUNSUPPORTED (count above
 * 2^31 - 1 warps' worth), BFM_ECUDA.
 */
bfm_status bfm_trace(bfm_design_t d, const void *Y, int dtype, const uint32_t *mask_bits, int64_t m, int n_hist,
                     double h_frac, const int64_t *pixels, int64_t count, const uint8_t *status, float *mo,
                     float *resid, void *stream);

/* The form BFM_ALGO_AUTO takes for these arguments (BFM_ALGO_HYBRID,
 * BFM_ALGO_STREAM, BFM_ALGO_MMA or BFM_ALGO_SIMT; no work, no device
 * access).  Y and m matter only through Y's alignment and m; a NULL or
 * invalid design gives BFM_ALGO_SIMT. */
int bfm_algo_auto(bfm_design_t d, int dtype, int n_hist, double h_frac, const void *Y, int64_t m);

/* As bfm_monitor with an explicit algorithm (bfm_algo).  BFM_ALGO_MMA needs
 * what BFM_ALGO_AUTO checks for it (else BFM_EUNSUPPORTED). */
bfm_status bfm_monitor_ex(bfm_design_t d, const void *Y, int dtype, const uint32_t *mask_bits, int64_t m,
                          int n_hist, double h_frac, double lambda, int32_t *break_idx, float *mean_mosum,
                          float *sigma, float *beta, uint8_t *status, int algo, void *stream);

/*
 * bfm_monitor_host -- the same computation on HOST buffers (Algorithm 2,
 * steps 2 and 15: transfer Y in, breaks out).  Y_host [N][m] and mask_host
 * (nullable) are read, the five outputs are written to host memory, with the
 * pixel range cut into chunks whose host->device copy, kernel and
 * device->host copy overlap on internal streams.  Page-locked host memory is
 * needed for the copies to overlap.  Each chunk runs the form
 * BFM_ALGO_AUTO picks, so outputs equal bfm_monitor's bit for bit.
 * `workspace` is a device buffer of at
 * least bfm_monitor_host_workspace(d, dtype, chunk_px, with_mask) bytes,
 * owned by the caller; chunk_px > 0 is the pixels per chunk.  Returns once
 * the work is enqueued on `stream`; the outputs are ready when `stream` is.
 */
size_t bfm_monitor_host_workspace(bfm_design_t d, int dtype, int64_t chunk_px, int with_mask);
bfm_status bfm_monitor_host(bfm_design_t d, const void *Y_host, int dtype, const uint32_t *mask_host,
                            int64_t m, int n_hist, double h_frac, double lambda, int32_t *break_idx,
                            float *mean_mosum, float *sigma, float *beta, uint8_t *status, void *workspace,
                            size_t workspace_bytes, int64_t chunk_px, void *stream);

/*
 * Batched persistent launch -- many scene tiles of uneven pixel counts,
 * series lengths (their own designs), harmonics and storage types processed
 * by one CUDA-graph replay of persistent kernels: one per hybrid kernel
 * variant (k, storage, mask) and shared-memory layout for the tiles the
 * hybrid form takes (512-pixel blocks, taken in a fixed order), one
 * kernel node per tile the tensor-core form takes (the kernel of a single
 * call, over the tile's 128-pixel blocks), and one CUDA-core kernel for the
 * rest (32-pixel blocks); bfm_batch_form and bfm_batch_tile_form tell which.  The paper processes one scene per
 * call (Algorithm 2); batching is a serving extension with the same
 * per-pixel results: every pixel's outputs equal those of bfm_monitor_ex
 * with the form bfm_batch_form names, on its tile alone.
 *   bfm_batch_create    new empty batch on the current device (owned by the
 *                       caller, freed by bfm_batch_destroy).
 *   bfm_batch_add       appends one tile; arguments and errors as
 *                       bfm_monitor (device buffers, caller-owned and kept
 *                       alive while the batch runs).  *tile_id (nullable)
 *                       receives its index.  The batch holds a reference to
 *                       the design.
 *   bfm_batch_run       enqueues the whole batch on `stream`: a graph of the
 *                       work-counter reset, the hybrid kernels (one CTA per
 *                       SM; a chain), then in parallel branches the
 *                       tensor-core tile nodes and the CUDA-core kernel
 *                       (CTAs = SM count x CTAs per SM, taking `grab`
 *                       32-pixel blocks at a time).  The first run after adds uploads the tile
 *                       table and instantiates the graph; later runs replay it.
 *   bfm_batch_autotune  times every (CTAs per SM, grab in {1,2,4,8})
 *                       candidate on this batch (3 replays each, CUDA events on
 *                       `stream`, synchronising) and keeps the fastest; results
 *                       are cached per batch signature (N, K, dtype and pixel
 *                       count class of every tile) for later batches.  Outputs
 *                       (nullable): the chosen pair and its time in ms.
 *   bfm_batch_set_config  fixes the pair by hand (ctas_per_sm 0 = automatic).
 * The library allocates the device tile table and work counter.
 */
typedef struct bfm_batch_s *bfm_batch_t;
bfm_status bfm_batch_create(bfm_batch_t *out);
bfm_status bfm_batch_add(bfm_batch_t b, bfm_design_t d, const void *Y, int dtype, const uint32_t *mask_bits,
                         int64_t m, int n_hist, double h_frac, double lambda, int32_t *break_idx, float *mean_mosum,
                         float *sigma, float *beta, uint8_t *status, int *tile_id);
bfm_status bfm_batch_run(bfm_batch_t b, void *stream);
bfm_status bfm_batch_autotune(bfm_batch_t b, void *stream, int *ctas_per_sm, int *grab, float *best_ms);
bfm_status bfm_batch_set_config(bfm_batch_t b, int ctas_per_sm, int grab);
int bfm_batch_tiles(bfm_batch_t b);
/* The form a tile with these arguments takes in a batch whose forms are
 * BFM_ALGO_AUTO: BFM_ALGO_HYBRID, BFM_ALGO_MMA or BFM_ALGO_SIMT (no work, no
 * device access). */
int bfm_batch_form(bfm_design_t d, int dtype, int n_hist, double h_frac, const void *Y, int64_t m);
/* The forms tiles added later may take: BFM_ALGO_AUTO (the default: the
 * hybrid form where it applies, else the tensor-core form, else the
 * CUDA-core form), BFM_ALGO_HYBRID (hybrid, else CUDA-core), BFM_ALGO_MMA
 * (tensor-core, else CUDA-core) or BFM_ALGO_SIMT (CUDA-core only).
 * BFM_EINVAL for any other value or once the batch holds tiles. */
bfm_status bfm_batch_set_forms(bfm_batch_t b, int algo);
/* The form tile `tile_id` (bfm_batch_add's *tile_id) takes in this batch, a
 * BFM_ALGO_* value; -1 for a NULL batch or an unknown id. */
int bfm_batch_tile_form(bfm_batch_t b, int tile_id);
bfm_status bfm_batch_destroy(bfm_batch_t b);

/*
 * Serving loop (continuous admission under an HBM budget).  The paper runs
 * one scene at a time (Algorithm 2); this is the serving extension.
 *   bfm_serve_create   reserves `hbm_budget` bytes of device memory (one
 *                      allocation; BFM_ENOMEM if it cannot) and `slots`
 *                      streams (1..64), and starts the scheduler thread.
 *   bfm_serve_submit   queues a tile; *ticket identifies it.  Requests are
 *                      admitted in arrival order as soon as a slot is idle
 *                      and the arena has room for its buffers (the input copy
 *                      when y_on_host, and the five outputs); admitted
 *                      requests run concurrently on the GPU.  BFM_EBUSY if
 *                      the request alone exceeds the whole budget.
 *   bfm_serve_poll     state: 0 pending, 1 running, 2 done, 3 failed,
 *                      4 cancelled; latency from submission to completion
 *                      (ms, -1 until done).  Returns the failure's status.
 *   bfm_serve_result   device pointers of a done request's outputs (layout
 *                      as bfm_monitor), valid until bfm_serve_release.
 *   bfm_serve_release  frees a finished/failed/cancelled request's memory
 *                      (results are device-resident until then).
 *   bfm_serve_cancel   withdraws a request that is still pending.
 *   bfm_serve_wait_all waits (bounded) until no request is pending/running.
 *   bfm_serve_stats    p50/p99 latency of completed requests, their count
 *                      and pixels, and the span from first arrival to last
 *                      completion.
 * Request fields: design (kept alive by the caller), Y (host when y_on_host,
 * page-locked for the copy to overlap; else device), dtype, mask_bits
 * (device or NULL), m, n_hist, h_frac, lambda as bfm_monitor; algo as
 * bfm_monitor_ex (AUTO picks the streaming form, else the tensor-core form,
 * else the CUDA-core form; BFM_ALGO_MMA falls back to the CUDA-core form
 * when the tensor-core form does not take the request; an explicit
 * BFM_ALGO_STREAM the form does not take fails the request with
 * BFM_EUNSUPPORTED).  bfm_serve_submit returns BFM_EINVAL for an algo
 * outside the bfm_algo values.
 */
typedef struct bfm_server_s *bfm_server_t;
typedef struct {
    bfm_design_t design;
    const void *Y;
    int y_on_host;
    int dtype;
    const uint32_t *mask_bits;
    int64_t m;
    int n_hist;
    double h_frac;
    double lambda;
    int algo;
} bfm_serve_request;
bfm_status bfm_serve_create(size_t hbm_budget, int slots, bfm_server_t *out);
bfm_status bfm_serve_submit(bfm_server_t s, const bfm_serve_request *r, uint64_t *ticket);
bfm_status bfm_serve_poll(bfm_server_t s, uint64_t ticket, int *state, double *latency_ms);
bfm_status bfm_serve_result(bfm_server_t s, uint64_t ticket, int32_t **break_idx, float **mean_mosum,
                            float **sigma, float **beta, uint8_t **status);
bfm_status bfm_serve_release(bfm_server_t s, uint64_t ticket);
bfm_status bfm_serve_cancel(bfm_server_t s, uint64_t ticket);
bfm_status bfm_serve_wait_all(bfm_server_t s, double timeout_s);
bfm_status bfm_serve_stats(bfm_server_t s, double *p50_ms, double *p99_ms, int64_t *completed, int64_t *pixels,
                           double *span_ms);
bfm_status bfm_serve_destroy(bfm_server_t s);

/*
 * bfm_batch_run_static -- a batch run that allocates nothing.  The paper has
 * no counterpart; this is a deployment aid.
 *
 * Who needs it: callers that must not allocate device memory when they run
 * work -- e.g. a serving process whose device memory is entirely reserved by
 * its own pool allocator (a cudaMalloc outside the pool can fail or take
 * memory the pool has already promised), or a latency-critical loop in which
 * cudaMalloc/cudaFree would synchronise the device and stall other streams.
 * bfm_batch_create/bfm_batch_run allocate a tile table, a work counter and a
 * CUDA graph; this entry point instead keeps the tile table, the tensor maps
 * and the work counter in one fixed array compiled into the library (about
 * 17 KB of device memory, held by every GPU that loads the library until the
 * process exits), and calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 *   tiles   host array of ntiles tile descriptions (same meaning and checks as
 *           the arguments of bfm_batch_add; buffers are device pointers the
 *           caller owns, designs stay alive until the work is done).
 *   ntiles  0 <= ntiles <= BFM_STATIC_MAX_TILES; more is BFM_EINVAL with a
 *           message (split the batch).
 *   stream  work is enqueued on it: a small kernel that writes the tile table
 *           into the fixed array and resets its work counter, then the
 *           persistent kernel.  The table travels as that kernel's argument,
 *           so the call does not wait for earlier work in `stream`, and
 *           nothing of it refers to host memory once it returns.
 * Results equal those of bfm_monitor with BFM_ALGO_SIMT on each tile alone.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it.  Every call on a device
 * shares the one array and overwrites it: two calls whose work overlaps on
 * the GPU (different streams, no ordering between them) race and give wrong
 * results -- order them on one stream or with events.
 */
#define BFM_STATIC_MAX_TILES 64
typedef struct {
    bfm_design_t design;
    const void *Y;
    int dtype;
    const uint32_t *mask_bits;
    int64_t m;
    int n_hist;
    double h_frac;
    double lambda;
    int32_t *break_idx;
    float *mean_mosum;
    float *sigma;
    float *beta;
    uint8_t *status;
} bfm_tile_spec;
bfm_status bfm_batch_run_static(const bfm_tile_spec *tiles, int ntiles, void *stream);

/*
 * bfm_solve_rate -- measured device time of the per-pixel K x K solve of
 * Eq. 6 (Cholesky factor, forward and backward substitution) done twice per
 * system (as for beta0 and for the refinement delta), for `systems` synthetic
 * symmetric positive definite systems, in FP64 (fp64 != 0) or FP32.  A
 * diagnostic: it is the figure behind running the solves in FP32 with one
 * refinement step.  *ms_out receives the time of the solves alone (the same
 * launch without them subtracted).  K is 4, 6 or 8; 1 <= systems <= 2^31.
 * Synchronises `stream`.  BFM_EINVAL on bad arguments.
 */
bfm_status bfm_solve_rate(int K, int64_t systems, int fp64, void *stream, float *ms_out);

/* Reads and clears the library's device error word (bit 0: a tile load wait
 * gave up).  Synchronises `stream`. */
bfm_status bfm_device_errors(void *stream, uint32_t *bits);

/*
 * bfm_stage_wait_limit -- the bound, in nanoseconds, of the waits in which
 * the pixel warps of the streaming and hybrid forms (BFM_ALGO_STREAM,
 * BFM_ALGO_HYBRID) wait for a stage of Y to land in shared memory.  The paper has no counterpart: every wait of the
 * library is bounded so that a stalled copy ends the kernel with an error
 * instead of hanging the GPU, and this setter lets a test make such a wait run
 * out.  A wait that runs out stops its warp: the warp's pixels from that tile
 * on get BFM_PX_TIMEOUT, bit 0 of the device error word (bfm_device_errors) is
 * set, and the CTA's loader stops issuing copies and lets those in flight land
 * before the CTA ends.  A bound below 1000 ns makes each wait look at its
 * barrier once.  Process-wide; read at each launch; 0 restores the default of
 * 2 s.  The loader's own waits keep their 2 s bound.
 */
bfm_status bfm_stage_wait_limit(uint64_t consumer_wait_ns);

#ifdef __cplusplus
}
#endif

#endif /* BFM_H */
