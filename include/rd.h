/*
 * rd.h -- C ABI of the GB300 ridge-directed ring detector.
 *
 * The detector is the method of Afik, "Robust and highly performant ring
 * detection algorithm for 3d particle tracking using 2d microscope imaging"
 * (Sci. Rep. 5, 13584, 2015):
 *   frame -> Gaussian smoothing -> 5x5 second-order Sobel Hessian
 *   (Methods, "Algorithm implementation"; Detailed algorithm, step 1)
 *   -> least principal curvature k- and its direction X- (Results,
 *   "Directed ridge detection & votes collection")
 *   -> directed-ridge mask: k- < tau and k- a local minimum along X-
 *   (Detailed algorithm, step 2)
 *   -> ridge-directed circle Hough voting, (x, y) +/- r X- for every r in
 *   [r_min - 1, r_max + 1] (Results; Additional notes)
 *   -> integer hotspot threshold, radius-dependent Gaussian smoothing with
 *   sigma(r) = sig_a r + sig_b and 1/r normalisation (Results, "Local maxima
 *   detection in a noisy parameter space"; Methods; Detailed algorithm,
 *   step 4)
 *   -> float threshold peak_frac * 2 pi and 3x3x3 local maxima with r in
 *   [r_min, r_max] (Detailed algorithm, step 4; Additional notes)
 *   -> annulus classification of ridge pixels and a circle fit per peak
 *   (Results, "Ridge points classification & sub-pixel accuracy"; Detailed
 *   algorithm, step 5).
 *
 * Every stage runs as hand-written sm_103a CUDA kernels on one GPU.  Pointers
 * marked _dev are device pointers; all work is enqueued on the caller's
 * stream (a cudaStream_t passed as void*, NULL = legacy default stream) and
 * is asynchronous: outputs are valid once that stream has synchronised.
 * Functions return rd_status codes; they never abort, throw or trap.
 * A context is not thread-safe: one host thread (or external locking) per
 * context.  Distinct contexts are independent.
 */
#ifndef RD_H
#define RD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_ABI_VERSION 1

/* Pixel type of the frames.  Integer frames are smoothed with exact integer
 * arithmetic (quantised Gaussian taps), which makes the Hessian exact. */
typedef enum { RD_U8 = 0, RD_U16 = 1, RD_F32 = 2 /* soft-score entry points only */ } rd_dtype;

typedef enum {
  RD_OK = 0,
  RD_E_INVAL = 1,     /* bad argument: the call did nothing                      */
  RD_E_NOMEM = 2,     /* a device (or host) allocation failed                    */
  RD_E_CUDA = 3,      /* a CUDA runtime call failed; see rd_last_error           */
  RD_E_OVERFLOW = 4,  /* a capacity was exceeded; counts are true, lists truncated */
  RD_E_TIMEOUT = 5,   /* a bounded device wait gave up                           */
  RD_E_BUSY = 6,      /* the context is in use by an unfinished call             */
  RD_E_HOST = 7       /* another host-side failure (a thread could not start)    */
} rd_status;
/* No C++ exception leaves the library: a failure inside an entry point is
 * returned as RD_E_NOMEM or RD_E_HOST (-1 from the entry points that return a
 * count), with its message in that entry point's last-error string, and what
 * the call had acquired is released. */

/* Method parameters (the C struct holds floats; the detector widens them to
 * double wherever it computes in double). */
typedef struct rd_params {
  float sigma;        /* Gaussian smoothing scale in px, (0, 4]; taps |i| <= ceil(4 sigma)
                         (Results, scale selection)                              */
  int   r_min, r_max; /* radius search range in px, 2 <= r_min <= r_max <= 250;
                         votes cover r_min-1 .. r_max+1 (Additional notes)       */
  float ridge_thresh; /* curvature threshold tau <= 0 on k- in intensity/px^2
                         (Detailed algorithm, step 2)                            */
  float peak_frac;    /* float threshold: a peak needs S > peak_frac * 2 pi, >= 0
                         (Detailed algorithm, step 4)                            */
  int   vote_thresh;  /* integer hotspot threshold: a voxel is a hotspot when its
                         vote count exceeds this value, >= 0 (step 4)            */
  float annulus_w;    /* annulus half-width in px, >= 0: ridge pixels with
                         | |p - c| - r | <= annulus_w are fitted (step 5)       */
  float sig_a, sig_b; /* level smoothing sigma(r) = sig_a r + sig_b, > 0 for all
                         levels (Methods: 0.05, 0.25)                            */
  int   coarse;       /* cell edge c of the circle parameter space in px: 0 or 1
                         (full resolution), 2 or 4 (Additional notes: a lower
                         resolution of the parameter space for more speed per
                         processing unit).  A vote at a = p + s r X goes to the
                         cell floor((a + c/2) / c); the level window is the same
                         Gaussian in cells (sigma(r) / c); a cell is a hotspot
                         when its count exceeds vote_thresh c^2 (<= 65534); a
                         peak cell (u, v) is the centre (c u, c v) px, fitted
                         over the annulus of half-width annulus_w + c - 1.
                         Radii stay in 1 px steps.                               */
} rd_params;

/* One detected ring.  (ix, iy, ir) is the integer peak of the smoothed,
 * normalised circle parameter space; (cx, cy, r) the sub-pixel circle fitted
 * to the ridge pixels of its annulus.  x is the column, y the row. */
typedef struct rd_ring {
  int   frame;        /* index of the frame in the rd_detect batch                */
  float cx, cy, r;    /* fitted centre and radius (px)                            */
  int   ix, iy, ir;   /* integer peak                                             */
  float score;        /* S = smoothed votes / r at the peak (ideal ring ~ 2 pi)   */
  int   n_fit;        /* ridge pixels in the annulus                              */
  int   flags;        /* RD_RING_FIT_FAIL: fewer than 5 points or singular fit;
                         (cx, cy, r) then equal (ix, iy, ir)                      */
} rd_ring;

#define RD_RING_FIT_FAIL 1

/* Device-side status of the last rd_detect, read back by rd_get_stats. */
typedef struct rd_stats {
  int64_t ridge_pixels;     /* directed ridge pixels over the batch               */
  int64_t votes;            /* votes inside the image over all levels             */
  int64_t peaks;            /* integer peaks (true count, before any truncation)  */
  int64_t exact_fallbacks;  /* decisions re-taken in double precision             */
  int32_t overflow;         /* bit mask of RD_OVF_* capacities that overflowed    */
  int32_t n_frames;
  int64_t hotspots;         /* voxels above the integer vote threshold            */
  int64_t smooth_macs;      /* weight x count products of their smoothing windows */
} rd_stats;

#define RD_OVF_RIDGE 1      /* ridge list of a frame full                         */
#define RD_OVF_BINS  2      /* vote bin pool full                                 */
#define RD_OVF_PEAKS 4      /* peak list of a frame full                          */
#define RD_OVF_RINGS 8      /* caller's ring buffer too small                     */
#define RD_OVF_SCORE 16     /* a smoothed vote sum exceeded 32 bits               */
#define RD_OVF_CHECK 32     /* debug build only (compiled with RD_CHECK): a computed
                               index fell outside its buffer; the access was skipped */

typedef struct rd_ctx rd_ctx;

/* Create a detector.  Validates *params, builds the weight tables (Gaussian
 * taps, per-level smoothing weights, per-level peak thresholds) and allocates
 * every device workspace for frames up to max_H x max_W (12 <= size <= 65535)
 * and batches up to max_batch frames.  *out receives the context, or NULL on
 * failure.  Errors: RD_E_INVAL (bad params or sizes), RD_E_NOMEM, RD_E_CUDA. */
rd_status rd_create(const rd_params* params, int max_H, int max_W, int max_batch, rd_ctx** out);

/* Detect rings in n frames.
 *   frames_dev : n frames of H x W pixels of type dtype, row-major, frame i at
 *                frames_dev + i*H*W*sizeof(pixel); read only; caller-owned.
 *   rings_dev  : caller-owned array of ring_cap rd_ring; frame i's rings are
 *                rings_dev[offsets_dev[i] .. offsets_dev[i] + counts_dev[i]),
 *                sorted by (ir, iy, ix).  Rings past ring_cap are dropped and
 *                RD_OVF_RINGS is raised.
 *   counts_dev, offsets_dev : caller-owned int[n]; true ring count per frame
 *                and the exclusive prefix sum of the counts.
 * Enqueues every kernel on stream and returns without waiting.  Errors:
 * RD_E_INVAL (sizes above the rd_create maxima, bad dtype, NULL pointers;
 * nothing is enqueued), RD_E_CUDA (a launch failed).  Capacity overflows are
 * reported after the stream syncs, by rd_get_stats. */
rd_status rd_detect(rd_ctx* ctx, const void* frames_dev, int n, int H, int W, int dtype,
                    void* stream, rd_ring* rings_dev, int ring_cap,
                    int* counts_dev, int* offsets_dev);

/* rd_detect on HOST buffers: copies the n frames from frames_host (pinned
 * memory makes the copy asynchronous) into the context's device staging
 * buffer, runs rd_detect, copies counts, offsets and the rings back to the
 * host arrays (ring_cap rings, n counts, n offsets) and waits for the stream.
 * Returns like rd_get_stats (RD_E_OVERFLOW when a capacity overflowed; the
 * rings that fit are valid).  Staging buffers are sized at rd_create:
 * ring_cap may not exceed max_batch * 4096. */
rd_status rd_detect_host(rd_ctx* ctx, const void* frames_host, int n, int H, int W, int dtype,
                         void* stream, rd_ring* rings_host, int ring_cap,
                         int* counts_host, int* offsets_host);

/* Graph mode.  rd_set_graph(ctx, 1) makes rd_detect capture its whole launch
 * sequence (memsets and every kernel) into a CUDA graph the first time it is
 * called with a given argument set (frames_dev, n, H, W, dtype, stream,
 * rings_dev, ring_cap, counts_dev, offsets_dev) and replay that graph with
 * one cudaGraphLaunch on later calls with the same arguments; the frames'
 * contents may change between calls, their address may not (a different
 * address captures anew).  Graph mode needs a non-default stream (RD_E_INVAL
 * otherwise) and records no stage timing.  rd_set_graph(ctx, 0), the debug
 * settings and rd_destroy release the captured graph. */
rd_status rd_set_graph(rd_ctx* ctx, int on);

/* Synchronise the stream of the last rd_detect on ctx and copy its device
 * counters to *out.  Returns RD_E_OVERFLOW when any RD_OVF_* bit is set. */
rd_status rd_get_stats(rd_ctx* ctx, rd_stats* out);

/* Device memory the context holds: the sum of its allocations (workspaces
 * sized at rd_create, plus the soft path's and the edge variant's once
 * allocated).  Host-side, no GPU work.  RD_E_INVAL on NULL arguments. */
rd_status rd_get_device_bytes(const rd_ctx* ctx, long long* bytes);

rd_status rd_destroy(rd_ctx* ctx);

/* ---- differentiable soft score, its gradients and refinement --------------
 * Not in the paper: a smooth extension of its voting and scoring steps
 * (Results, "Directed ridge detection & votes collection" and "Local maxima
 * detection in a noisy parameter space") used to refine rings by gradient
 * ascent and to differentiate a ring's score with respect to the image:
 *   Score(c, rho) = (1/rho) sum_{p in ridge} m(p) a(p) sum_{s = +-1} sum_{q in corners(v)}
 *                   bil(v, q) exp(-|q - c|^2 / (2 sigma(rho)^2)),
 *   v = p + s rho X-(p), m(p) = logistic((tau - k-(p)) / T), T = |tau| / 4,
 *   a(p) = exp(-(|p - c| - rho)^2 / (2 (w/2)^2)),
 * where the directed-ridge set of the frame (the rd_detect rule, evaluated on
 * the frame in double precision) is held fixed, bil(v, q) are the bilinear
 * weights of the four grid points of v's cell (points outside the image get
 * nothing), sigma(rho) = sig_a rho + sig_b, and a(p) is the ring's soft
 * annulus of half-width w = rd_params.annulus_w (the paper's ridge-point
 * classification, Results: it keeps the pixels of neighbouring rings, which
 * lie off the circle, out of the score).  c = (cx, cy) and rho = r
 * are read from the rings' float fields; frame i's rings are the counts_dev[i]
 * rings that follow frame i - 1's in rings_dev.  Computed in double
 * precision; outputs are float.  Frames may be RD_U8, RD_U16 or RD_F32
 * (rd_backward: RD_F32).  The first call on a context allocates its FP64
 * workspaces (about 64 bytes per pixel of max_batch x max_H x max_W).
 * Errors: RD_E_INVAL (NULL pointers, sizes above the rd_create maxima, bad
 * dtype), RD_E_NOMEM, RD_E_CUDA.
 *
 * rd_soft_score writes Score of every ring to score_dev and, when
 * dparams_dev is not NULL, (dScore/dcx, dScore/dcy, dScore/dr) per ring.
 * rd_backward takes dscore_dev (one float per ring) and writes
 * dimage_dev[n][H][W] = sum_i dscore_i dScore_i/dframe and, when dparams_dev
 * is not NULL, dscore_i times each ring's parameter gradient.
 * rd_refine ascends the unnormalised vote mass r * Score of every ring (the
 * 1/r normalisation compares rings of different radii; for one ring it
 * would pull r inward by about sigma(r)^2 / r), iters steps of
 *   delta = step * se^2 / Score * (dScore/dcx, dScore/dcy, dScore/dr + Score / r),
 *   1 / se^2 = 1 / sigma(r)^2 + 1 / (w/2)^2
 * (each component at most 0.5 px; r at least 1), updating cx, cy, r of
 * rings_dev in place; at most 4096 rings per frame. */
rd_status rd_soft_score(rd_ctx* ctx, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                        const rd_ring* rings_dev, const int* counts_dev, float* score_dev, float* dparams_dev);
rd_status rd_backward(rd_ctx* ctx, const float* frames_dev, int n, int H, int W, void* stream,
                      const rd_ring* rings_dev, const int* counts_dev, const float* dscore_dev,
                      float* dimage_dev, float* dparams_dev);
rd_status rd_refine(rd_ctx* ctx, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                    rd_ring* rings_dev, const int* counts_dev, int iters, float step);

/* ---- feature stage: directed ridges (the method) or directed edges ----------
 * The Additional notes of the paper describe a variant for images whose
 * features are better described by edges: the gradient replaces the
 * Hessian, and the gradient magnitude, replacing k-, must be a local maximum
 * along the gradient direction.  rd_set_features(ctx, RD_FEATURES_EDGE, t)
 * makes the following rd_detect calls use directed edges: (Gx, Gy) = the
 * first-order 5x5 Sobel of the smoothed frame / 128 (exact integers, then one
 * division), an edge pixel has |grad| > t (intensity / px), |grad| > its
 * bilinear sample at p + X and >= its sample at p - X, X = grad / |grad|
 * (canonical sign); each edge pixel then votes, is scored and fitted exactly
 * like a ridge pixel.  RD_FEATURES_RIDGE restores the method.  The first
 * switch to edges allocates the records' exact directions (16 bytes per
 * record of max_batch frames).  Errors: RD_E_INVAL
 * (unknown features, t < 0), RD_E_NOMEM.  rd_debug_ridges then returns the
 * edge pixels and their directions (hess = 0). */
#define RD_FEATURES_RIDGE 0
#define RD_FEATURES_EDGE  1
rd_status rd_set_features(rd_ctx* ctx, int features, float edge_thresh);

/* ---- accumulator geometry and its autotuner --------------------------------
 * The voting stage works on (frame, tile, slab) bins: tile x tile pixels of
 * the accumulator and slab_levels consecutive peak levels, each held in one
 * SM's shared memory (Results, "Directed ridge detection & votes
 * collection"; the paper streams whole equi-radius levels instead).  The
 * geometry changes speed only: results are bit-identical for every valid
 * geometry.  tile is 64, 80, 96 or 128; slab_levels is 4 .. 64; 0 in both
 * fields asks for the automatic choice (the autotuner's cached choice for
 * this frame size and radius range if there is one, else the first of
 * 128 x 32 levels, 96 x 12 and 64 x 12 whose per-tile storage fits the
 * radius range's smoothing windows). */
typedef struct rd_geometry {
  int tile;
  int slab_levels;
} rd_geometry;

/* rd_create with an explicit geometry (NULL = automatic).  Errors as
 * rd_create, plus RD_E_INVAL for a geometry outside the ranges above or one
 * whose per-tile storage exceeds one SM's shared memory for this radius
 * range. */
rd_status rd_create_ex(const rd_params* params, int max_H, int max_W, int max_batch, const rd_geometry* geometry,
                       rd_ctx** out);

/* The geometry a context uses. */
rd_status rd_get_geometry(const rd_ctx* ctx, rd_geometry* out);

/* Time rd_detect on the caller's n device frames (1 <= n <= 65535; H x W,
 * dtype, as for rd_detect) for every geometry that fits (tile 64/80/96/128 x
 * slab 8/16/24/32), with one warm-up and two timed calls each on stream, and
 * return the fastest in *best.  The choice is also cached for this process
 * under (H, W, r_min, r_max, coarse), where rd_create and rd_create_ex with an
 * automatic geometry find it.  Allocates and frees a temporary context per candidate
 * and synchronises stream.  Errors: RD_E_INVAL (as rd_create / rd_detect),
 * RD_E_NOMEM (no candidate could allocate), RD_E_CUDA. */
rd_status rd_autotune(const rd_params* params, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                      rd_geometry* best);

/* Last error message of ctx (or of the last failed rd_create when ctx is
 * NULL).  The string lives until the next call on the same context. */
const char* rd_last_error(const rd_ctx* ctx);

/* ---- host-only helpers (no GPU work): the exact weight tables -------------
 * rd_gaussian_taps writes the integer Gaussian taps Q_i = floor(2^19 g_i + 1/2),
 * |i| <= ceil(4 sigma), of the smoothing step and returns their count (or -1
 * if cap is too small).  rd_level_weights writes the (2R+1)^2 integer level
 * smoothing weights floor(2^16 exp(-(dx^2+dy^2) / (2 sigma(r)^2)) + 1/2),
 * R = ceil(3 sigma(r)), row-major over (dy, dx), and returns their count (or
 * -1).  rd_peak_threshold returns the smallest smoothed vote sum N that
 * passes the float threshold at level r: N > ((peak_frac 2 pi) 2^16) r. */
int     rd_gaussian_taps(float sigma, int32_t* taps, int cap);
int     rd_level_weights(float sig_a, float sig_b, int r, int32_t* w, int cap);
int64_t rd_peak_threshold(float peak_frac, int r);

/* ---- stage timing ----------------------------------------------------------
 * rd_set_timing(ctx, 1) makes every following rd_detect record CUDA events on
 * its stream around its stages; rd_get_timing waits for the last call and
 * writes the stage durations in milliseconds to ms[0 .. RD_N_STAGES-1]:
 * stencil + ridge mask, direction refinement, vote binning, voting + peak
 * epilogue, sort + circle fit.  Returns the number of stages written,
 * min(cap, RD_N_STAGES), or -1 (timing off, no call yet, or cap < 0). */
#define RD_N_STAGES 5
rd_status rd_set_timing(rd_ctx* ctx, int on);
int       rd_get_timing(rd_ctx* ctx, float* ms, int cap);

/* ---- diagnostics (test and profiling use) ---------------------------------
 * rd_debug_ridges copies frame f's ridge pixels of the last rd_detect (after
 * the stream syncs) to host arrays of capacity cap: xy[2i], xy[2i+1] = x, y;
 * dir[2i], dir[2i+1] = X-, Y- (float, canonical sign); hess[3i..3i+2] = the
 * exact integer Hessian (Hxx', Hyy', Hxy') = 64 S^2 (Lxx, Lyy, Lxy).  Any
 * pointer may be NULL.  Returns the number of ridge pixels of frame f (which
 * may exceed cap), or -1 on error.  Order: by 32 x 32 stencil tile; the
 * order inside a tile is unspecified.
 * rd_debug_capture makes the next rd_detect write frame 0's raw accumulator
 * (acc_dev, int32) and smoothed accumulator (sm_dev, uint32) for every voting
 * level r_min-1 .. r_max+1 as [level][Hc][Wc] device arrays, Hc = ceil(H / c)
 * and Wc = ceil(W / c) cells of the parameter space (c = params.coarse; the
 * frame size when c = 1; either array may be NULL; NULL for both turns
 * capture off).  The smoothed accumulator is written at hotspots only; the
 * caller zero-fills the arrays. */
int       rd_debug_ridges(rd_ctx* ctx, int f, int32_t* xy, float* dir, int64_t* hess, int cap);
/* rd_debug_route(ctx, flags) changes the routing of the following rd_detect
 * calls; the results are identical.  Bit 0 processes every accumulator tile
 * with the dense-storage voting kernel (normally used only for tiles whose
 * hotspots exceed the sparse kernel's capacities).  Bit 1 bins with global
 * atomic counters (normally used only for frames of more than 8192
 * accumulator bins) instead of per-CTA counters in shared memory.  0
 * restores the normal routing; other bits: RD_E_INVAL. */
rd_status rd_debug_route(rd_ctx* ctx, int flags);
rd_status rd_debug_capture(rd_ctx* ctx, int32_t* acc_dev, uint32_t* sm_dev);

/* ---- measured peak of the voting unit --------------------------------------
 * rd_probe_smem_atomics measures the rate of shared-memory atomic adds on the
 * current device, the operation that accumulates votes (Results, "Directed
 * ridge detection & votes collection"; Detailed algorithm step 4).  Every
 * CTA (256 threads, ctas_per_sm per SM) adds 8 x iters times per thread into
 * a 32 KB shared array with one address pattern: 0 conflict-free (a warp's
 * lanes in 32 distinct banks), 1 packed u16 pairs (two lanes per word, as
 * votes for horizontally adjacent voxels), 2 pseudo-random words (the
 * address spread of a warp's votes).  One warm-up launch, then one launch
 * timed with CUDA events on stream; the call waits for it.  Writes the adds
 * per second to *atomics_per_s and the timed launch's milliseconds to *ms (may
 * be NULL).  Allocates and frees 4 bytes of device memory.  Errors:
 * RD_E_INVAL (pattern not 0-2, ctas_per_sm not 1-8, iters not 1-2^20, NULL
 * atomics_per_s), RD_E_CUDA; message in rd_probe_last_error. */
rd_status   rd_probe_smem_atomics(int pattern, int ctas_per_sm, int iters, void* stream, double* atomics_per_s,
                                  float* ms);
const char* rd_probe_last_error(void);

/* ---- allocation-free directed-ridge stages --------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory where they call the detector: acquisition
 * loops that forbid cudaMalloc on the per-frame path (it can synchronise the
 * whole device and its latency is unbounded), plug-ins whose host
 * application owns every device allocation through its own pool, and
 * processes whose device memory another framework has already reserved.
 *
 * rd_ridges_static runs the first stages of rd_detect on ONE frame --
 * Gaussian smoothing, exact Hessian, directed-ridge mask, direction
 * refinement -- and allocates nothing.  Its intermediate data (exact
 * Hessians, per-tile record index, vote-rounding margins, counters; about
 * 8.4 MB) live in one fixed device array inside the library, which every GPU
 * that loads the library holds until the process exits.
 *   params    : only sigma and ridge_thresh are read (ranges as in rd_params).
 *   frame_dev : H x W pixels of type dtype, row-major, device, read only,
 *               caller-owned; H, W in [max(12, ceil(4 sigma) + 4), 65535] and
 *               H * W <= RD_STATIC_MAX_PIXELS.
 *   xy_dev    : caller-owned device uint32[cap]: x | y << 16 per ridge pixel.
 *   dir_dev   : caller-owned device float[4 * cap], 16-byte aligned:
 *               (Xhi, Yhi, Xlo, Ylo) per ridge pixel, the unit direction
 *               X- = (Xhi + Xlo, Yhi + Ylo) with canonical sign (X > 0, or
 *               X == 0 and Y > 0).
 *   cap       : record capacity, 0 <= cap <= RD_STATIC_MAX_RIDGE.
 *   count_dev : caller-owned device int: the true number of ridge pixels;
 *               when it exceeds cap, the records past cap are dropped.
 * The records are the ridge pixels rd_detect finds in the same frame with
 * the same parameters (rd_debug_ridges), in an unspecified order.  Work is
 * enqueued on stream; outputs are valid once the stream has synchronised.
 * Errors: RD_E_INVAL (NULL pointer, bad parameter, frame or cap beyond the
 * limits, a pointer not aligned to its element -- dir_dev to 16 bytes, xy_dev
 * and count_dev to 4, a RD_U16 frame_dev to 2: nothing is enqueued),
 * RD_E_CUDA (set-up or a launch failed).  The message is in
 * rd_static_last_error (per host thread).
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress) and the SM count; make
 * that first call before any stream capture on that device.  The address
 * belongs to the CUDA context current at that call; a call made while
 * another context is current on the device (a context created with the
 * driver API, or the primary context rebuilt after cudaDeviceReset) repeats
 * the look-up, so the first call in each such context must also come before
 * any stream capture.
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents (each call clears its counters on its stream before use).
 * Calls whose GPU work overlaps -- on streams with no ordering between them,
 * or from several host threads -- race on the array and give wrong results:
 * order them on one stream. */
#define RD_STATIC_MAX_PIXELS (1 << 20)  /* e.g. 1024 x 1024 */
#define RD_STATIC_MAX_RIDGE  (1 << 18)
rd_status   rd_ridges_static(const rd_params* params, const void* frame_dev, int H, int W, int dtype,
                             void* stream, uint32_t* xy_dev, float* dir_dev, int cap, int* count_dev);
const char* rd_static_last_error(void);

/* ---- continuous-batching request server ------------------------------------
 * One server serves single-frame requests of several size classes on the
 * current GPU (the paper's producer-consumer processing, Methods, made a
 * device-resident request loop).  Each class runs its batches on up to
 * `slots` detector contexts ("slots"), each with its own stream, pinned
 * staging and mapped pinned outputs.  A scheduler thread admits queued
 * requests, the class of the oldest request first, into a free slot, up to
 * max_batch frames per launch, so requests arriving while others are on the
 * GPU are admitted as slots and memory free up, and the slots' work overlaps.
 * A frame's rings are the ones rd_detect gives for that frame alone.
 * Memory: a slot holds its context's workspaces (rd_get_device_bytes) and
 * the device copy of its frames; the slots alive never hold more than
 * mem_budget bytes together (0: no limit).  A new slot is made only when it
 * fits beside the others; idle slots of other classes are destroyed, least
 * recently used first, to make room; otherwise the class waits until
 * batches in flight finish, and classes with newer requests take no new
 * memory meanwhile.  rd_serve_create makes one slot per class (RD_E_NOMEM
 * when one slot of some class exceeds the budget).  The detector writes
 * rings, counts and offsets straight into mapped host memory, so only the
 * rings found leave the device.
 *   rd_serve_submit copies the class's H x W frame (dtype of the class) from
 *     frame_host and queues it (RD_E_BUSY: queue_cap requests are waiting, or
 *     completed results wait to be polled; RD_E_INVAL: bad class or
 *     pointer).  Thread-safe.
 *   rd_serve_poll waits up to wait_ms for completed requests and returns up
 *     to max_results of them (-1 on bad arguments): ids, class, status
 *     (RD_OK; the error of its batch; RD_E_NOMEM when a host allocation for
 *     its result failed, or no slot could be made for its class), ring
 *     count, latency from submission to results on the host (microseconds);
 *     their rings are concatenated in rings (a result whose rings do not fit
 *     stays for the next poll, unless it is the first, which is then
 *     truncated).  Thread-safe.
 *   rd_serve_stats writes submitted, completed, batches launched and device
 *     bytes of the slots alive; rd_serve_stats_ex writes up to cap of the
 *     RD_SERVE_N_STATS values below and returns how many (-1: bad
 *     arguments).
 *   rd_serve_debug_inject makes the next `count` host allocations of one
 *     kind fail as if the host were out of memory, for tests of the failure
 *     path: RD_SERVE_FAIL_RESULT, a completed request's ring vector (that
 *     request gets RD_E_NOMEM); RD_SERVE_FAIL_SLOT, the making of a new slot
 *     (a class with no slot left fails its queued requests with RD_E_NOMEM).
 *   rd_serve_destroy stops admitting, waits for the batches in flight and
 *     frees everything; results not polled are dropped.
 * Errors of rd_serve_create / rd_serve_submit: rd_serve_last_error (per
 * host thread). */
#define RD_SERVE_N_STATS 10  /* submitted, completed, batches, device bytes of the slots alive,
                                their peak, slots made, slots destroyed to make room, scheduling
                                rounds that waited for memory, failed requests, the budget      */
#define RD_SERVE_FAIL_RESULT 1
#define RD_SERVE_FAIL_SLOT   2
typedef struct rd_serve_class {
  rd_params params;
  int H, W;       /* frame size of the class's requests                       */
  int dtype;      /* RD_U8 or RD_U16                                          */
  int max_batch;  /* frames per launch, 1..65535                              */
  int slots;      /* batches in flight at once (contexts and streams), 1..16   */
} rd_serve_class;

typedef struct rd_server rd_server;

rd_status   rd_serve_create(const rd_serve_class* classes, int n_classes, long long mem_budget, int queue_cap,
                            rd_server** out);
rd_status   rd_serve_submit(rd_server* server, int cls, const void* frame_host, long long request_id);
int         rd_serve_poll(rd_server* server, long long* ids, int* classes, int* status, int* n_rings,
                          rd_ring* rings, int rings_cap, double* latency_us, int max_results, int wait_ms);
rd_status   rd_serve_stats(rd_server* server, long long* out4);
int         rd_serve_stats_ex(rd_server* server, long long* out, int cap);
rd_status   rd_serve_debug_inject(rd_server* server, int kind, int count);
rd_status   rd_serve_destroy(rd_server* server);
const char* rd_serve_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RD_H */
