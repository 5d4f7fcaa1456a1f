/*
 * ht.h — C ABI of the GB300 Hough-transform track finder (libht.so).
 *
 * Method: Lujan et al., "GPU Enhancement of the Trigger to Extend Physics
 * Reach at the LHC" (arXiv:1311.2769), Section 3.  Every parameter instance
 * starts with zero votes, each hit adds one vote to every instance that
 * contains it, local maxima of the vote array are track candidates, and the
 * candidates' hits are collected for a confirmation fit.  Instances are the
 * cells of a (phi0, d0, kappa) perigee-helix grid (the curved, displaced
 * three-parameter model Section 3 calls for).  Section 4 notes that each
 * hit's parameter-space computation is independent of all other hits, which
 * is the parallelism this library maps onto the GPU.
 *
 * Geometry of a cell column (phi0_i, d0_j): n = (-sin phi0, cos phi0),
 * q = h . n = y cos phi0 - x sin phi0, and the circle through the hit with
 * that perigee has curvature kappa = 2 (q - d0) / (r^2 + d0^2 - 2 d0 q).
 * The hit votes into kappa bin floor(w), w = (kappa - kappa_min) * n_kappa /
 * (kappa_max - kappa_min), when the denominator is positive and
 * 0 <= w < n_kappa.  The bin is defined by binary64 IEEE arithmetic on the
 * float32 hit coordinates and float32 bin-centre tables (cos/sin phi0_i,
 * d0_j); the library reproduces that definition bit for bit (it evaluates in
 * float32 with a certified error bound and falls back to higher precision
 * only when the bound cannot decide the bin).
 *
 * Conventions for every function:
 *   - returns HT_OK (0) or a negative HT_ERR_* status; ht_strerror() names it
 *     and ht_last_error() returns a message for the context's last failure;
 *   - the caller owns every buffer it passes; device pointers are borrowed
 *     for the duration of the call or, for asynchronous calls, until the
 *     stream reaches the work (call ht_sync or synchronise the stream);
 *   - a context is not thread-safe: one host thread at a time;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef HT_H
#define HT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HT_OK 0
#define HT_ERR_INVALID_ARG (-1) /* bad pointer, size, grid, NaN/Inf coordinate, layer id, offsets */
#define HT_ERR_OOM (-2)         /* device or pinned allocation failed */
#define HT_ERR_OVERFLOW (-3)    /* an output cap was hit; the true count is still returned */
#define HT_ERR_CUDA (-4)        /* a CUDA runtime call failed (see ht_last_error) */
#define HT_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define HT_ERR_BUDGET (-6)      /* the work does not fit the accumulator memory budget */
#define HT_ERR_STATE (-7)       /* call out of order (e.g. ht_peaks before ht_vote) */

/* ---- memory kinds ---- */
#define HT_HOST 0
#define HT_DEVICE 1

typedef struct ht_ctx ht_ctx;

/* Barrel layers: n_layers radii in cm (host memory, copied at ht_create).
 * Used to validate hit layer ids; the vote itself uses only (x, y). */
typedef struct {
    int32_t n_layers;
    const float *layer_r;
} ht_geometry;

/* Accumulator binning.  phi0 covers [0, 2 pi) in n_phi bins (bin centres
 * (i + 1/2) 2 pi / n_phi); d0 in [d0_min, d0_max) cm and kappa in
 * [kappa_min, kappa_max) 1/cm are split into n_d0 and n_kappa equal bins.
 * Limits: 1 <= n_phi, n_d0 <= 65535; 1 <= n_kappa <= 4096;
 * n_d0 * n_kappa <= 2^24; d0_min < d0_max; kappa_min < kappa_max. */
typedef struct {
    int32_t n_phi, n_d0, n_kappa;
    float d0_min, d0_max, kappa_min, kappa_max;
} ht_grid;

/* Ragged-packed SoA hits of n_events events: event e owns hits
 * [event_offsets[e], event_offsets[e+1]).  event_offsets has n_events + 1
 * entries, starts at 0, is non-decreasing and ends at n_hits.  x, y, z in cm
 * (finite, |x|, |y| <= 1e4), layer in [0, n_layers).  All six pointers are in
 * the memory named by `mem` (HT_HOST or HT_DEVICE).  z may be NULL (it is
 * carried for the caller, not used by the vote).  Host inputs are validated
 * on the host before any launch; device inputs are validated by a kernel and
 * an invalid batch is reported by the next synchronising call. */
typedef struct {
    const float *x, *y, *z;
    const int8_t *layer;
    const int32_t *event_offsets;
    int32_t n_events;
    int32_t mem;
    int64_t n_hits;
} ht_hits;

/* One track candidate: event index within the batch, cell indices, votes. */
typedef struct {
    int32_t event, i_phi, i_d0, i_kappa;
    uint32_t votes;
} ht_peak;

/* Output buffers of ht_process, all in the memory named by `mem`.
 * peaks[peak_cap]; peak_offsets[peak_cap + 1] (CSR row pointers into hit_idx);
 * hit_idx[pair_cap] (global hit indices of the batch, ascending within each
 * peak); counts[2] = {n_peaks, n_pairs}, the true totals even on overflow.
 * Peaks beyond peak_cap and pairs beyond pair_cap are dropped and the call
 * reports HT_ERR_OVERFLOW (at ht_sync for device outputs): the first
 * peak_cap peaks and every CSR row that ends at or below pair_cap are still
 * exact; the one row that crosses pair_cap holds the first (lowest) of its
 * hits in its slots below the cap.  Re-run with larger caps for the rest. */
typedef struct {
    ht_peak *peaks;
    int64_t peak_cap;
    int64_t *peak_offsets;
    int32_t *hit_idx;
    int64_t pair_cap;
    int64_t *counts;
    int32_t mem;
} ht_results;

/* ---- options (ht_set_option / ht_get_option) ---- */
#define HT_OPT_MODE 1              /* HT_MODE_BATCHED (default) or HT_MODE_PLAIN */
#define HT_OPT_TILE_PHI 2          /* phi0 rows per vote tile: 1, 2, 4 or 8 (0 = auto) */
#define HT_OPT_TILE_D0 3           /* d0 columns per vote tile, 1..n_d0 (0 = auto) */
#define HT_OPT_THREADS 4           /* threads per vote CTA: 128 or 256 (0 = auto) */
#define HT_OPT_ACC_BUDGET 5        /* accumulator memory budget in bytes (0 = 40 GB) */
#define HT_OPT_COUNT_STAGES 6      /* 1 = count precision-stage usage (ht_filter_stats) */
#define HT_OPT_USE_GRAPH 7         /* 1 = replay the batched step as a CUDA graph (default 1; host
                                      results copied in chunks, HT_OPT_HOST_CHUNKS > 1, launch directly) */
#define HT_OPT_PHASE_TIMING 8      /* 1 = time vote / peaks+association with device events */
#define HT_OPT_LAUNCHES 9          /* read-only: kernels launched by the last ht_process */
#define HT_OPT_ATILE_PHI 10        /* phi0 rows per association item: 1, 2, 4 or 8 (0 = auto);
                                      more than 1 only with HT_OPT_ATILE_D0 = n_d0 */
#define HT_OPT_ATILE_D0 11         /* d0 columns per association item (0 = auto); rows x
                                      columns of an item at most 32 */
#define HT_OPT_PRUNE 12            /* bit 0: the vote, bit 1: the association first drop the hits
                                      whose d0 band (a proven superset of the columns where a hit
                                      can vote) misses the tile's rows, then evaluate the remaining
                                      hits over the hull (vote) or union (association) of their
                                      bands; same results.  Default 3; no effect when the kappa
                                      range does not contain 0. */

#define HT_OPT_VOTE_MODE 13        /* HT_VOTE_POINT (default), HT_VOTE_RANGE or HT_VOTE_LINE */
#define HT_OPT_ASSOC_CURSORS 14    /* association row cursors per warp, a multiple of 32 (0 = auto:
                                      as many as fit 9 KB of shared memory per warp, 256..1024);
                                      a column block with more peaks is walked once per block of
                                      cursors.  Reading gives the resolved value. */
#define HT_OPT_HOST_CHUNKS 15      /* ht_process with host results (batched mode): run the batch in at
                                      least this many waves and copy each wave's peaks and CSR to the
                                      host while later waves compute (1..64, default 8; 1 = copy after
                                      the whole batch) */
#define HT_OPT_ASSOC_INDEX 16      /* 1: ht_process associates point votes through a per-(event,
                                      layer) index of hit angles, binning only the hits whose exact
                                      curvature can fall in a peak's window (needs layer ids and at
                                      most 32 layers); 0 (default): every hit in every column.  Same
                                      rows either way. */
#define HT_OPT_RECORDS 17          /* 1 (default): in ht_process the band vote also writes, for every
                                      hit whose d0 band meets a tile, the tile's bins (one byte per
                                      cell) and the association reads them instead of binning every
                                      cell again; used with point voting, band pruning of the vote,
                                      n_kappa <= 255 and a vote tile of 32, 64, 128 or 256 cells
                                      (other cases, and 0, bin again).  Same rows either way. */
#define HT_OPT_VOTE_ITEMS 20       /* band-pruned point vote: 1 each warp expands 32 hits' bands into
                                      (hit, d0 column) items and bins 32 items at a time; 0 (default)
                                      bins every column of the hull of 32 queued hits' bands.  Same
                                      accumulators either way; ht_autotune tries both. */
#define HT_OPT_HIT_STAGING 21      /* 1: the band vote (HT_OPT_VOTE_ITEMS 0) copies each event's hits
                                      into shared memory in 512-hit blocks with 1-D bulk copies (TMA),
                                      double-buffered, instead of loading them per warp; used when x
                                      and y are 16-byte aligned.  A copy that never completes (a bounded
                                      wait) is reported as HT_ERR_TIMEOUT.  Default 0; same results. */
#define HT_OPT_BAND_SPLIT 22      /* hull band vote (HT_OPT_VOTE_ITEMS 0, hits loaded per warp): hits
                                      whose d0 band spans at most this many of the tile's columns are
                                      queued apart from the rest, and each of them walks its own band
                                      instead of the hull of 32 hits' bands; 0: one queue for all.
                                      -1 (default): tile_d0 * 5 / 16, at least 3.  Reads back the value
                                      in use.  Same accumulators and records either way. */
#define HT_OPT_HOST_COPY 23        /* ht_process with host results in page-locked host memory
                                      (cudaHostAlloc, cudaHostRegister): n >= 1 (default 32) copies them
                                      with a kernel of n 64-thread blocks beside the next wave's
                                      kernels; 0, and pageable memory always, use the copy engines
                                      (cudaMemcpyAsync).  0..4096; same bytes either way. */
#define HT_OPT_WAVES 19            /* read-only: waves (kernel sequences over groups of events) of the
                                      last ht_process */
#define HT_OPT_RECORD_BUDGET 18    /* device memory for those records in bytes (0 = 72 GB): a wave of
                                      events needs (its hits) x (vote tiles per event) x (cells per
                                      tile) bytes, and ht_process splits the batch into waves that fit
                                      (for device hits whose records exceed it, the event offsets are
                                      read back once, synchronously); an event too large for it alone
                                      is binned again instead. */

/* Vote modes.  HT_VOTE_POINT: a hit votes, in each (phi0, d0) column, for the
 * kappa bin of its curve at the column's centre (Section 3's vote, point
 * sampled).  HT_VOTE_RANGE: a hit votes, in each (phi0, d0) cell, for every
 * kappa bin from the lowest to the highest bin of its curve at the cell's
 * four corners (phi0 edges m 2pi/n_phi, periodic; d0 edges d0_min +
 * n (d0_max - d0_min)/n_d0), clipped to the kappa range, and for none when a
 * corner is the hit's own perigee point (a non-positive denominator); it
 * joins peak (i, j, k) when those bins reach within `window` of k.  Range
 * voting collects every hit of an unsmeared off-centre track in the track's
 * own cell, which point sampling misses.  Bins are defined in binary64 as for
 * the point vote. */
#define HT_VOTE_POINT 0
#define HT_VOTE_RANGE 1
/* HT_VOTE_LINE: the paper's straight displaced model (kappa = 0), on a grid
 * with n_kappa = 1: each hit votes, in every phi0 row, for the d0 bin of
 * q = y cos phi_i - x sin phi_i, floor((q - d0_min) n_d0 / (d0_max - d0_min))
 * in binary64 (the two products of float values are exact); it joins peak
 * (i, j, 0) when its d0 bin in row i lies within `window` of j.  Peaks are
 * the local maxima of the [n_phi][n_d0] accumulator by the usual rule. */
#define HT_VOTE_LINE 2

#define HT_MODE_BATCHED 0 /* one persistent launch per kernel over all (event, tile) items */
#define HT_MODE_PLAIN 1   /* one launch sequence per event */

/* Create a context for one geometry and grid.  Builds the bin-centre tables
 * (float32 cos/sin of phi0_i, d0_j) and the float32-filter constants on the
 * current CUDA device.  *out receives the context; HT_ERR_INVALID_ARG for a
 * grid outside the limits above. */
int ht_create(const ht_geometry *geometry, const ht_grid *grid, ht_ctx **out);

/* Release every device/pinned buffer, graph and stream the context owns. */
int ht_destroy(ht_ctx *ctx);

int ht_set_option(ht_ctx *ctx, int32_t key, int64_t value);
int ht_get_option(ht_ctx *ctx, int32_t key, int64_t *value);

/* Section 3 voting: fill one accumulator per event, uint32
 * [n_phi][n_d0][n_kappa] (kappa fastest), owned by the context.  Asynchronous
 * on `stream`; host hits are validated and staged first.  HT_ERR_BUDGET when
 * n_events accumulators exceed HT_OPT_ACC_BUDGET (use ht_process, which runs
 * in waves).  The accumulators stay valid until the next ht_vote/ht_process. */
int ht_vote(ht_ctx *ctx, const ht_hits *hits, void *stream);

/* Section 3 "local maxima": cells with votes >= threshold that are strictly
 * greater than every neighbour preceding them in linear (phi0, d0, kappa)
 * order and >= every neighbour following them; neighbours are the distinct
 * other cells at offsets {-1,0,1}^3, phi0 periodic, d0/kappa not.  Writes at
 * most `cap` peaks to host memory `out`, ascending (event, linear index), and
 * the true count to *n_out (HT_ERR_OVERFLOW if it exceeds cap).  Synchronous.
 * The full peak list is kept on the device for ht_associate. */
int ht_peaks(ht_ctx *ctx, uint32_t threshold, ht_peak *out, int64_t cap, int64_t *n_out);

/* Hit-to-candidate association for the peaks of the last ht_peaks: hit h of
 * a peak's event belongs to peak (i, j, k) when it votes in column (i, j) into
 * a bin within `window` of k.  CSR into host memory: peak_offsets[n_peaks + 1]
 * (caller sizes it from ht_peaks' count) and hit_idx[cap] (global hit indices,
 * ascending within each peak); *n_pairs = true total (HT_ERR_OVERFLOW if it
 * exceeds cap).  Synchronous. */
int ht_associate(ht_ctx *ctx, int32_t window, int64_t *peak_offsets, int32_t *hit_idx,
                 int64_t cap, int64_t *n_pairs);

/* The whole path — vote, peaks, association — for a batch, in waves that
 * respect HT_OPT_ACC_BUDGET.  With device results the call is asynchronous
 * on `stream` (status of the device-side checks and overflow at ht_sync);
 * with host results it synchronises before returning. */
int ht_process(ht_ctx *ctx, const ht_hits *hits, uint32_t threshold, int32_t window,
               const ht_results *results, void *stream);

/* Copy event `event`'s accumulator from the last ht_vote to host memory
 * `out` (n_phi * n_d0 * n_kappa uint32).  Synchronous. */
int ht_get_accumulator(ht_ctx *ctx, int32_t event, uint32_t *out);

/* Copy the bin-centre tables to host memory (any pointer may be NULL):
 * cos_phi[n_phi], sin_phi[n_phi], d0[n_d0]. */
int ht_get_tables(ht_ctx *ctx, float *cos_phi, float *sin_phi, float *d0);

/* Wait for the context's outstanding work; returns the first deferred error
 * (device-side validation, overflow of device outputs, CUDA errors). */
int ht_sync(ht_ctx *ctx);

/* Time the vote for a few tile shapes on `hits` and keep the fastest
 * (HT_OPT_TILE_PHI / HT_OPT_TILE_D0 / HT_OPT_THREADS), then time the peaks +
 * association phase for a few association tiles (HT_OPT_ATILE_PHI /
 * HT_OPT_ATILE_D0, measured at threshold 9 and window 1).  Synchronous;
 * the sample must fit the accumulator budget. */
int ht_autotune(ht_ctx *ctx, const ht_hits *hits, void *stream);

/* Circle fit of the candidates of the last ht_process, whose outputs are
 * `res` (the confirmation fit Section 3 hands the candidates to; this
 * library's reading, not a formula of the paper): for each stored candidate
 * c < min(n_peaks, peak_cap, cap), the algebraic least-squares circle
 * x^2 + y^2 + D x + E y + F = 0 through the hits of its CSR row (sums over
 * the row in order, Cramer's rule, every step one binary64 IEEE operation),
 * as perigee parameters with the turning sign s of the peak's kappa bin
 * centre: kappa = s / R, unit normal n = s C / |C| = (-sin phi0, cos phi0),
 * d0 = s (|C| - R), chi2 = sum (|h - C| - R)^2.  status 1 fitted; 0 fewer
 * than 3 hits, a singular system, R^2 <= 0 or a centre at the origin; -1 the
 * row lost hits to pair_cap.  The hits are those of that ht_process (device
 * hits must still be valid).  out[cap] lives in res->mem: with device
 * results the call is asynchronous on `stream`, with host results it
 * synchronises. */
typedef struct {
    int32_t status, n_hits;
    double cos_phi0, sin_phi0, d0, kappa, chi2;
} ht_track;
int ht_fit(ht_ctx *ctx, const ht_results *res, ht_track *out, int64_t cap, void *stream);

/* Duplicate and mirror merging of the fitted candidates of the last
 * ht_process (Section 3's confirmation step; this library's reading, not a
 * formula of the paper).  For each stored candidate c < min(n_peaks,
 * peak_cap, cap), with fits[c] from ht_fit on the same `res`:
 *   HT_MERGE_UNFITTED  fits[c].status != 1;
 *   HT_MERGE_BACKWARD  its hits do not lie ahead of its perigee: the
 *                      binary64 sum over its CSR row, in row order, of
 *                      x cos phi0 + y sin phi0 is not > 0 (the mirror cell
 *                      (phi0 + pi, -d0, -kappa) of a forward track);
 *   HT_MERGE_DUPLICATE another forward fitted candidate of the same event
 *                      lies within `radius` cells in phi0 (periodic), d0 and
 *                      kappa and is better: more votes, or as many and a
 *                      smaller index;
 *   HT_MERGE_KEPT      otherwise.
 * Radius 0 and 1 merge mirrors only (peaks are never neighbours).  fits[cap]
 * and state[cap] (int32) and *n_kept (the number KEPT) live in res->mem:
 * with device results the call is asynchronous on `stream`, with host
 * results it synchronises.  0 <= radius <= 64, else HT_ERR_INVALID_ARG; no
 * preceding ht_process: HT_ERR_STATE. */
#define HT_MERGE_KEPT 1
#define HT_MERGE_DUPLICATE 0
#define HT_MERGE_BACKWARD (-1)
#define HT_MERGE_UNFITTED (-2)
int ht_merge(ht_ctx *ctx, const ht_results *res, const ht_track *fits, int32_t radius, int32_t *state,
             int64_t cap, int64_t *n_kept, void *stream);

/* Second Hough transform for displaced vertices (Section "Displaced vertex
 * identification": tracks from a common vertex (xv, yv) satisfy
 * d0 = yv cos phi0 - xv sin phi0, and a second transform of the first one's
 * maxima finds it).  The stored candidates of the last ht_process, whose
 * outputs are `res`, vote with their cells' centre tables for the cells of
 * the (x, y) grid `vg` that their line y cos phi_i - x sin phi_i = d0_j
 * crosses, walking the axis along which the line is less steep (one vote per
 * bin of that axis whose other coordinate lies inside the grid; binary64).
 * Vertices are the local maxima of each event's [n_x][n_y] accumulator at or
 * above `threshold`: strictly above the neighbours preceding in linear
 * (x, y) order, at least the ones following, 8-neighbourhood, no wrap;
 * written to out[cap] in ascending (event, linear index) order, the true
 * number to *count.  out and count live in res->mem (device: asynchronous on
 * `stream`; host: synchronous).  The accumulators stay in the context. */
typedef struct {
    int32_t n_x, n_y;
    float x_min, x_max, y_min, y_max;
} ht_vgrid;

typedef struct {
    int32_t event, i_x, i_y;
    uint32_t votes;
} ht_vertex;

int ht_vertices(ht_ctx *ctx, const ht_vgrid *vg, const ht_results *res, uint32_t threshold, ht_vertex *out,
                int64_t cap, int64_t *count, void *stream);

/* Device time of the last single-wave ht_process (needs HT_OPT_PHASE_TIMING=1,
 * read after ht_sync), into ms[4]: ms[0] vote kernel, ms[1] peaks +
 * association, ms[2] whole device step, ms[3] association kernel (with its
 * work-counter reset).  Events are recorded on the step's stream, so the
 * numbers hold inside a replayed CUDA graph too. */
int ht_phase_times(ht_ctx *ctx, float *ms);

/* Precision-stage counters since the last reset (needs HT_OPT_COUNT_STAGES=1):
 * out[0] cells evaluated, out[1] cells decided by the double-float stage,
 * out[2] cells decided in binary64.  reset != 0 zeroes them after reading. */
int ht_filter_stats(ht_ctx *ctx, int64_t *out, int32_t reset);

/* Peak finding that allocates nothing (no paper counterpart: a service for
 * callers that cannot call cudaMalloc where they need peaks — code inside a
 * framework that owns every device allocation, a real-time path that must
 * not block on an allocation, code without a context to keep buffers in).
 * Same rule and output order as ht_peaks, for n_events accumulators the
 * caller already holds on the device: acc is uint32
 * [n_events][n_phi][n_d0][n_kappa] (device), peaks[cap] and *count (true
 * number of peaks, int64) are device outputs; asynchronous on `stream`.
 * Scratch (per-column peak counts and bitmasks, scan partials) lives in one
 * fixed device array of HT_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit; a call needs
 * n_events * n_phi * n_d0 * (12 + 6 * ceil(n_kappa / 32)) bytes plus ~5 KB of
 * it (256 x 32 x 128 grid: about 113 events per call) and returns
 * HT_ERR_BUDGET when that does not fit (nothing runs).  The array is looked
 * up on the first call on each device (make that first call before any
 * stream capture); every call on a device shares it and starts by clearing
 * what must be zero, so calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Calls no
 * cudaMalloc/cudaFree.  Alignment: acc 16-byte aligned when n_kappa is a
 * multiple of 4 (rows are read with 16-byte loads), else 4-byte; peaks 4-byte,
 * count 8-byte.  HT_ERR_INVALID_ARG for a bad grid, a NULL or misaligned
 * pointer, HT_ERR_CUDA if a launch fails.  The kernels' shared-memory limits
 * are only ever raised, so a call never lowers what a context relies on. */
#define HT_NOALLOC_SCRATCH_BYTES (32u << 20)
int ht_peaks_noalloc(const ht_grid *grid, const uint32_t *acc, int32_t n_events, uint32_t threshold,
                     ht_peak *peaks, int64_t cap, int64_t *count, void *stream);

/* Diagnostic (no paper counterpart): accuracy of the float32 reciprocal
 * approximation the stage-1 bound relies on, over `count` consecutive float
 * bit patterns starting at first_bits (positive normal floats).
 * out[0] = max |rcp(x) * x - 1| scaled by 2^40, out[1] = patterns checked.
 * Synchronous; allocates 16 bytes of device memory. */
int ht_check_rcp(uint32_t first_bits, uint32_t count, uint64_t *out);

/* Diagnostic (no paper counterpart): throughput ceilings of the operations
 * the vote is made of, measured on the current device with CUDA events over
 * one launch of 8 blocks of 256 threads per SM after a warm-up launch.
 *   HT_MB_FP32     independent FP32 multiplies and adds (lane operations/s);
 *   HT_MB_SHARED_RED  red.shared.add.u32 at random addresses of a 16 KB
 *                  tile (increments/s, bank conflicts included);
 *   HT_MB_FDIV     IEEE float32 divisions (divisions/s);
 *   HT_MB_FP64     independent binary64 multiplies and adds (operations/s).
 * `iters` is the per-thread iteration count (>= 1; each does 8 operations of
 * the kind, FP32 and FP64 16).  *rate receives operations per second.  Synchronous on
 * the legacy default stream; allocates a few KB of device memory. */
#define HT_MB_FP32 0
#define HT_MB_SHARED_RED 1
#define HT_MB_FDIV 2
#define HT_MB_FP64 3
int ht_microbench(int32_t kind, int64_t iters, double *rate);

const char *ht_strerror(int status);
const char *ht_last_error(ht_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
