/*
 * tnn.h -- C ABI of the exact Trajectory Nearest Neighbours (TNN) library.
 *
 * Method: "Efficient Wind Speed Nowcasting with GPU-Accelerated Nearest
 * Neighbors Algorithm" (Pannatier, Picatoste, Fleuret), Sec. 3.
 *
 * Problem (Sec. 3.4): N measurements x_i = (x_i, y_i, z_i, t_i) grouped by
 * trajectory; for a query at (x, y, z, t) find the k nearest points under the
 * scalable metric
 *     d2 = sx (dx)^2 + sy (dy)^2 + sz (dz)^2 + st (dt)^2
 * among the points measured strictly more than `lag` (t_w) before it
 * (Sec. 3.1, Eq. of the masked temporal part): valid iff t_j < t - lag.
 * The result is exact: the ranking is that of the FP64 value
 *     ((sx dx^2 + sy dy^2) + sz dz^2) + st dt^2    (dx = (double)x_j - (double)x)
 * with ties broken by the smaller point index.
 *
 * Conventions for every entry point:
 *  - Pointers prefixed d_ are device pointers (CUDA global memory on the
 *    current device), h_ are host pointers.  The caller owns every buffer it
 *    passes; the library never frees or retains caller memory beyond the call,
 *    except where an object (tnn_index, tnn_batch, tnn_mlp) documents a copy.
 *  - Points are float32 rows (x, y, z, t): x, y, z in km (any consistent
 *    unit), t in s.  Rows of one trajectory are contiguous and sorted by
 *    non-decreasing t.  N < 2^31.
 *  - Every call is asynchronous on `stream` unless it says it synchronises;
 *    outputs are valid once the stream reaches the call.  Errors are status
 *    codes, never aborts; the message of the last failure on the calling
 *    thread is returned by tnn_last_error().
 *  - Output neighbour lists are rows of k entries sorted by (d2, index);
 *    missing neighbours (fewer than k valid points) are index -1, d2 +inf.
 */
#ifndef TNN_H
#define TNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *tnn_stream_t;

typedef enum {
    TNN_OK = 0,
    TNN_ERR_INVALID_ARG = 1, /* bad size, pointer, parameter or input value */
    TNN_ERR_OOM = 2,         /* device allocation failed                    */
    TNN_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed        */
    TNN_ERR_TIMEOUT = 4,     /* a bounded device wait expired (1 s)         */
    TNN_ERR_UNSUPPORTED = 5  /* the device is not sm_103 or lacks a feature */
} tnn_status;

const char *tnn_status_string(tnn_status s);
/* Message of the last failing call on this thread ("" if none). */
const char *tnn_last_error(void);

/* ------------------------------------------------------------------ index */

typedef struct tnn_index tnn_index;

typedef struct {
    double sigma[4]; /* weights (sx, sy, sz, st) on squared differences,
                        finite, 0 <= s <= 1e6 (Sec. 3.4, the scalable metric) */
    int32_t seg_len; /* K, points per segment, 2..64 (Sec. 3.4)            */
} tnn_build_params;

typedef struct {
    int64_t n_points;
    int64_t n_traj;
    int64_t n_segments;
    int32_t seg_len;
    float coord_max;   /* largest |sqrt(s) * coordinate| over x, y, z        */
    float max_radius;  /* largest segment cylinder radius (scaled units)     */
} tnn_index_info;

/*
 * Build the TNN index (Sec. 3.4 partitioning; Fig. 2 caption: segment
 * matrices A, t_A, B, t_B, U, E).  Each trajectory is cut into consecutive
 * sets of seg_len points (the last set keeps the remainder, no padding);
 * every set becomes a segment from its first point A to its last point B in
 * sqrt(sigma)-scaled space with U = AB / |AB|^2 and a cylinder radius r that
 * bounds the distance of every member to the segment (computed in FP64 and
 * rounded up).  Segments are then ordered by t_A.
 *   d_xyzt      [n][4] float, device; copied into the index.
 *   h_traj_off  [n_traj + 1] int64, host; 0 = off[0] <= ... <= off[n_traj] = n.
 * Validates the input on the device (finite, |coordinate| <= 1e15, times
 * sorted within each trajectory) and therefore SYNCHRONISES `stream` once,
 * after the validation (the grid's geometry is chosen from the points'
 * bounding box and durations read back at the same time); the segment fit,
 * the sorts and the grid are enqueued after it and run on in stream order
 * after the call returns.  On success *out owns device memory until
 * tnn_index_destroy.
 */
tnn_status tnn_build_segments(const float *d_xyzt, int64_t n,
                              const int64_t *h_traj_off, int64_t n_traj,
                              const tnn_build_params *params,
                              tnn_stream_t stream, tnn_index **out);

void tnn_index_destroy(tnn_index *index);
/* Sizes of the index.  The first call waits for the build to finish (for
   max_radius, the segment fit's largest radius). */
tnn_status tnn_index_get_info(const tnn_index *index, tnn_index_info *out);

/*
 * Copy the t_A-ordered segment table out of the index (for inspection and
 * tests).  d_seg receives [n_segments][16] floats per segment:
 *   0-2 A (scaled), 3 t_A, 4-6 U = AB/|AB|^2 (scaled), 7 t_B,
 *   8-10 AB (scaled), 11 r, 12 first point (int32 bits), 13 count (int32
 *   bits), 14 trajectory (int32 bits), 15 build-order id (int32 bits).
 * d_pm (optional) receives [n_segments] floats, the running maximum of t_B
 * in that order.
 */
tnn_status tnn_index_export(const tnn_index *index, float *d_seg, float *d_pm,
                            tnn_stream_t stream);

/* ------------------------------------------------------------------- k-NN */

enum {
    /* Output (float) of the FP64 distance for every neighbour (each one is
       recomputed in FP64).  Without it, neighbours whose FP32 distance is
       separated from their rank neighbours report the FP32 distance, which is
       within 2^-20 relative of the FP64 value; the neighbour set and order
       are exact either way. */
    TNN_FLAG_EXACT_D2 = 1,
    /* Visit the segments by walking the t_A order backwards (the sweep)
       instead of through the time-bucketed spatial grid of the index.  Both
       give the same exact result; the grid skips whole groups of segments
       and is the default. */
    TNN_FLAG_SWEEP = 2,
    /* tnn_knn_bruteforce only: compute the pair distances on the CUDA cores
       (direct differences) instead of screening them with the tensor-core
       distance matrix.  Same exact result. */
    TNN_FLAG_FFMA = 4,
    /* tnn_knn, grid order: form the distances of the fetched candidate
       points as 128 x 128 tensor-core tiles (tcgen05, TF32 operands, FP32
       accumulation) and screen them with a certified margin; points that
       pass are scored again in FP32 and the ranking settled in FP64 as
       usual.  128 queries share a traversal.  The first such call builds a
       grid-key-ordered copy of the points in the index (16 B per point).
       Same exact result. */
    TNN_FLAG_TC_TILES = 8,
    /* tnn_knn_host only (other calls ignore it): h_idx and h_d2 are
       page-locked host memory mapped into the device's address space over
       their whole extent (cudaHostAlloc, or cudaHostRegister of the whole
       range).  The shared-tile kernel then writes each finished tile's rows
       into them itself (coalesced stores), so the transfer runs under the
       search, and a kernel writes the few rows finished later (queries
       handed to a warp of their own, or settled exactly).  The call checks
       the first and the last element of each (TNN_ERR_INVALID_ARG when
       they are not mapped); the caller vouches for the rest.  Ignored
       together with TNN_FLAG_TC_TILES. */
    TNN_FLAG_MAPPED_OUT = 16
};

typedef struct {
    int32_t k;             /* neighbours per query, 1..64                    */
    double lag;            /* t_w >= 0 (s): valid iff t_j < t_q - lag        */
    int32_t seed_segments; /* F: the F segments of smallest bound are scanned
                              first (Algorithm 2 fetches F segments, nearest
                              first), 1..6 (0 = default 4)                    */
    int32_t seed_window;   /* at most this many of the most recent causal
                              segments are searched for those F
                              (0 = no limit, the default)                     */
    int32_t extra;         /* candidate slots kept beyond k, 2..32 (0 = 4)   */
    int32_t flags;         /* TNN_FLAG_*                                      */
    float defer_cells;     /* grid order: a query whose k-th candidate after
                              seeding is farther than defer_cells grid cells
                              (beyond the sigma_t lag^2 every key carries)
                              leaves its shared query tile and is finished
                              by a warp of its own (Algorithm 2 puts finished
                              lines aside; here the slow ones are) -- 0 =
                              default 1.5, < 0 = never                       */
} tnn_knn_params;

typedef struct {
    uint64_t queries;          /* queries answered                           */
    uint64_t lb_evals;         /* query-to-cylinder lower bounds evaluated   */
    uint64_t pairs;            /* point distances computed ("comparisons",
                                  Table 3)                                   */
    uint64_t segs_scanned;     /* (query, segment) scans                     */
    uint64_t fp64_rechecks;    /* distances recomputed in FP64               */
    uint64_t warp_queries;     /* queries finished by a warp of their own    */
    uint64_t exact_queries;    /* queries ranked by the FP64 definition      */
} tnn_stats;

/*
 * Exact causal k-NN with TNN (Algorithm 1 lower bounds, Algorithm 2 search
 * and stop rule).  For every query: lower bounds to the cylinders of the
 * causally valid segments, most recent first; a segment's points are scanned
 * only while its bound does not exceed the current k-th candidate; the
 * search stops once the running maximum of t_B certifies that every
 * remaining segment is farther than that candidate.  Candidates are ranked
 * in FP32 with a certified error bound; ranks the FP32 values cannot
 * separate are settled in FP64 on the GPU.
 *   d_q     [m][4] float queries (device), or NULL for self-query: every
 *           indexed point is a query (m must equal n_points).  Self-queries
 *           are taken in tiles of consecutive samples of one trajectory;
 *           queries the caller passes, in tiles of 32 in the given order
 *           (queries near one another in space-time and next to one
 *           another in the array share work best).
 *   d_idx   [m][k] int32 out, d_d2 [m][k] float out (device).
 *   h_stats optional; when non-NULL the call SYNCHRONISES `stream`, fills
 *           the counters and reports what the kernels flagged (see
 *           tnn_sync_status).  Without it the call does not wait, and a flag
 *           raised by its kernels is reported by the next call that
 *           synchronises and checks the device's fault word.
 * Device scratch (a few bytes per query) is taken from the stream-ordered
 * allocator and released on the stream.
 */
tnn_status tnn_knn(const tnn_index *index, const float *d_q, int64_t m,
                   const tnn_knn_params *params, int32_t *d_idx, float *d_d2,
                   tnn_stats *h_stats, tnn_stream_t stream);

/*
 * The comparator: the same exact causal k-NN by linear search (Sec. 3.6,
 * Table 1 "Linear search"; Table 3 "Lin. Search") over the time-ordered
 * copy of the points kept in the index, with the same FP32 ranking and FP64
 * settlement.  Arguments as tnn_knn (seed_* fields are ignored).
 * By default the distance matrix of 128 queries x 128 points is formed on
 * the tensor cores (tcgen05, expansion |q|^2 + |p|^2 - 2 q.p, split TF32
 * operands) and used only to screen out points: every point within the
 * current k-th candidate plus a certified margin is scored again with the
 * exact FP32 distance, so the result is the one tnn_knn returns.
 * TNN_FLAG_FFMA computes every distance directly on the CUDA cores.
 * counters: lb_evals = points scored again, pairs = causal point pairs
 * screened, segs_scanned = 128 x 128 distance tiles multiplied.
 */
tnn_status tnn_knn_bruteforce(const tnn_index *index, const float *d_q,
                              int64_t m, const tnn_knn_params *params,
                              int32_t *d_idx, float *d_d2, tnn_stats *h_stats,
                              tnn_stream_t stream);

/*
 * tnn_knn for callers that cannot allocate device memory: a plugin whose
 * host framework owns every device allocation, or a real-time loop that must
 * not call an allocator that may block or fail under memory pressure.  (The
 * paper has no counterpart: this is a deployment variant of tnn_knn.)
 * Arguments and results as tnn_knn, without statistics.  It allocates
 * nothing: its scratch -- work-queue counter, counters and the lists of
 * queries handed to the fallback scans, 256 B + 20 B x 65,536 = 1,310,976 B
 * (1.25 MiB + 256 B) -- is a static array of this library in device memory,
 * held by every GPU that loads the library until the process exits.
 *  - At most 65,536 queries per call (TNN_ERR_INVALID_ARG beyond, before any
 *    device work); answer more by calling it on slices of the queries.
 *  - The first call on a device looks up the array's device address, with
 *    that device current, and keeps it; make that first call before any
 *    stream capture.  After cudaDeviceReset the kept address is stale: do not
 *    call it again in that process.
 *  - Every call uses the same array and clears its counters first: calls
 *    whose work overlaps on the GPU (other streams, other threads) race and
 *    corrupt each other's results.  Order them, e.g. on one stream.
 *  - It does not wait for its kernels; what they flag is reported by
 *    tnn_sync_status (or any other call that checks the fault word).
 */
tnn_status tnn_knn_noalloc(const tnn_index *index, const float *d_q, int64_t m,
                           const tnn_knn_params *params, int32_t *d_idx,
                           float *d_d2, tnn_stream_t stream);

/*
 * Lower bounds used by the search (Algorithm 1 with the cylinder reading of
 * the exclusion criterion of Sec. 3.4): d_lb [m][n_segments] float (device),
 * column j for the j-th segment of the t_A order; +inf where the segment
 * holds no valid point.  Every valid point p of segment j satisfies
 * lb <= the FP32 distance the search computes for p.
 */
tnn_status tnn_segment_lower_bounds(const tnn_index *index, const float *d_q,
                                    int64_t m, double lag, float *d_lb,
                                    tnn_stream_t stream);

/*
 * The work any exact search over this index must do for each query once its
 * k-th distance d_k is known (the "comparisons" of Table 3 reduced to the
 * necessary ones), summed over the queries:
 *   h_work[0] = cylinder bounds: segments of the grid keys whose key bound
 *               does not exceed d_k;
 *   h_work[1] = point distances: members of the segments whose cylinder bound
 *               does not exceed d_k;
 *   h_work[2] = key bounds: non-empty keys of the causal buckets whose
 *               temporal bound does not exceed d_k, within reach of d_k.
 * d_d2 [m][k] is the output of tnn_knn for the same queries (d_k = column
 * k-1, +inf when fewer than k points are valid).  Synchronises `stream`.
 */
tnn_status tnn_knn_work(const tnn_index *index, const float *d_q, int64_t m,
                        int32_t k, double lag, const float *d_d2,
                        uint64_t *h_work, tnn_stream_t stream);

/*
 * tnn_knn_work per kernel: the same sums, split by the kernel that finished
 * each query.  d_path [m] (uint8, device) as tnn_knn_trace writes it, or
 * NULL (every query in class 0).  h_work [3][3]: row c = the three sums of
 * tnn_knn_work over the queries of class c.  Synchronises `stream`.
 */
tnn_status tnn_knn_work_split(const tnn_index *index, const float *d_q, int64_t m,
                              int32_t k, double lag, const float *d_d2,
                              const uint8_t *d_path, uint64_t *h_work,
                              tnn_stream_t stream);

/*
 * tnn_knn (without statistics) that also records, per query, which kernel
 * finished it: d_path [m] (uint8, device) = 0 for the 32-query tile kernel,
 * 1 for the warp-per-query kernel (queries deferred from their tile, or whose
 * tie chain needed a longer list), 2 for the FP64 definition.  For
 * measurement tools (it attributes the necessary work to the kernels) and
 * tests.  d_seen (optional, grid order only): [m][(n_points + 31) / 32]
 * uint32 (device), zeroed by the call; bit j of row q is set when the
 * search scanned the segment holding point j for query q (the FP64
 * definition, path 2, records nothing) -- the segments it skipped are those
 * its stop rule and exclusion criterion certified.
 */
tnn_status tnn_knn_trace(const tnn_index *index, const float *d_q, int64_t m,
                         const tnn_knn_params *params, int32_t *d_idx, float *d_d2,
                         uint8_t *d_path, uint32_t *d_seen, tnn_stream_t stream);

/*
 * Kernel timing for measurement tools.  While enabled, every launch of the
 * search kernels (TNN or linear search) is bracketed by CUDA events recorded
 * on the stream it is launched on: before the main kernel, before the
 * warp-per-query kernel, before the FP64 kernel and after it.
 * tnn_profile_read synchronises on those events and returns the summed
 * device time in ms and the number of launches since the last reset
 * (reset != 0 clears them); tnn_profile_read_kernels returns the three
 * kernels' times separately, h_ms [3] = (main kernel -- the tile kernel, or
 * the query order and the linear-search kernel --, warp-per-query kernel,
 * FP64 kernel).
 */
tnn_status tnn_profile_enable(int32_t on);
tnn_status tnn_profile_read(double *ms, int64_t *launches, int32_t reset);
tnn_status tnn_profile_read_kernels(double *h_ms, int64_t *launches, int32_t reset);

/*
 * FP32 issue throughput of this GPU, measured: every SM runs warps of
 * independent FFMA chains (`iters` fused multiply-adds per chain, 8 chains
 * per thread) and the launch is timed with CUDA events on `stream`.
 * *h_lane_ops = FFMA lane-operations per second (one per thread and
 * instruction); *h_ms = the launch's duration.  The roofline peak of the
 * ALU-bound search kernels.  Synchronises `stream`.
 */
tnn_status tnn_probe_fp32(int32_t iters, double *h_lane_ops, double *h_ms,
                          tnn_stream_t stream);

/* ------------------------------------------------------ device faults */

/*
 * Device-side faults.  The search kernels flag what they cannot recover
 * from -- a bounded device wait that expired (1 s), an internal list that
 * overflowed -- in a fault word of the device, kept until reported.
 * tnn_sync_status synchronises `stream`, then reports and clears that word:
 * TNN_ERR_TIMEOUT for an expired wait, TNN_ERR_CUDA for an overflow (the
 * outputs of the flagged search are incomplete), TNN_OK otherwise.  The
 * calls that synchronise anyway check it too: tnn_knn and
 * tnn_knn_bruteforce with statistics, tnn_batch_stats, tnn_autotune,
 * tnn_knn_host.
 */
tnn_status tnn_sync_status(tnn_stream_t stream);

/*
 * Self-test of that path (the paper has no counterpart): one warp waits, at
 * most limit_us microseconds (1..10^6), on an mbarrier that nothing arrives
 * on -- with no copy or tensor-core operation in flight -- then raises the
 * timeout flag as an expired wait of the search kernels does.  The next
 * tnn_sync_status on `stream` returns TNN_ERR_TIMEOUT.  Asynchronous.
 */
tnn_status tnn_selftest_bounded_wait(int32_t limit_us, tnn_stream_t stream);

/* -------------------------------------------------------- host pipeline */

/*
 * The whole pipeline on host buffers: the points of Sec. 3.5's batch are
 * copied in, indexed (as tnn_build_segments with *bp) and every point is
 * answered as its own query (as tnn_knn with d_q = NULL and *kp); the
 * neighbour lists land in host memory.  The queries are answered in `chunks`
 * consecutive slices of rows (at most 64), shrinking by 2/3 from one to the
 * next: a second stream copies a slice's lists out while the search works
 * on the next slice.  0 = the library's choice: 2 slices, 3 from 2^20
 * points.  With TNN_FLAG_MAPPED_OUT there are no slices (`chunks` is
 * ignored): the search kernels write the lists into host memory as they go.
 *   h_xyzt [n][4] float, h_traj_off [n_traj + 1]: as tnn_build_segments,
 *     host memory (page-locked memory is copied faster).
 *   h_idx [n][k] int32, h_d2 [n][k] float: host outputs, layout as tnn_knn.
 *   stream: where the copies in, the build and the searches run; the copies
 *     out run on a second stream the library keeps per device.
 * Device memory: 16 n + 8 n k bytes of scratch and the index, from the
 * library pool; all of it is returned before the call ends.  Synchronous:
 * returns when the outputs are complete.  Errors as tnn_build_segments and
 * tnn_knn; on an error the outputs are undefined.
 */
tnn_status tnn_knn_host(const float *h_xyzt, int64_t n, const int64_t *h_traj_off,
                        int64_t n_traj, const tnn_build_params *bp,
                        const tnn_knn_params *kp, int32_t chunks, int32_t *h_idx,
                        float *h_d2, tnn_stream_t stream);

/* ----------------------------------------------------------------- memory */

/*
 * Device memory.  The index arrays and every call's scratch are taken, in
 * stream order, from a memory pool private to the library (one per device)
 * that keeps freed memory reserved for the next call: a build or a search
 * maps no new pages and does not synchronise the device.  Destroying an
 * index waits for the device (as cudaFree does) and returns its arrays to
 * the pool.
 * tnn_memory_trim: wait for the device, then release reserved memory not in
 *   use down to keep_bytes (0: all of it).  keep_bytes < 0 is an error.
 * tnn_memory_reserved: bytes the pool of the current device holds
 *   (*h_reserved) and hands out (*h_used, may be NULL).
 */
tnn_status tnn_memory_trim(int64_t keep_bytes);
tnn_status tnn_memory_reserved(int64_t *h_reserved, int64_t *h_used);

/* ---------------------------------------------------------------- batched */

typedef struct tnn_batch tnn_batch;

/*
 * Many independent windows (each its own index, query set and k) answered by
 * one persistent launch that pulls (window, query tile) items from a device
 * work queue -- the row compaction of Algorithm 2 ("put completed lines at
 * the end of the batch") done by letting finished warps take new work.
 *   indexes[w], d_q[w] (NULL = self-query), m[w], params[w], d_idx[w],
 *   d_d2[w]: as tnn_knn, per window.  The arrays are read at creation; the
 *   device buffers must stay valid while the batch is run.  All windows
 *   take the same segment order (TNN_FLAG_SWEEP set in all or in none;
 *   otherwise TNN_ERR_INVALID_ARG); TNN_FLAG_TC_TILES is not accepted.
 * The launch is captured once into a CUDA graph; tnn_batch_run replays it.
 * This is the batched k-NN call of the library (create once, run many
 * times).
 */
tnn_status tnn_batch_create(const tnn_index *const *indexes,
                            const float *const *d_q, const int64_t *m,
                            const tnn_knn_params *params, int32_t n_windows,
                            int32_t *const *d_idx, float *const *d_d2,
                            tnn_batch **out);
tnn_status tnn_batch_run(tnn_batch *batch, tnn_stream_t stream);
/* Counters of the last completed run (synchronises `stream`). */
tnn_status tnn_batch_stats(tnn_batch *batch, tnn_stats *h_stats,
                           tnn_stream_t stream);
void tnn_batch_destroy(tnn_batch *batch);

/* -------------------------------------------------------------- autotune */

/*
 * Choose the segment order (TNN_FLAG_SWEEP), seed_segments, extra and
 * defer_cells for one index and k by timing
 * the search on a sample of self-queries (CUDA events): one run of
 * max(m_sample, 262,144) consecutive indexed points (at most all n) from
 * the middle of the index, so that the sample fills the GPU and takes the
 * per-trajectory tiles of a self-query.  Writes the best into *params (k,
 * lag, flags untouched).
 * Synchronises `stream`.
 */
tnn_status tnn_autotune(const tnn_index *index, tnn_knn_params *params,
                        int64_t m_sample, tnn_stream_t stream);

/* --------------------------------------------------------------- nowcast */

#define TNN_N_FEAT 6

/*
 * Context features and inverse-distance-weighted wind (the context of
 * Sec. 3.1-3.2: neighbours retrieved by TNN feed an aggregator; the paper's
 * GKA weights by a kernel of the scaled distance, this library's fallback
 * weights by 1 / (d2 + eps)).
 *   d_wind [n_points][2] float (u, v) of the indexed points, device.
 *   d_q    [m][4] queries or NULL (self-query), d_idx/d_d2 [m][k] from tnn_knn.
 *   h_mean, h_std [6] host: per-channel standardisation of the features
 *     (dx, dy, dz, dt scaled by sqrt(sigma), u, v); NULL = none.
 *   d_feat [m][k*6] bf16 out (device) or NULL; missing neighbours give 0.
 *   d_idw  [m][2] float out (device) or NULL; NaN when no neighbour exists.
 */
tnn_status tnn_context_features(const tnn_index *index, const float *d_wind,
                                const float *d_q, int64_t m,
                                const int32_t *d_idx, const float *d_d2,
                                int32_t k, const float *h_mean,
                                const float *h_std, float idw_eps,
                                uint16_t *d_feat, float *d_idw,
                                tnn_stream_t stream);

/*
 * The averaging baselines of the nowcasting comparison (Sec. 4.1, Table 2):
 * d_uv [m][2] = the mean wind (u, v) of every indexed point measured in
 *     t_q - before_lo <= t_j <= t_q - before_hi      (FP64 comparisons)
 * NaN where no point falls in that window.  before_lo = 5400, before_hi =
 * 1800 is the paper's hour average over [t - 1 h 30, t - 30 min];
 * before_lo = +inf, before_hi = -inf the (non-causal) day average.  d_wind
 * [n_points][2] float (device), d_q [m][4] queries or NULL (self-query).
 * Scratch (16 B per indexed point) from the stream-ordered allocator.
 */
tnn_status tnn_window_average(const tnn_index *index, const float *d_wind,
                              const float *d_q, int64_t m, double before_lo,
                              double before_hi, float *d_uv, tnn_stream_t stream);

typedef struct tnn_mlp tnn_mlp;

typedef struct {
    float lr, beta1, beta2, eps, weight_decay;
} tnn_adamw_params;

/*
 * Two-layer GELU MLP aggregator, d_in -> d_hidden -> 2 (the MLP of Sec. 3.2
 * used here to map a context to the wind at the query).  FP32 master
 * weights and AdamW moments on the device; the two products with the batch
 * (X W1 and dW1 = X^T dZ) run on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation in TMEM), the head and the gradient epilogue in FP32.
 * Kaiming-uniform initialisation from `seed`.  d_in a multiple of 16
 * (<= 1024), d_hidden a multiple of 64 (<= 512).  A device wait of these
 * kernels that times out (1 s) is reported by the next tnn_mlp_get_params
 * as TNN_ERR_TIMEOUT.
 */
tnn_status tnn_mlp_create(int32_t d_in, int32_t d_hidden, uint64_t seed,
                          tnn_mlp **out);
void tnn_mlp_destroy(tnn_mlp *mlp);
/* Number of floats in the flat parameter layout [W1 (d_in x d_hidden,
   row-major) | b1 | W2 (d_hidden x 2) | b2]. */
int64_t tnn_mlp_num_params(const tnn_mlp *mlp);
/* Host copies of the parameters, optionally the AdamW moments and step
   (checkpoint / resume).  Synchronous. */
tnn_status tnn_mlp_get_params(const tnn_mlp *mlp, float *h_params,
                              float *h_m, float *h_v, int64_t *h_step);
tnn_status tnn_mlp_set_params(tnn_mlp *mlp, const float *h_params,
                              const float *h_m, const float *h_v,
                              int64_t step);
/*
 * Checkpoint: tnn_mlp_save writes the parameters, both AdamW moments and the
 * step to `path`; tnn_mlp_load reads such a file into an MLP of the same
 * d_in and d_hidden (TNN_ERR_INVALID_ARG for another shape, a foreign or a
 * truncated file).  Format, little-endian on every host: int64 magic
 * 0x544E4E4D ("TNNM"), int64 version 1, int64 d_in, int64 d_hidden, int64
 * step, then P float32 parameters (flat layout above), P float32 first
 * moments, P float32 second moments.  Both synchronise the device.
 */
tnn_status tnn_mlp_save(const tnn_mlp *mlp, const char *path);
tnn_status tnn_mlp_load(tnn_mlp *mlp, const char *path);
/* y [B][2] = MLP(x), x [B][d_in] bf16 (device, 16-byte aligned).  Needs no
   workspace. */
tnn_status tnn_mlp_forward(const tnn_mlp *mlp, const uint16_t *d_x, int64_t B,
                           float *d_y, tnn_stream_t stream);
/* Loss mean((y - target)^2) over B x 2 and its gradient in the flat layout
   (d_grad, device, tnn_mlp_num_params floats); no update. */
tnn_status tnn_mlp_gradients(tnn_mlp *mlp, const uint16_t *d_x,
                             const float *d_target, int64_t B, float *d_loss,
                             float *d_grad, tnn_stream_t stream);
/* One AdamW step (decoupled weight decay) on that loss; d_loss optional. */
tnn_status tnn_mlp_train_step(tnn_mlp *mlp, const uint16_t *d_x,
                              const float *d_target, int64_t B,
                              const tnn_adamw_params *opt, float *d_loss,
                              tnn_stream_t stream);

/* ------------------------------------------------------------------- GKA */

typedef struct tnn_gka tnn_gka;

/*
 * Gaussian kernel averaging over the TNN context (Sec. 3.2, Eq. GKA; the
 * GKA-TNN model of Sec. 4.1): the nowcast at q is
 *     s_hat(q) = sum_k w_k s_k / sum_k w_k,
 *     w_k = exp(-(s_xy ((x - x_k)^2 + (y - y_k)^2) + s_z (z - z_k)^2
 *                 + s_t (t - t_k)^2))
 * over the valid neighbours k of q (NaN for an empty context).  The three
 * scales are kept on the device as theta = log(s) (so they stay positive)
 * and trained with Adam on the mean squared error of the nowcast.
 *   h_sigma  [3] floats (s_xy, s_z, s_t) > 0, host.
 */
tnn_status tnn_gka_create(const float *h_sigma, tnn_gka **out);
void tnn_gka_destroy(tnn_gka *gka);
/* Current scales (host) and Adam step count.  Synchronous. */
tnn_status tnn_gka_get_params(const tnn_gka *gka, float *h_sigma, int64_t *h_step);
/* Set the scales and restart Adam (moments and step zeroed).  Synchronous. */
tnn_status tnn_gka_set_params(tnn_gka *gka, const float *h_sigma);
/*
 * d_uv [m][2] float (device) = GKA nowcast at the queries d_q [m][4] (or the
 * indexed points when d_q is NULL, m == n_points) from their neighbour
 * lists d_idx [m][k] (int32, -1 = missing, as tnn_knn writes them) and the
 * measured wind d_wind [n_points][2] (device, in the index's point order).
 */
tnn_status tnn_gka_forward(const tnn_gka *gka, const tnn_index *index, const float *d_wind,
                           const float *d_q, int64_t m, const int32_t *d_idx, int32_t k,
                           float *d_uv, tnn_stream_t stream);
/*
 * One training step on the batch of dataset rows d_rows [B] (int32,
 * device): each row is its own query (self-query contexts d_idx
 * [n_points][k], target its measured wind).  Loss = mean over B x 2 of
 * (s_hat - s)^2 into d_loss (optional, device float); its gradient with
 * respect to theta into d_grad (optional, device [3]).  With opt non-NULL
 * one Adam step (weight_decay acts on theta) follows on the device;
 * opt == NULL requires d_grad.  Rows with an empty context contribute
 * nothing.
 */
tnn_status tnn_gka_train_step(tnn_gka *gka, const tnn_index *index, const float *d_wind,
                              const int32_t *d_rows, int64_t B, const int32_t *d_idx, int32_t k,
                              const tnn_adamw_params *opt, float *d_loss, float *d_grad,
                              tnn_stream_t stream);

/* --------------------------------------------------------------- GKA-MLP */

typedef struct tnn_gkamlp tnn_gkamlp;

/*
 * GKA with scales that depend on the location (Sec. 3.2: the scales as a
 * function of space, modelled by an MLP; the GKA-MLP-TNN model of Table 2):
 *     theta(q) = tanh(u W1 + b1) W2 + b2,  u = (q_xyz - lo) / (hi - lo),
 *     s(q) = exp(theta(q)) = (s_xy, s_z, s_t) at q,
 * then the nowcast of tnn_gka_forward with s(q).  lo and hi are the bounding
 * box of the index's points.  Flat parameters (float32):
 *     W1 [3][H] | b1 [H] | W2 [H][3] | b2 [3],  H = hidden in [1, 32].
 * Initialisation from `seed`: W1, b1 ~ U(-1/sqrt(3), 1/sqrt(3)), W2 = 0 and
 * b2 = log(h_sigma), so the model starts as tnn_gka with h_sigma.
 */
tnn_status tnn_gkamlp_create(const float *h_sigma, int32_t hidden, uint64_t seed,
                             tnn_gkamlp **out);
void tnn_gkamlp_destroy(tnn_gkamlp *model);
int64_t tnn_gkamlp_num_params(const tnn_gkamlp *model);
/* Host copy of the flat parameters and the Adam step.  Synchronous. */
tnn_status tnn_gkamlp_get_params(const tnn_gkamlp *model, float *h_params, int64_t *h_step);
/* Set the parameters and restart Adam.  Synchronous. */
tnn_status tnn_gkamlp_set_params(tnn_gkamlp *model, const float *h_params);
/* Arguments and results as tnn_gka_forward. */
tnn_status tnn_gkamlp_forward(const tnn_gkamlp *model, const tnn_index *index,
                              const float *d_wind, const float *d_q, int64_t m,
                              const int32_t *d_idx, int32_t k, float *d_uv,
                              tnn_stream_t stream);
/* Arguments and results as tnn_gka_train_step; d_grad (optional) receives
   tnn_gkamlp_num_params floats in the flat layout. */
tnn_status tnn_gkamlp_train_step(tnn_gkamlp *model, const tnn_index *index,
                                 const float *d_wind, const int32_t *d_rows, int64_t B,
                                 const int32_t *d_idx, int32_t k,
                                 const tnn_adamw_params *opt, float *d_loss, float *d_grad,
                                 tnn_stream_t stream);

/*
 * Nowcast wind at the queries: TNN context (tnn_knn), features and IDW
 * (tnn_context_features), then the MLP when `mlp` is non-NULL (its input
 * width must be k * 6), else the IDW average.
 *   d_uv [m][2] float out (device).  Temporaries come from the
 *   stream-ordered allocator.
 */
tnn_status tnn_nowcast(const tnn_index *index, const float *d_wind,
                       const float *d_q, int64_t m,
                       const tnn_knn_params *params, const tnn_mlp *mlp,
                       const float *h_mean, const float *h_std, float idw_eps,
                       float *d_uv, tnn_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TNN_H */
