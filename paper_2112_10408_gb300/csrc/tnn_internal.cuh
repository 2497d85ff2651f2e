// Internal declarations shared by the translation units of libtnn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tnn.h"

// ------------------------------------------------------------------ errors

void tnn_set_error(const char *fmt, ...);
void tnn_clear_error();

#define TNN_CUDA_TRY(call)                                                    \
    do {                                                                      \
        cudaError_t e__ = (call);                                             \
        if (e__ != cudaSuccess) {                                             \
            tnn_set_error("%s failed: %s (%s:%d)", #call,                     \
                          cudaGetErrorString(e__), __FILE__, __LINE__);       \
            return e__ == cudaErrorMemoryAllocation ? TNN_ERR_OOM             \
                                                    : TNN_ERR_CUDA;           \
        }                                                                     \
    } while (0)

#define TNN_ARG_CHECK(cond, ...)                                              \
    do {                                                                      \
        if (!(cond)) {                                                        \
            tnn_set_error(__VA_ARGS__);                                       \
            return TNN_ERR_INVALID_ARG;                                       \
        }                                                                     \
    } while (0)

// ------------------------------------------------------------------- index

// Floats per exported / stored segment record (4 x float4).
#define TNN_SEG_FLOATS 16

// Time-bucketed spatial grid over the segments.  Every segment belongs to
// exactly one key = (bucket of t_A, cell of its midpoint in the scaled x-y
// plane); per key the search reads the CSR range of its segments, an extent
// e such that every point of every member cylinder lies within e of the
// key's cell rectangle, and the largest t_B of the members.
struct GridDesc {
    float x0, y0;       // scaled-space corner of cell (0, 0)
    float cell, inv_cell;
    float t0, dt, inv_dt; // bucket b covers t_A in [t0 + b dt, t0 + (b+1) dt)
    const float *ext_max; // [1] device: largest extent over the keys
    int32_t nx, ny, ncell, nb;
    const int32_t *off; // [nb * ncell + 1]
    const int32_t *ids; // [S] segment positions (t_A order) grouped by key
    const float4 *gseg; // [S][4] the same segments' records in that key order;
                        // record 3 carries the t_A position in .z
    const float *ext;   // [nb * ncell]
    const float *tB;    // [nb * ncell]
    const float *bpm;   // [nb] running max over buckets <= b of the max t_B
    const int4 *krec;   // [nb * ncell] (off[k], off[k + 1], ext bits, tB bits):
                        // one 16-byte load per key in the search
};

struct tnn_index {
    int device;
    int64_t n;      // points
    int64_t n_traj; // trajectories
    int64_t S;      // segments
    int32_t K;      // points per segment
    double sigma[4];
    float sig_f[4];  // sigma rounded to float
    float ssq_f[3];  // sqrt(sigma) rounded to float, spatial axes
    float coord_max; // max |ssq * coordinate| over the points
    float max_radius;
    float4 *pts;     // [n] raw (x, y, z, t) in input order
    float4 *seg;     // [S][4] records ordered by t_A (see tnn_index_export)
    float *segTA;    // [S] t_A in that order
    float *segPM;    // [S] running max of t_B in that order
    float4 *pts_t;   // [n] points ordered by (t, index) (linear search; built
                     // by tnn_index_time_order on first use)
    int32_t *idx_t;  // [n + 4] their input index (4 entries of padding)
    // Points in grid-key order (tensor-core member scan; built by
    // tnn_index_key_order on first use): the members of every key's segments,
    // key after key, each key's run padded to a multiple of 4 points with
    // copies of its first point whose index is -1.
    float4 *pts_k;   // [nk]
    int32_t *idx_k;  // [nk + 4] input index, -1 for padding
    int32_t *kp_start; // [nb * ncell + 1] start of each key's run
    int64_t nk;
    // Points in space-time order (the Morton key of x, y, t below; linear
    // search thresholds; built by tnn_index_space_order on first use).
    float4 *pts_m;    // [n]
    int32_t *idx_m;   // [n] input index
    uint32_t *code_m; // [n] Morton key, ascending
    GridDesc grid;   // views of the arrays below
    int32_t *g_off, *g_ids;
    float4 *g_seg;
    float *g_ext, *g_tB, *g_bpm;
    int4 *g_krec;
    float *g_ext_max; // [1]
    float bb_lo[4], bb_hi[4]; // bounding box of the points (x, y, z, t)
    // Query tiles of the self-queries: every trajectory cut into runs of up
    // to 32 consecutive points (a tile never spans two trajectories, whose
    // regions may lie far apart); [n_tiles + 1] starts, the last is n.
    int32_t *d_tiles;
    int32_t *h_tiles;
    int64_t n_tiles;
    unsigned int *d_rmax;     // [1] max_radius bits, written by the segment fit
    cudaEvent_t built;        // recorded after the build's last kernel
    bool rmax_known;          // max_radius has been read back
};

// Parameters of one independent k-NN problem, read by the search kernels.
struct KnnWin {
    const float4 *pts;
    const float4 *seg;
    const float *segTA;
    const float *segPM;
    const float4 *pts_t;
    const int32_t *idx_t;
    const float4 *q; // queries (== pts for self-query)
    int32_t *out_idx;
    float *out_d2;
    int64_t m;
    int64_t tile_begin; // first global tile of this window
    // Self-queries over the index's rows [row0, row0 + m): tile t of the
    // window is the index tile tile_first + t clipped to that range (see
    // tnn_index::d_tiles); NULL: tiles of 32 consecutive queries.
    const int32_t *tile_rows;
    int64_t row0;
    int64_t tile_first;
    GridDesc grid;
    const float4 *pts_k;      // key-ordered points (tensor-core member scan)
    const int32_t *idx_k;
    const int32_t *kp_start;
    float bb_lo[4], bb_hi[4]; // bounding box of the points
    double sigd[4];
    double lag;
    float sig[4];
    float ssq[3];
    float coord_max;
    int32_t n;
    int32_t S;
    int32_t k;
    int32_t L; // candidate slots per query (k + extra)
    int32_t F; // seed segments
    int32_t W0; // seed window
    float tau_defer; // lanes whose key exceeds this after seeding are deferred
    int32_t flags;
    int32_t pad_;
};

#define TNN_MAX_WINDOWS_PARAM 1

struct KnnScratch {
    unsigned long long tile_counter;
    unsigned long long stats[8]; // queries, lb, pairs, segs, fp64, fallback
    unsigned int n_fallback;  // queries handed to the FP32 warp scan
    unsigned int status;
    unsigned int n_fallback3; // queries handed to the exact FP64 warp scan
    unsigned int fb_next;     // work queue over fb_list
    unsigned int fb_next3;    // work queue over fb_list3
    unsigned int pad_;
};

struct KnnLaunch {
    KnnWin w0;            // used when nwin == 1
    const KnnWin *wins;   // device array when nwin > 1
    int32_t nwin;
    int32_t L_max;
    int32_t kseg_max;     // largest segment length over the windows
    int32_t pad_;
    int64_t total_tiles;
    KnnScratch *scr;
    int2 *fb_list;        // (window, query) for the FP32 warp scan
    int2 *fb_list3;       // (window, query) for the exact FP64 warp scan
    int64_t fb_cap;       // capacity of each list
    float *fb_tau;        // [fb_cap] pruning key of a deferred query when the
                          // tile kernel handed it over (parallel to fb_list)
    const unsigned long long *qorder; // tensor-core linear search: sorted
                                      // (space-time key << 32 | query row)
    const float4 *seed_pts;   // linear search: the points in space-time order
    const int32_t *seed_idx;  // (tnn_index pts_m, idx_m, code_m), or NULL
    const uint32_t *seed_code;
    uint32_t *dbg_seen;   // tests only (tnn_knn_trace), else NULL: bit j of
                          // row q = point j's distance to query q was taken
    int64_t dbg_words;    // 32-bit words per row of dbg_seen
    // When set (one window), a grid or sweep tile kernel copies the rows of
    // each finished tile, handed-over rows included as they stand, from
    // out_idx / out_d2 to the same rows of these: mapped page-locked host
    // lists, written with coalesced stores.
    int32_t *mirror_idx;
    float *mirror_d2;
    int32_t mirror_vec; // k % 4 == 0 and all four lists 16-byte aligned
    int32_t pad2_;
};

// Ascending sort of n2 (a power of two, >= 2048) 64-bit keys in place
// (tnn_index.cu); tnn_next_pow2_sort gives the n2 for n keys.
int tnn_next_pow2_sort(int64_t n);
void tnn_bitonic_sort(unsigned long long *keys, int n2, cudaStream_t st);

// Stream-ordered device memory from the library's pool (tnn_memory.cu):
// no device synchronisation, memory kept reserved between calls.
cudaError_t tnn_alloc(void **p, size_t bytes, cudaStream_t st);
void tnn_free(void *p, cudaStream_t st);

// Points in (t, index) order for the linear search, built on first use
// (stream-ordered on `st`).
tnn_status tnn_index_time_order(const tnn_index *ix, cudaStream_t st);
// Sets the window's tiles (self-queries: per-trajectory tiles of the index;
// otherwise 32 consecutive queries) and returns how many there are.
int64_t tnn_window_tiles(const tnn_index *ix, KnnWin *w);

// Points in space-time (Morton) order, built on first use.
tnn_status tnn_index_space_order(const tnn_index *ix, cudaStream_t st);

// Morton key of (x, y, t): 10 bits per axis over the points' bounding box
// (lo, and sc = 1024 / extent, 0 for a flat axis), interleaved x, y, t.
__device__ __forceinline__ uint32_t tnn_spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t tnn_morton_xyt(const float4 &v, const float4 &lo, const float4 &sc)
{
    const uint32_t ix = (uint32_t)fminf(fmaxf((v.x - lo.x) * sc.x, 0.0f), 1023.0f);
    const uint32_t iy = (uint32_t)fminf(fmaxf((v.y - lo.y) * sc.y, 0.0f), 1023.0f);
    const uint32_t it = (uint32_t)fminf(fmaxf((v.w - lo.w) * sc.w, 0.0f), 1023.0f);
    return tnn_spread3(ix) | (tnn_spread3(iy) << 1) | (tnn_spread3(it) << 2);
}
inline void tnn_morton_frame(const float *lo, const float *hi, float4 *l4, float4 *s4)
{
    *l4 = make_float4(lo[0], lo[1], lo[2], lo[3]);
    s4->x = hi[0] > lo[0] ? 1024.0f / (hi[0] - lo[0]) : 0.0f;
    s4->y = hi[1] > lo[1] ? 1024.0f / (hi[1] - lo[1]) : 0.0f;
    s4->z = 0.0f;
    s4->w = hi[3] > lo[3] ? 1024.0f / (hi[3] - lo[3]) : 0.0f;
}
// Points in grid-key order for the tensor-core member scan, built on first
// use (stream-ordered on `st`).
tnn_status tnn_index_key_order(const tnn_index *ix, cudaStream_t st);

// Launch helpers (tnn_knn.cu).
tnn_status tnn_fill_window(const tnn_index *ix, const float *d_q, int64_t m,
                           const tnn_knn_params *p, int32_t *d_idx,
                           float *d_d2, KnnWin *w);
tnn_status tnn_launch_search(const KnnLaunch &L, bool brute,
                             cudaStream_t stream);
// The two halves of a grid- or sweep-order search: the tile kernel alone,
// and the warp-per-query and exact kernels over what it handed over.
tnn_status tnn_launch_tiles(const KnnLaunch &L, cudaStream_t stream);
tnn_status tnn_launch_finish(const KnnLaunch &L, cudaStream_t stream);
size_t tnn_search_smem_per_warp(int L_max, int kseg_max, int mode);

// Search faults flagged on the device since the last report: synchronise
// `st`, then read and clear the device's fault word (tnn_knn.cu).
tnn_status tnn_take_search_faults(cudaStream_t st);
// Enqueue on `st` a copy of the device's fault word into page-locked *h_word
// (nonzero: tnn_take_search_faults has something to report).
cudaError_t tnn_fault_word_async(unsigned int *h_word, cudaStream_t st);
// Free an index whose every use is ordered before the end of `st`: the
// arrays go back to the pool in stream order, with no synchronisation
// (tnn_index.cu).
void tnn_index_release(tnn_index *ix, cudaStream_t st);

#define TNN_WARPS_PER_CTA 4
#define TNN_TILE 32
#define TNN_MAX_DEVICES 64
