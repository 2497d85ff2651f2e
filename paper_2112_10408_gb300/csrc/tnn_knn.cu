// Exact causal k-NN search: TNN (Sec. 3.5, Algorithms 1 and 2) and the
// linear-search comparator (Sec. 3.6, Table 1), both with the same FP32
// ranking, certified error bounds and FP64 settlement.
//
// Execution model.  One warp answers a tile of 32 queries, one query per
// lane, so that every segment record and every candidate point is loaded
// once into shared memory and read by all 32 lanes as a broadcast.  Warps
// pull tiles from a device work queue (an atomic counter) until none is
// left; a finished warp immediately takes new work, which is the GPU form of
// Algorithm 2's "put completed lines at the end of the batch".
//
// TNN per query (lane):
//   1. seed: among the W0 most recent causally valid segments, the F with
//      the smallest lower bound are scanned first (Algorithm 2 fetches F
//      segments at a time, nearest first);
//   2. sweep: segments are visited from the most recent t_A backwards in
//      chunks of 32; a segment's points are scanned only if its lower bound
//      does not exceed the current k-th candidate (exclusion criterion of
//      Sec. 3.4); the sweep stops once the time-only bound of every remaining
//      segment, taken from the running maximum of t_B, exceeds it (the stop
//      rule of Algorithm 2 with the temporal part of the bound).
//   3. settle: rank ties the FP32 values cannot separate are re-ranked in
//      FP64 (the canonical formula of the oracle), output sorted by
//      (d2, index).
//
// Numerical contract (u = 2^-24).
//   d32 = the FP32 distance below; with Delta rounded once and at most seven
//   further roundings of non-negative terms, |d32 - d2| <= 8u d2 (+ an
//   absolute underflow term below 2^-120).  Let eps1 = 2^-20 >= 16u.
//   Lower bound: for every valid point p of a segment, the value returned by
//   seg_lb is <= d32(p):
//     - spatial part: with q' = sqrt(sigma) q, every member lies within r of
//       the stored segment [A', A' + AB'] (r from FP64, rounded up), so
//       |q' - p'| >= dist(q', segment) - r; the FP32 evaluation of that
//       distance errs by at most 5u|v| (projection parameter), 2u|q'| (q'
//       rounding) and a few u of |v| + |AB| (arithmetic), all below
//       delta = 2^-18 (max|q'| + max|p'|), plus a relative 2^-20 for the
//       approximate square root;
//     - temporal part: t_q - min(t_B, T32) rounded down never exceeds
//       t_q - t_j for a valid point (t_j <= t_B, t_j < T32);
//     - the sum is multiplied by (1 - 2^-19), which covers the roundings of
//       the bound itself and the 8u of d32.
//   A candidate is inserted iff its key (d32, index) is below the largest
//   key kept, so a segment whose bound exceeds that key cannot contribute.
//   Settlement: if d32(b) > d32(a)(1 + 2^-17) + 2^-100 then d2(b) > d2(a);
//   maximal chains of keys closer than that are re-ranked in FP64.  When the
//   chain holding rank k reaches the last kept slot of a full candidate
//   list, points outside the list could belong to it: that query is
//   answered again by the warp scans of tnn_fallback.cuh.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tnn_internal.cuh"

#include "tnn_device.cuh"
#include "tnn_search.cuh"
#include "tnn_grid.cuh"
#include "tnn_linear.cuh"
#include "tnn_fallback.cuh"
#include "tnn_linear_tc.cuh"
#include "tnn_tctiles.cuh"

// ------------------------------------------------------ lower-bound export

__global__ void k_segment_lb(const __grid_constant__ KnnWin W, float *out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W.m * (long long)W.S)
        return;
    const long long qi = t / W.S;
    const int s = (int)(t % W.S);
    const QCtx c = make_qctx(&W, W.q[qi], true);
    const float lb = seg_lb(c, W.sig[3], W.seg[4 * (size_t)s], W.seg[4 * (size_t)s + 1],
                            W.seg[4 * (size_t)s + 2]);
    out[t] = isnan(lb) ? INFINITY : lb;
}

// -------------------------------------------------------------- host side

static int g_num_sms = 0;
static int g_smem_per_sm = 0; // shared memory of one SM (bytes)

// ---- kernel timing for measurement tools (tnn_profile_*): four events per
// search launch, on its stream -- before the main kernel (tile kernel, or
// query order + tensor-core kernel), before the warp-per-query kernel,
// before the exact kernel, after it.
struct ProfEv {
    cudaEvent_t e[4];
};
static bool g_prof_on = false;
static std::vector<ProfEv> g_prof_ev;   // recorded
static std::vector<ProfEv> g_prof_pool; // free

static cudaError_t prof_begin(cudaStream_t st, ProfEv *pr)
{
    if (!g_prof_pool.empty()) {
        *pr = g_prof_pool.back();
        g_prof_pool.pop_back();
    } else {
        for (int i = 0; i < 4; ++i) {
            cudaError_t e = cudaEventCreate(&pr->e[i]);
            if (e != cudaSuccess)
                return e;
        }
    }
    return cudaEventRecord(pr->e[0], st);
}

static tnn_status device_setup()
{
    int dev = 0;
    TNN_CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    TNN_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3) {
        tnn_set_error("libtnn is built for sm_103 (GB300); device %d is sm_%d%d",
                      dev, prop.major, prop.minor);
        return TNN_ERR_UNSUPPORTED;
    }
    g_num_sms = prop.multiProcessorCount;
    g_smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    // The shared-memory limit of a kernel is a per-device attribute: raised
    // once on every device that runs a search.
    static std::mutex mu;
    static bool attrs[TNN_MAX_DEVICES];
    if (dev < 0 || dev >= TNN_MAX_DEVICES) {
        tnn_set_error("device ids must be below %d, got %d", TNN_MAX_DEVICES, dev);
        return TNN_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!attrs[dev]) {
        const int maxs = 227 * 1024;
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_search<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_search<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_grid_search<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_grid_search<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_linear_search, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_linear_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_fallback_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        attrs[dev] = true;
    }
    return TNN_OK;
}

tnn_status tnn_fill_window(const tnn_index *ix, const float *d_q, int64_t m,
                           const tnn_knn_params *p, int32_t *d_idx, float *d_d2,
                           KnnWin *w)
{
    TNN_ARG_CHECK(ix != nullptr && p != nullptr && w != nullptr, "NULL argument");
    TNN_ARG_CHECK(p->k >= 1 && p->k <= 64, "k must be in [1, 64], got %d", p->k);
    TNN_ARG_CHECK(isfinite(p->lag) && p->lag >= 0.0, "lag must be finite and >= 0");
    const int F = p->seed_segments == 0 ? 4 : p->seed_segments;
    const int W0 = p->seed_window;
    const int E = p->extra == 0 ? 4 : p->extra;
    TNN_ARG_CHECK(F >= 1 && F <= 6, "seed_segments must be in [1, 6]");
    TNN_ARG_CHECK(W0 >= 0, "seed_window must be >= 0 (0 = no limit)");
    TNN_ARG_CHECK(E >= 2 && E <= 32, "extra must be in [2, 32]");
    TNN_ARG_CHECK(m >= 0, "m must be >= 0");
    if (d_q == nullptr)
        TNN_ARG_CHECK(m == ix->n, "self-query needs m == n_points (%lld), got %lld",
                      (long long)ix->n, (long long)m);
    else
        TNN_ARG_CHECK(((uintptr_t)d_q & 15) == 0, "d_q must be 16-byte aligned");
    TNN_ARG_CHECK(m < (1ll << 31), "m must be < 2^31");
    int dev = -1;
    cudaGetDevice(&dev);
    TNN_ARG_CHECK(dev == ix->device, "index lives on device %d, current is %d", ix->device, dev);
    memset(w, 0, sizeof(*w));
    w->pts = ix->pts;
    w->seg = ix->seg;
    w->segTA = ix->segTA;
    w->segPM = ix->segPM;
    w->pts_t = ix->pts_t;
    w->idx_t = ix->idx_t;
    w->pts_k = ix->pts_k;
    w->idx_k = ix->idx_k;
    w->kp_start = ix->kp_start;
    w->grid = ix->grid;
    for (int i = 0; i < 4; ++i) {
        w->bb_lo[i] = ix->bb_lo[i];
        w->bb_hi[i] = ix->bb_hi[i];
    }
    w->q = d_q ? (const float4 *)d_q : ix->pts;
    // self-queries (all points, or a run of them as tnn_knn_host passes):
    // per-trajectory tiles
    {
        const float4 *q4 = w->q;
        const bool self = q4 >= ix->pts && q4 < ix->pts + ix->n && m <= (ix->pts + ix->n) - q4;
        w->tile_rows = self && ix->d_tiles ? ix->d_tiles : nullptr;
        w->row0 = self ? (int64_t)(q4 - ix->pts) : 0;
        w->tile_first = 0;
    }
    w->out_idx = d_idx;
    w->out_d2 = d_d2;
    w->m = m;
    for (int i = 0; i < 4; ++i) {
        w->sigd[i] = ix->sigma[i];
        w->sig[i] = ix->sig_f[i];
    }
    for (int i = 0; i < 3; ++i)
        w->ssq[i] = ix->ssq_f[i];
    w->coord_max = ix->coord_max;
    w->lag = p->lag;
    w->n = (int32_t)ix->n;
    w->S = (int32_t)ix->S;
    w->k = p->k;
    w->L = p->k + E;
    w->F = F;
    w->W0 = W0;
    {
        // Deferral: a key that still reaches beyond defer_cells grid cells
        // in space.  Every valid point is at least lag before the query, so
        // every key carries at least sigma_t lag^2 of temporal distance;
        // that floor is added so that a lag does not defer every query.
        const double dc = p->defer_cells == 0.0f ? 1.5 : (double)p->defer_cells;
        const double side = dc * (double)ix->grid.cell;
        w->tau_defer = dc > 0.0 ? (float)(side * side + ix->sigma[3] * p->lag * p->lag) : INFINITY;
    }
    w->flags = p->flags;
    return TNN_OK;
}

// Space-time order of the queries for the tensor-core linear search: a
// Morton key of (x, y, t) above the query row; rows [m, n2) are padding that
// sorts last.
__global__ void k_query_order_keys(const float4 *__restrict__ q, int64_t m, int64_t n2,
                                   float4 lo, float4 sc, unsigned long long *__restrict__ keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2)
        return;
    if (i >= m) {
        keys[i] = ~0ull;
        return;
    }
    keys[i] = ((unsigned long long)tnn_morton_xyt(q[i], lo, sc) << 32) | (unsigned long long)i;
}

int64_t tnn_window_tiles(const tnn_index *ix, KnnWin *w)
{
    if (w->m <= 0)
        return 0;
    if (!w->tile_rows)
        return (w->m + TNN_TILE - 1) / TNN_TILE;
    // the index tiles holding the first and the last row of the range
    const int32_t *b = ix->h_tiles, *e = ix->h_tiles + ix->n_tiles;
    const int64_t t0 = (std::upper_bound(b, e, (int32_t)w->row0) - b) - 1;
    const int64_t t1 = (std::upper_bound(b, e, (int32_t)(w->row0 + w->m - 1)) - b) - 1;
    w->tile_first = t0;
    return t1 - t0 + 1;
}

// The per-query kernels that finish the tile kernel's deferred and
// unsettled queries; the measured interval covers the whole search.
static tnn_status finish_search(const KnnLaunch &L, cudaStream_t st, bool prof, ProfEv &pr)
{
    if (prof)
        TNN_CUDA_TRY(cudaEventRecord(pr.e[1], st));
    {
        const size_t wsm = wq_smem_per_warp() * TNN_WARPS_PER_CTA;
        int nbw = 0;
        TNN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbw, k_tnn_warp, TNN_WARPS_PER_CTA * 32, wsm));
        k_tnn_warp<<<(unsigned)(std::max(nbw, 1) * g_num_sms), TNN_WARPS_PER_CTA * 32, wsm, st>>>(L);
    }
    TNN_CUDA_TRY(cudaGetLastError());
    if (prof)
        TNN_CUDA_TRY(cudaEventRecord(pr.e[2], st));
    k_fallback_exact<<<(unsigned)g_num_sms, TNN_WARPS_PER_CTA * 32,
                       fb_exact_smem_per_warp(L.L_max) * TNN_WARPS_PER_CTA, st>>>(L);
    TNN_CUDA_TRY(cudaGetLastError());
    if (prof) {
        TNN_CUDA_TRY(cudaEventRecord(pr.e[3], st));
        g_prof_ev.push_back(pr);
    }
    return TNN_OK;
}

// The grid- or sweep-order tile kernel.
static tnn_status launch_tiles(const KnnLaunch &L, cudaStream_t st)
{
    const bool sweep = (L.w0.flags & TNN_FLAG_SWEEP) != 0;
    const size_t smem = smem_per_warp(L.L_max, L.kseg_max, sweep ? SMEM_SWEEP : SMEM_GRID) *
                        TNN_WARPS_PER_CTA;
    const bool mirror = L.mirror_idx != nullptr;
    const void *kern = sweep ? (mirror ? (const void *)k_tnn_search<true> : (const void *)k_tnn_search<false>)
                             : (mirror ? (const void *)k_tnn_grid_search<true> : (const void *)k_tnn_grid_search<false>);
    int nb = 0;
    TNN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, TNN_WARPS_PER_CTA * 32, smem));
    if (nb < 1) {
        tnn_set_error("search kernel does not fit on an SM (%zu B shared memory)", smem);
        return TNN_ERR_UNSUPPORTED;
    }
    const long long need = (L.total_tiles + TNN_WARPS_PER_CTA - 1) / TNN_WARPS_PER_CTA;
    long long grid = std::min<long long>(need, (long long)nb * g_num_sms);
    if (grid < 1)
        grid = 1;
    if (sweep && mirror)
        k_tnn_search<true><<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    else if (sweep)
        k_tnn_search<false><<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    else if (mirror)
        k_tnn_grid_search<true><<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    else
        k_tnn_grid_search<false><<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

tnn_status tnn_launch_search(const KnnLaunch &L, bool brute, cudaStream_t st)
{
    tnn_status s = device_setup();
    if (s != TNN_OK)
        return s;
    int nb = 0;
    const bool sweep = (L.w0.flags & TNN_FLAG_SWEEP) != 0;
    // Tensor-core linear search: one window, 128 queries per CTA, 256 TMEM
    // columns per CTA.  At least 80 KB of shared memory keeps at most 2 CTAs
    // (512 columns) on an SM, so every TMEM allocation is granted at once; the
    // grid is sized from that bound (the occupancy query answers 1 block per
    // SM for this kernel).
    const bool tc = brute && (L.w0.flags & TNN_FLAG_FFMA) == 0 && L.nwin <= 1 &&
                    tc_smem_bytes(L.L_max) <= (size_t)227 * 1024;
    if (tc) {
        const size_t smem = std::max<size_t>(tc_smem_bytes(L.L_max), 80 * 1024);
        nb = std::min<int>(2, (int)(g_smem_per_sm / (smem + 1024)));
        if (nb < 1) {
            tnn_set_error("tensor-core search kernel does not fit on an SM (%zu B shared memory)", smem);
            return TNN_ERR_UNSUPPORTED;
        }
        KnnLaunch Lt = L;
        Lt.total_tiles = (L.w0.m + TC_Q - 1) / TC_Q;
        long long grid = std::min<long long>(Lt.total_tiles, (long long)nb * g_num_sms);
        if (grid < 1)
            grid = 1;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        const bool prof = g_prof_on && cap == cudaStreamCaptureStatusNone;
        ProfEv pr;
        if (prof)
            TNN_CUDA_TRY(prof_begin(st, &pr));
        // queries in space-time order (skipped beyond 2^29 queries)
        unsigned long long *keys = nullptr;
        if (L.w0.m <= (1ll << 29)) {
            const int n2 = tnn_next_pow2_sort(L.w0.m);
            TNN_CUDA_TRY(tnn_alloc((void **)&keys, (size_t)n2 * 8, st));
            float4 l4, s4;
            tnn_morton_frame(L.w0.bb_lo, L.w0.bb_hi, &l4, &s4);
            k_query_order_keys<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(L.w0.q, L.w0.m, n2, l4, s4,
                                                                           keys);
            tnn_bitonic_sort(keys, n2, st);
            Lt.qorder = keys;
        }
        k_linear_tc<<<(unsigned)grid, TC_THREADS, smem, st>>>(Lt);
        const cudaError_t le = cudaGetLastError();
        if (keys)
            tnn_free(keys, st);
        TNN_CUDA_TRY(le);
        return finish_search(L, st, prof, pr);
    }
    // TNN with tensor-core candidate tiles: one window, 128 queries per CTA,
    // 256 TMEM columns per CTA; at least 80 KB of shared memory keeps at most
    // 2 CTAs (512 columns) on an SM
    if (!brute && !sweep && (L.w0.flags & TNN_FLAG_TC_TILES) && L.nwin <= 1) {
        const size_t smem = std::max<size_t>(tt_smem_bytes(L.L_max), 80 * 1024);
        if (smem > (size_t)227 * 1024) {
            tnn_set_error("tensor-core TNN kernel does not fit on an SM (%zu B shared memory)", smem);
            return TNN_ERR_UNSUPPORTED;
        }
        nb = std::min<int>(2, (int)(g_smem_per_sm / (smem + 1024)));
        KnnLaunch Lt = L;
        Lt.total_tiles = (L.w0.m + TT_Q - 1) / TT_Q;
        long long grid = std::min<long long>(Lt.total_tiles, (long long)std::max(nb, 1) * g_num_sms);
        if (grid < 1)
            grid = 1;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        const bool prof = g_prof_on && cap == cudaStreamCaptureStatusNone;
        ProfEv pr;
        if (prof)
            TNN_CUDA_TRY(prof_begin(st, &pr));
        k_tnn_tc<<<(unsigned)grid, TT_THREADS, smem, st>>>(Lt);
        TNN_CUDA_TRY(cudaGetLastError());
        return finish_search(L, st, prof, pr);
    }
    if (!brute) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        const bool prof = g_prof_on && cap == cudaStreamCaptureStatusNone;
        ProfEv pr;
        if (prof)
            TNN_CUDA_TRY(prof_begin(st, &pr));
        s = launch_tiles(L, st);
        if (s != TNN_OK) {
            if (prof)
                g_prof_pool.push_back(pr);
            return s;
        }
        return finish_search(L, st, prof, pr);
    }
    const size_t smem = smem_per_warp(L.L_max, L.kseg_max, SMEM_LINEAR) * TNN_WARPS_PER_CTA;
    TNN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_linear_search, TNN_WARPS_PER_CTA * 32, smem));
    if (nb < 1) {
        tnn_set_error("search kernel does not fit on an SM (%zu B shared memory)", smem);
        return TNN_ERR_UNSUPPORTED;
    }
    long long need = (L.total_tiles + TNN_WARPS_PER_CTA - 1) / TNN_WARPS_PER_CTA;
    long long grid = std::min<long long>(need, (long long)nb * g_num_sms);
    if (grid < 1)
        grid = 1;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool prof = g_prof_on && cap == cudaStreamCaptureStatusNone;
    ProfEv pr;
    if (prof)
        TNN_CUDA_TRY(prof_begin(st, &pr));
    k_linear_search<<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    TNN_CUDA_TRY(cudaGetLastError());
    return finish_search(L, st, prof, pr);
}

tnn_status tnn_launch_tiles(const KnnLaunch &L, cudaStream_t st)
{
    tnn_status s = device_setup();
    if (s != TNN_OK)
        return s;
    return launch_tiles(L, st);
}

tnn_status tnn_launch_finish(const KnnLaunch &L, cudaStream_t st)
{
    ProfEv pr;
    return finish_search(L, st, false, pr);
}

// ------------------------------------------------------------- faults

tnn_status tnn_take_search_faults(cudaStream_t st)
{
    unsigned int f = 0;
    TNN_CUDA_TRY(cudaStreamSynchronize(st));
    TNN_CUDA_TRY(cudaMemcpyFromSymbol(&f, g_search_fault, sizeof(f)));
    if (!f)
        return TNN_OK;
    const unsigned int zero = 0;
    TNN_CUDA_TRY(cudaMemcpyToSymbol(g_search_fault, &zero, sizeof(zero)));
    if (f & 4u) {
        tnn_set_error("a bounded device wait of a search timed out (1 s); its outputs are incomplete");
        return TNN_ERR_TIMEOUT;
    }
    tnn_set_error("a search overflowed an internal list (flags %u); its outputs are incomplete", f);
    return TNN_ERR_CUDA;
}

cudaError_t tnn_fault_word_async(unsigned int *h_word, cudaStream_t st)
{
    return cudaMemcpyFromSymbolAsync(h_word, g_search_fault, sizeof(unsigned int), 0,
                                     cudaMemcpyDeviceToHost, st);
}

extern "C" tnn_status tnn_sync_status(tnn_stream_t stream)
{
    tnn_clear_error();
    return tnn_take_search_faults((cudaStream_t)stream);
}

// Self-test of the bounded-wait path: one warp waits on an mbarrier that no
// thread and no copy ever arrives on (nothing else is in flight), gives up
// after limit_ns and raises the timeout flag exactly as the tensor-core
// kernels do.
__global__ void k_selftest_wait(uint64_t limit_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_err;
    if (threadIdx.x == 0) {
        s_err = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_try(su32(&bar), 0u) ||
                    mbar_wait_slow(su32(&bar), 0u, (volatile int *)&s_err, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok)
            atomicOr(&g_search_fault, 4u);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(&bar)) : "memory");
    }
}

extern "C" tnn_status tnn_selftest_bounded_wait(int32_t limit_us, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(limit_us >= 1 && limit_us <= 1000000, "limit_us must be in [1, 10^6]");
    k_selftest_wait<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_us * 1000ull);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

// Which kernel finished each query: 1 for the entries of the list of the
// warp-per-query kernel, then 2 for those of the exact kernel.
__global__ void k_mark_paths(const int2 *__restrict__ list, const unsigned *__restrict__ count,
                             int64_t cap, uint8_t v, uint8_t *__restrict__ path)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = min((int64_t)*count, cap);
    if (i < n)
        path[list[i].y] = v;
}

static tnn_status run_single(const tnn_index *ix, const float *d_q, int64_t m,
                             const tnn_knn_params *p, int32_t *d_idx, float *d_d2,
                             tnn_stats *h_stats, tnn_stream_t stream, bool brute,
                             uint8_t *d_path = nullptr, uint32_t *d_seen = nullptr)
{
    tnn_clear_error();
    if (brute && ix) {
        tnn_status ts = tnn_index_time_order(ix, (cudaStream_t)stream);
        if (ts == TNN_OK && !(p && (p->flags & TNN_FLAG_FFMA))) // threshold seeds of the tensor-core form
            ts = tnn_index_space_order(ix, (cudaStream_t)stream);
        if (ts != TNN_OK)
            return ts;
    }
    if (!brute && ix && p && (p->flags & TNN_FLAG_TC_TILES) && !(p->flags & TNN_FLAG_SWEEP)) {
        tnn_status ts = tnn_index_key_order(ix, (cudaStream_t)stream);
        if (ts != TNN_OK)
            return ts;
    }
    KnnLaunch L;
    memset(&L, 0, sizeof(L));
    tnn_status s = tnn_fill_window(ix, d_q, m, p, d_idx, d_d2, &L.w0);
    if (s != TNN_OK)
        return s;
    TNN_ARG_CHECK(m == 0 || (d_idx != nullptr && d_d2 != nullptr), "NULL output");
    if (h_stats)
        memset(h_stats, 0, sizeof(*h_stats));
    if (m == 0)
        return TNN_OK;
    cudaStream_t st = (cudaStream_t)stream;
    L.nwin = 1;
    L.L_max = L.w0.L;
    L.kseg_max = ix->K;
    if (brute)
        L.w0.tile_rows = nullptr; // the linear search gains nothing from trajectory tiles
    L.total_tiles = tnn_window_tiles(ix, &L.w0);
    L.fb_cap = m;
    if (brute) {
        L.seed_pts = ix->pts_m;
        L.seed_idx = ix->idx_m;
        L.seed_code = ix->code_m;
    }
    const size_t hdr = 256;
    void *buf = nullptr;
    TNN_CUDA_TRY(tnn_alloc(&buf, hdr + (2 * sizeof(int2) + sizeof(float)) * (size_t)m, st));
    L.scr = (KnnScratch *)buf;
    L.fb_list = (int2 *)((char *)buf + hdr);
    L.fb_list3 = L.fb_list + m;
    L.fb_tau = (float *)(L.fb_list3 + m);
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(KnnScratch), st);
    if (e == cudaSuccess && d_seen) {
        L.dbg_seen = d_seen;
        L.dbg_words = (ix->n + 31) / 32;
        e = cudaMemsetAsync(d_seen, 0, sizeof(uint32_t) * (size_t)(m * L.dbg_words), st);
    }
    if (e != cudaSuccess) {
        tnn_free(buf, st);
        TNN_CUDA_TRY(e);
    }
    s = tnn_launch_search(L, brute, st);
    if (s == TNN_OK && d_path) {
        e = cudaMemsetAsync(d_path, 0, (size_t)m, st);
        if (e == cudaSuccess) {
            const unsigned nb = (unsigned)((m + 255) / 256);
            k_mark_paths<<<nb, 256, 0, st>>>(L.fb_list, &L.scr->n_fallback, m, 1, d_path);
            k_mark_paths<<<nb, 256, 0, st>>>(L.fb_list3, &L.scr->n_fallback3, m, 2, d_path);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            tnn_set_error("marking the query paths failed: %s", cudaGetErrorString(e));
            s = TNN_ERR_CUDA;
        }
    }
    KnnScratch hs;
    if (s == TNN_OK && h_stats) {
        e = cudaMemcpyAsync(&hs, buf, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            tnn_set_error("reading search counters failed: %s", cudaGetErrorString(e));
            s = TNN_ERR_CUDA;
        } else {
            h_stats->queries = hs.stats[0];
            h_stats->lb_evals = hs.stats[1];
            h_stats->pairs = hs.stats[2];
            h_stats->segs_scanned = hs.stats[3];
            h_stats->fp64_rechecks = hs.stats[4];
            h_stats->warp_queries = hs.stats[5];
            h_stats->exact_queries = hs.stats[6];
            // this call's flags (folded into the device's fault word by
            // its last kernel) and any earlier unreported ones
            s = tnn_take_search_faults(st);
        }
    }
    tnn_free(buf, st);
    return s;
}

extern "C" tnn_status tnn_knn(const tnn_index *index, const float *d_q, int64_t m,
                              const tnn_knn_params *params, int32_t *d_idx,
                              float *d_d2, tnn_stats *h_stats, tnn_stream_t stream)
{
    return run_single(index, d_q, m, params, d_idx, d_d2, h_stats, stream, false);
}

extern "C" tnn_status tnn_knn_trace(const tnn_index *index, const float *d_q, int64_t m,
                                    const tnn_knn_params *params, int32_t *d_idx, float *d_d2,
                                    uint8_t *d_path, uint32_t *d_seen, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(d_path != nullptr || m == 0, "d_path is NULL");
    TNN_ARG_CHECK(d_seen == nullptr || (params && (params->flags & TNN_FLAG_SWEEP) == 0),
                  "d_seen records the grid order only");
    return run_single(index, d_q, m, params, d_idx, d_d2, nullptr, stream, false, d_path, d_seen);
}

extern "C" tnn_status tnn_knn_bruteforce(const tnn_index *index, const float *d_q,
                                         int64_t m, const tnn_knn_params *params,
                                         int32_t *d_idx, float *d_d2,
                                         tnn_stats *h_stats, tnn_stream_t stream)
{
    return run_single(index, d_q, m, params, d_idx, d_d2, h_stats, stream, true);
}

extern "C" tnn_status tnn_segment_lower_bounds(const tnn_index *index, const float *d_q,
                                               int64_t m, double lag, float *d_lb,
                                               tnn_stream_t stream)
{
    tnn_clear_error();
    tnn_knn_params p;
    memset(&p, 0, sizeof(p));
    p.k = 1;
    p.lag = lag;
    KnnWin w;
    tnn_status s = tnn_fill_window(index, d_q, m, &p, nullptr, nullptr, &w);
    if (s != TNN_OK)
        return s;
    if (m == 0)
        return TNN_OK;
    TNN_ARG_CHECK(d_lb != nullptr, "d_lb is NULL");
    const long long total = m * (long long)index->S;
    k_segment_lb<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(w, d_lb);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

// ------------------------------------------------------------------ batch

struct tnn_batch {
    int device;
    KnnLaunch L;
    KnnWin *d_wins;
    void *scratch;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" void tnn_batch_destroy(tnn_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    cudaFree(b->d_wins);
    cudaFree(b->scratch);
    delete b;
}

extern "C" tnn_status tnn_batch_create(const tnn_index *const *indexes,
                                       const float *const *d_q, const int64_t *m,
                                       const tnn_knn_params *params, int32_t n_windows,
                                       int32_t *const *d_idx, float *const *d_d2,
                                       tnn_batch **out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    TNN_ARG_CHECK(indexes && m && params && d_idx && d_d2, "NULL argument");
    TNN_ARG_CHECK(n_windows >= 1 && n_windows <= (1 << 20), "n_windows must be in [1, 2^20]");
    tnn_status s = device_setup();
    if (s != TNN_OK)
        return s;
    std::vector<KnnWin> wins(n_windows);
    long long tiles = 0, fb = 0;
    int L_max = 0, kseg = 0;
    for (int w = 0; w < n_windows; ++w) {
        s = tnn_fill_window(indexes[w], d_q ? d_q[w] : nullptr, m[w], &params[w],
                            d_idx[w], d_d2[w], &wins[w]);
        if (s != TNN_OK)
            return s;
        TNN_ARG_CHECK(m[w] == 0 || (d_idx[w] != nullptr && d_d2[w] != nullptr),
                      "NULL output for window %d", w);
        TNN_ARG_CHECK((params[w].flags & TNN_FLAG_TC_TILES) == 0,
                      "TNN_FLAG_TC_TILES is for tnn_knn (window %d)", w);
        TNN_ARG_CHECK((params[w].flags & TNN_FLAG_SWEEP) == (params[0].flags & TNN_FLAG_SWEEP),
                      "all windows of a batch take the same segment order (TNN_FLAG_SWEEP; window %d "
                      "differs from window 0)", w);
        wins[w].tile_begin = tiles;
        tiles += tnn_window_tiles(indexes[w], &wins[w]);
        fb += m[w];
        L_max = std::max(L_max, wins[w].L);
        kseg = std::max(kseg, (int)indexes[w]->K);
    }
    tnn_batch *b = new tnn_batch();
    memset(b, 0, sizeof(*b));
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->d_wins, sizeof(KnnWin) * n_windows);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->scratch, 256 + (2 * sizeof(int2) + sizeof(float)) * (size_t)std::max(fb, 1ll));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_wins, wins.data(), sizeof(KnnWin) * n_windows, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tnn_batch_destroy(b);
        tnn_set_error("batch allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    KnnLaunch &L = b->L;
    memset(&L, 0, sizeof(L));
    L.w0 = wins[0];
    L.wins = b->d_wins;
    L.nwin = n_windows;
    L.L_max = L_max;
    L.kseg_max = kseg;
    L.total_tiles = tiles;
    L.scr = (KnnScratch *)b->scratch;
    L.fb_list = (int2 *)((char *)b->scratch + 256);
    L.fb_list3 = L.fb_list + std::max(fb, 1ll);
    L.fb_tau = (float *)(L.fb_list3 + std::max(fb, 1ll));
    L.fb_cap = fb;
    if (n_windows == 1)
        L.nwin = 1;

    // Capture: reset the queue, search, fallback.
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->scratch, 0, sizeof(KnnScratch), cs);
            s = tnn_launch_search(L, false, cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
            if (s == TNN_OK && e2 == cudaSuccess)
                e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            else if (e2 != cudaSuccess)
                e = e2;
        }
        cudaStreamDestroy(cs);
    }
    if (s != TNN_OK || e != cudaSuccess) {
        tnn_batch_destroy(b);
        if (s == TNN_OK) {
            tnn_set_error("batch graph capture failed: %s", cudaGetErrorString(e));
            s = TNN_ERR_CUDA;
        }
        return s;
    }
    *out = b;
    return TNN_OK;
}

extern "C" tnn_status tnn_batch_run(tnn_batch *b, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(b != nullptr, "batch is NULL");
    TNN_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return TNN_OK;
}

extern "C" tnn_status tnn_batch_stats(tnn_batch *b, tnn_stats *h, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(b != nullptr && h != nullptr, "NULL argument");
    KnnScratch hs;
    TNN_CUDA_TRY(cudaMemcpyAsync(&hs, b->scratch, sizeof(hs), cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream));
    TNN_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    h->queries = hs.stats[0];
    h->lb_evals = hs.stats[1];
    h->pairs = hs.stats[2];
    h->segs_scanned = hs.stats[3];
    h->fp64_rechecks = hs.stats[4];
    h->warp_queries = hs.stats[5];
    h->exact_queries = hs.stats[6];
    return tnn_take_search_faults((cudaStream_t)stream);
}

// --------------------------------------------------------------- autotune

extern "C" tnn_status tnn_autotune(const tnn_index *ix, tnn_knn_params *params,
                                   int64_t m_sample, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && params, "NULL argument");
    TNN_ARG_CHECK(m_sample >= 32, "m_sample must be >= 32");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = ix->n;
    // A sample too small to fill the GPU times the slowest warp, not the
    // throughput: at least 262,144 queries (or all of them).  The sample is
    // one run of the index's own rows from its middle, searched as
    // self-queries, so that it takes the same per-trajectory tiles as a
    // self-query of every point.
    m_sample = std::max<int64_t>(m_sample, 262144);
    const int64_t m = std::min<int64_t>(m_sample, n);
    const int64_t r0 = (n - m) / 2;
    const float4 *dq = ix->pts + r0;
    int32_t *di = nullptr;
    float *dd = nullptr;
    cudaError_t e = cudaMalloc(&di, sizeof(int32_t) * m * params->k);
    if (e == cudaSuccess)
        e = cudaMalloc(&dd, sizeof(float) * m * params->k);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    tnn_status s = TNN_OK;
    if (e != cudaSuccess) {
        tnn_set_error("autotune setup failed: %s", cudaGetErrorString(e));
        s = TNN_ERR_CUDA;
    }
    // Candidates: the grid order over seed count F, spare slots and the
    // deferral threshold, plus the sweep order with two seed counts.
    struct Cand {
        int F, E, flags;
        float defer;
    };
    std::vector<Cand> cands;
    for (int F : {2, 3, 4})
        for (int E : {4, 8})
            for (float dfr : {0.6f, 0.75f, 1.0f, 1.5f, 2.0f, 3.0f, 6.0f})
                cands.push_back({F, E, 0, dfr});
    for (int F : {3, 4})
        cands.push_back({F, 4, TNN_FLAG_SWEEP, 0.0f});
    float best = 1e30f;
    tnn_knn_params bestp = *params;
    for (size_t ci = 0; ci < cands.size() && s == TNN_OK; ++ci) {
        tnn_knn_params p = *params;
        p.seed_segments = cands[ci].F;
        p.seed_window = 0;
        p.extra = cands[ci].E;
        p.flags = (params->flags & ~TNN_FLAG_SWEEP) | cands[ci].flags;
        p.defer_cells = cands[ci].defer;
        s = tnn_knn(ix, (const float *)dq, m, &p, di, dd, nullptr, stream);
        if (s != TNN_OK)
            break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && s == TNN_OK; ++r)
            s = tnn_knn(ix, (const float *)dq, m, &p, di, dd, nullptr, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            tnn_set_error("autotune timing failed");
            s = TNN_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bestp = p;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(di);
    cudaFree(dd);
    if (s == TNN_OK)
        s = tnn_take_search_faults(st);
    if (s == TNN_OK) {
        params->seed_segments = bestp.seed_segments;
        params->seed_window = bestp.seed_window;
        params->flags = bestp.flags;
        params->defer_cells = bestp.defer_cells;
        params->extra = bestp.extra;
    }
    return s;
}

extern "C" tnn_status tnn_profile_enable(int32_t on)
{
    tnn_clear_error();
    g_prof_on = on != 0;
    return TNN_OK;
}

extern "C" tnn_status tnn_profile_read_kernels(double *h_ms, int64_t *launches, int32_t reset)
{
    tnn_clear_error();
    double tot[3] = {0.0, 0.0, 0.0};
    for (auto &pr : g_prof_ev) {
        TNN_CUDA_TRY(cudaEventSynchronize(pr.e[3]));
        for (int i = 0; i < 3; ++i) {
            float x = 0.f;
            TNN_CUDA_TRY(cudaEventElapsedTime(&x, pr.e[i], pr.e[i + 1]));
            tot[i] += x;
        }
    }
    if (h_ms)
        for (int i = 0; i < 3; ++i)
            h_ms[i] = tot[i];
    if (launches)
        *launches = (int64_t)g_prof_ev.size();
    if (reset) {
        for (auto &pr : g_prof_ev)
            g_prof_pool.push_back(pr);
        g_prof_ev.clear();
    }
    return TNN_OK;
}

extern "C" tnn_status tnn_profile_read(double *ms, int64_t *launches, int32_t reset)
{
    double k3[3];
    tnn_status s = tnn_profile_read_kernels(k3, launches, reset);
    if (s == TNN_OK && ms)
        *ms = k3[0] + k3[1] + k3[2];
    return s;
}

// ------------------------------------------------------- necessary work

// One thread per query, with its final k-th distance d_k: the work any
// exact search over this index must do -- evaluate the bound of every
// non-empty grid key of the causal buckets whose temporal bound does not
// exceed d_k and whose cell lies within reach, the cylinder bound of every
// segment of the keys whose bound does not exceed d_k, and the distance of
// every member of the segments whose bound does not exceed d_k.
__global__ void k_knn_work(const __grid_constant__ KnnWin W, const float *__restrict__ d2,
                           int k, const uint8_t *__restrict__ path, unsigned long long *out)
{
    const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nlb = 0, npairs = 0, nkeys = 0;
    const int cls = (qi < W.m && path) ? min((int)path[qi], 2) : 0;
    if (qi < W.m) {
        const QCtx c = make_qctx(&W, W.q[qi], true);
        const float dk = d2[qi * k + (k - 1)];
        const GridDesc &G = W.grid;
        const float fb = (c.T32 - G.t0) * G.inv_dt;
        const int bhi = fb >= 0.0f ? (int)fminf(floorf(fb), (float)(G.nb - 1)) : -1;
        for (int b = bhi; b >= 0; --b) {
            if (!(time_lb(c, W.sig[3], G.bpm[b]) <= dk))
                break;
            const float R = sqrtf(dk) * (1.0f + 0x1p-18f) + __ldg(G.ext_max) + c.delta;
            int cx0, cx1, cy0, cy1;
            reach_cells(c.sx, c.sx, R, G.x0, G.inv_cell, G.nx, cx0, cx1);
            reach_cells(c.sy, c.sy, R, G.y0, G.inv_cell, G.ny, cy0, cy1);
            for (int cy = cy0; cy <= cy1; ++cy)
                for (int cx = cx0; cx <= cx1; ++cx) {
                    const int key = b * G.ncell + cy * G.nx + cx;
                    const int lo = G.off[key], hi = G.off[key + 1];
                    if (hi <= lo)
                        continue;
                    ++nkeys;
                    const float rx0 = G.x0 + (float)cx * G.cell, ry0 = G.y0 + (float)cy * G.cell;
                    if (!(cell_lb(c, W.sig[3], rx0, rx0 + G.cell, ry0, ry0 + G.cell, G.ext[key],
                                  G.tB[key]) <= dk))
                        continue;
                    for (int i = lo; i < hi; ++i) {
                        const float4 *r = W.seg + 4 * (size_t)G.ids[i];
                        ++nlb;
                        if (seg_lb(c, W.sig[3], r[0], r[1], r[2]) <= dk)
                            npairs += (unsigned)__float_as_int(r[3].y);
                    }
                }
        }
    }
    // per class of query (the kernel that finished it), summed over the warp
    for (int c = 0; c < 3; ++c) {
        unsigned long long v0 = cls == c ? nlb : 0, v1 = cls == c ? npairs : 0, v2 = cls == c ? nkeys : 0;
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(FULLMASK, v0, o);
            v1 += __shfl_xor_sync(FULLMASK, v1, o);
            v2 += __shfl_xor_sync(FULLMASK, v2, o);
        }
        if ((threadIdx.x & 31) == 0 && (v0 | v1 | v2)) {
            atomicAdd(out + 3 * c, v0);
            atomicAdd(out + 3 * c + 1, v1);
            atomicAdd(out + 3 * c + 2, v2);
        }
    }
}

extern "C" tnn_status tnn_knn_work_split(const tnn_index *index, const float *d_q, int64_t m,
                                         int32_t k, double lag, const float *d_d2,
                                         const uint8_t *d_path, uint64_t *h_work,
                                         tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(h_work != nullptr, "h_work is NULL");
    tnn_knn_params p;
    memset(&p, 0, sizeof(p));
    p.k = k;
    p.lag = lag;
    KnnWin w;
    tnn_status s = tnn_fill_window(index, d_q, m, &p, nullptr, nullptr, &w);
    if (s != TNN_OK)
        return s;
    for (int i = 0; i < 9; ++i)
        h_work[i] = 0;
    if (m == 0)
        return TNN_OK;
    TNN_ARG_CHECK(d_d2 != nullptr, "d_d2 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *buf = nullptr;
    TNN_CUDA_TRY(tnn_alloc((void **)&buf, 72, st));
    cudaError_t e = cudaMemsetAsync(buf, 0, 72, st);
    if (e == cudaSuccess) {
        k_knn_work<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(w, d_d2, k, d_path, buf);
        e = cudaGetLastError();
    }
    unsigned long long h[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, buf, 72, cudaMemcpyDeviceToHost, st);
    tnn_free(buf, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    TNN_CUDA_TRY(e);
    for (int i = 0; i < 9; ++i)
        h_work[i] = h[i];
    return TNN_OK;
}

extern "C" tnn_status tnn_knn_work(const tnn_index *index, const float *d_q, int64_t m,
                                   int32_t k, double lag, const float *d_d2,
                                   uint64_t *h_work, tnn_stream_t stream)
{
    TNN_ARG_CHECK(h_work != nullptr, "h_work is NULL");
    uint64_t h9[9];
    tnn_status s = tnn_knn_work_split(index, d_q, m, k, lag, d_d2, nullptr, h9, stream);
    if (s == TNN_OK)
        for (int i = 0; i < 3; ++i)
            h_work[i] = h9[i];
    return s;
}
