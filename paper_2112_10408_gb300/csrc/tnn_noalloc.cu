// tnn_knn_noalloc: the exact causal k-NN search of tnn_knn for callers that
// must not allocate device memory -- for example a plugin whose host
// framework owns every device allocation, or a real-time nowcasting loop
// that cannot afford an allocator call that may block or fail under memory
// pressure.  The search needs a little scratch (the work-queue counter, the
// counters, and the lists of queries handed to the fallback scans); here it
// lives in a static device array of this library instead of coming from an
// allocator.  The paper has no counterpart to this entry point.
#include <mutex>
#include <string.h>

#include "tnn_internal.cuh"

// Largest number of queries one call may answer; the array holds the
// scratch header and the two fallback lists for that many queries.
#define TNN_NOALLOC_MAX_QUERIES 65536
#define TNN_NOALLOC_HEADER 256
#define TNN_NOALLOC_BYTES (TNN_NOALLOC_HEADER + (2 * 8 + 4) * TNN_NOALLOC_MAX_QUERIES)

// Resident on every device that loads the library, until the process exits:
// 256 B + 20 B x 65,536 = 1,310,976 B (1.25 MiB + 256 B).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TNN_NOALLOC_BYTES];

#define TNN_NOALLOC_MAX_DEVICES 64
static void *g_noalloc_addr[TNN_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Device address of the array on the current device.  The name of the array
// in host code only stands for it; the address is looked up once per device,
// with that device current, and kept (so a call inside a stream capture does
// no lookup, provided an earlier call on the device did it).  cudaDeviceReset
// reloads the module, after which the kept address is stale: the header
// tells callers not to call again after a reset.
static tnn_status noalloc_scratch(void **out)
{
    int dev = 0;
    TNN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= TNN_NOALLOC_MAX_DEVICES) {
        tnn_set_error("tnn_knn_noalloc supports device ids below %d", TNN_NOALLOC_MAX_DEVICES);
        return TNN_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        TNN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return TNN_OK;
}

extern "C" tnn_status tnn_knn_noalloc(const tnn_index *index, const float *d_q, int64_t m,
                                      const tnn_knn_params *params, int32_t *d_idx,
                                      float *d_d2, tnn_stream_t stream)
{
    tnn_clear_error();
    KnnLaunch L;
    memset(&L, 0, sizeof(L));
    tnn_status s = tnn_fill_window(index, d_q, m, params, d_idx, d_d2, &L.w0);
    if (s != TNN_OK)
        return s;
    TNN_ARG_CHECK(m == 0 || (d_idx != nullptr && d_d2 != nullptr), "NULL output");
    TNN_ARG_CHECK((params->flags & TNN_FLAG_TC_TILES) == 0,
                  "TNN_FLAG_TC_TILES is for tnn_knn (its key-ordered copy is allocated on first use)");
    TNN_ARG_CHECK(m <= TNN_NOALLOC_MAX_QUERIES,
                  "tnn_knn_noalloc answers at most %d queries per call, got %lld; "
                  "call it on slices of the queries",
                  TNN_NOALLOC_MAX_QUERIES, (long long)m);
    if (m == 0)
        return TNN_OK;
    void *scr = nullptr;
    s = noalloc_scratch(&scr);
    if (s != TNN_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    L.nwin = 1;
    L.L_max = L.w0.L;
    L.kseg_max = index->K;
    L.total_tiles = tnn_window_tiles(index, &L.w0);
    L.fb_cap = m;
    L.scr = (KnnScratch *)scr;
    L.fb_list = (int2 *)((char *)scr + TNN_NOALLOC_HEADER);
    L.fb_list3 = L.fb_list + m;
    L.fb_tau = (float *)(L.fb_list3 + m);
    // The array keeps the previous call's contents: the queue counter, the
    // counters and the list lengths must start at zero.
    TNN_CUDA_TRY(cudaMemsetAsync(scr, 0, sizeof(KnnScratch), st));
    // Each of the two fallback lists holds m entries and a query is appended
    // to each at most once, so neither can overflow here; the kernels'
    // flags (an overflow, should that ever change, or an expired wait) go to
    // the device's fault word, which tnn_sync_status reports.
    return tnn_launch_search(L, false, st);
}
