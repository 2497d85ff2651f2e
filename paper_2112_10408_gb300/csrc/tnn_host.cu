// The whole pipeline on host buffers: points in, index build, the causal
// k-NN of every point (Sec. 3.5 answers a batch of M points, each its own
// query), neighbour lists out.  Two ways out for the lists:
//   copied  the queries are answered in consecutive slices; as each slice is
//           answered, a second stream copies its lists to the host.
//   mapped  (outputs in mapped page-locked memory) the shared-tile kernel
//           writes each finished tile's rows into the host lists itself, so
//           the transfer runs under the search; the few rows the per-query
//           kernels finish afterwards are written by a kernel at the end.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "tnn_internal.cuh"

#define TNN_HOST_MAX_DEVICES 64
#ifndef TNN_SLICE_RATIO
#define TNN_SLICE_RATIO (2.0 / 3.0) // size of a slice over the one before it
#endif

// One copy stream per device, created on first use (non-blocking: it does
// not serialise with the legacy default stream).
static std::mutex g_copy_mu;
static cudaStream_t g_copy_stream[TNN_HOST_MAX_DEVICES];

static cudaError_t copy_stream(int dev, cudaStream_t *out)
{
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[dev]) {
        cudaError_t e = cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return e;
    }
    *out = g_copy_stream[dev];
    return cudaSuccess;
}

// Events and a page-locked fault word of this host thread on each device,
// created on first use and kept (creating them costs more host time than
// the rest of a call's set-up).
struct HostCallState {
    cudaEvent_t ev[65];
    unsigned int *fault; // page-locked
};

static cudaError_t call_state(int dev, HostCallState **out)
{
    static thread_local HostCallState *t_state[TNN_HOST_MAX_DEVICES];
    if (!t_state[dev]) {
        HostCallState *h = new HostCallState();
        memset(h, 0, sizeof(*h));
        cudaError_t e = cudaHostAlloc((void **)&h->fault, sizeof(unsigned int), cudaHostAllocPortable);
        for (int i = 0; i < 65 && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int i = 0; i < 65; ++i)
                if (h->ev[i])
                    cudaEventDestroy(h->ev[i]);
            if (h->fault)
                cudaFreeHost(h->fault);
            delete h;
            return e;
        }
        t_state[dev] = h;
    }
    *out = t_state[dev];
    return cudaSuccess;
}

// Device address of host range [p, p + bytes) when both of its ends lie in
// page-locked memory mapped into the device's address space at one offset;
// NULL otherwise.
static void *mapped_address(const void *p, size_t bytes)
{
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, (const char *)p + bytes - 1) != cudaSuccess) {
        cudaGetLastError(); // an unknown host pointer is not an error here
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
        (char *)b.devicePointer != (char *)a.devicePointer + (bytes - 1))
        return nullptr;
    return a.devicePointer;
}

// Rows the per-query kernels finished (every entry of the tile kernel's
// hand-over list: deferred or unsettled), copied from the device lists into
// the mapped host lists, one warp per row.
__global__ void k_patch_rows(const int2 *__restrict__ list, const unsigned *__restrict__ count,
                             int64_t cap, int k, const int32_t *__restrict__ d_idx,
                             const float *__restrict__ d_d2, int32_t *m_idx, float *m_d2)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n = min((int64_t)*count, cap);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int64_t o = (int64_t)list[i].y * k;
        for (int j = lane; j < k; j += 32) {
            m_idx[o + j] = d_idx[o + j];
            m_d2[o + j] = d_d2[o + j];
        }
    }
}

// Slice bounds: nc consecutive parts of [0, n), each TNN_SLICE_RATIO times
// the one before it.
static void slice_bounds(int64_t n, int nc, int64_t *bound)
{
    double wsum = 0.0, w = 1.0;
    for (int c = 0; c < nc; ++c, w *= TNN_SLICE_RATIO)
        wsum += w;
    double acc = 0.0;
    w = 1.0;
    bound[0] = 0;
    for (int c = 0; c < nc; ++c, w *= TNN_SLICE_RATIO) {
        acc += w;
        bound[c + 1] = c + 1 == nc ? n : std::min<int64_t>(n, (int64_t)(n * (acc / wsum)));
    }
}

// Slices of complete searches: each slice is a tnn_knn call on `st`, its
// lists copied out on `cs` once answered.
static tnn_status run_copied(tnn_index *ix, int64_t n, const tnn_knn_params *kp, int nc,
                             int32_t *d_idx, float *d_d2, int32_t *h_idx, float *h_d2,
                             cudaStream_t st, cudaStream_t cs, cudaEvent_t *ev)
{
    const int64_t k = kp->k;
    int64_t bound[65];
    slice_bounds(n, nc, bound);
    for (int c = 0; c < nc; ++c) {
        const int64_t r0 = bound[c], r1 = bound[c + 1];
        if (r1 <= r0)
            continue;
        tnn_status s = tnn_knn(ix, (const float *)(ix->pts + r0), r1 - r0, kp, d_idx + r0 * k,
                               d_d2 + r0 * k, nullptr, (tnn_stream_t)st);
        if (s != TNN_OK)
            return s;
        cudaError_t e = cudaEventRecord(ev[c], st);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(cs, ev[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_idx + r0 * k, d_idx + r0 * k, sizeof(int32_t) * (size_t)((r1 - r0) * k),
                                cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_d2 + r0 * k, d_d2 + r0 * k, sizeof(float) * (size_t)((r1 - r0) * k),
                                cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) {
            tnn_set_error("tnn_knn_host copy failed: %s", cudaGetErrorString(e));
            return TNN_ERR_CUDA;
        }
    }
    return TNN_OK;
}

// One window of all n self-queries: the tile kernel mirrors every finished
// tile's rows into the mapped outputs m_idx, m_d2 as it goes, the per-query
// kernels then finish the handed-over queries in the device lists, and
// k_patch_rows writes those rows into the mapped outputs.  All on `st`.
static tnn_status run_mapped(tnn_index *ix, int64_t n, const tnn_knn_params *kp, int32_t *d_idx,
                             float *d_d2, int32_t *m_idx, float *m_d2, cudaStream_t st)
{
    KnnLaunch L;
    memset(&L, 0, sizeof(L));
    tnn_status s = tnn_fill_window(ix, (const float *)ix->pts, n, kp, d_idx, d_d2, &L.w0);
    if (s != TNN_OK)
        return s;
    L.nwin = 1;
    L.L_max = L.w0.L;
    L.kseg_max = ix->K;
    L.total_tiles = tnn_window_tiles(ix, &L.w0);
    L.fb_cap = n;
    L.mirror_idx = m_idx;
    L.mirror_d2 = m_d2;
    L.mirror_vec = kp->k % 4 == 0 && (((uintptr_t)m_idx | (uintptr_t)m_d2 | (uintptr_t)d_idx | (uintptr_t)d_d2) & 15) == 0;
    const size_t hdr = 256;
    void *buf = nullptr;
    TNN_CUDA_TRY(tnn_alloc(&buf, hdr + (2 * sizeof(int2) + sizeof(float)) * (size_t)n, st));
    L.scr = (KnnScratch *)buf;
    L.fb_list = (int2 *)((char *)buf + hdr);
    L.fb_list3 = L.fb_list + n;
    L.fb_tau = (float *)(L.fb_list3 + n);
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(KnnScratch), st);
    if (e != cudaSuccess) {
        tnn_free(buf, st);
        TNN_CUDA_TRY(e);
    }
    s = tnn_launch_tiles(L, st);
    if (s == TNN_OK)
        s = tnn_launch_finish(L, st);
    if (s == TNN_OK) {
        k_patch_rows<<<1024, 256, 0, st>>>(L.fb_list, &L.scr->n_fallback, L.fb_cap, (int)kp->k, d_idx,
                                            d_d2, m_idx, m_d2);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            tnn_set_error("tnn_knn_host row patch failed: %s", cudaGetErrorString(e));
            s = TNN_ERR_CUDA;
        }
    }
    tnn_free(buf, st);
    return s;
}

extern "C" tnn_status tnn_knn_host(const float *h_xyzt, int64_t n, const int64_t *h_traj_off,
                                   int64_t n_traj, const tnn_build_params *bp,
                                   const tnn_knn_params *kp, int32_t chunks, int32_t *h_idx,
                                   float *h_d2, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(h_xyzt && h_traj_off && bp && kp && h_idx && h_d2, "NULL argument");
    TNN_ARG_CHECK(n >= 1 && n < (1ll << 31) - 64, "n must be in [1, 2^31-64), got %lld",
                  (long long)n);
    TNN_ARG_CHECK(kp->k >= 1 && kp->k <= 64, "k must be in [1, 64], got %d", kp->k);
    TNN_ARG_CHECK(chunks >= 0 && chunks <= 64, "chunks must be in [0, 64]");
    const int64_t k = kp->k;
    const bool mapped = (kp->flags & TNN_FLAG_MAPPED_OUT) && !(kp->flags & TNN_FLAG_TC_TILES);
    int dev = 0;
    TNN_CUDA_TRY(cudaGetDevice(&dev));
    TNN_ARG_CHECK(dev >= 0 && dev < TNN_HOST_MAX_DEVICES, "device ordinal out of range");
    int32_t *m_idx = nullptr;
    float *m_d2 = nullptr;
    if (mapped) {
        m_idx = (int32_t *)mapped_address(h_idx, sizeof(int32_t) * (size_t)(n * k));
        m_d2 = (float *)mapped_address(h_d2, sizeof(float) * (size_t)(n * k));
        TNN_ARG_CHECK(m_idx && m_d2,
                      "TNN_FLAG_MAPPED_OUT: h_idx and h_d2 must be mapped page-locked host memory");
    }
    // the library's choice: 2 slices, 3 from 2^20 queries (the fixed costs of
    // a slice weigh less against a longer search); mapped outputs: no slices
    const int nc = mapped ? 1 : (int)std::min<int64_t>(chunks != 0 ? chunks : (n >= (1 << 20) ? 3 : 2), n);
    cudaStream_t st = (cudaStream_t)stream, cs = nullptr;
    TNN_CUDA_TRY(copy_stream(dev, &cs));
    HostCallState *hs = nullptr;
    TNN_CUDA_TRY(call_state(dev, &hs));
    // ev[c]: slice c answered; ev[nc]: last copy done
    cudaEvent_t *ev = hs->ev;

    float *d_x = nullptr;
    int32_t *d_idx = nullptr;
    float *d_d2 = nullptr;
    tnn_index *ix = nullptr;
    tnn_status s = TNN_OK;
    cudaError_t e = tnn_alloc((void **)&d_x, sizeof(float4) * (size_t)n, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&d_idx, sizeof(int32_t) * (size_t)(n * k), st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&d_d2, sizeof(float) * (size_t)(n * k), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_x, h_xyzt, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        tnn_set_error("tnn_knn_host set-up failed: %s", cudaGetErrorString(e));
        s = e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    if (s == TNN_OK)
        s = tnn_build_segments(d_x, n, h_traj_off, n_traj, bp, stream, &ix);
    if (s == TNN_OK)
        s = mapped ? run_mapped(ix, n, kp, d_idx, d_d2, m_idx, m_d2, st)
                   : run_copied(ix, n, kp, nc, d_idx, d_d2, h_idx, h_d2, st, cs, ev);
    // `st` joins the copy stream; then the scratch and the index go back to
    // the pool in its order, the device's fault word is read back, and one
    // synchronisation ends the call
    const bool joined =
        cudaEventRecord(ev[nc], cs) == cudaSuccess && cudaStreamWaitEvent(st, ev[nc], 0) == cudaSuccess;
    if (!joined)
        cudaStreamSynchronize(cs);
    tnn_free(d_idx, st);
    tnn_free(d_d2, st);
    tnn_free(d_x, st);
    tnn_index_release(ix, st);
    *hs->fault = 0;
    const cudaError_t e1 = tnn_fault_word_async(hs->fault, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == TNN_OK && (!joined || e1 != cudaSuccess || e2 != cudaSuccess)) {
        tnn_set_error("tnn_knn_host failed: %s",
                      cudaGetErrorString(e2 != cudaSuccess ? e2 : e1 != cudaSuccess ? e1 : cudaGetLastError()));
        s = TNN_ERR_CUDA;
    }
    if (s == TNN_OK && *hs->fault != 0)
        s = tnn_take_search_faults(st);
    return s;
}
