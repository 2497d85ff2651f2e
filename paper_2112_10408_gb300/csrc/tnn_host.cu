// The whole pipeline on host buffers: points in, index build, the causal
// k-NN of every point (Sec. 3.5 answers a batch of M points, each its own
// query), neighbour lists out.  The queries are answered in consecutive
// slices; while the search works on one slice, a second stream copies the
// lists of the previous one to the host.
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

static cudaError_t copy_stream(cudaStream_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= TNN_HOST_MAX_DEVICES)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[dev]) {
        e = cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return e;
    }
    *out = g_copy_stream[dev];
    return cudaSuccess;
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
    // the library's choice: 2 slices, 3 from 2^20 queries (the fixed costs of
    // a slice weigh less against a longer search)
    const int nc = (int)std::min<int64_t>(chunks == 0 ? (n >= (1 << 20) ? 3 : 2) : chunks, n);
    const int64_t k = kp->k;
    cudaStream_t st = (cudaStream_t)stream, cs = nullptr;
    TNN_CUDA_TRY(copy_stream(&cs));

    float *d_x = nullptr;
    int32_t *d_idx = nullptr;
    float *d_d2 = nullptr;
    tnn_index *ix = nullptr;
    cudaEvent_t ev[65] = {};
    tnn_status s = TNN_OK;
    cudaError_t e = tnn_alloc((void **)&d_x, sizeof(float4) * (size_t)n, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&d_idx, sizeof(int32_t) * (size_t)(n * k), st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&d_d2, sizeof(float) * (size_t)(n * k), st);
    for (int c = 0; c <= nc && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_x, h_xyzt, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        tnn_set_error("tnn_knn_host set-up failed: %s", cudaGetErrorString(e));
        s = e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    if (s == TNN_OK)
        s = tnn_build_segments(d_x, n, h_traj_off, n_traj, bp, stream, &ix);
    // Slices shrink geometrically (ratio 2/3, about the time a row's lists
    // take to copy over the time its search takes), so that the copy of one
    // slice ends under the search of the next; each slice's lists go out on
    // the copy stream once the search stream has answered it.
    int64_t bound[65];
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
    for (int c = 0; c < nc && s == TNN_OK; ++c) {
        const int64_t r0 = bound[c], r1 = bound[c + 1];
        if (r1 <= r0)
            continue;
        s = tnn_knn(ix, (const float *)(ix->pts + r0), r1 - r0, kp, d_idx + r0 * k,
                    d_d2 + r0 * k, nullptr, stream);
        if (s != TNN_OK)
            break;
        e = cudaEventRecord(ev[c], st);
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
            s = TNN_ERR_CUDA;
        }
    }
    // the scratch goes back to the pool after the last copy has read it
    if (ev[nc] && cudaEventRecord(ev[nc], cs) == cudaSuccess)
        cudaStreamWaitEvent(st, ev[nc], 0);
    else
        cudaStreamSynchronize(cs);
    tnn_free(d_idx, st);
    tnn_free(d_d2, st);
    tnn_free(d_x, st);
    cudaError_t e1 = cudaStreamSynchronize(cs);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == TNN_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) {
        tnn_set_error("tnn_knn_host failed: %s",
                      cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        s = TNN_ERR_CUDA;
    }
    if (s == TNN_OK)
        s = tnn_take_search_faults(st);
    for (int c = 0; c <= nc; ++c)
        if (ev[c])
            cudaEventDestroy(ev[c]);
    if (ix)
        tnn_index_destroy(ix);
    return s;
}
