// Stream-ordered device memory of the library.
//
// Index arrays and per-call scratch come from one private memory pool per
// device whose release threshold is unlimited: memory freed by a call stays
// reserved for the next one, so building an index or answering a search maps
// no new pages and never synchronises the device (cudaMalloc / cudaFree do
// both).  tnn_memory_trim hands the reserve back.
#include <string.h>

#include <mutex>

#include "tnn_internal.cuh"

#define TNN_MAX_POOL_DEVICES 64

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[TNN_MAX_POOL_DEVICES];

static cudaError_t pool_of(int dev, cudaMemPool_t *out)
{
    if (dev < 0 || dev >= TNN_MAX_POOL_DEVICES)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess)
            return e;
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t tnn_alloc(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    cudaMemPool_t pool;
    e = pool_of(dev, &pool);
    if (e != cudaSuccess)
        return e;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
}

void tnn_free(void *p, cudaStream_t st)
{
    if (p)
        cudaFreeAsync(p, st);
}

extern "C" tnn_status tnn_memory_trim(int64_t keep_bytes)
{
    tnn_clear_error();
    TNN_ARG_CHECK(keep_bytes >= 0, "keep_bytes must be >= 0");
    int dev = 0;
    TNN_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    TNN_CUDA_TRY(pool_of(dev, &pool));
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    TNN_CUDA_TRY(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
    return TNN_OK;
}

extern "C" tnn_status tnn_memory_reserved(int64_t *h_reserved, int64_t *h_used)
{
    tnn_clear_error();
    TNN_ARG_CHECK(h_reserved != nullptr, "h_reserved is NULL");
    int dev = 0;
    TNN_CUDA_TRY(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    TNN_CUDA_TRY(pool_of(dev, &pool));
    unsigned long long r = 0, u = 0;
    TNN_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
    TNN_CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
    *h_reserved = (int64_t)r;
    if (h_used)
        *h_used = (int64_t)u;
    return TNN_OK;
}
