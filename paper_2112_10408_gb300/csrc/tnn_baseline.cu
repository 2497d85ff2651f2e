// The causal averaging baselines of the nowcasting comparison (Sec. 4.1,
// Table 2): the hour average predicts, for a point measured at time t, the
// mean wind of every point measured in [t - 1 h 30, t - 30 min]; the day
// average (non-causal) takes the mean over the whole day.  Both are one
// entry point: the mean of the points with
//     t_q - before_lo <= t_j <= t_q - before_hi
// (comparisons in FP64 on the float times), which is the day average for
// before_lo = +inf, before_hi = -inf.
//
// GPU form.  The points in (t, index) order (kept by the index for the
// linear search) give every window as a contiguous range; the wind is
// gathered in that order and summed into an FP64 prefix array P (P[0] = 0,
// P[i + 1] = P[i] + wind of the i-th point), so a query costs two binary
// searches over the sorted times and one difference:
//     mean = (P[hi] - P[lo]) / (hi - lo).
// The prefix sum is a chunked scan: per 4,096-point chunk a block total,
// a scan of the totals, then each chunk again with its offset.
#include <math.h>
#include <string.h>

#include "tnn_internal.cuh"

#define WAVG_THREADS 256
#define WAVG_ITEMS 16
#define WAVG_CHUNK (WAVG_THREADS * WAVG_ITEMS)

__device__ __forceinline__ double2 wind_at(const float2 *__restrict__ wind,
                                           const int32_t *__restrict__ idx_t, int64_t i)
{
    const float2 w = __ldg(wind + __ldg(idx_t + i));
    return make_double2((double)w.x, (double)w.y);
}

__device__ __forceinline__ double2 dadd2(double2 a, double2 b)
{
    return make_double2(a.x + b.x, a.y + b.y);
}

// Inclusive scan of one double2 per thread over the block; returns this
// thread's inclusive value, *total the block's sum.
__device__ double2 block_scan_d2(double2 v, double2 *total)
{
    __shared__ double2 warp_sum[WAVG_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double ox = __shfl_up_sync(0xffffffffu, v.x, o);
        const double oy = __shfl_up_sync(0xffffffffu, v.y, o);
        if (lane >= o) {
            v.x += ox;
            v.y += oy;
        }
    }
    if (lane == 31)
        warp_sum[wid] = v;
    __syncthreads();
    double2 off = make_double2(0.0, 0.0), tot = make_double2(0.0, 0.0);
    for (int w = 0; w < WAVG_THREADS / 32; ++w) {
        if (w < wid)
            off = dadd2(off, warp_sum[w]);
        tot = dadd2(tot, warp_sum[w]);
    }
    __syncthreads();
    *total = tot;
    return dadd2(v, off);
}

// Pass 1: the sum of every chunk.
__global__ void __launch_bounds__(WAVG_THREADS)
    k_wavg_chunk_sums(const float2 *__restrict__ wind, const int32_t *__restrict__ idx_t,
                      int64_t n, double2 *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * WAVG_CHUNK + (int64_t)threadIdx.x * WAVG_ITEMS;
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < WAVG_ITEMS; ++j)
        if (base + j < n)
            s = dadd2(s, wind_at(wind, idx_t, base + j));
    double2 tot;
    block_scan_d2(s, &tot);
    if (threadIdx.x == 0)
        sums[blockIdx.x] = tot;
}

// Pass 2: exclusive scan of the chunk sums, in place (one block).
__global__ void __launch_bounds__(WAVG_THREADS) k_wavg_scan_sums(double2 *__restrict__ sums, int64_t nchunk)
{
    double2 carry = make_double2(0.0, 0.0);
    for (int64_t b = 0; b < nchunk; b += WAVG_THREADS) {
        const int64_t i = b + threadIdx.x;
        const double2 v = i < nchunk ? sums[i] : make_double2(0.0, 0.0);
        double2 tot;
        const double2 inc = block_scan_d2(v, &tot);
        if (i < nchunk)
            sums[i] = make_double2(carry.x + (inc.x - v.x), carry.y + (inc.y - v.y));
        carry = dadd2(carry, tot);
    }
}

// Pass 3: P[i + 1] for every point of the chunk (P[0] = 0 by block 0).
__global__ void __launch_bounds__(WAVG_THREADS)
    k_wavg_prefix(const float2 *__restrict__ wind, const int32_t *__restrict__ idx_t, int64_t n,
                  const double2 *__restrict__ offs, double2 *__restrict__ P)
{
    const int64_t base = (int64_t)blockIdx.x * WAVG_CHUNK + (int64_t)threadIdx.x * WAVG_ITEMS;
    double2 v[WAVG_ITEMS];
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < WAVG_ITEMS; ++j) {
        v[j] = base + j < n ? wind_at(wind, idx_t, base + j) : make_double2(0.0, 0.0);
        s = dadd2(s, v[j]);
    }
    double2 tot;
    const double2 inc = block_scan_d2(s, &tot);
    double2 run = dadd2(offs[blockIdx.x], make_double2(inc.x - s.x, inc.y - s.y));
#pragma unroll
    for (int j = 0; j < WAVG_ITEMS; ++j) {
        run = dadd2(run, v[j]);
        if (base + j < n)
            P[base + j + 1] = run;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        P[0] = make_double2(0.0, 0.0);
}

// Number of sorted times that do not reach the threshold: strict (t < thr)
// or not (t <= thr).
__device__ __forceinline__ int64_t count_below(const float4 *__restrict__ pts_t, int64_t n, double thr,
                                               bool inclusive)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const double t = (double)__ldg(&pts_t[mid].w);
        if (inclusive ? t <= thr : t < thr)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Pass 4: one thread per query.
__global__ void k_wavg_query(const float4 *__restrict__ pts_t, int64_t n, const double2 *__restrict__ P,
                             const float4 *__restrict__ q, int64_t m, double before_lo,
                             double before_hi, float2 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m)
        return;
    const double tq = (double)q[i].w;
    const int64_t lo = count_below(pts_t, n, tq - before_lo, false); // first t_j >= t_q - before_lo
    const int64_t hi = count_below(pts_t, n, tq - before_hi, true);  // first t_j >  t_q - before_hi
    float2 r = make_float2(__int_as_float(0x7fffffff), __int_as_float(0x7fffffff));
    if (hi > lo) {
        const double c = (double)(hi - lo);
        const double2 a = P[lo], b = P[hi];
        r = make_float2((float)((b.x - a.x) / c), (float)((b.y - a.y) / c));
    }
    out[i] = r;
}

extern "C" tnn_status tnn_window_average(const tnn_index *ix, const float *d_wind,
                                         const float *d_q, int64_t m, double before_lo,
                                         double before_hi, float *d_uv, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && d_wind, "NULL argument");
    TNN_ARG_CHECK(m >= 0, "m must be >= 0");
    TNN_ARG_CHECK(d_q != nullptr || m == ix->n, "self-query needs m == n_points");
    TNN_ARG_CHECK(!isnan(before_lo) && !isnan(before_hi), "window bounds must not be NaN");
    TNN_ARG_CHECK(((uintptr_t)d_wind & 7) == 0, "d_wind must be 8-byte aligned");
    TNN_ARG_CHECK(d_q == nullptr || ((uintptr_t)d_q & 15) == 0, "d_q must be 16-byte aligned");
    if (m == 0)
        return TNN_OK;
    TNN_ARG_CHECK(d_uv != nullptr && ((uintptr_t)d_uv & 7) == 0, "d_uv must be non-NULL and 8-byte aligned");
    int dev = -1;
    cudaGetDevice(&dev);
    TNN_ARG_CHECK(dev == ix->device, "index lives on device %d, current is %d", ix->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    tnn_status s = tnn_index_time_order(ix, st);
    if (s != TNN_OK)
        return s;
    const int64_t n = ix->n;
    const int64_t nchunk = (n + WAVG_CHUNK - 1) / WAVG_CHUNK;
    void *buf = nullptr;
    TNN_CUDA_TRY(tnn_alloc(&buf, sizeof(double2) * (size_t)(nchunk + n + 1), st));
    double2 *sums = (double2 *)buf;
    double2 *P = sums + nchunk;
    const float2 *wind = (const float2 *)d_wind;
    k_wavg_chunk_sums<<<(unsigned)nchunk, WAVG_THREADS, 0, st>>>(wind, ix->idx_t, n, sums);
    k_wavg_scan_sums<<<1, WAVG_THREADS, 0, st>>>(sums, nchunk);
    k_wavg_prefix<<<(unsigned)nchunk, WAVG_THREADS, 0, st>>>(wind, ix->idx_t, n, sums, P);
    const float4 *q = d_q ? (const float4 *)d_q : ix->pts;
    k_wavg_query<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(ix->pts_t, n, P, q, m, before_lo, before_hi,
                                                             (float2 *)d_uv);
    const cudaError_t e = cudaGetLastError();
    tnn_free(buf, st);
    TNN_CUDA_TRY(e);
    return TNN_OK;
}
