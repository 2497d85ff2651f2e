// Index construction: Sec. 3.4 (partitioning trajectories into sets of K
// points approximated by segments, the approximation error) and the segment
// matrices A, t_A, B, t_B, U, E of the Fig. 2 caption.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "tnn_internal.cuh"

namespace cg = cooperative_groups;

// ------------------------------------------------------------------ errors

static thread_local char g_err[512];

void tnn_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void tnn_clear_error() { g_err[0] = 0; }

extern "C" const char *tnn_last_error(void) { return g_err; }

extern "C" const char *tnn_status_string(tnn_status s)
{
    switch (s) {
    case TNN_OK: return "ok";
    case TNN_ERR_INVALID_ARG: return "invalid argument";
    case TNN_ERR_OOM: return "out of device memory";
    case TNN_ERR_CUDA: return "CUDA error";
    case TNN_ERR_TIMEOUT: return "device wait timed out";
    case TNN_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

// ----------------------------------------------------------- device helpers

// Order-preserving map of a float to uint32 (negative values included).
__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

enum { BAD_VALUE = 1, BAD_ORDER = 2 };

// Every coordinate finite with |v| <= 1e15 (so every FP32 squared
// difference stays finite); largest |sqrt(sigma) * x| over the spatial axes.
__global__ void k_validate_points(const float4 *__restrict__ p, int n,
                                  float s0, float s1, float s2,
                                  unsigned int *flag, unsigned int *cmax_bits)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < n) {
        float4 v = p[i];
        bool ok = fabsf(v.x) <= 1e15f && fabsf(v.y) <= 1e15f &&
                  fabsf(v.z) <= 1e15f && fabsf(v.w) <= 1e15f;
        if (!ok)
            atomicOr(flag, (unsigned)BAD_VALUE);
        else
            m = fmaxf(fmaxf(fabsf(s0 * v.x), fabsf(s1 * v.y)), fabsf(s2 * v.z));
    }
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f)
        atomicMax(cmax_bits, __float_as_uint(m)); // m >= 0: bits are monotone
}

// Times non-decreasing inside each trajectory, and the summed duration
// t_last - t_first of its K-point sets, which sizes the grid's time buckets
// (one warp per trajectory).
__global__ void k_validate_traj(const float4 *__restrict__ p,
                                const int32_t *__restrict__ traj_off,
                                int n_traj, int K, unsigned int *flag, double *dur_sum)
{
    const int tr = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (tr >= n_traj) // the same for the whole warp
        return;
    const int b = traj_off[tr], e = traj_off[tr + 1];
    bool bad = false;
    for (int i = b + 1 + lane; i < e; i += 32)
        bad |= !(p[i].w >= p[i - 1].w);
    double dur = 0.0;
    for (int f = b + lane * K; f < e; f += 32 * K)
        dur += (double)p[min(f + K - 1, e - 1)].w - (double)p[f].w;
    for (int o = 16; o > 0; o >>= 1)
        dur += __shfl_xor_sync(0xffffffffu, dur, o);
    if (__any_sync(0xffffffffu, bad) && lane == 0)
        atomicOr(flag, (unsigned)BAD_ORDER);
    if (lane == 0 && dur != 0.0)
        atomicAdd(dur_sum, dur);
}

// SF_LANES lanes per segment (build order).  FP64 throughout, rounded once to
// the stored FP32 record:
//   A' = fl(sqrt(s) A),  AB' = fl(sqrt(s) B - A'),  U' = fl(AB' / |AB'|^2)
// The stored segment is [A', A' + AB'] (both exactly representable);
// r bounds, with upward rounding, the distance of every member's scaled
// position sqrt(s) p_j to it (Sec. 3.4 E_app, in the cylinder reading).
#ifndef SF_LANES
#define SF_LANES 4 // a power of two, at most 32
#endif
__global__ void k_segment_fit(const float4 *__restrict__ p,
                              const int32_t *__restrict__ traj_off,
                              const int32_t *__restrict__ seg_off, int n_traj,
                              int S, int K, double q0, double q1, double q2,
                              float4 *__restrict__ rec,
                              unsigned long long *__restrict__ keys,
                              unsigned int *rmax_bits)
{
    // SF_LANES lanes per segment, splitting its members (FP64 is scarce:
    // the per-segment set-up is repeated by each of them)
    const int s_raw = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / SF_LANES);
    const int sub = threadIdx.x % SF_LANES;
    const bool valid = s_raw < S;
    const int s = valid ? s_raw : S - 1;
    // trajectory of segment s: largest tr with seg_off[tr] <= s
    int lo = 0, hi = n_traj; // seg_off[lo] <= s < seg_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (seg_off[mid] <= s)
            lo = mid;
        else
            hi = mid;
    }
    int tr = lo;
    int first = traj_off[tr] + (s - seg_off[tr]) * K;
    int count = min(K, traj_off[tr + 1] - first);
    float4 pa = p[first], pb = p[first + count - 1];
    double A[3], E[3], AB[3];
    float Af[3], ABf[3], Uf[3];
    const double qq[3] = {q0, q1, q2};
    const float pav[3] = {pa.x, pa.y, pa.z}, pbv[3] = {pb.x, pb.y, pb.z};
    for (int i = 0; i < 3; ++i) {
        Af[i] = (float)(qq[i] * (double)pav[i]);
        A[i] = (double)Af[i];
        ABf[i] = (float)(qq[i] * (double)pbv[i] - A[i]);
        AB[i] = (double)ABf[i];
        E[i] = A[i] + AB[i];
    }
    const double ab2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
    // Any lam in [0, 1] names a point of the segment, so the distance to it
    // bounds the distance to the segment from above: lam = dot / |AB|^2 may
    // take the reciprocal (one division per lane, not one per member).
    const double inv_ab2 = ab2 > 0.0 ? 1.0 / ab2 : 0.0;
    // mag only scales the rounding slack below, which is about a thousand
    // times the FP64 error of the distances; FP32 is ample for it.
    const float qf[3] = {(float)q0, (float)q1, (float)q2};
    float mag = fabsf(Af[0]) + fabsf(Af[1]) + fabsf(Af[2]) + fabsf((float)E[0]) +
                fabsf((float)E[1]) + fabsf((float)E[2]);
    double r2 = 0.0;
    for (int j = sub; j < (valid ? count : 0); j += SF_LANES) {
        const float4 v = p[first + j];
        const double D0 = qq[0] * (double)v.x - A[0], D1 = qq[1] * (double)v.y - A[1],
                     D2 = qq[2] * (double)v.z - A[2];
        const double lam = fmin(fmax((D0 * AB[0] + D1 * AB[1] + D2 * AB[2]) * inv_ab2, 0.0), 1.0);
        const double e0 = D0 - lam * AB[0], e1 = D1 - lam * AB[1], e2 = D2 - lam * AB[2];
        r2 = fmax(r2, e0 * e0 + e1 * e1 + e2 * e2);
        mag = fmaxf(mag, fabsf(qf[0] * v.x) + fabsf(qf[1] * v.y) + fabsf(qf[2] * v.z));
    }
    for (int o = 1; o < SF_LANES; o <<= 1) {
        r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
        mag = fmaxf(mag, __shfl_xor_sync(0xffffffffu, mag, o));
    }
    const bool writer = valid && sub == 0;
    unsigned int rbits = 0u;
    if (writer) {
        for (int i = 0; i < 3; ++i)
            Uf[i] = ab2 > 1e-30 ? (float)(AB[i] / ab2) : 0.f;
        // FP64 rounding of the distances above is far below 1e-12 * mag.
        const double r = sqrt(r2) + 1e-12 * (1.0 + (double)mag);
        const float rf = __double2float_ru(r);
        rbits = __float_as_uint(rf); // rf >= 0: the bits order like the values
        rec[4 * s + 0] = make_float4(Af[0], Af[1], Af[2], pa.w);
        rec[4 * s + 1] = make_float4(Uf[0], Uf[1], Uf[2], pb.w);
        rec[4 * s + 2] = make_float4(ABf[0], ABf[1], ABf[2], rf);
        rec[4 * s + 3] = make_float4(__int_as_float(first), __int_as_float(count),
                                     __int_as_float(tr), __int_as_float(s));
        keys[s] = ((unsigned long long)f2ord(pa.w) << 32) | (unsigned)s;
    }
    rbits = __reduce_max_sync(0xffffffffu, rbits); // one atomic per warp
    if ((threadIdx.x & 31) == 0 && rbits != 0u)
        atomicMax(rmax_bits, rbits);
}

__global__ void k_time_keys(const float4 *__restrict__ p, int n,
                            unsigned long long *__restrict__ keys, int n2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        keys[i] = ((unsigned long long)f2ord(p[i].w) << 32) | (unsigned)i;
    else if (i < n2)
        keys[i] = ~0ull;
}

__global__ void k_fill(unsigned long long *keys, int from, int n2)
{
    int i = from + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2)
        keys[i] = ~0ull;
}

// ------------------------------------------------------------ bitonic sort
//
// Batcher's bitonic network on n2 = 2^p 64-bit keys, ascending.  Step (k, j)
// compares positions i and i + j (bit j of i clear) and puts the smaller key
// first when bit k of i is clear, last otherwise.  Every kernel below keeps
// four consecutive keys per thread in registers: steps j = 1, 2 stay inside a
// thread, steps 4 <= j <= 64 inside a warp (shuffles, no barrier), steps
// 128 <= j < block size go through shared memory, and larger steps through
// distributed shared memory (cluster) or global memory.

#define BS_MIN 2048  // smallest n2 handed out (a cluster of 8 x 256 keys)
#define BS_BLOCK 4096 // keys per CTA of the multi-launch path (1024 threads)

__device__ __forceinline__ void cmpx(unsigned long long &a,
                                     unsigned long long &b, bool asc)
{
    if ((a > b) == asc) {
        unsigned long long t = a;
        a = b;
        b = t;
    }
}

__device__ __forceinline__ void bs_load4(unsigned long long (&r)[4], const unsigned long long *p)
{
    const ulonglong2 a = ((const ulonglong2 *)p)[0], b = ((const ulonglong2 *)p)[1];
    r[0] = a.x;
    r[1] = a.y;
    r[2] = b.x;
    r[3] = b.y;
}

__device__ __forceinline__ void bs_store4(unsigned long long *p, const unsigned long long (&r)[4])
{
    ((ulonglong2 *)p)[0] = make_ulonglong2(r[0], r[1]);
    ((ulonglong2 *)p)[1] = make_ulonglong2(r[2], r[3]);
}

// Steps j, j/2, ..., 1 (j <= 64) of stage k on the four keys at global
// positions g0 .. g0 + 3 (g0 a multiple of 4); the partner of a key at
// distance j >= 4 sits in lane ^ (j / 4) of the same warp.
__device__ __forceinline__ void bs_warp_steps(unsigned long long (&r)[4], int g0, int k, int j)
{
    for (; j >= 4; j >>= 1) {
        const int ld = j >> 2;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, r[e], ld);
            const int g = g0 + e;
            const bool take_min = ((g & j) == 0) == ((g & k) == 0);
            const bool w_lt = w < r[e];
            r[e] = (take_min == w_lt) ? w : r[e];
        }
    }
    if (j >= 2) { // k >= 4: the four keys share bit k
        const bool asc = (g0 & k) == 0;
        cmpx(r[0], r[2], asc);
        cmpx(r[1], r[3], asc);
    }
    cmpx(r[0], r[1], (g0 & k) == 0);
    cmpx(r[2], r[3], ((g0 + 2) & k) == 0);
}

// Steps j, j/2, ..., 1 (j < nl) of stage k on a CTA's nl consecutive keys
// starting at global position gb, held four per thread (nl / 4 threads);
// s has room for nl keys.
__device__ __forceinline__ void bs_local_steps(unsigned long long (&r)[4], unsigned long long *s,
                                               int nl, int gb, int k, int j)
{
    const int t = threadIdx.x, nt = nl >> 2;
    if (j >= 128) {
        bs_store4(s + 4 * t, r);
        __syncthreads();
        for (; j >= 128; j >>= 1) {
            for (int q = t; q < (nl >> 1); q += nt) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1)); // j is a power of two
                cmpx(s[i], s[i + j], ((gb + i) & k) == 0);
            }
            __syncthreads();
        }
        bs_load4(r, s + 4 * t); // each thread rereads only its own four slots
    }
    bs_warp_steps(r, gb + 4 * t, k, j);
}

// Stages 2 .. BS_BLOCK, each 4096-key block on its own (the direction of a
// block follows its global position, as the network requires).
__global__ void __launch_bounds__(BS_BLOCK / 4) k_bitonic_block(unsigned long long *keys)
{
    __shared__ __align__(16) unsigned long long s[BS_BLOCK];
    const int base = blockIdx.x * BS_BLOCK;
    unsigned long long r[4];
    bs_load4(r, keys + base + 4 * threadIdx.x);
    for (int k = 2; k <= BS_BLOCK; k <<= 1)
        bs_local_steps(r, s, BS_BLOCK, base, k, k >> 1);
    bs_store4(keys + base + 4 * threadIdx.x, r);
}

// Steps j < BS_BLOCK of stage k, inside each block.
__global__ void __launch_bounds__(BS_BLOCK / 4) k_bitonic_merge_local(unsigned long long *keys, int k)
{
    __shared__ __align__(16) unsigned long long s[BS_BLOCK];
    const int base = blockIdx.x * BS_BLOCK;
    unsigned long long r[4];
    bs_load4(r, keys + base + 4 * threadIdx.x);
    bs_local_steps(r, s, BS_BLOCK, base, k, BS_BLOCK >> 1);
    bs_store4(keys + base + 4 * threadIdx.x, r);
}

__global__ void k_bitonic_global(unsigned long long *keys, int j, int k)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x; // one per pair
    int i = ((t & ~(j - 1)) << 1) | (t & (j - 1)); // j is a power of two
    bool asc = (i & k) == 0;
    unsigned long long a = keys[i], b = keys[i + j];
    if ((a > b) == asc) {
        keys[i] = b;
        keys[i + j] = a;
    }
}

int tnn_next_pow2_sort(int64_t n)
{
    int64_t p = BS_MIN;
    while (p < n)
        p <<= 1;
    return (int)p;
}

// The whole network for n2 <= 32768 keys in one launch: a cluster of 8 CTAs
// of n2 / 32 threads, CTA c holding keys c * n2 / 8 .. (c + 1) * n2 / 8 - 1.
// A step whose partner lies in another CTA (j >= n2 / 8) publishes the keys
// in shared memory and reads the partner's through distributed shared memory
// between two cluster barriers: the first makes every key visible, the
// second keeps a CTA from overwriting (or leaving) its buffer while its
// partner still reads it.
#define BS_CLUSTER 8
#define BS_CLUSTER_MAX (BS_CLUSTER * 4096)

__global__ void __cluster_dims__(BS_CLUSTER, 1, 1) __launch_bounds__(1024)
    k_bitonic_cluster(unsigned long long *keys, int n2)
{
    __shared__ __align__(16) unsigned long long s[4096];
    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)cluster.block_rank(), nl = n2 / BS_CLUSTER, base = c * nl;
    const int g0 = base + 4 * threadIdx.x;
    unsigned long long r[4];
    bs_load4(r, keys + g0);
    for (int k = 2; k <= n2; k <<= 1) {
        int j = k >> 1;
        for (; j >= nl; j >>= 1) {
            const unsigned long long *peer = cluster.map_shared_rank(s, c ^ (j / nl));
            bs_store4(s + 4 * threadIdx.x, r);
            cluster.sync();
            unsigned long long w[4];
            bs_load4(w, peer + 4 * threadIdx.x);
            const bool take_min = ((g0 & j) == 0) == ((g0 & k) == 0); // same for g0 .. g0 + 3
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool w_lt = w[e] < r[e];
                r[e] = (take_min == w_lt) ? w[e] : r[e];
            }
            cluster.sync();
        }
        bs_local_steps(r, s, nl, base, k, j);
    }
    bs_store4(keys + g0, r);
}

void tnn_bitonic_sort(unsigned long long *keys, int n2, cudaStream_t st)
{
    if (n2 <= BS_CLUSTER_MAX) {
        k_bitonic_cluster<<<BS_CLUSTER, n2 / (4 * BS_CLUSTER), 0, st>>>(keys, n2);
        return;
    }
    k_bitonic_block<<<n2 / BS_BLOCK, BS_BLOCK / 4, 0, st>>>(keys);
    for (int k = 2 * BS_BLOCK; k <= n2; k <<= 1) {
        for (int j = k >> 1; j >= BS_BLOCK; j >>= 1)
            k_bitonic_global<<<(n2 / 2 + 255) / 256, 256, 0, st>>>(keys, j, k);
        k_bitonic_merge_local<<<n2 / BS_BLOCK, BS_BLOCK / 4, 0, st>>>(keys, k);
    }
}

// --------------------------------------------------------- gather / scans

__global__ void k_gather_segments(const unsigned long long *__restrict__ keys,
                                  const float4 *__restrict__ rec, int S,
                                  float4 *__restrict__ out,
                                  float *__restrict__ tA, int32_t *__restrict__ pos)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S)
        return;
    int s = (int)(keys[i] & 0xffffffffu);
    pos[s] = i;
    float4 a = rec[4 * s];
    out[4 * i + 0] = a;
    out[4 * i + 1] = rec[4 * s + 1];
    out[4 * i + 2] = rec[4 * s + 2];
    out[4 * i + 3] = rec[4 * s + 3];
    tA[i] = a.w;
}

// Running maximum of t_B over the t_A order, in two passes over blocks of
// 1024 segments: the maximum of every block, then per block the maxima of
// the blocks before it and a block-wide inclusive scan.
__device__ __forceinline__ float block_max_1024(float v, float *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0)
        sh[w] = v;
    __syncthreads();
    v = sh[lane];
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    return v;
}

__global__ void __launch_bounds__(1024) k_pm_block_max(const float4 *__restrict__ seg, int S,
                                                       float *__restrict__ bmax)
{
    __shared__ float sh[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const float v = block_max_1024(i < S ? seg[4 * i + 1].w : -INFINITY, sh);
    if (threadIdx.x == 0)
        bmax[blockIdx.x] = v;
}

__global__ void __launch_bounds__(1024) k_pm_apply(const float4 *__restrict__ seg, int S,
                                                   const float *__restrict__ bmax,
                                                   float *__restrict__ pm)
{
    __shared__ float sh[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float c = -INFINITY;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += 1024)
        c = fmaxf(c, bmax[b]);
    const float carry = block_max_1024(c, sh);
    const int i = blockIdx.x * 1024 + threadIdx.x;
    float v = i < S ? seg[4 * i + 1].w : -INFINITY;
    for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v = fmaxf(v, u);
    }
    if (lane == 31)
        sh[w] = v;
    __syncthreads();
    if (w == 0) {
        float y = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const float u = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o)
                y = fmaxf(y, u);
        }
        sh[lane] = y;
    }
    __syncthreads();
    if (w > 0)
        v = fmaxf(v, sh[w - 1]);
    if (i < S)
        pm[i] = fmaxf(v, carry);
}

__global__ void k_gather_points(const unsigned long long *__restrict__ keys,
                                const float4 *__restrict__ p, int n,
                                float4 *__restrict__ out,
                                int32_t *__restrict__ idx)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int j = (int)(keys[i] & 0xffffffffu);
    out[i] = p[j];
    idx[i] = j;
}

// ------------------------------------------------------------------- grid

__device__ __forceinline__ float ord2f(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Bounding box of the raw points (x, y, z, t): ordered min/max per axis,
// reduced over the block (grid-stride) before one atomic per value.
__global__ void k_point_bbox(const float4 *__restrict__ p, int n, unsigned int *ord)
{
    __shared__ unsigned int s[32][8];
    unsigned int m[8] = {0xffffffffu, 0u, 0xffffffffu, 0u, 0xffffffffu, 0u, 0xffffffffu, 0u};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 v = p[i];
        const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const unsigned int u = f2ord(c[d]);
            m[2 * d] = min(m[2 * d], u);
            m[2 * d + 1] = max(m[2 * d + 1], u);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 0; d < 8; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned int x = __shfl_xor_sync(0xffffffffu, m[d], o);
            m[d] = (d & 1) ? max(m[d], x) : min(m[d], x);
        }
    if (lane == 0)
        for (int d = 0; d < 8; ++d)
            s[w][d] = m[d];
    __syncthreads();
    if (threadIdx.x < 8) {
        const int d = threadIdx.x;
        unsigned int r = s[0][d];
        for (int j = 1; j < nw; ++j)
            r = (d & 1) ? max(r, s[j][d]) : min(r, s[j][d]);
        if (d & 1)
            atomicMax(ord + d, r);
        else
            atomicMin(ord + d, r);
    }
}

struct GridBuild {
    float x0, y0, cell, inv_cell, t0, dt, inv_dt;
    int nx, ny, ncell, nb;
};

// Key of every segment (records in build order; the key's low half is the
// build id, so the keys sort without the t_A order and the two sorts run
// side by side) and the per-key aggregates: the extent (FP64, rounded up) of
// the member cylinders around the key's cell rectangle and the largest t_B;
// the per-bucket largest t_B.
__global__ void k_grid_keys(const float4 *__restrict__ seg, int S, GridBuild g,
                            unsigned long long *__restrict__ keys,
                            unsigned int *__restrict__ ext_bits,
                            unsigned int *__restrict__ tB_ord,
                            unsigned int *__restrict__ bmax_ord)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x; // build id
    if (p >= S)
        return;
    const float4 a = seg[4 * p], u = seg[4 * p + 1], b = seg[4 * p + 2];
    const float mx = fmaf(0.5f, b.x, a.x), my = fmaf(0.5f, b.y, a.y);
    const int bk = min(max((int)floorf((a.w - g.t0) * g.inv_dt), 0), g.nb - 1);
    const int cx = min(max((int)floorf((mx - g.x0) * g.inv_cell), 0), g.nx - 1);
    const int cy = min(max((int)floorf((my - g.y0) * g.inv_cell), 0), g.ny - 1);
    const int key = bk * g.ncell + cy * g.nx + cx;
    keys[p] = ((unsigned long long)(unsigned)key << 32) | (unsigned)p;
    // every cylinder point is within |AB|/2 + r of the midpoint
    const double ax = a.x, ay = a.y, bx = b.x, by = b.y, bz = b.z;
    const double half = 0.5 * sqrt(bx * bx + by * by + bz * bz) + (double)b.w;
    const double Mx = ax + 0.5 * bx, My = ay + 0.5 * by;
    const double rx0 = (double)g.x0 + cx * (double)g.cell, rx1 = rx0 + g.cell;
    const double ry0 = (double)g.y0 + cy * (double)g.cell, ry1 = ry0 + g.cell;
    const double dx = fmax(fmax(rx0 - Mx, Mx - rx1), 0.0);
    const double dy = fmax(fmax(ry0 - My, My - ry1), 0.0);
    // margin for the FP32 evaluation of the rectangle corners at query time
    const double margin = 1e-6 * (fabs((double)g.x0) + fabs((double)g.y0) +
                                  (double)g.cell * (g.nx + g.ny + 2)) + 1e-9;
    const float e = __double2float_ru(sqrt(dx * dx + dy * dy) + half + margin);
    atomicMax(ext_bits + key, __float_as_uint(e));
    atomicMax(tB_ord + key, f2ord(u.w));
    atomicMax(bmax_ord + bk, f2ord(u.w));
}

// off[k] = number of sorted keys below k.
__global__ void k_grid_offsets(const unsigned long long *__restrict__ keys, int S,
                               int nkeys, int32_t *__restrict__ off)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nkeys)
        return;
    const unsigned long long t = (unsigned long long)(unsigned)k << 32;
    int lo = 0, hi = S;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < t)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[k] = lo;
}

// t_A position of the segment of every sorted grid key (keys hold build ids).
__global__ void k_grid_ids(const unsigned long long *__restrict__ keys, int S,
                           const int32_t *__restrict__ pos, int32_t *__restrict__ ids)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S)
        ids[i] = pos[(int)(keys[i] & 0xffffffffu)];
}

// Segment records in grid-key order (record 3's trajectory field replaced by
// the t_A position), so that the search reads a key's segments without an
// indirection.
__global__ void k_grid_records(const float4 *__restrict__ seg, const int32_t *__restrict__ ids, int S,
                               float4 *__restrict__ gseg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S)
        return;
    const int p = ids[i];
    gseg[4 * (size_t)i] = seg[4 * (size_t)p];
    gseg[4 * (size_t)i + 1] = seg[4 * (size_t)p + 1];
    gseg[4 * (size_t)i + 2] = seg[4 * (size_t)p + 2];
    float4 r3 = seg[4 * (size_t)p + 3];
    r3.z = __int_as_float(p);
    gseg[4 * (size_t)i + 3] = r3;
}

__global__ void k_decode_ord(unsigned int *__restrict__ v, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const unsigned int u = v[i];
        v[i] = u ? __float_as_uint(ord2f(u)) : __float_as_uint(-INFINITY);
    }
}

// Per key, its CSR range, extent and largest t_B packed in one record.
__global__ void k_key_records(const int32_t *__restrict__ off, const float *__restrict__ ext,
                              const float *__restrict__ tB, int nkeys, int4 *__restrict__ kr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nkeys)
        kr[i] = make_int4(off[i], off[i + 1], __float_as_int(ext[i]), __float_as_int(tB[i]));
}

// Maximum of non-negative floats given as their bits (the bits order them).
__global__ void k_max_bits(const unsigned int *__restrict__ v, int n, unsigned int *out)
{
    unsigned int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, v[i]);
    for (int o = 16; o > 0; o >>= 1)
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m)
        atomicMax(out, m);
}

// Running maximum over buckets (one block).
__global__ void k_prefix_max(float *__restrict__ v, int n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float m = -INFINITY;
        for (int i = 0; i < n; ++i) {
            m = fmaxf(m, v[i]);
            v[i] = m;
        }
    }
}

// ---------------------------------------------------------------- host API

// The index may still be read by work queued on any stream: wait for the
// device (as cudaFree would), then return the arrays to the pool.
// Arrays back to the pool in the order of `st`, host parts freed.
static void release_index(tnn_index *ix, cudaStream_t st)
{
    void *arrays[] = {ix->pts,   ix->seg,   ix->segTA, ix->segPM, ix->pts_t,
                      ix->idx_t, ix->g_off, ix->g_ids, ix->g_seg, ix->g_ext,
                      ix->g_tB,  ix->g_krec, ix->g_bpm, ix->g_ext_max,
                      ix->pts_k, ix->idx_k, ix->kp_start, ix->pts_m,
                      ix->idx_m, ix->code_m};
    for (void *p : arrays)
        tnn_free(p, st);
    tnn_free(ix->d_rmax, st);
    tnn_free(ix->d_tiles, st);
    free(ix->h_tiles);
    if (ix->built)
        cudaEventDestroy(ix->built);
    delete ix;
}

static void free_index(tnn_index *ix)
{
    if (!ix)
        return;
    cudaDeviceSynchronize();
    release_index(ix, 0);
}

void tnn_index_release(tnn_index *ix, cudaStream_t st)
{
    if (ix)
        release_index(ix, st);
}

// The build's second stream per device (non-blocking, created on first
// use): the grid keys and their sort run there beside the t_A sort.
#define TNN_BUILD_MAX_DEVICES 64
static std::mutex g_side_mu;
static cudaStream_t g_side_stream[TNN_BUILD_MAX_DEVICES];

static cudaError_t side_stream(cudaStream_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= TNN_BUILD_MAX_DEVICES)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_side_mu);
    if (!g_side_stream[dev]) {
        e = cudaStreamCreateWithFlags(&g_side_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return e;
    }
    *out = g_side_stream[dev];
    return cudaSuccess;
}

// Build-time scratch, returned to the pool in stream order.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t st = 0;
    cudaError_t alloc(size_t bytes, cudaStream_t s)
    {
        st = s;
        return tnn_alloc(&p, bytes, s);
    }
    ~DevBuf() { tnn_free(p, st); }
};

static float host_ord2f(uint32_t u)
{
    uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

// Grid geometry from the points' bounding box in sqrt(sigma)-scaled x, y
// (it holds every segment midpoint up to rounding, and keys are clamped to
// the grid), their time range and the summed segment duration.  Buckets span
// about five mean segment durations (at most 4096 of them); cells are square,
// about one segment per (bucket, cell) on average, at most 65,536 cells and
// 2^22 keys.
#ifndef TNN_BUCKET_SEGS
#define TNN_BUCKET_SEGS 5.0 // bucket span in mean segment durations
#endif
#ifndef TNN_KEY_SEGS
#define TNN_KEY_SEGS 1.0 // mean segments per (bucket, cell)
#endif
static GridBuild grid_geometry(double xmn, double xmx, double ymn, double ymx, double tmn,
                               double tmx, double dur, int64_t S)
{
    const double T = tmx - tmn;
    double dt = TNN_BUCKET_SEGS * dur / S;
    if (!(dt > 0.0))
        dt = T > 0.0 ? T / 64.0 : 1.0;
    if (T / dt > 4095.0)
        dt = T / 4095.0;
    const int nb = (int)std::min(4096.0, floor(T / dt) + 1.0);
    const double Wd = xmx - xmn, Hd = ymx - ymn;
    const double target = std::min(65536.0, std::max(1.0, TNN_KEY_SEGS * S / nb));
    double cell = sqrt(std::max(Wd * Hd, 1e-12) / target);
    cell = std::max(cell, std::max(std::max(Wd, Hd) / 1024.0, 1e-6));
    int nx = 1, ny = 1;
    for (;;) {
        nx = (int)floor(Wd / cell) + 1;
        ny = (int)floor(Hd / cell) + 1;
        if ((double)nx * ny <= 65536.0 && (double)nb * nx * ny <= (double)(1 << 22))
            break;
        cell *= 1.25;
    }
    GridBuild g;
    g.x0 = (float)xmn;
    g.y0 = (float)ymn;
    g.cell = (float)cell;
    g.inv_cell = (float)(1.0 / cell);
    g.t0 = (float)tmn;
    g.dt = (float)dt;
    g.inv_dt = (float)(1.0 / dt);
    g.nx = nx;
    g.ny = ny;
    g.ncell = nx * ny;
    g.nb = nb;
    return g;
}

// The grid's arrays, zeroed where the key kernel takes maxima.
static tnn_status grid_alloc(tnn_index *ix, const GridBuild &g, cudaStream_t st)
{
    const int S = (int)ix->S, nb = g.nb, nkeys = nb * g.ncell;
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_off, sizeof(int32_t) * (nkeys + 1), st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_ids, sizeof(int32_t) * S, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_seg, sizeof(float4) * 4 * (size_t)S, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_ext, sizeof(float) * nkeys, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_tB, sizeof(float) * nkeys, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_bpm, sizeof(float) * nb, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_krec, sizeof(int4) * (size_t)nkeys, st));
    TNN_CUDA_TRY(tnn_alloc((void **)&ix->g_ext_max, sizeof(float), st));
    TNN_CUDA_TRY(cudaMemsetAsync(ix->g_ext_max, 0, sizeof(float), st));
    TNN_CUDA_TRY(cudaMemsetAsync(ix->g_ext, 0, sizeof(float) * nkeys, st));
    TNN_CUDA_TRY(cudaMemsetAsync(ix->g_tB, 0, sizeof(float) * nkeys, st));
    TNN_CUDA_TRY(cudaMemsetAsync(ix->g_bpm, 0, sizeof(float) * nb, st));
    return TNN_OK;
}

// The grid from its sorted keys (build ids; pos = t_A position of each).
static tnn_status build_grid(tnn_index *ix, const unsigned long long *keys, const int32_t *pos,
                             const GridBuild &g, cudaStream_t st)
{
    const int S = (int)ix->S, tb = 256;
    const int nx = g.nx, ny = g.ny, nb = g.nb;
    const int nkeys = nb * g.ncell;
    k_grid_offsets<<<(nkeys + 1 + tb - 1) / tb, tb, 0, st>>>(keys, S, nkeys, ix->g_off);
    k_grid_ids<<<(S + tb - 1) / tb, tb, 0, st>>>(keys, S, pos, ix->g_ids);
    k_grid_records<<<(S + tb - 1) / tb, tb, 0, st>>>(ix->seg, ix->g_ids, S, ix->g_seg);
    k_decode_ord<<<(nkeys + tb - 1) / tb, tb, 0, st>>>((unsigned int *)ix->g_tB, nkeys);
    k_decode_ord<<<(nb + tb - 1) / tb, tb, 0, st>>>((unsigned int *)ix->g_bpm, nb);
    k_prefix_max<<<1, 32, 0, st>>>(ix->g_bpm, nb);
    k_key_records<<<(nkeys + tb - 1) / tb, tb, 0, st>>>(ix->g_off, ix->g_ext, ix->g_tB, nkeys,
                                                       ix->g_krec);
    // largest extent (for the search region)
    k_max_bits<<<std::min((nkeys + tb - 1) / tb, 1024), tb, 0, st>>>(
        (const unsigned int *)ix->g_ext, nkeys, (unsigned int *)ix->g_ext_max);
    TNN_CUDA_TRY(cudaGetLastError());
    GridDesc &G = ix->grid;
    G.x0 = g.x0;
    G.y0 = g.y0;
    G.cell = g.cell;
    G.inv_cell = g.inv_cell;
    G.t0 = g.t0;
    G.dt = g.dt;
    G.inv_dt = g.inv_dt;
    G.ext_max = ix->g_ext_max;
    G.nx = nx;
    G.ny = ny;
    G.ncell = g.ncell;
    G.nb = nb;
    G.off = ix->g_off;
    G.ids = ix->g_ids;
    G.gseg = ix->g_seg;
    G.ext = ix->g_ext;
    G.tB = ix->g_tB;
    G.bpm = ix->g_bpm;
    G.krec = ix->g_krec;
    return TNN_OK;
}

extern "C" tnn_status tnn_build_segments(const float *d_xyzt, int64_t n,
                                         const int64_t *h_traj_off,
                                         int64_t n_traj,
                                         const tnn_build_params *params,
                                         tnn_stream_t stream, tnn_index **out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    TNN_ARG_CHECK(params != nullptr, "params is NULL");
    TNN_ARG_CHECK(n >= 1 && n < (1ll << 31) - 64, "n must be in [1, 2^31-64), got %lld",
                  (long long)n);
    TNN_ARG_CHECK(d_xyzt != nullptr && h_traj_off != nullptr, "NULL input");
    TNN_ARG_CHECK(((uintptr_t)d_xyzt & 15) == 0, "d_xyzt must be 16-byte aligned");
    TNN_ARG_CHECK(n_traj >= 1 && n_traj <= n, "n_traj must be in [1, n]");
    const int K = params->seg_len;
    TNN_ARG_CHECK(K >= 2 && K <= 64, "seg_len must be in [2, 64], got %d", K);
    for (int i = 0; i < 4; ++i) {
        double s = params->sigma[i];
        TNN_ARG_CHECK(isfinite(s) && s >= 0.0 && s <= 1e6,
                      "sigma[%d] must be finite in [0, 1e6]", i);
    }
    TNN_ARG_CHECK(h_traj_off[0] == 0 && h_traj_off[n_traj] == n,
                  "traj_off must start at 0 and end at n");
    std::vector<int32_t> toff(n_traj + 1), soff(n_traj + 1);
    int64_t S = 0;
    for (int64_t t = 0; t < n_traj; ++t) {
        int64_t len = h_traj_off[t + 1] - h_traj_off[t];
        TNN_ARG_CHECK(len >= 0, "traj_off must be non-decreasing");
        toff[t] = (int32_t)h_traj_off[t];
        soff[t] = (int32_t)S;
        S += (len + K - 1) / K;
    }
    toff[n_traj] = (int32_t)n;
    soff[n_traj] = (int32_t)S;
    cudaStream_t st = (cudaStream_t)stream;

    tnn_index *ix = new tnn_index();
    memset(ix, 0, sizeof(*ix));
    cudaGetDevice(&ix->device);
    ix->n = n;
    ix->n_traj = n_traj;
    ix->S = S;
    ix->K = K;
    for (int i = 0; i < 4; ++i) {
        ix->sigma[i] = params->sigma[i];
        ix->sig_f[i] = (float)params->sigma[i];
    }
    for (int i = 0; i < 3; ++i)
        ix->ssq_f[i] = (float)sqrt(params->sigma[i]);

    const int s2 = tnn_next_pow2_sort(S);
    DevBuf toff_d, soff_d, rec_d, keys_d, flags_d;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                                     \
    if (e == cudaSuccess)                                                     \
        e = tnn_alloc((void **)&(ptr), (bytes), st);
    ALLOC(ix->pts, sizeof(float4) * n);
    ALLOC(ix->seg, sizeof(float4) * 4 * S);
    ALLOC(ix->segTA, sizeof(float) * S);
    ALLOC(ix->segPM, sizeof(float) * S);
#undef ALLOC
    if (e == cudaSuccess)
        e = toff_d.alloc(sizeof(int32_t) * (n_traj + 1), st);
    if (e == cudaSuccess)
        e = soff_d.alloc(sizeof(int32_t) * (n_traj + 1), st);
    if (e == cudaSuccess)
        e = rec_d.alloc(sizeof(float4) * 4 * S, st);
    if (e == cudaSuccess)
        e = keys_d.alloc(sizeof(unsigned long long) * s2, st);
    if (e == cudaSuccess)
        e = flags_d.alloc(sizeof(unsigned int) * 12, st);
    if (e != cudaSuccess) {
        free_index(ix);
        tnn_set_error("index allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    // flags_d: [0] validation flags, [1] largest |scaled coordinate| bits,
    // [2..9] point bounding box (ordered min, max per axis), [10..11] summed
    // segment duration (double)
    static const unsigned int meta_init[12] = {0u, 0u, 0xffffffffu, 0u, 0xffffffffu, 0u,
                                               0xffffffffu, 0u, 0xffffffffu, 0u, 0u, 0u};
    unsigned int *flag = (unsigned int *)flags_d.p;
    unsigned long long *keys = (unsigned long long *)keys_d.p;
    const int tb = 256;
    e = cudaMemcpyAsync(ix->pts, d_xyzt, sizeof(float4) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(toff_d.p, toff.data(), sizeof(int32_t) * (n_traj + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(soff_d.p, soff.data(), sizeof(int32_t) * (n_traj + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flag, meta_init, sizeof(meta_init), cudaMemcpyHostToDevice, st);
    // query tiles of the self-queries: runs of up to 32 points of one trajectory
    {
        int64_t nt = 0;
        for (int64_t t = 0; t < n_traj; ++t)
            nt += (h_traj_off[t + 1] - h_traj_off[t] + 31) / 32;
        ix->n_tiles = nt;
        ix->h_tiles = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt + 1));
        if (!ix->h_tiles) {
            free_index(ix);
            tnn_set_error("index allocation failed (host tile table)");
            return TNN_ERR_OOM;
        }
        int64_t j = 0;
        for (int64_t t = 0; t < n_traj; ++t)
            for (int64_t r = h_traj_off[t]; r < h_traj_off[t + 1]; r += 32)
                ix->h_tiles[j++] = (int32_t)r;
        ix->h_tiles[nt] = (int32_t)n;
    }
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&ix->d_tiles, sizeof(int32_t) * (size_t)(ix->n_tiles + 1), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ix->d_tiles, ix->h_tiles, sizeof(int32_t) * (size_t)(ix->n_tiles + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&ix->d_rmax, sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ix->d_rmax, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ix->built, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_index(ix);
        tnn_set_error("index upload failed: %s", cudaGetErrorString(e));
        return TNN_ERR_CUDA;
    }
    const int ni = (int)n, Si = (int)S, Ti = (int)n_traj;
    // ---- validation, and what the grid geometry needs: the build's only
    // host synchronisation; everything after it is enqueued at once
    k_validate_points<<<(ni + tb - 1) / tb, tb, 0, st>>>(
        ix->pts, ni, ix->ssq_f[0], ix->ssq_f[1], ix->ssq_f[2], flag, flag + 1);
    k_validate_traj<<<(int)(((int64_t)Ti * 32 + tb - 1) / tb), tb, 0, st>>>(
        ix->pts, (const int32_t *)toff_d.p, Ti, K, flag, (double *)(flag + 10));
    k_point_bbox<<<(int)std::min<int64_t>((ix->n + tb - 1) / tb, 608), tb, 0, st>>>(
        ix->pts, (int)ix->n, flag + 2);
    // The values come back through a page-locked buffer of this host thread
    // and an event: the segment fit (which needs neither the geometry nor
    // the validation result) is enqueued before the host waits, so it runs while the
    // host chooses the geometry and enqueues the rest.  Invalid input is
    // still reported here; the fit's output is then dropped.
    static thread_local unsigned int *t_meta = nullptr;
    unsigned int hm[12];
    cudaEvent_t ev_meta = nullptr;
    e = cudaGetLastError();
    if (e == cudaSuccess && !t_meta)
        e = cudaHostAlloc((void **)&t_meta, sizeof(hm), cudaHostAllocPortable);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ev_meta, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t_meta, flag, sizeof(hm), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev_meta, st);
    const double q0 = sqrt(params->sigma[0]), q1 = sqrt(params->sigma[1]);
    if (e == cudaSuccess) {
        k_segment_fit<<<(int)(((int64_t)Si * SF_LANES + tb - 1) / tb), tb, 0, st>>>(
            ix->pts, (const int32_t *)toff_d.p, (const int32_t *)soff_d.p, Ti, Si, K,
            q0, q1, sqrt(params->sigma[2]), (float4 *)rec_d.p, keys, ix->d_rmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaEventSynchronize(ev_meta);
    if (ev_meta)
        cudaEventDestroy(ev_meta);
    if (e != cudaSuccess) {
        free_index(ix);
        tnn_set_error("index validation failed: %s", cudaGetErrorString(e));
        return TNN_ERR_CUDA;
    }
    memcpy(hm, t_meta, sizeof(hm));
    if (hm[0] & BAD_VALUE) {
        free_index(ix);
        tnn_set_error("non-finite or too large (|v| > 1e15) coordinate in input");
        return TNN_ERR_INVALID_ARG;
    }
    if (hm[0] & BAD_ORDER) {
        free_index(ix);
        tnn_set_error("times are not sorted inside a trajectory");
        return TNN_ERR_INVALID_ARG;
    }
    memcpy(&ix->coord_max, &hm[1], sizeof(float));
    for (int d = 0; d < 4; ++d) {
        ix->bb_lo[d] = host_ord2f(hm[2 + 2 * d]);
        ix->bb_hi[d] = host_ord2f(hm[3 + 2 * d]);
    }
    double dur = 0.0;
    memcpy(&dur, &hm[10], sizeof(double));
    const GridBuild geo = grid_geometry(q0 * ix->bb_lo[0], q0 * ix->bb_hi[0], q1 * ix->bb_lo[1],
                                        q1 * ix->bb_hi[1], ix->bb_lo[3], ix->bb_hi[3], dur, S);

    // ---- segments, their t_A order, the running maximum of t_B, the grid.
    // The grid keys come from the build-order records, so their sort runs on
    // a second stream beside the t_A sort; the two join before the grid's
    // offsets and records.
    {
        DevBuf keys2_d, pos_d, bmax_d;
        cudaStream_t st2 = nullptr;
        cudaEvent_t ev_fit = nullptr, ev_keys = nullptr;
        const int nblk = (Si + 1023) / 1024;
        e = side_stream(&st2);
        if (e == cudaSuccess)
            e = keys2_d.alloc(sizeof(unsigned long long) * s2, st);
        if (e == cudaSuccess)
            e = pos_d.alloc(sizeof(int32_t) * (size_t)Si, st);
        if (e == cudaSuccess)
            e = bmax_d.alloc(sizeof(float) * (size_t)nblk, st);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ev_fit, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ev_keys, cudaEventDisableTiming);
        tnn_status gs = e == cudaSuccess ? grid_alloc(ix, geo, st) : TNN_ERR_CUDA;
        if (gs == TNN_OK) {
            unsigned long long *keys2 = (unsigned long long *)keys2_d.p;
            e = cudaEventRecord(ev_fit, st); // the fit (enqueued above) and the grid's zeroing
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(st2, ev_fit, 0);
            if (e == cudaSuccess) {
                // second stream: grid keys of the build-order records, sorted
                k_fill<<<(s2 - Si + tb - 1) / tb + 1, tb, 0, st2>>>(keys2, Si, s2);
                k_grid_keys<<<(Si + tb - 1) / tb, tb, 0, st2>>>(
                    (const float4 *)rec_d.p, Si, geo, keys2, (unsigned int *)ix->g_ext,
                    (unsigned int *)ix->g_tB, (unsigned int *)ix->g_bpm);
                tnn_bitonic_sort(keys2, s2, st2);
                e = cudaEventRecord(ev_keys, st2);
            }
            // this stream: the t_A order and the running maximum of t_B
            k_fill<<<(s2 - Si + tb - 1) / tb + 1, tb, 0, st>>>(keys, Si, s2);
            tnn_bitonic_sort(keys, s2, st);
            k_gather_segments<<<(Si + tb - 1) / tb, tb, 0, st>>>(keys, (const float4 *)rec_d.p, Si,
                                                                 ix->seg, ix->segTA, (int32_t *)pos_d.p);
            k_pm_block_max<<<nblk, 1024, 0, st>>>(ix->seg, Si, (float *)bmax_d.p);
            k_pm_apply<<<nblk, 1024, 0, st>>>(ix->seg, Si, (const float *)bmax_d.p, ix->segPM);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(st, ev_keys, 0);
            if (e == cudaSuccess)
                gs = build_grid(ix, keys2, (const int32_t *)pos_d.p, geo, st);
            else
                gs = TNN_ERR_CUDA;
        }
        if (ev_fit)
            cudaEventDestroy(ev_fit);
        if (ev_keys)
            cudaEventDestroy(ev_keys);
        if (gs != TNN_OK) {
            if (e != cudaSuccess)
                tnn_set_error("index build failed: %s", cudaGetErrorString(e));
            cudaStreamSynchronize(st2);
            free_index(ix);
            return gs;
        }
    }
    // The build runs on after this call returns (stream order); a failure
    // there surfaces at the next synchronising call.
    e = cudaEventRecord(ix->built, st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess) {
        free_index(ix);
        tnn_set_error("index build failed: %s", cudaGetErrorString(e));
        return TNN_ERR_CUDA;
    }
    *out = ix;
    return TNN_OK;
}

extern "C" void tnn_index_destroy(tnn_index *index) { free_index(index); }

static std::mutex g_time_order_mu;

tnn_status tnn_index_time_order(const tnn_index *cix, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_time_order_mu);
    tnn_index *ix = const_cast<tnn_index *>(cix);
    if (ix->pts_t)
        return TNN_OK;
    const int n = (int)ix->n, n2 = tnn_next_pow2_sort(n), tb = 256;
    float4 *pts_t = nullptr;
    int32_t *idx_t = nullptr;
    DevBuf keys_d;
    cudaError_t e = tnn_alloc((void **)&pts_t, sizeof(float4) * n, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&idx_t, sizeof(int32_t) * (n + 4), st); // padding for 16-byte copies
    if (e == cudaSuccess)
        e = keys_d.alloc(sizeof(unsigned long long) * n2, st);
    if (e != cudaSuccess) {
        tnn_free(pts_t, st);
        tnn_free(idx_t, st);
        tnn_set_error("time-order allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    unsigned long long *keys = (unsigned long long *)keys_d.p;
    k_time_keys<<<(n2 + tb - 1) / tb, tb, 0, st>>>(ix->pts, n, keys, n2);
    tnn_bitonic_sort(keys, n2, st);
    k_gather_points<<<(n + tb - 1) / tb, tb, 0, st>>>(keys, ix->pts, n, pts_t, idx_t);
    e = cudaMemsetAsync(idx_t + n, 0, 4 * sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess) {
        tnn_free(pts_t, st);
        tnn_free(idx_t, st);
        tnn_set_error("time order failed: %s", cudaGetErrorString(e));
        return TNN_ERR_CUDA;
    }
    ix->pts_t = pts_t;
    ix->idx_t = idx_t;
    return TNN_OK;
}

// ------------------------------------------------------------ space order

__global__ void k_space_keys(const float4 *__restrict__ p, int n, float4 lo, float4 sc,
                             unsigned long long *__restrict__ keys, int n2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        keys[i] = ((unsigned long long)tnn_morton_xyt(p[i], lo, sc) << 32) | (unsigned)i;
    else if (i < n2)
        keys[i] = ~0ull;
}

__global__ void k_gather_space(const unsigned long long *__restrict__ keys, const float4 *__restrict__ p,
                               int n, float4 *__restrict__ pm, int32_t *__restrict__ im,
                               uint32_t *__restrict__ cm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const unsigned long long k = keys[i];
        const int j = (int)(k & 0xffffffffull);
        pm[i] = p[j];
        im[i] = j;
        cm[i] = (uint32_t)(k >> 32);
    }
}

static std::mutex g_space_order_mu;

tnn_status tnn_index_space_order(const tnn_index *cix, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_space_order_mu);
    tnn_index *ix = const_cast<tnn_index *>(cix);
    if (ix->pts_m)
        return TNN_OK;
    const int n = (int)ix->n, n2 = tnn_next_pow2_sort(n), tb = 256;
    float4 *pm = nullptr;
    int32_t *im = nullptr;
    uint32_t *cm = nullptr;
    DevBuf keys_d;
    cudaError_t e = tnn_alloc((void **)&pm, sizeof(float4) * n, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&im, sizeof(int32_t) * n, st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&cm, sizeof(uint32_t) * n, st);
    if (e == cudaSuccess)
        e = keys_d.alloc(sizeof(unsigned long long) * n2, st);
    if (e != cudaSuccess) {
        tnn_free(pm, st);
        tnn_free(im, st);
        tnn_free(cm, st);
        tnn_set_error("space-order allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    float4 l4, s4;
    tnn_morton_frame(ix->bb_lo, ix->bb_hi, &l4, &s4);
    unsigned long long *keys = (unsigned long long *)keys_d.p;
    k_space_keys<<<(n2 + tb - 1) / tb, tb, 0, st>>>(ix->pts, n, l4, s4, keys, n2);
    tnn_bitonic_sort(keys, n2, st);
    k_gather_space<<<(n + tb - 1) / tb, tb, 0, st>>>(keys, ix->pts, n, pm, im, cm);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        tnn_free(pm, st);
        tnn_free(im, st);
        tnn_free(cm, st);
        tnn_set_error("space order failed: %s", cudaGetErrorString(e));
        return TNN_ERR_CUDA;
    }
    ix->pts_m = pm;
    ix->idx_m = im;
    ix->code_m = cm;
    return TNN_OK;
}

// ------------------------------------------------------------- key order

// Padded run length of every key: its segments' member count rounded up to
// a multiple of 4 (so every run starts on a 16-byte boundary of idx_k).
__global__ void k_key_runs(const int32_t *__restrict__ off, const float4 *__restrict__ gseg, int nkeys,
                           int64_t *__restrict__ len)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys)
        return;
    int64_t c = 0;
    for (int i = off[k]; i < off[k + 1]; ++i)
        c += __float_as_int(gseg[4 * (size_t)i + 3].y);
    len[k] = (c + 3) & ~3ll;
}

// Exclusive prefix sum of n int64 values by one block, in place, with the
// total appended at v[n] (n + 1 entries).
__global__ void __launch_bounds__(1024) k_scan_i64(int64_t *__restrict__ v, int n)
{
    __shared__ int64_t part[1024];
    const int per = (n + 1023) / 1024;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i)
        s += v[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t a = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += a;
        __syncthreads();
    }
    int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        const int64_t x = v[i];
        v[i] = run;
        run += x;
    }
    if (threadIdx.x == 1023)
        v[n] = part[1023];
}

// Every key's members into its run, then the padding.
__global__ void k_key_gather(const int32_t *__restrict__ off, const float4 *__restrict__ gseg,
                             const int64_t *__restrict__ start, int nkeys, const float4 *__restrict__ pts,
                             float4 *__restrict__ pk, int32_t *__restrict__ ik, int32_t *__restrict__ ks)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nkeys)
        return;
    ks[k] = (int32_t)start[k];
    if (k == nkeys)
        return;
    int64_t o = start[k];
    float4 first = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = off[k]; i < off[k + 1]; ++i) {
        const float4 r = gseg[4 * (size_t)i + 3];
        const int f = __float_as_int(r.x), c = __float_as_int(r.y);
        if (i == off[k])
            first = pts[f];
        for (int j = 0; j < c; ++j, ++o) {
            pk[o] = pts[f + j];
            ik[o] = f + j;
        }
    }
    for (; o < start[k + 1]; ++o) {
        pk[o] = first;
        ik[o] = -1;
    }
}

static std::mutex g_key_order_mu;

tnn_status tnn_index_key_order(const tnn_index *cix, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_key_order_mu);
    tnn_index *ix = const_cast<tnn_index *>(cix);
    if (ix->pts_k)
        return TNN_OK;
    const int nkeys = ix->grid.nb * ix->grid.ncell, tb = 256;
    DevBuf len_d;
    TNN_CUDA_TRY(len_d.alloc(sizeof(int64_t) * (nkeys + 1), st));
    int64_t *len = (int64_t *)len_d.p;
    k_key_runs<<<(nkeys + tb - 1) / tb, tb, 0, st>>>(ix->g_off, ix->g_seg, nkeys, len);
    k_scan_i64<<<1, 1024, 0, st>>>(len, nkeys);
    int64_t nk = 0;
    TNN_CUDA_TRY(cudaMemcpyAsync(&nk, len + nkeys, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    TNN_CUDA_TRY(cudaStreamSynchronize(st));
    if (nk >= (1ll << 31) - 256) {
        tnn_set_error("the key-ordered copy (%lld points with padding) exceeds 2^31", (long long)nk);
        return TNN_ERR_UNSUPPORTED;
    }
    float4 *pk = nullptr;
    int32_t *ik = nullptr, *ks = nullptr;
    cudaError_t e = tnn_alloc((void **)&pk, sizeof(float4) * (size_t)std::max<int64_t>(nk, 1), st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&ik, sizeof(int32_t) * (size_t)(nk + 4), st);
    if (e == cudaSuccess)
        e = tnn_alloc((void **)&ks, sizeof(int32_t) * (size_t)(nkeys + 1), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ik + nk, 0xff, 4 * sizeof(int32_t), st);
    if (e == cudaSuccess) {
        k_key_gather<<<(nkeys + 1 + tb - 1) / tb, tb, 0, st>>>(ix->g_off, ix->g_seg, len, nkeys, ix->pts, pk,
                                                             ik, ks);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        tnn_free(pk, st);
        tnn_free(ik, st);
        tnn_free(ks, st);
        tnn_set_error("key order failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    ix->pts_k = pk;
    ix->idx_k = ik;
    ix->kp_start = ks;
    ix->nk = nk;
    return TNN_OK;
}

extern "C" tnn_status tnn_index_get_info(const tnn_index *ix, tnn_index_info *out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && out, "NULL argument");
    out->n_points = ix->n;
    out->n_traj = ix->n_traj;
    out->n_segments = ix->S;
    out->seg_len = ix->K;
    out->coord_max = ix->coord_max;
    if (!ix->rmax_known) {
        // the segment fit's largest radius: wait for the build to finish
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        tnn_index *w = const_cast<tnn_index *>(ix);
        unsigned int bits = 0u;
        cudaError_t e = ix->built ? cudaEventSynchronize(ix->built) : cudaSuccess;
        if (e == cudaSuccess)
            e = cudaMemcpy(&bits, ix->d_rmax, sizeof(bits), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            tnn_set_error("reading the index radius failed: %s", cudaGetErrorString(e));
            return TNN_ERR_CUDA;
        }
        memcpy(&w->max_radius, &bits, sizeof(float));
        w->rmax_known = true;
    }
    out->max_radius = ix->max_radius;
    return TNN_OK;
}

extern "C" tnn_status tnn_index_export(const tnn_index *ix, float *d_seg,
                                       float *d_pm, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && d_seg, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    TNN_CUDA_TRY(cudaMemcpyAsync(d_seg, ix->seg, sizeof(float4) * 4 * ix->S,
                                 cudaMemcpyDeviceToDevice, st));
    if (d_pm)
        TNN_CUDA_TRY(cudaMemcpyAsync(d_pm, ix->segPM, sizeof(float) * ix->S,
                                     cudaMemcpyDeviceToDevice, st));
    return TNN_OK;
}
