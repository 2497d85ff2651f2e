// Queries whose ranking the search could not settle (the chain of FP32 keys
// that FP32 cannot order reaches the last candidate slot kept) are answered
// again here, one warp per query:
//
//   k_fallback_scan   every causally valid point (time-ordered copy, newest
//                     first, lanes interleaved) in FP32 with a candidate list
//                     of k + 32 per lane; a lane stops once the temporal part
//                     alone exceeds its list's largest key; the 32 lists are
//                     merged and settled exactly like the search.  A query
//                     whose near-tie chain still reaches the end of the
//                     merged list moves on to
//   k_fallback_exact  the definition itself: the FP64 distance of every
//                     valid point, ranked by (d2, index).
#pragma once
#include "tnn_device.cuh"

#define FB_EXTRA 32

__host__ __device__ inline size_t fb_scan_smem_per_warp(int k_max)
{
    const size_t C = (size_t)k_max + FB_EXTRA;
    return C * 32 * 8 + C * 8 + (size_t)CMAX * 32 * 12;
}

__host__ __device__ inline size_t fb_exact_smem_per_warp(int k_max)
{
    return (size_t)k_max * 32 * 12;
}

// Warp minimum of 64-bit keys.
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(FULLMASK, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_fallback_scan(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int kmax = L.L_max;
    const int Cmax = kmax + FB_EXTRA;
    unsigned char *ws = smem + (threadIdx.x >> 5) * fb_scan_smem_per_warp(kmax);
    unsigned long long *K = (unsigned long long *)ws + lane;          // [Cmax][32]
    unsigned long long *merged = (unsigned long long *)ws + (size_t)Cmax * 32; // [Cmax]
    unsigned char *cl = ws + (size_t)Cmax * 32 * 8 + (size_t)Cmax * 8;
    unsigned long long *cl_d = (unsigned long long *)cl; // lane 0's columns
    int *cl_i = (int *)(cl + CMAX * 32 * 8);

    unsigned nfb = *(volatile unsigned *)&L.scr->n_fallback;
    if ((long long)nfb > L.fb_cap)
        nfb = (unsigned)L.fb_cap;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    LaneStats st = {0, 0, 0, 0, 0};
    for (unsigned e = gw; e < nfb; e += nw) {
        const int2 ent = L.fb_list[e];
        const KnnWin *W = L.nwin <= 1 ? &L.w0 : L.wins + ent.x;
        const float4 q = W->q[ent.y];
        const QCtx c = make_qctx(W, q, true);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float4 *__restrict__ pts_t = W->pts_t;
        const int32_t *__restrict__ idx_t = W->idx_t;
        const int C = W->k + FB_EXTRA;
        for (int i = 0; i < C; ++i)
            K[i * 32] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY;
        const int hi = warp_count_less([&](int p) { return __ldg(&pts_t[p].w); }, W->n, c.T32, lane);
        for (int base = hi - 1; base >= 0; base -= 32) {
            const float tb = __ldg(&pts_t[base].w); // newest remaining time
            if (__all_sync(FULLMASK, !(time_lb(c, s3, tb) <= tau)))
                break;
            const int j = base - lane;
            if (j >= 0) {
                const float4 p = __ldg(pts_t + j);
                const float d = dist32(c, s0, s1, s2, s3, p);
                st.pairs++;
                if (p.w < c.T32 && d <= tau) {
                    const unsigned long long key = pack_key(d, __ldg(idx_t + j));
                    if (key < tauk) {
                        tauk = lane_push(K, C, nv, key);
                        tau = key_d(tauk);
                    }
                }
            }
        }
        // merge the 32 sorted lists into the C smallest keys
        int h = 0;
        for (int r = 0; r < C; ++r) {
            const unsigned long long v = h < nv ? K[h * 32] : SENT;
            const unsigned long long mn = warp_min_u64(v);
            if (lane == 0)
                merged[r] = mn;
            if (v == mn && mn != SENT)
                ++h;
        }
        __syncwarp();
        if (lane == 0) {
            st.q++;
            if (!finalize_query(W, q, merged, C, cl_d, cl_i, ent.y, st, 1)) {
                const unsigned slot = atomicAdd(&L.scr->n_fallback3, 1u);
                if (slot < (unsigned long long)L.fb_cap)
                    L.fb_list3[slot] = ent;
                else
                    atomicOr(&L.scr->status, 2u);
            }
        }
        __syncwarp();
    }
    unsigned long long x = st.pairs, f = st.fp64;
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(FULLMASK, x, o);
        f += __shfl_xor_sync(FULLMASK, f, o);
    }
    if (lane == 0 && x)
        atomicAdd(&L.scr->stats[2], x);
    if (lane == 0 && f)
        atomicAdd(&L.scr->stats[4], f);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        L.scr->stats[5] = nfb;
}

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_fallback_exact(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int kmax = L.L_max;
    unsigned char *ws = smem + (threadIdx.x >> 5) * fb_exact_smem_per_warp(kmax);
    unsigned long long *kd = (unsigned long long *)ws + lane;   // [kmax][32]
    int *ki = (int *)(ws + (size_t)kmax * 32 * 8) + lane;       // [kmax][32]
    unsigned nfb = *(volatile unsigned *)&L.scr->n_fallback3;
    if ((long long)nfb > L.fb_cap)
        nfb = (unsigned)L.fb_cap;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long INF64 = 0x7ff0000000000000ull;
    unsigned long long nfp = 0;
    for (unsigned e = gw; e < nfb; e += nw) {
        const int2 ent = L.fb_list3[e];
        const KnnWin *W = L.nwin <= 1 ? &L.w0 : L.wins + ent.x;
        const float4 q = W->q[ent.y];
        const float T32 = __double2float_ru((double)q.w - W->lag);
        const int k = W->k;
        for (int r = 0; r < k; ++r) {
            kd[r * 32] = INF64;
            ki[r * 32] = 0x7fffffff;
        }
        int cnt = 0;
        for (int j = lane; j < W->n; j += 32) {
            const float4 p = W->pts[j];
            if (!(p.w < T32))
                continue;
            const unsigned long long db =
                (unsigned long long)__double_as_longlong(dist64(W->sigd, q, p));
            nfp++;
            const unsigned long long wd = kd[(k - 1) * 32];
            if (!(db < wd || (db == wd && j < ki[(k - 1) * 32])))
                continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0) {
                const unsigned long long pd = kd[(pos - 1) * 32];
                const int pi = ki[(pos - 1) * 32];
                if (pd < db || (pd == db && pi < j))
                    break;
                kd[pos * 32] = pd;
                ki[pos * 32] = pi;
                --pos;
            }
            kd[pos * 32] = db;
            ki[pos * 32] = j;
            if (cnt < k)
                ++cnt;
        }
        // merge by (d2, index)
        int h = 0;
        int32_t *oi = W->out_idx + (int64_t)ent.y * k;
        float *od = W->out_d2 + (int64_t)ent.y * k;
        for (int r = 0; r < k; ++r) {
            unsigned long long vd = h < cnt ? kd[h * 32] : INF64;
            int vi = h < cnt ? ki[h * 32] : 0x7fffffff;
            unsigned long long md = vd;
            int mi = vi;
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long od_ = __shfl_xor_sync(FULLMASK, md, o);
                const int oi_ = __shfl_xor_sync(FULLMASK, mi, o);
                if (od_ < md || (od_ == md && oi_ < mi)) {
                    md = od_;
                    mi = oi_;
                }
            }
            if (vd == md && vi == mi && h < cnt)
                ++h;
            if (lane == 0) {
                const bool ok = md != INF64;
                oi[r] = ok ? mi : -1;
                od[r] = ok ? (float)__longlong_as_double((long long)md) : INFINITY;
            }
        }
        __syncwarp();
    }
    unsigned long long x = nfp;
    for (int o = 16; o > 0; o >>= 1)
        x += __shfl_xor_sync(FULLMASK, x, o);
    if (lane == 0 && x)
        atomicAdd(&L.scr->stats[4], x);
}
