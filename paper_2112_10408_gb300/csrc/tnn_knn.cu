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
//   re-answered by the exact FP64 linear scan (k_fallback).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tnn_internal.cuh"

#define FULLMASK 0xffffffffu
#define CMAX 8

static const unsigned long long SENT = (0x7f800000ull << 32) | 0xffffffffull;

__host__ __device__ inline size_t smem_per_warp(int L_max, int kseg_max, bool brute)
{
    size_t base = (size_t)L_max * 32 * 8;
    size_t rest = brute ? (32 * 16 + 32 * 4) : (2048 + (size_t)kseg_max * 16 + 32);
    size_t cl = (size_t)CMAX * 32 * 12;
    if (rest < cl)
        rest = cl;
    return (base + rest + 15) & ~(size_t)15;
}

size_t tnn_search_smem_per_warp(int L_max, int kseg_max, bool brute)
{
    return smem_per_warp(L_max, kseg_max, brute);
}

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned long long pack_key(float d, int idx)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)idx;
}
__device__ __forceinline__ float key_d(unsigned long long k)
{
    return __uint_as_float((unsigned)(k >> 32));
}
__device__ __forceinline__ int key_i(unsigned long long k)
{
    return (int)(unsigned)(k & 0xffffffffull);
}

struct QCtx {
    float qx, qy, qz, qt; // raw query
    float sx, sy, sz;     // sqrt(sigma)-scaled spatial query
    float T32;            // valid iff t_j < T32  (== t_j < t_q - lag exactly)
    float delta;          // absolute slack of the spatial bound
};

__device__ __forceinline__ QCtx make_qctx(const KnnWin *W, float4 q, bool active)
{
    QCtx c;
    c.qx = q.x;
    c.qy = q.y;
    c.qz = q.z;
    c.qt = q.w;
    c.sx = W->ssq[0] * q.x;
    c.sy = W->ssq[1] * q.y;
    c.sz = W->ssq[2] * q.z;
    // For float t_j, t_j < t_q - lag (evaluated in FP64) iff t_j < RU(t_q - lag).
    c.T32 = active ? __double2float_ru((double)q.w - W->lag) : -INFINITY;
    float qmax = fmaxf(fabsf(c.sx), fmaxf(fabsf(c.sy), fabsf(c.sz)));
    c.delta = (qmax + W->coord_max) * 0x1p-18f;
    return c;
}

// Scalable metric of Sec. 3.4 in FP32 on raw differences.
__device__ __forceinline__ float dist32(const QCtx &c, float s0, float s1,
                                        float s2, float s3, float4 p)
{
    float dx = p.x - c.qx, dy = p.y - c.qy, dz = p.z - c.qz, dt = p.w - c.qt;
    float d = (s0 * dx) * dx;
    d = fmaf(s1 * dy, dy, d);
    d = fmaf(s2 * dz, dz, d);
    d = fmaf(s3 * dt, dt, d);
    return d;
}

// The canonical FP64 distance (same operations and order as the oracle;
// explicit round-to-nearest intrinsics forbid contraction).
__device__ __forceinline__ double dist64(const double *s, float4 q, float4 p)
{
    double dx = __dsub_rn((double)p.x, (double)q.x);
    double dy = __dsub_rn((double)p.y, (double)q.y);
    double dz = __dsub_rn((double)p.z, (double)q.z);
    double dt = __dsub_rn((double)p.w, (double)q.w);
    double r = __dmul_rn(s[0], __dmul_rn(dx, dx));
    r = __dadd_rn(r, __dmul_rn(s[1], __dmul_rn(dy, dy)));
    r = __dadd_rn(r, __dmul_rn(s[2], __dmul_rn(dz, dz)));
    r = __dadd_rn(r, __dmul_rn(s[3], __dmul_rn(dt, dt)));
    return r;
}

// Query-to-cylinder lower bound (Algorithm 1 with the cylinder reading of
// the exclusion criterion): NaN when the segment holds no valid point
// (Eq. masked temporal part: t_A >= t_q - lag), so every "<=" test fails.
// a = (A', t_A), u = (U', t_B), b = (AB', r).
__device__ __forceinline__ float seg_lb(const QCtx &c, float st, float4 a,
                                        float4 u, float4 b)
{
    float vx = c.sx - a.x, vy = c.sy - a.y, vz = c.sz - a.z;
    float lam = __saturatef(fmaf(vz, u.z, fmaf(vy, u.y, vx * u.x)));
    float ex = fmaf(-lam, b.x, vx), ey = fmaf(-lam, b.y, vy), ez = fmaf(-lam, b.z, vz);
    float a2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
    float dist = a2 * rsqrtf(fmaxf(a2, 1e-37f));
    float sp = fmaxf(fmaf(dist, 1.0f - 0x1p-20f, -(b.w + c.delta)), 0.0f);
    float et = fmaxf(__fsub_rd(c.qt, fminf(u.w, c.T32)), 0.0f);
    float lb = fmaf(sp, sp, (st * et) * et) * (1.0f - 0x1p-19f);
    return (a.w < c.T32) ? lb : __int_as_float(0x7fffffff);
}

// Temporal part alone for a segment that ended at or before tB_max; a lower
// bound of seg_lb for every such segment.
__device__ __forceinline__ float time_lb(const QCtx &c, float st, float tB_max)
{
    float et = fmaxf(__fsub_rd(c.qt, fminf(tB_max, c.T32)), 0.0f);
    return ((st * et) * et) * (1.0f - 0x1p-19f);
}

// Number of entries < T of a sorted array, by a 32-way search of the warp.
template <typename Get>
__device__ __forceinline__ int warp_count_less(Get get, int n, float T, int lane)
{
    int lo = 0, hi = n; // every index < lo is < T, every index >= hi is >= T
    while (hi - lo > 32) {
        int step = (hi - lo + 31) >> 5;
        int p = lo + (lane + 1) * step - 1;
        bool lt = p < hi && get(p) < T;
        int nlt = __popc(__ballot_sync(FULLMASK, lt));
        int nlo = lo + nlt * step;
        int nhi = lo + (nlt + 1) * step - 1;
        hi = nhi < hi ? nhi : hi;
        lo = nlo < hi ? nlo : hi;
    }
    bool lt = lo + lane < hi && get(lo + lane) < T;
    return lo + __popc(__ballot_sync(FULLMASK, lt));
}

__device__ __forceinline__ void lane_insert(unsigned long long *K, int L,
                                            unsigned long long key)
{
    int i = L - 1;
#pragma unroll 1
    while (i > 0) {
        unsigned long long pv = K[(i - 1) * 32];
        if (pv < key)
            break;
        K[i * 32] = pv;
        --i;
    }
    K[i * 32] = key;
}

struct LaneStats {
    unsigned long long q, lb, pairs, segs, fp64;
};

// Write the k results of one query from its sorted candidate list K
// (stride 32), settling close ranks in FP64.  Returns false when the query
// needs the exact fallback.
__device__ bool finalize_query(const KnnWin *W, float4 q, const unsigned long long *K,
                               int L, unsigned long long *cl_d, int *cl_i,
                               int64_t qrow, LaneStats &st)
{
    const int k = W->k;
    int32_t *oi = W->out_idx + qrow * k;
    float *od = W->out_d2 + qrow * k;
    const bool exact_all = (W->flags & TNN_FLAG_EXACT_D2) != 0;
    const bool full = K[(L - 1) * 32] != SENT;
    int r = 0, i = 0;
    while (r < k && i < L) {
        unsigned long long ki = K[i * 32];
        if (ki == SENT)
            break;
        int e = i;
        float de = key_d(ki);
        while (e + 1 < L) {
            unsigned long long kn = K[(e + 1) * 32];
            if (kn == SENT)
                break;
            float dn = key_d(kn);
            if (dn <= fmaf(de, 0x1p-17f, de) + 0x1p-100f) {
                ++e;
                de = dn;
            } else {
                break;
            }
        }
        if (e == i && !exact_all) {
            oi[r] = key_i(ki);
            od[r] = key_d(ki);
            ++r;
            ++i;
            continue;
        }
        const int c = e - i + 1;
        if ((full && e == L - 1) || c > CMAX)
            return false;
        for (int t = 0; t < c; ++t) {
            int j = key_i(K[(i + t) * 32]);
            double dd = dist64(W->sigd, q, W->pts[j]);
            st.fp64++;
            unsigned long long db = (unsigned long long)__double_as_longlong(dd);
            int pos = t;
            while (pos > 0) {
                unsigned long long pd = cl_d[(pos - 1) * 32];
                int pi = cl_i[(pos - 1) * 32];
                if (pd < db || (pd == db && pi < j))
                    break;
                cl_d[pos * 32] = pd;
                cl_i[pos * 32] = pi;
                --pos;
            }
            cl_d[pos * 32] = db;
            cl_i[pos * 32] = j;
        }
        for (int t = 0; t < c && r < k; ++t) {
            oi[r] = cl_i[t * 32];
            od[r] = (float)__longlong_as_double((long long)cl_d[t * 32]);
            ++r;
        }
        i = e + 1;
    }
    for (; r < k; ++r) {
        oi[r] = -1;
        od[r] = INFINITY;
    }
    return true;
}

__device__ __forceinline__ void flush_stats(KnnScratch *scr, LaneStats &s)
{
    unsigned long long v[5] = {s.q, s.lb, s.pairs, s.segs, s.fp64};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        unsigned long long x = v[i];
        for (int o = 16; o > 0; o >>= 1)
            x += __shfl_xor_sync(FULLMASK, x, o);
        if ((threadIdx.x & 31) == 0 && x)
            atomicAdd(&scr->stats[i], x);
    }
}

__device__ __forceinline__ const KnnWin *find_window(const KnnLaunch &L, long long tile)
{
    if (L.nwin <= 1)
        return &L.w0;
    int lo = 0, hi = L.nwin;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (L.wins[mid].tile_begin <= tile)
            lo = mid;
        else
            hi = mid;
    }
    return L.wins + lo;
}

__device__ __forceinline__ int window_id(const KnnLaunch &L, const KnnWin *W)
{
    return L.nwin <= 1 ? 0 : (int)(W - L.wins);
}

// -------------------------------------------------------------- TNN kernel

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_tnn_search(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const size_t pw = smem_per_warp(L.L_max, L.kseg_max, false);
    unsigned char *ws = smem + (threadIdx.x >> 5) * pw;
    unsigned long long *K = (unsigned long long *)ws + lane;
    unsigned char *rest = ws + (size_t)L.L_max * 256;
    float4 *segbuf = (float4 *)rest;                        // [32][4]
    float4 *pbuf = (float4 *)(rest + 2048);                 // [kseg_max]
    unsigned *seedbits = (unsigned *)(rest + 2048 + 16 * L.kseg_max); // [8]
    unsigned long long *cl_d = (unsigned long long *)rest + lane; // aliases
    int *cl_i = (int *)(rest + CMAX * 32 * 8) + lane;

    LaneStats st = {0, 0, 0, 0, 0};
    for (;;) {
        long long tile = 0;
        if (lane == 0)
            tile = (long long)atomicAdd(&L.scr->tile_counter, 1ull);
        tile = __shfl_sync(FULLMASK, tile, 0);
        if (tile >= L.total_tiles)
            break;
        const KnnWin *W = find_window(L, tile);
        const int64_t qrow = (tile - W->tile_begin) * 32 + lane;
        const bool active = qrow < W->m;
        const float4 q = active ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, active);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float4 *__restrict__ seg = W->seg;
        const float4 *__restrict__ pts = W->pts;
        const int Lw = W->L, F = W->F, W0 = W->W0;

        float tmax = c.T32;
        for (int o = 16; o > 0; o >>= 1)
            tmax = fmaxf(tmax, __shfl_xor_sync(FULLMASK, tmax, o));
        const float *__restrict__ segTA = W->segTA;
        const int hi = warp_count_less([&](int p) { return __ldg(segTA + p); }, W->S, tmax, lane);

        for (int i = 0; i < Lw; ++i)
            K[i * 32] = SENT;
        if (lane < 8)
            seedbits[lane] = 0u;
        unsigned long long tauk = SENT;
        float tau = INFINITY;
        __syncwarp();

        // Scan all points of one segment for the lanes that need it.
        auto scan_segment = [&](float4 meta, bool need) {
            const int first = __float_as_int(meta.x), cnt = __float_as_int(meta.y);
            for (int j = lane; j < cnt; j += 32)
                pbuf[j] = __ldg(pts + first + j);
            __syncwarp();
            if (need) {
                st.segs++;
                st.pairs += cnt;
                for (int j = 0; j < cnt; ++j) {
                    const float4 p = pbuf[j];
                    const float d = dist32(c, s0, s1, s2, s3, p);
                    if (p.w < c.T32 && d <= tau) {
                        unsigned long long key = pack_key(d, first + j);
                        if (key < tauk) {
                            lane_insert(K, Lw, key);
                            tauk = K[(Lw - 1) * 32];
                            tau = key_d(tauk);
                        }
                    }
                }
            }
            __syncwarp();
        };

        // 1. seed: the F smallest bounds among the W0 most recent segments.
        const int lo0 = hi > W0 ? hi - W0 : 0;
        if (F > 0 && hi > 0) {
            float bl[8];
            int bp[8];
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                bl[f] = INFINITY;
                bp[f] = -1;
            }
            for (int c0 = lo0; c0 < hi; c0 += 32) {
                const int cnt = min(32, hi - c0);
                if (lane < cnt) {
                    const float4 *src = seg + 4 * (size_t)(c0 + lane);
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        segbuf[4 * lane + v] = __ldg(src + v);
                }
                __syncwarp();
                for (int i = 0; i < cnt; ++i) {
                    float cur = seg_lb(c, s3, segbuf[4 * i], segbuf[4 * i + 1], segbuf[4 * i + 2]);
                    int cp = c0 + i;
#pragma unroll
                    for (int f = 0; f < 8; ++f) {
                        if (f < F && cur < bl[f]) {
                            float tf = bl[f];
                            bl[f] = cur;
                            cur = tf;
                            int tp = bp[f];
                            bp[f] = cp;
                            cp = tp;
                        }
                    }
                }
                st.lb += active ? cnt : 0;
                __syncwarp();
            }
#pragma unroll
            for (int f = 0; f < 8; ++f)
                if (f < F && bp[f] >= 0)
                    atomicOr(&seedbits[(bp[f] - lo0) >> 5], 1u << ((bp[f] - lo0) & 31));
            __syncwarp();
            const int nwords = (hi - lo0 + 31) >> 5;
            for (int wd = 0; wd < nwords; ++wd) {
                unsigned bits = seedbits[wd];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int pos = lo0 + wd * 32 + b;
                    scan_segment(__ldg(seg + 4 * (size_t)pos + 3), active);
                }
            }
        }

        // 2. sweep from the most recent segment backwards.
        int pos_hi = hi;
        while (pos_hi > 0) {
            const float pm = __ldg(W->segPM + pos_hi - 1);
            const bool done = !active || !(time_lb(c, s3, pm) <= tau);
            if (__all_sync(FULLMASK, done))
                break;
            const int c0 = pos_hi > 32 ? pos_hi - 32 : 0;
            const int cnt = pos_hi - c0;
            if (lane < cnt) {
                const float4 *src = seg + 4 * (size_t)(c0 + lane);
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    segbuf[4 * lane + v] = __ldg(src + v);
            }
            __syncwarp();
            unsigned need = 0;
            if (!done) {
#pragma unroll 4
                for (int i = 0; i < cnt; ++i) {
                    const float lb = seg_lb(c, s3, segbuf[4 * i], segbuf[4 * i + 1], segbuf[4 * i + 2]);
                    const int rel = c0 + i - lo0;
                    const bool seeded = rel >= 0 && ((seedbits[rel >> 5] >> (rel & 31)) & 1u);
                    if (lb <= tau && !seeded)
                        need |= 1u << i;
                }
                st.lb += cnt;
            }
            unsigned any = __reduce_or_sync(FULLMASK, need);
            while (any) {
                const int i = 31 - __clz(any);
                any &= ~(1u << i);
                scan_segment(segbuf[4 * i + 3], (need >> i) & 1u);
            }
            __syncwarp();
            pos_hi = c0;
        }

        // 3. settle and write.
        __syncwarp();
        if (active) {
            st.q++;
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st)) {
                unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
                if (slot < (unsigned long long)L.fb_cap)
                    L.fb_list[slot] = make_int2(window_id(L, W), (int)qrow);
                else
                    atomicOr(&L.scr->status, 1u);
            }
        }
        __syncwarp();
    }
    flush_stats(L.scr, st);
}

// ---------------------------------------------------- linear-search kernel

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_linear_search(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const size_t pw = smem_per_warp(L.L_max, L.kseg_max, true);
    unsigned char *ws = smem + (threadIdx.x >> 5) * pw;
    unsigned long long *K = (unsigned long long *)ws + lane;
    unsigned char *rest = ws + (size_t)L.L_max * 256;
    float4 *pb = (float4 *)rest;          // [32]
    int *ib = (int *)(rest + 512);        // [32]
    unsigned long long *cl_d = (unsigned long long *)rest + lane;
    int *cl_i = (int *)(rest + CMAX * 32 * 8) + lane;

    LaneStats st = {0, 0, 0, 0, 0};
    for (;;) {
        long long tile = 0;
        if (lane == 0)
            tile = (long long)atomicAdd(&L.scr->tile_counter, 1ull);
        tile = __shfl_sync(FULLMASK, tile, 0);
        if (tile >= L.total_tiles)
            break;
        const KnnWin *W = find_window(L, tile);
        const int64_t qrow = (tile - W->tile_begin) * 32 + lane;
        const bool active = qrow < W->m;
        const float4 q = active ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, active);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float4 *__restrict__ pts_t = W->pts_t;
        const int32_t *__restrict__ idx_t = W->idx_t;
        const int Lw = W->L;

        float tmax = c.T32;
        for (int o = 16; o > 0; o >>= 1)
            tmax = fmaxf(tmax, __shfl_xor_sync(FULLMASK, tmax, o));
        const int hi = warp_count_less([&](int p) { return __ldg(&pts_t[p].w); }, W->n, tmax, lane);

        for (int i = 0; i < Lw; ++i)
            K[i * 32] = SENT;
        unsigned long long tauk = SENT;
        float tau = INFINITY;
        __syncwarp();

        for (int pos_hi = hi; pos_hi > 0;) {
            const int c0 = pos_hi > 32 ? pos_hi - 32 : 0;
            const int cnt = pos_hi - c0;
            if (lane < cnt) {
                pb[lane] = __ldg(pts_t + c0 + lane);
                ib[lane] = __ldg(idx_t + c0 + lane);
            }
            __syncwarp();
#pragma unroll 4
            for (int i = cnt - 1; i >= 0; --i) {
                const float4 p = pb[i];
                const float d = dist32(c, s0, s1, s2, s3, p);
                if (p.w < c.T32 && d <= tau) {
                    unsigned long long key = pack_key(d, ib[i]);
                    if (key < tauk) {
                        lane_insert(K, Lw, key);
                        tauk = K[(Lw - 1) * 32];
                        tau = key_d(tauk);
                    }
                }
            }
            if (active)
                st.pairs += cnt;
            __syncwarp();
            pos_hi = c0;
        }

        __syncwarp();
        if (active) {
            st.q++;
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st)) {
                unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
                if (slot < (unsigned long long)L.fb_cap)
                    L.fb_list[slot] = make_int2(window_id(L, W), (int)qrow);
                else
                    atomicOr(&L.scr->status, 1u);
            }
        }
        __syncwarp();
    }
    flush_stats(L.scr, st);
}

// ------------------------------------------------------- exact FP64 scan

// Queries whose FP32 ranking could not be settled: rank every valid point by
// the canonical FP64 distance and index (the oracle's definition).
__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_fallback(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int kmax = L.L_max;
    unsigned char *ws = smem + (threadIdx.x >> 5) * ((size_t)kmax * 32 * 12);
    unsigned long long *kd = (unsigned long long *)ws + lane;
    int *ki = (int *)(ws + (size_t)kmax * 32 * 8) + lane;
    unsigned nfb = *(volatile unsigned *)&L.scr->n_fallback;
    if ((long long)nfb > L.fb_cap)
        nfb = (unsigned)L.fb_cap;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long nfp = 0;
    for (unsigned base = (unsigned)gw * 32; base < nfb; base += (unsigned)nw * 32) {
        const unsigned slot = base + lane;
        if (slot < nfb) {
            const int2 e = L.fb_list[slot];
            const KnnWin *W = L.nwin <= 1 ? &L.w0 : L.wins + e.x;
            const float4 q = W->q[e.y];
            const float T32 = __double2float_ru((double)q.w - W->lag);
            const int k = W->k;
            const unsigned long long INF64 = 0x7ff0000000000000ull;
            for (int r = 0; r < k; ++r) {
                kd[r * 32] = INF64;
                ki[r * 32] = 0x7fffffff;
            }
            for (int j = 0; j < W->n; ++j) {
                const float4 p = W->pts[j];
                if (!(p.w < T32))
                    continue;
                const unsigned long long db =
                    (unsigned long long)__double_as_longlong(dist64(W->sigd, q, p));
                nfp++;
                const unsigned long long wd = kd[(k - 1) * 32];
                if (!(db < wd || (db == wd && j < ki[(k - 1) * 32])))
                    continue;
                int pos = k - 1;
                while (pos > 0) {
                    unsigned long long pd = kd[(pos - 1) * 32];
                    int pi = ki[(pos - 1) * 32];
                    if (pd < db || (pd == db && pi < j))
                        break;
                    kd[pos * 32] = pd;
                    ki[pos * 32] = pi;
                    --pos;
                }
                kd[pos * 32] = db;
                ki[pos * 32] = j;
            }
            int32_t *oi = W->out_idx + (int64_t)e.y * k;
            float *od = W->out_d2 + (int64_t)e.y * k;
            for (int r = 0; r < k; ++r) {
                const bool ok = kd[r * 32] != INF64;
                oi[r] = ok ? ki[r * 32] : -1;
                od[r] = ok ? (float)__longlong_as_double((long long)kd[r * 32]) : INFINITY;
            }
        }
    }
    unsigned long long x = nfp;
    for (int o = 16; o > 0; o >>= 1)
        x += __shfl_xor_sync(FULLMASK, x, o);
    if (lane == 0 && x)
        atomicAdd(&L.scr->stats[4], x);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        L.scr->stats[5] = nfb;
}

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

// ---- kernel timing for measurement tools (tnn_profile_*)
static bool g_prof_on = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_ev; // recorded pairs
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_pool; // free pairs

static cudaError_t prof_begin(cudaStream_t st, std::pair<cudaEvent_t, cudaEvent_t> *pr)
{
    if (!g_prof_pool.empty()) {
        *pr = g_prof_pool.back();
        g_prof_pool.pop_back();
    } else {
        cudaError_t e = cudaEventCreate(&pr->first);
        if (e != cudaSuccess)
            return e;
        e = cudaEventCreate(&pr->second);
        if (e != cudaSuccess)
            return e;
    }
    return cudaEventRecord(pr->first, st);
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
    static bool attrs = false;
    if (!attrs) {
        const int maxs = 227 * 1024;
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_tnn_search, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_linear_search, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_fallback, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs));
        attrs = true;
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
    const int W0 = p->seed_window == 0 ? 64 : p->seed_window;
    const int E = p->extra == 0 ? 8 : p->extra;
    TNN_ARG_CHECK(F >= 1 && F <= 8, "seed_segments must be in [1, 8]");
    TNN_ARG_CHECK(W0 >= 1 && W0 <= 256, "seed_window must be in [1, 256]");
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
    w->q = d_q ? (const float4 *)d_q : ix->pts;
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
    w->flags = p->flags;
    return TNN_OK;
}

tnn_status tnn_launch_search(const KnnLaunch &L, bool brute, cudaStream_t st)
{
    tnn_status s = device_setup();
    if (s != TNN_OK)
        return s;
    const size_t smem = smem_per_warp(L.L_max, L.kseg_max, brute) * TNN_WARPS_PER_CTA;
    int nb = 0;
    if (brute)
        TNN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_linear_search, TNN_WARPS_PER_CTA * 32, smem));
    else
        TNN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tnn_search, TNN_WARPS_PER_CTA * 32, smem));
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
    std::pair<cudaEvent_t, cudaEvent_t> pr;
    if (prof)
        TNN_CUDA_TRY(prof_begin(st, &pr));
    if (brute)
        k_linear_search<<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    else
        k_tnn_search<<<(unsigned)grid, TNN_WARPS_PER_CTA * 32, smem, st>>>(L);
    TNN_CUDA_TRY(cudaGetLastError());
    if (prof) {
        TNN_CUDA_TRY(cudaEventRecord(pr.second, st));
        g_prof_ev.push_back(pr);
    }
    const size_t fsm = (size_t)L.L_max * 32 * 12 * TNN_WARPS_PER_CTA;
    k_fallback<<<(unsigned)(2 * g_num_sms), TNN_WARPS_PER_CTA * 32, fsm, st>>>(L);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

static tnn_status run_single(const tnn_index *ix, const float *d_q, int64_t m,
                             const tnn_knn_params *p, int32_t *d_idx, float *d_d2,
                             tnn_stats *h_stats, tnn_stream_t stream, bool brute)
{
    tnn_clear_error();
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
    L.total_tiles = (m + TNN_TILE - 1) / TNN_TILE;
    L.fb_cap = m;
    const size_t hdr = 256;
    void *buf = nullptr;
    TNN_CUDA_TRY(cudaMallocAsync(&buf, hdr + sizeof(int2) * (size_t)m, st));
    L.scr = (KnnScratch *)buf;
    L.fb_list = (int2 *)((char *)buf + hdr);
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(KnnScratch), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(buf, st);
        TNN_CUDA_TRY(e);
    }
    s = tnn_launch_search(L, brute, st);
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
            h_stats->fallback_queries = hs.stats[5];
        }
    }
    cudaFreeAsync(buf, st);
    return s;
}

extern "C" tnn_status tnn_knn(const tnn_index *index, const float *d_q, int64_t m,
                              const tnn_knn_params *params, int32_t *d_idx,
                              float *d_d2, tnn_stats *h_stats, tnn_stream_t stream)
{
    return run_single(index, d_q, m, params, d_idx, d_d2, h_stats, stream, false);
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
        wins[w].tile_begin = tiles;
        tiles += (m[w] + TNN_TILE - 1) / TNN_TILE;
        fb += m[w];
        L_max = std::max(L_max, wins[w].L);
        kseg = std::max(kseg, (int)indexes[w]->K);
    }
    tnn_batch *b = new tnn_batch();
    memset(b, 0, sizeof(*b));
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->d_wins, sizeof(KnnWin) * n_windows);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->scratch, 256 + sizeof(int2) * (size_t)std::max(fb, 1ll));
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
    h->fallback_queries = hs.stats[5];
    return TNN_OK;
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
    int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(m_sample / 32, n / 32));
    if (n < 32)
        nblk = 1;
    const int64_t rows = std::min<int64_t>(32, n);
    const int64_t m = nblk * rows;
    const int64_t step = nblk > 1 ? (n - rows) / (nblk - 1) : 0;
    float4 *dq = nullptr;
    int32_t *di = nullptr;
    float *dd = nullptr;
    cudaError_t e = cudaMalloc(&dq, sizeof(float4) * m);
    if (e == cudaSuccess)
        e = cudaMalloc(&di, sizeof(int32_t) * m * params->k);
    if (e == cudaSuccess)
        e = cudaMalloc(&dd, sizeof(float) * m * params->k);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dq, rows * sizeof(float4), ix->pts,
                              (step > 0 ? step : rows) * sizeof(float4),
                              rows * sizeof(float4), nblk, cudaMemcpyDeviceToDevice, st);
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
    const int Fs[] = {2, 4, 6};
    const int Ws[] = {32, 64, 128};
    const int Es[] = {4, 8, 16};
    float best = 1e30f;
    tnn_knn_params bestp = *params;
    for (int a = 0; a < 3 && s == TNN_OK; ++a)
        for (int b = 0; b < 3 && s == TNN_OK; ++b)
            for (int c = 0; c < 3 && s == TNN_OK; ++c) {
                tnn_knn_params p = *params;
                p.seed_segments = Fs[a];
                p.seed_window = Ws[b];
                p.extra = Es[c];
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
    cudaFree(dq);
    cudaFree(di);
    cudaFree(dd);
    if (s == TNN_OK) {
        params->seed_segments = bestp.seed_segments;
        params->seed_window = bestp.seed_window;
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

extern "C" tnn_status tnn_profile_read(double *ms, int64_t *launches, int32_t reset)
{
    tnn_clear_error();
    double tot = 0.0;
    for (auto &pr : g_prof_ev) {
        TNN_CUDA_TRY(cudaEventSynchronize(pr.second));
        float x = 0.f;
        TNN_CUDA_TRY(cudaEventElapsedTime(&x, pr.first, pr.second));
        tot += x;
    }
    if (ms)
        *ms = tot;
    if (launches)
        *launches = (int64_t)g_prof_ev.size();
    if (reset) {
        for (auto &pr : g_prof_ev)
            g_prof_pool.push_back(pr);
        g_prof_ev.clear();
    }
    return TNN_OK;
}

// ------------------------------------------------------- necessary work

// One thread per query: walk the t_A order backwards from the causal end,
// stop when the temporal bound of every remaining segment exceeds d_k,
// count the bounds needed and the members of the segments within d_k.
__global__ void k_knn_work(const __grid_constant__ KnnWin W, const float *__restrict__ d2,
                           int k, unsigned long long *out)
{
    const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nlb = 0, npairs = 0;
    if (qi < W.m) {
        const QCtx c = make_qctx(&W, W.q[qi], true);
        const float dk = d2[qi * k + (k - 1)];
        int lo = 0, hi = W.S; // count of t_A < T32
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (W.segTA[mid] < c.T32)
                lo = mid + 1;
            else
                hi = mid;
        }
        for (int pos = lo - 1; pos >= 0; --pos) {
            if (!(time_lb(c, W.sig[3], W.segPM[pos]) <= dk))
                break;
            const float4 *r = W.seg + 4 * (size_t)pos;
            if (!(time_lb(c, W.sig[3], r[1].w) <= dk))
                continue;
            ++nlb;
            const float lb = seg_lb(c, W.sig[3], r[0], r[1], r[2]);
            if (lb <= dk)
                npairs += (unsigned)__float_as_int(r[3].y);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nlb += __shfl_xor_sync(FULLMASK, nlb, o);
        npairs += __shfl_xor_sync(FULLMASK, npairs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, nlb);
        atomicAdd(out + 1, npairs);
    }
}

extern "C" tnn_status tnn_knn_work(const tnn_index *index, const float *d_q, int64_t m,
                                   int32_t k, double lag, const float *d_d2,
                                   uint64_t *h_work, tnn_stream_t stream)
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
    h_work[0] = h_work[1] = 0;
    if (m == 0)
        return TNN_OK;
    TNN_ARG_CHECK(d_d2 != nullptr, "d_d2 is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *buf = nullptr;
    TNN_CUDA_TRY(cudaMallocAsync((void **)&buf, 16, st));
    cudaError_t e = cudaMemsetAsync(buf, 0, 16, st);
    if (e == cudaSuccess) {
        k_knn_work<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(w, d_d2, k, buf);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, buf, 16, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    TNN_CUDA_TRY(e);
    h_work[0] = h[0];
    h_work[1] = h[1];
    return TNN_OK;
}
