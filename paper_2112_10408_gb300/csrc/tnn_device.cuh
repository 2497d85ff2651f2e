// Device helpers shared by the search kernels (see tnn_knn.cu for the
// execution model and the numerical contract).
#pragma once

#include <math.h>

#include "tnn_internal.cuh"

#define FULLMASK 0xffffffffu
#define CMAX 8
#define TNN_UCAP 128 // seed segments scanned in pass 2 (per warp)
#define TNN_WCAP 384 // segments recorded by pass 1 (per warp)

static const unsigned long long SENT = (0x7f800000ull << 32) | 0xffffffffull;

// Shared-memory layout per warp of the tile kernels.
enum { SMEM_SWEEP = 0, SMEM_LINEAR = 1, SMEM_GRID = 2 };

__host__ __device__ inline size_t smem_per_warp(int L_max, int kseg_max, int mode)
{
    // candidate lists [L_max][32] keys, then: sweep and grid: segment chunk
    // [32][4] float4 | points [kseg_max] float4 | seed union [TNN_UCAP] int
    // (| pass-1 list [TNN_WCAP] int for the sweep); linear search: points
    // [32] float4 | indices [32] int.  The FP64 settlement scratch
    // ([CMAX][32] u64 + [CMAX][32] int) reuses that area.
    size_t base = (size_t)L_max * 32 * 8;
    size_t rest = mode == SMEM_LINEAR
                      ? (32 * 16 + 32 * 4)
                      : (2048 + (size_t)kseg_max * 16 +
                         4 * (TNN_UCAP + (mode == SMEM_SWEEP ? TNN_WCAP : 0)));
    size_t cl = (size_t)CMAX * 32 * 12;
    if (rest < cl)
        rest = cl;
    return (base + rest + 15) & ~(size_t)15;
}

size_t tnn_search_smem_per_warp(int L_max, int kseg_max, int mode)
{
    return smem_per_warp(L_max, kseg_max, mode);
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

// Candidate list of one query held as a heap (used where one thread serves
// one query without warp-wide divergence costs, e.g. the tensor-core linear
// search): at most L keys in a shared-memory column whose slots are S keys
// apart.  While fewer than L are kept a key is appended (slots beyond hold
// SENT); at L keys the column becomes a binary max-heap, and from then on a
// smaller key replaces the root and sinks (log2 L levels of two independent
// loads).  list_sort restores ascending order for the settlement.
template <int S>
__device__ __forceinline__ void heap_sink(unsigned long long *K, int n, int i, unsigned long long v)
{
#pragma unroll 1
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= n)
            break;
        unsigned long long cv = K[l * S];
        int c = l;
        if (l + 1 < n) {
            const unsigned long long rv = K[(l + 1) * S];
            if (rv > cv) {
                cv = rv;
                c = l + 1;
            }
        }
        if (cv <= v)
            break;
        K[i * S] = cv;
        i = c;
    }
    K[i * S] = v;
}

// Add `key` (the caller checked key < the returned bound) and return the new
// pruning key: the L-th smallest key kept, SENT while fewer than L are kept.
template <int S>
__device__ __forceinline__ unsigned long long list_push(unsigned long long *K, int L, int &nv,
                                                        unsigned long long key)
{
    if (nv < L) {
        K[nv * S] = key;
        if (++nv < L)
            return SENT;
#pragma unroll 1
        for (int i = L / 2 - 1; i >= 0; --i)
            heap_sink<S>(K, L, i, K[i * S]);
    } else {
        heap_sink<S>(K, L, 0, key);
    }
    return K[0];
}

// Ascending order of the nv kept keys (heapsort; slots nv.. keep SENT).
template <int S>
__device__ __forceinline__ void list_sort(unsigned long long *K, int nv)
{
#pragma unroll 1
    for (int i = nv / 2 - 1; i >= 0; --i)
        heap_sink<S>(K, nv, i, K[i * S]);
#pragma unroll 1
    for (int end = nv - 1; end > 0; --end) {
        const unsigned long long top = K[0];
        const unsigned long long last = K[end * S];
        K[end * S] = top;
        heap_sink<S>(K, end, 0, last);
    }
}

// Sorted candidate list of one lane (stride 32 in shared memory) holding
// nv <= L keys; slots nv..L-1 hold SENT.  Insert `key` (the caller checked
// key < the returned bound) and return the new pruning key: the L-th smallest
// key kept, SENT while fewer than L are kept.  The lanes of a warp insert at
// different moments, so the cost that matters is the latency of one
// insertion: the shift reads four slots ahead, so that its loads do not wait
// on one another.  (A heap has a one-time build and data-dependent sift
// depths that serialise across the warp's lanes.)
__device__ __forceinline__ unsigned long long lane_push(unsigned long long *K, int L, int &nv,
                                                        unsigned long long key)
{
    int i = nv < L ? nv : L - 1;
#pragma unroll 1
    while (i >= 4) {
        const unsigned long long a = K[(i - 1) * 32], b = K[(i - 2) * 32];
        const unsigned long long c = K[(i - 3) * 32], d = K[(i - 4) * 32];
        if (a < key)
            goto place;
        K[i * 32] = a;
        if (b < key) {
            i -= 1;
            goto place;
        }
        K[(i - 1) * 32] = b;
        if (c < key) {
            i -= 2;
            goto place;
        }
        K[(i - 2) * 32] = c;
        if (d < key) {
            i -= 3;
            goto place;
        }
        K[(i - 3) * 32] = d;
        i -= 4;
    }
#pragma unroll 1
    while (i > 0) {
        const unsigned long long pv = K[(i - 1) * 32];
        if (pv < key)
            break;
        K[i * 32] = pv;
        --i;
    }
place:
    K[i * 32] = key;
    if (nv < L)
        ++nv;
    return nv == L ? K[(L - 1) * 32] : SENT;
}

// Points of one segment held in registers (lane j keeps members j and
// j + 32) so that the global load of the next segment overlaps the scan of
// the current one.
struct SegPoints {
    float4 a, b;
    int first, cnt;
};

__device__ __forceinline__ void seg_points_load(SegPoints &sp, const float4 *__restrict__ pts,
                                                float4 meta, int lane)
{
    sp.first = __float_as_int(meta.x);
    sp.cnt = __float_as_int(meta.y);
    if (lane < sp.cnt)
        sp.a = __ldg(pts + sp.first + lane);
    if (lane + 32 < sp.cnt)
        sp.b = __ldg(pts + sp.first + lane + 32);
}

__device__ __forceinline__ void seg_points_store(const SegPoints &sp, float4 *pbuf, int lane)
{
    if (lane < sp.cnt)
        pbuf[lane] = sp.a;
    if (lane + 32 < sp.cnt)
        pbuf[lane + 32] = sp.b;
}

// Tests only: record that the distances of points [first, first + cnt) to
// query `row` were taken (the segment was scanned for it).
__device__ __forceinline__ void dbg_mark_seen(const KnnLaunch &L, int64_t row, int first, int cnt)
{
    uint32_t *r = L.dbg_seen + row * L.dbg_words;
    for (int j = first; j < first + cnt; ++j)
        atomicOr(r + (j >> 5), 1u << (j & 31));
}

// The query row of this lane in global tile `tile` of window W, and whether
// the lane has one: a run of consecutive rows of one trajectory for
// self-queries (W->tile_rows), else 32 consecutive queries.
__device__ __forceinline__ bool tile_query(const KnnWin *W, long long tile, int lane, int64_t &qrow)
{
    const int64_t t = tile - W->tile_begin;
    if (W->tile_rows) {
        const int64_t gt = W->tile_first + t;
        const int64_t a = max((int64_t)__ldg(W->tile_rows + gt), W->row0);
        const int64_t b = min((int64_t)__ldg(W->tile_rows + gt + 1), W->row0 + W->m);
        qrow = a - W->row0 + lane;
        return a + lane < b;
    }
    qrow = t * 32 + lane;
    return qrow < W->m;
}

// Copy rows [row0, row0 + cnt) of a finished tile from the window's lists
// (just written by this warp) to the mirror lists (KnnLaunch::mirror_idx):
// consecutive words across the lanes, so every store instruction writes
// contiguous bytes (16 per lane when KnnLaunch::mirror_vec, else 4); two
// words of each list in flight per lane before their stores (more would
// take registers from the search loops).
template <typename T>
__device__ __forceinline__ void mirror_words(const T *__restrict__ si, const T *__restrict__ sd,
                                             T *__restrict__ di, T *__restrict__ dd, int64_t nw, int lane)
{
    for (int64_t j0 = 0; j0 < nw; j0 += 2 * 32) {
        T vi[2], vd[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t j = j0 + u * 32 + lane;
            if (j < nw) {
                vi[u] = __ldcg(si + j);
                vd[u] = __ldcg(sd + j);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t j = j0 + u * 32 + lane;
            if (j < nw) {
                di[j] = vi[u];
                dd[j] = vd[u];
            }
        }
    }
}

__device__ __forceinline__ void mirror_tile(const KnnLaunch &L, const KnnWin *W, int64_t row0, int cnt,
                                            int lane)
{
    __syncwarp();
    const int64_t o = row0 * W->k, nw = (int64_t)cnt * W->k;
    if (L.mirror_vec) // k % 4 == 0 and 16-byte aligned lists: whole int4 words
        mirror_words((const int4 *)(W->out_idx + o), (const int4 *)(W->out_d2 + o),
                     (int4 *)(L.mirror_idx + o), (int4 *)(L.mirror_d2 + o), nw / 4, lane);
    else
        mirror_words((const int *)(W->out_idx + o), (const int *)(W->out_d2 + o), (int *)(L.mirror_idx + o),
                     (int *)(L.mirror_d2 + o), nw, lane);
}

struct LaneStats {
    unsigned long long q, lb, pairs, segs, fp64;
};

// Write the k results of one query from its sorted candidate list K
// (stride 32), settling close ranks in FP64.  Returns false when the query
// needs the exact fallback.
__device__ bool finalize_query(const KnnWin *W, float4 q, const unsigned long long *K,
                               int L, unsigned long long *cl_d, int *cl_i,
                               int64_t qrow, LaneStats &st, int stride = 32)
{
    const int k = W->k;
    int32_t *oi = W->out_idx + qrow * k;
    float *od = W->out_d2 + qrow * k;
    const bool exact_all = (W->flags & TNN_FLAG_EXACT_D2) != 0;
    const bool full = K[(L - 1) * stride] != SENT;
    int r = 0, i = 0;
    while (r < k && i < L) {
        unsigned long long ki = K[i * stride];
        if (ki == SENT)
            break;
        int e = i;
        float de = key_d(ki);
        while (e + 1 < L) {
            unsigned long long kn = K[(e + 1) * stride];
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
            int j = key_i(K[(i + t) * stride]);
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

