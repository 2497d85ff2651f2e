// Queries answered one warp per query.  Two kinds arrive here:
//   - deferred: in the lane-per-query kernel their pruning key after seeding
//     was too large for a shared tile (e.g. a flight's first samples, whose
//     neighbours are far away); Algorithm 2 puts such unfinished lines
//     aside and carries on with the others -- they are finished here, where
//     the whole warp works on one query (list of k + extra candidates);
//   - unsettled (window id stored as -1 - w): the chain of FP32 keys that FP32
//     cannot order reached the last candidate slot; here the list keeps
//     k + 32 candidates (a deferred query that ends the same way is run
//     again at once with k + 32).
//
// k_tnn_warp: the 32 lanes split the grid keys, the member segments and the
// member points of one query.  Candidates below the pruning key are sorted
// across the warp (bitonic) and merged into a sorted list in shared memory
// (merge path).  Seeding visits cubes of keys of growing radius around the
// query's own key (cells in the plane, buckets backwards in time) until the
// list is full; inside a chunk of segments, while the list is not full, the
// segment of smallest bound is scanned first (Algorithm 2's nearest-first
// fetch), so the pruning key is tight as soon as it exists.  The main phase
// is the exclusion criterion and stop rule of Algorithm 2 over the other
// keys, scanning the needed segments of a chunk 32 points at a time.
// A query still unsettled goes to k_fallback_exact: the definition, with the
// FP64 distance taken only for the points that FP32 cannot rule out.
#pragma once
#include "tnn_device.cuh"
#include "tnn_grid.cuh"

#define FB_EXTRA 32
#define WQ_CMAX (64 + FB_EXTRA)
#ifndef WQ_RSEED
#define WQ_RSEED 4 // largest radius of the seeding shells
#endif

__host__ __device__ inline size_t wq_smem_per_warp()
{
    // list [WQ_CMAX] + merge output [WQ_CMAX] + batch [32] (u64), packed
    // segment starts and firsts, packed key starts and ranges [4][32] (int),
    // and the settlement scratch
    // ([CMAX][32] u64 + [CMAX][32] int) after them
    return (size_t)(2 * WQ_CMAX + 32) * 8 + 128 * 4 + (size_t)CMAX * 32 * 12;
}

__host__ __device__ inline size_t fb_exact_smem_per_warp(int k_max)
{
    return (size_t)k_max * 32 * 12;
}

// The settlement of the warp-per-query kernel, out of line (lane 0 only,
// and only for queries with close ranks): bit 0 = settled, the rest the
// FP64 rechecks made.  Keeps its body out of the kernel's hot loop code.
static __device__ __noinline__ unsigned finalize_query_ool(const KnnWin *W, float4 q,
                                                          const unsigned long long *K, int L,
                                                          unsigned long long *cl_d, int *cl_i,
                                                          int64_t qrow)
{
    LaneStats st = {0, 0, 0, 0, 0};
    const bool ok = finalize_query(W, q, K, L, cl_d, cl_i, qrow, st, 1);
    return ((unsigned)st.fp64 << 1) | (ok ? 1u : 0u);
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m)
{
    return __shfl_xor_sync(FULLMASK, v, m);
}

// Ascending bitonic sort of one key per lane across the warp.
__device__ __forceinline__ unsigned long long warp_sort_u64(unsigned long long v, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = shfl_xor_u64(v, j);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            const unsigned long long mn = o < v ? o : v, mx = o < v ? v : o;
            v = (lower == up) ? mn : mx;
        }
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = shfl_xor_u64(v, o);
        v = w < v ? w : v;
    }
    return v;
}

struct WarpList {
    unsigned long long *L;   // [C] sorted keys, SENT beyond nv
    unsigned long long *tmp; // [C]
    unsigned long long *B;   // [32]
    int C, nv;
    unsigned long long tauk; // largest key kept once full, else bound0
    unsigned long long bound0; // no key above it can enter the list
};

// Merge the keys below the pruning key (at most one per lane) into the list.
__device__ __forceinline__ void wl_merge(WarpList &w, unsigned long long ck, int lane)
{
    const bool take = ck < w.tauk;
    const unsigned m = __ballot_sync(FULLMASK, take);
    if (!m)
        return;
    const int nb = __popc(m);
    const unsigned long long v = warp_sort_u64(take ? ck : SENT, lane);
    w.B[lane] = v;
    __syncwarp();
    const int na = w.nv;
    for (int p = lane; p < w.C; p += 32) {
        int lo = max(0, p - nb), hi = min(p, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (w.L[mid] < w.B[p - mid - 1])
                lo = mid + 1;
            else
                hi = mid;
        }
        const int i = lo, j = p - lo;
        unsigned long long out = SENT;
        if (i < na && (j >= nb || w.L[i] < w.B[j]))
            out = w.L[i];
        else if (j < nb)
            out = w.B[j];
        w.tmp[p] = out;
    }
    __syncwarp();
    for (int p = lane; p < w.C; p += 32)
        w.L[p] = w.tmp[p];
    __syncwarp();
    w.nv = min(na + nb, w.C);
    w.tauk = w.nv == w.C ? w.L[w.C - 1] : w.bound0;
}

#ifndef TNN_WARP_MINB
#define TNN_WARP_MINB 7 // 7 CTAs (28 warps, 73 registers) per SM: fewer spills than 8 at 64 registers
#endif
__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32, TNN_WARP_MINB)
    k_tnn_warp(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    unsigned char *ws = smem + (threadIdx.x >> 5) * wq_smem_per_warp();
    WarpList wl;
    wl.L = (unsigned long long *)ws;
    wl.tmp = wl.L + WQ_CMAX;
    wl.B = wl.tmp + WQ_CMAX;
    int *Sstart = (int *)(wl.B + 32);
    int *Sfirst = Sstart + 32;
    int *Kstart = Sfirst + 32;
    int *Klo = Kstart + 32;
    unsigned long long *cl_d = (unsigned long long *)(Klo + 32);
    int *cl_i = (int *)((unsigned char *)cl_d + CMAX * 32 * 8);

    unsigned nfb = *(volatile unsigned *)&L.scr->n_fallback;
    if ((long long)nfb > L.fb_cap)
        nfb = (unsigned)L.fb_cap;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    (void)gw;
    (void)nw;
    LaneStats st = {0, 0, 0, 0, 0};
    int2 ent = make_int2(0, 0);
    bool retry = false; // the same query again with the larger list
    float tau0 = INFINITY;
    for (;;) {
        if (!retry) {
            // dynamic queue: query costs differ by orders of magnitude
            unsigned e = 0;
            if (lane == 0)
                e = atomicAdd(&L.scr->fb_next, 1u);
            e = __shfl_sync(FULLMASK, e, 0);
            if (e >= nfb)
                break;
            ent = L.fb_list[e];
            tau0 = L.fb_tau[e];
        }
        const bool unsettled = retry || ent.x < 0;
        const int wid = ent.x < 0 ? -1 - ent.x : ent.x;
        const KnnWin *W = L.nwin <= 1 ? &L.w0 : L.wins + wid;
        const float4 q = W->q[ent.y];
        const QCtx c = make_qctx(W, q, true);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float4 *__restrict__ seg = W->seg;
        const float4 *__restrict__ pts = W->pts;
        const GridDesc &G = W->grid;
        wl.C = unsettled ? W->k + FB_EXTRA : W->L;
        wl.nv = 0;
        // A deferred query arrives with the pruning key tau0 of the tile
        // kernel's list of the same length (the same FP32 keys): its final
        // list holds no key with a distance above tau0.
        wl.bound0 = (unsettled || !(tau0 < INFINITY))
                        ? SENT
                        : (((unsigned long long)__float_as_uint(tau0) << 32) | 0xffffffffull);
        wl.tauk = wl.bound0;
        for (int p = lane; p < wl.C; p += 32)
            wl.L[p] = SENT;
        __syncwarp();

        // all points of one segment, 32 at a time
        auto scan_seg = [&](int first, int cnt) {
            if (lane == 0)
                st.segs++;
            if (L.dbg_seen && lane == 0)
                dbg_mark_seen(L, ent.y, first, cnt);
            for (int o = 0; o < cnt; o += 32) {
                const int j = o + lane;
                unsigned long long ck = SENT;
                if (j < cnt) {
                    const float4 p = __ldg(pts + first + j);
                    const float d = dist32(c, s0, s1, s2, s3, p);
                    if (p.w < c.T32)
                        ck = pack_key(d, first + j);
                    st.pairs++;
                }
                wl_merge(wl, ck, lane);
            }
        };
        // the points of every lane's segment with `need`, packed 32 per step
        auto scan_packed = [&](bool need, float4 meta) {
            const unsigned m = __ballot_sync(FULLMASK, need);
            const int cnt = need ? __float_as_int(meta.y) : 0;
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULLMASK, incl, o);
                if (lane >= o)
                    incl += t;
            }
            const int total = __shfl_sync(FULLMASK, incl, 31);
            const int nseg = __popc(m);
            if (need) {
                const int rank = __popc(m & ((1u << lane) - 1u));
                Sstart[rank] = incl - cnt;
                Sfirst[rank] = __float_as_int(meta.x);
                if (L.dbg_seen)
                    dbg_mark_seen(L, ent.y, __float_as_int(meta.x), cnt);
            }
            if (lane == 0)
                st.segs += nseg;
            __syncwarp();
            for (int s = 0; s < total; s += 32) {
                const int g = s + lane;
                unsigned long long ck = SENT;
                if (g < total) {
                    int lo = 0, hi = nseg - 1; // largest r with Sstart[r] <= g
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (Sstart[mid] <= g)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    const int j = Sfirst[lo] + (g - Sstart[lo]);
                    const float4 p = __ldg(pts + j);
                    const float d = dist32(c, s0, s1, s2, s3, p);
                    if (p.w < c.T32)
                        ck = pack_key(d, j);
                    st.pairs++;
                }
                wl_merge(wl, ck, lane);
            }
            __syncwarp();
        };
        // the member segments of one key whose cylinder bound does not exceed
        // the pruning key; nearest first while the list is not full
        // The member segments of every lane's key (key < 0: none; [klo, khi)
        // its range of G.ids) are handled together, 32 segments per step
        // whatever key they belong to.
        auto visit_keys = [&](bool has, int klo, int khi) {
            const unsigned km = __ballot_sync(FULLMASK, has);
            if (!km)
                return;
            const int kc = has ? khi - klo : 0;
            int incl = kc;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULLMASK, incl, o);
                if (lane >= o)
                    incl += t;
            }
            const int total = __shfl_sync(FULLMASK, incl, 31);
            const int nk = __popc(km);
            __syncwarp();
            if (has) {
                const int rank = __popc(km & ((1u << lane) - 1u));
                Kstart[rank] = incl - kc;
                Klo[rank] = klo;
            }
            __syncwarp();
            for (int base = 0; base < total; base += 32) {
                const int g = base + lane;
                float lb = __int_as_float(0x7fffffff);
                float4 meta = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < total) {
                    int a = 0, z = nk - 1; // largest r with Kstart[r] <= g
                    while (a < z) {
                        const int mid = (a + z + 1) >> 1;
                        if (Kstart[mid] <= g)
                            a = mid;
                        else
                            z = mid - 1;
                    }
                    const float4 *src = G.gseg + 4 * (size_t)(Klo[a] + (g - Kstart[a]));
                    meta = __ldg(src + 3);
                    lb = seg_lb(c, s3, __ldg(src), __ldg(src + 1), __ldg(src + 2));
                    st.lb++;
                }
                while (wl.nv < wl.C) {
                    const bool need = lb <= key_d(wl.tauk);
                    const unsigned long long arg = warp_min_u64(
                        need ? (((unsigned long long)__float_as_uint(lb) << 32) | (unsigned)lane) : ~0ull);
                    if (arg == ~0ull)
                        break;
                    const int who = (int)(arg & 31u);
                    scan_seg(__float_as_int(__shfl_sync(FULLMASK, meta.x, who)),
                             __float_as_int(__shfl_sync(FULLMASK, meta.y, who)));
                    if (lane == who)
                        lb = __int_as_float(0x7fffffff);
                }
                const bool need = lb <= key_d(wl.tauk);
                if (__any_sync(FULLMASK, need))
                    scan_packed(need, meta);
            }
        };

        int bhi = -1;
        {
            const float fb = (c.T32 - G.t0) * G.inv_dt;
            if (fb >= 0.0f)
                bhi = (int)fminf(floorf(fb), (float)(G.nb - 1));
        }
        if (bhi >= 0) {
            const int hx = min(max((int)floorf((c.sx - G.x0) * G.inv_cell), 0), G.nx - 1);
            const int hy = min(max((int)floorf((c.sy - G.y0) * G.inv_cell), 0), G.ny - 1);
            const int rcover = max(max(max(hx, G.nx - 1 - hx), max(hy, G.ny - 1 - hy)), bhi);
            const float ext_max = __ldg(G.ext_max);
            // One loop hands visit_keys the keys of both phases, up to 32 per
            // round (a single inlined copy of the visit and its merges):
            // ---- seeding: shells of growing radius around the query's key, at
            // most WQ_RSEED + 1 of them (a query with fewer than C valid points
            // would otherwise grow the cube over the whole grid; the main
            // phase visits each causal bucket once instead);
            // ---- main: buckets backwards, keys within reach, by bound.
            bool seeding = true;
            int rs = -1, side = 1, nk = 0, t0 = 0; // shell rs of side x side x (rs + 1) positions
            int b = bhi + 1, cx0 = 0, cy0 = 0, wx = 1; // main: bucket b, its reach rectangle
            bool bseed = false;
            float bpm_next = 0.0f;
            for (;;) {
                int klo = 0, khi = 0;
                if (seeding) {
                    if (t0 >= nk) {
                        if (!(wl.nv < wl.C && rs < rcover && rs < WQ_RSEED)) {
                            seeding = false;
                            if (rs >= rcover)
                                break; // the shells covered every causal key
                            bpm_next = __ldg(G.bpm + bhi); // one bucket ahead
                            nk = 0;
                            t0 = 0;
                            continue;
                        }
                        ++rs;
                        side = 2 * rs + 1;
                        nk = side * side * (rs + 1);
                        t0 = 0;
                    }
                    const int t = t0 + lane, r = rs;
                    if (t < nk) {
                        const int db = t / (side * side), rem = t % (side * side);
                        const int dy = rem / side - r, dx = rem % side - r;
                        const int bk = bhi - db, cx = hx + dx, cy = hy + dy;
                        const bool shell = max(max(abs(dx), abs(dy)), db) == r;
                        if (shell && bk >= 0 && cx >= 0 && cx < G.nx && cy >= 0 && cy < G.ny) {
                            const int k2 = bk * G.ncell + cy * G.nx + cx;
                            klo = __ldg(G.off + k2);
                            khi = __ldg(G.off + k2 + 1);
                        }
                    }
                } else {
                    if (t0 >= nk) {
                        if (--b < 0)
                            break;
                        const float tau = key_d(wl.tauk);
                        const float bpm_b = bpm_next;
                        if (b > 0)
                            bpm_next = __ldg(G.bpm + b - 1);
                        if (!(time_lb(c, s3, bpm_b) <= tau))
                            break;
                        const float R = sqrtf(tau) * (1.0f + 0x1p-18f) + ext_max + c.delta;
                        int cx1, cy1;
                        reach_cells(c.sx, c.sx, R, G.x0, G.inv_cell, G.nx, cx0, cx1);
                        reach_cells(c.sy, c.sy, R, G.y0, G.inv_cell, G.ny, cy0, cy1);
                        wx = cx1 - cx0 + 1;
                        nk = wx * (cy1 - cy0 + 1);
                        bseed = bhi - b <= rs;
                        t0 = 0;
                    }
                    const int t = t0 + lane;
                    if (t < nk) {
                        const int cx = cx0 + t % wx, cy = cy0 + t / wx;
                        const bool seeded = bseed && abs(cx - hx) <= rs && abs(cy - hy) <= rs;
                        if (!seeded) {
                            const int k2 = b * G.ncell + cy * G.nx + cx;
                            const int4 kr = __ldg(G.krec + k2);
                            const int a0 = kr.x, a1 = kr.y;
                            if (a1 > a0) {
                                const float rx0 = G.x0 + (float)cx * G.cell;
                                const float ry0 = G.y0 + (float)cy * G.cell;
                                if (cell_lb(c, s3, rx0, rx0 + G.cell, ry0, ry0 + G.cell,
                                            __int_as_float(kr.z), __int_as_float(kr.w)) <= key_d(wl.tauk)) {
                                    klo = a0;
                                    khi = a1;
                                }
                            }
                        }
                    }
                }
                t0 += 32;
                visit_keys(khi > klo, klo, khi);
            }
        }
        __syncwarp();
        // Settle.  When no two of the first k keys are close enough to need
        // FP64 (no chain), the answer is the first k keys as they are and the
        // warp writes it; otherwise lane 0 settles the chains.
        bool ok = true;
        {
            const int k = W->k;
            bool chain = (W->flags & TNN_FLAG_EXACT_D2) != 0;
            for (int i = lane; i < k; i += 32) {
                const unsigned long long ki = wl.L[i];
                if (ki != SENT && i + 1 < wl.C) {
                    const unsigned long long kn = wl.L[i + 1];
                    const float de = key_d(ki);
                    chain |= kn != SENT && key_d(kn) <= fmaf(de, 0x1p-17f, de) + 0x1p-100f;
                }
            }
            if (!__any_sync(FULLMASK, chain)) {
                int32_t *oi = W->out_idx + (int64_t)ent.y * k;
                float *od = W->out_d2 + (int64_t)ent.y * k;
                for (int i = lane; i < k; i += 32) {
                    const unsigned long long ki = wl.L[i];
                    oi[i] = ki == SENT ? -1 : key_i(ki);
                    od[i] = ki == SENT ? INFINITY : key_d(ki);
                }
            } else {
                if (lane == 0) {
                    const unsigned r = finalize_query_ool(W, q, wl.L, wl.C, cl_d, cl_i, ent.y);
                    ok = (r & 1u) != 0;
                    st.fp64 += r >> 1;
                }
                ok = __shfl_sync(FULLMASK, ok, 0);
            }
        }
        // a tie chain ran past the end of a k + extra list: once more with
        // k + FB_EXTRA slots before the FP64 definition is used
        retry = !ok && wl.C < W->k + FB_EXTRA;
        if (!ok && !retry && lane == 0) {
            const unsigned slot = atomicAdd(&L.scr->n_fallback3, 1u);
            if (slot < (unsigned long long)L.fb_cap)
                L.fb_list3[slot] = make_int2(wid, ent.y);
            else
                atomicOr(&L.scr->status, 2u);
        }
        __syncwarp();
    }
    unsigned long long v[4] = {st.lb, st.pairs, st.segs, st.fp64};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long x = v[i];
        for (int o = 16; o > 0; o >>= 1)
            x += __shfl_xor_sync(FULLMASK, x, o);
        if (lane == 0 && x)
            atomicAdd(&L.scr->stats[1 + i], x);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        L.scr->stats[5] = nfb;
}

// Fault flags of the search launches on this device (the bits of
// KnnScratch::status: 1 and 2 a fallback list overflowed, 4 a bounded wait
// timed out), ORed in by the last kernel of every search and kept until a
// synchronising call reports and clears them (tnn_sync_status).  Searches
// without statistics and tnn_knn_noalloc report through it.
static __device__ unsigned int g_search_fault;

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_fallback_exact(const __grid_constant__ KnnLaunch L)
{
    // The kernels before this one on the stream have completed: their flags
    // are final.  Nothing below sets a flag.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned f = *(volatile unsigned *)&L.scr->status;
        if (f)
            atomicOr(&g_search_fault, f);
    }
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
    (void)gw;
    (void)nw;
    for (;;) {
        unsigned e = 0;
        if (lane == 0)
            e = atomicAdd(&L.scr->fb_next3, 1u);
        e = __shfl_sync(FULLMASK, e, 0);
        if (e >= nfb)
            break;
        const int2 ent = L.fb_list3[e];
        const KnnWin *W = L.nwin <= 1 ? &L.w0 : L.wins + ent.x;
        const float4 q = W->q[ent.y];
        const QCtx c = make_qctx(W, q, true);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float T32 = c.T32;
        const int k = W->k;
        // pass 1: the k-th smallest FP32 key over the valid points (each lane
        // keeps its k smallest, then a k-round warp merge)
        for (int r = 0; r < k; ++r)
            kd[r * 32] = SENT;
        int cnt = 0;
        for (int j = lane; j < W->n; j += 32) {
            const float4 p = W->pts[j];
            if (!(p.w < T32))
                continue;
            const unsigned long long key = pack_key(dist32(c, s0, s1, s2, s3, p), j);
            if (!(key < kd[(k - 1) * 32]))
                continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0) {
                const unsigned long long pk = kd[(pos - 1) * 32];
                if (pk < key)
                    break;
                kd[pos * 32] = pk;
                --pos;
            }
            kd[pos * 32] = key;
            if (cnt < k)
                ++cnt;
        }
        unsigned long long kth = SENT;
        {
            int h = 0;
            for (int r = 0; r < k; ++r) {
                const unsigned long long v = h < cnt ? kd[h * 32] : SENT;
                unsigned long long mv = v;
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long ov = shfl_xor_u64(mv, o);
                    mv = ov < mv ? ov : mv;
                }
                if (v == mv && h < cnt)
                    ++h;
                kth = mv;
            }
        }
        // Every point of the exact top k has d32 <= tau32 (1 + 2^-20): at
        // least k points have d32 <= tau32, so d64 of the k-th is at most
        // tau32 / (1 - 2^-21), and d32 <= d64 (1 + 2^-21).
        const float tau32 = key_d(kth);
        const float lim = fmaf(tau32, 0x1p-19f, tau32);
        // pass 2: FP64 distances of the points within that bound only
        for (int r = 0; r < k; ++r) {
            kd[r * 32] = INF64;
            ki[r * 32] = 0x7fffffff;
        }
        cnt = 0;
        for (int j = lane; j < W->n; j += 32) {
            const float4 p = W->pts[j];
            if (!(p.w < T32) || !(dist32(c, s0, s1, s2, s3, p) <= lim))
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
        // merge the 32 lists by (d2, index)
        int h = 0;
        int32_t *oi = W->out_idx + (int64_t)ent.y * k;
        float *od = W->out_d2 + (int64_t)ent.y * k;
        for (int r = 0; r < k; ++r) {
            const unsigned long long vd = h < cnt ? kd[h * 32] : INF64;
            const int vi = h < cnt ? ki[h * 32] : 0x7fffffff;
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
    if (blockIdx.x == 0 && threadIdx.x == 0)
        L.scr->stats[6] = nfb;
}
