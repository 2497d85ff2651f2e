// TNN search over the time-bucketed spatial grid of the index.
//
// Same tiles, candidate lists, seeds and settlement as the sweep kernel
// (tnn_search.cuh); only the order in which segments are considered
// changes.  A key of the grid (bucket of t_A, cell of the midpoint) has its
// own lower bound -- distance from the query to the cell rectangle minus the
// key's extent, plus the temporal part from the key's largest t_B -- which
// never exceeds the cylinder bound of any member segment, so whole keys are
// excluded at once by the exclusion criterion of Sec. 3.4.
//
//   seeds   the 3 x 3 cells around the warp in the three most recent buckets:
//           every lane keeps its F smallest cylinder bounds there; the union
//           of those segments is scanned first (Algorithm 2's first fetch).
//   main    buckets from the causal end backwards; a bucket is visited while
//           the temporal bound of its running maximum of t_B does not exceed
//           some lane's pruning key (Algorithm 2's stop rule); inside it, the
//           cells within reach of the warp's queries, and inside a cell whose
//           bound does not exceed a lane's key, the member segments whose
//           cylinder bound does not exceed it are scanned for that lane.
#pragma once
#include "tnn_device.cuh"

#ifndef TNN_GMAX_F
#define TNN_GMAX_F 6
#endif
#ifndef TNN_SEED_BUCKETS
#define TNN_SEED_BUCKETS 3 // newest buckets whose 3 x 3 cells seed a tile (at most 3)
#endif

// Lower bound on the cylinder bound (and so on the FP32 distance of any
// valid member) of every segment of one key.
__device__ __forceinline__ float cell_lb(const QCtx &c, float st, float rx0, float rx1,
                                         float ry0, float ry1, float ext, float tBk)
{
    const float dx = fmaxf(fmaxf(rx0 - c.sx, c.sx - rx1), 0.0f);
    const float dy = fmaxf(fmaxf(ry0 - c.sy, c.sy - ry1), 0.0f);
    const float a2 = fmaf(dy, dy, dx * dx);
    const float dist = a2 * rsqrtf(fmaxf(a2, 1e-37f));
    const float sp = fmaxf(fmaf(dist, 1.0f - 0x1p-20f, -(ext + c.delta)), 0.0f);
    const float et = fmaxf(__fsub_rd(c.qt, fminf(tBk, c.T32)), 0.0f);
    return fmaf(sp, sp, (st * et) * et) * (1.0f - 0x1p-19f);
}

// Cells [c0, c1] of one axis (n cells of size 1 / inv_cell from o) whose
// span can come within R of the interval [s0, s1].  The FP32 evaluation of
// the indices here and of the cell corners at query time errs by at most
// 2^-21 ((|s0| + R + 2|o|) inv_cell + n) cells; the slack is twice that plus
// 2^-10.  (A whole cell of margin on each side would triple the cells
// examined at the usual cell sizes, and still fall short for coordinates far
// from the origin.)
__device__ __forceinline__ void reach_cells(float s0, float s1, float R, float o, float inv_cell, int n,
                                            int &c0, int &c1)
{
    const float slack =
        fmaf(0x1p-20f, fmaf(fabsf(s0) + fabsf(s1) + R + 2.0f * fabsf(o), inv_cell, (float)n), 0x1p-10f);
    c0 = max((int)floorf(fmaxf(fmaf(s0 - R - o, inv_cell, -slack), -1.0f)), 0);
    c1 = min((int)floorf(fminf(fmaf(s1 + R - o, inv_cell, slack), (float)n)), n - 1);
}

__device__ __forceinline__ float warp_minf(float v)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fminf(v, __shfl_xor_sync(FULLMASK, v, o));
    return v;
}
__device__ __forceinline__ float warp_maxf(float v)
{
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(FULLMASK, v, o));
    return v;
}

#ifndef TNN_GRID_MINB
#define TNN_GRID_MINB 4
#endif

// MIRROR: also copy each finished tile's rows to KnnLaunch::mirror_idx /
// mirror_d2 (a separate instantiation, so that the plain search compiles
// without that code).
template <bool MIRROR>
__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32, TNN_GRID_MINB)
    k_tnn_grid_search(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const size_t pw = smem_per_warp(L.L_max, L.kseg_max, SMEM_GRID);
    unsigned char *ws = smem + (threadIdx.x >> 5) * pw;
    unsigned long long *K = (unsigned long long *)ws + lane;
    unsigned char *rest = ws + (size_t)L.L_max * 256;
    float4 *segbuf = (float4 *)rest;                     // [32][4]
    float4 *pbuf = (float4 *)(rest + 2048);              // [kseg_max]
    int *ulist = (int *)(rest + 2048 + 16 * L.kseg_max); // [TNN_UCAP] seeds
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
        int64_t qrow;
        const bool active = tile_query(W, tile, lane, qrow);
        const float4 q = active ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, active);
        const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
        const float4 *__restrict__ seg = W->seg;
        const float4 *__restrict__ pts = W->pts;
        const GridDesc &G = W->grid;
        const int32_t *__restrict__ goff = G.off;
        const int Lw = W->L, F = W->F;

        const float tmax = warp_maxf(c.T32);
        const float bx0 = warp_minf(active ? c.sx : INFINITY);
        const float bx1 = warp_maxf(active ? c.sx : -INFINITY);
        const float by0 = warp_minf(active ? c.sy : INFINITY);
        const float by1 = warp_maxf(active ? c.sy : -INFINITY);
        const float dmax = warp_maxf(active ? c.delta : 0.0f);
        const float ext_max = __ldg(G.ext_max);
        int bhi = -1;
        {
            const float fb = (tmax - G.t0) * G.inv_dt;
            if (fb >= 0.0f)
                bhi = (int)fminf(floorf(fb), (float)(G.nb - 1));
        }

        for (int i = 0; i < Lw; ++i)
            K[i * 32] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY;
        bool done = !active;

        auto scan_pbuf = [&](int first, int cnt, bool need) {
            if (!need)
                return;
            st.segs++;
            st.pairs += cnt;
            if (L.dbg_seen)
                dbg_mark_seen(L, qrow, first, cnt);
            // newest member first: along a trajectory the members nearest a
            // later query come last, and keys arriving in ascending order
            // make the sorted insertion an append
            auto consider = [&](const float4 &p, float d, int id) {
                if (p.w < c.T32 && d <= tau) {
                    const unsigned long long key = pack_key(d, id);
                    if (key < tauk) {
                        tauk = lane_push(K, Lw, nv, key);
                        tau = key_d(tauk);
                    }
                }
            };
            int j = cnt - 1;
            // four members per step: their loads and distance chains overlap
            for (; j >= 3; j -= 4) {
                const float4 pa = pbuf[j], pb = pbuf[j - 1], pc = pbuf[j - 2], pd = pbuf[j - 3];
                const float da = dist32(c, s0, s1, s2, s3, pa), db = dist32(c, s0, s1, s2, s3, pb);
                const float dc = dist32(c, s0, s1, s2, s3, pc), dd = dist32(c, s0, s1, s2, s3, pd);
                consider(pa, da, first + j);
                consider(pb, db, first + j - 1);
                consider(pc, dc, first + j - 2);
                consider(pd, dd, first + j - 3);
            }
            for (; j >= 0; --j) {
                const float4 p = pbuf[j];
                consider(p, dist32(c, s0, s1, s2, s3, p), first + j);
            }
        };
        auto scan_chunk = [&](unsigned any, unsigned need) {
            if (!any)
                return;
            SegPoints cur, nxt;
            int i = 31 - __clz(any);
            any &= ~(1u << i);
            seg_points_load(cur, pts, segbuf[4 * i + 3], lane);
            for (;;) {
                int inx = -1;
                if (any) {
                    inx = 31 - __clz(any);
                    any &= ~(1u << inx);
                    seg_points_load(nxt, pts, segbuf[4 * inx + 3], lane);
                }
                __syncwarp();
                seg_points_store(cur, pbuf, lane);
                __syncwarp();
                scan_pbuf(cur.first, cur.cnt, (need >> i) & 1u);
                if (inx < 0)
                    break;
                cur = nxt;
                i = inx;
            }
        };

        float bl[TNN_GMAX_F];
        int bp[TNN_GMAX_F];
#pragma unroll
        for (int f = 0; f < TNN_GMAX_F; ++f) {
            bl[f] = INFINITY;
            bp[f] = -1;
        }
        float wF = INFINITY;
        int nu = 0;

        // Records of up to 32 segments into segbuf (lane j loads gseg[src_j]);
        // returns this lane's segment position in the t_A order.
        auto load_records = [&](int src, bool have) -> int {
            __syncwarp();
            int mypos = -1;
            if (have) {
                const float4 *r = G.gseg + 4 * (size_t)src;
                segbuf[4 * lane] = __ldg(r);
                segbuf[4 * lane + 1] = __ldg(r + 1);
                segbuf[4 * lane + 2] = __ldg(r + 2);
                const float4 r3 = __ldg(r + 3);
                segbuf[4 * lane + 3] = r3;
                mypos = __float_as_int(r3.z);
            }
            __syncwarp();
            return mypos;
        };
        // Seed selection over the cnt staged segments: every lane keeps its F
        // smallest cylinder bounds.
        auto seed_pick = [&](int cnt, int mypos) {
            for (int i = 0; i < cnt; ++i) {
                const int pos = __shfl_sync(FULLMASK, mypos, i);
                const float lb = seg_lb(c, s3, segbuf[4 * i], segbuf[4 * i + 1], segbuf[4 * i + 2]);
                if (active && lb < wF) {
                    float cur = lb;
                    int cp = pos;
#pragma unroll
                    for (int f = 0; f < TNN_GMAX_F; ++f) {
                        if (f < F && cur < bl[f]) {
                            const float tf = bl[f];
                            bl[f] = cur;
                            cur = tf;
                            const int tp = bp[f];
                            bp[f] = cp;
                            cp = tp;
                        }
                    }
#pragma unroll
                    for (int f = 0; f < TNN_GMAX_F; ++f)
                        if (f == F - 1)
                            wF = bl[f];
                }
            }
            if (active)
                st.lb += cnt;
        };

        // Main mode over the member segments [lo, hi) (key order) of one key:
        // scan those whose bound allows.
        auto visit = [&](int lo, int hi) {
            for (int base = lo; base < hi; base += 32) {
                const int cnt = min(32, hi - base);
                const int mypos = load_records(base + lane, lane < cnt);
                {
                    bool sd = false;
                    if (lane < cnt)
                        for (int u = 0; u < nu; ++u)
                            sd |= ulist[u] == mypos;
                    const unsigned smask = __ballot_sync(FULLMASK, sd);
                    unsigned need = 0;
                    if (!done) {
#pragma unroll 4
                        for (int i = 0; i < cnt; ++i) {
                            const float lb = seg_lb(c, s3, segbuf[4 * i], segbuf[4 * i + 1],
                                                    segbuf[4 * i + 2]);
                            if (lb <= tau)
                                need |= 1u << i;
                        }
                        need &= ~smask;
                        st.lb += cnt;
                    }
                    scan_chunk(__reduce_or_sync(FULLMASK, need), need);
                }
            }
        };

        // ---- seeds: 3 x 3 cells around the warp, two most recent buckets
        if (bhi >= 0) {
            const int hx = min(max((int)floorf((0.5f * (bx0 + bx1) - G.x0) * G.inv_cell), 0), G.nx - 1);
            const int hy = min(max((int)floorf((0.5f * (by0 + by1) - G.y0) * G.inv_cell), 0), G.ny - 1);
            // lanes 0..9 TNN_SEED_BUCKETS - 1 hold the 3 x 3 cells of the
            // newest buckets bhi, bhi - 1, ...; the member segments of all
            // those keys are staged 32 at a time
            const int bq = bhi - lane / 9, cl = lane % 9;
            const int cx = hx + cl % 3 - 1, cy = hy + cl / 3 - 1;
            const bool ok = lane < 9 * TNN_SEED_BUCKETS && bq >= 0 && cx >= 0 && cx < G.nx && cy >= 0 &&
                            cy < G.ny;
            int lo = 0, n = 0;
            if (ok) {
                const int key = bq * G.ncell + cy * G.nx + cx;
                lo = __ldg(goff + key);
                n = __ldg(goff + key + 1) - lo;
            }
            int inc = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULLMASK, inc, o);
                if (lane >= o)
                    inc += v;
            }
            const int total = __shfl_sync(FULLMASK, inc, 31);
            const int rel = lo - (inc - n); // record index = rel_j + position in the batch
            for (int base = 0; base < total; base += 32) {
                const int t = base + lane;
                int src = 0;
#pragma unroll
                for (int j = 0; j < 9 * TNN_SEED_BUCKETS; ++j) {
                    const int ij = __shfl_sync(FULLMASK, inc, j);
                    const int rj = __shfl_sync(FULLMASK, rel, j);
                    if (src == 0 && t < ij)
                        src = rj + t + 1; // +1 keeps 0 as "unset"
                }
                const int cnt = min(32, total - base);
                const int mypos = load_records(src - 1, lane < cnt);
                seed_pick(cnt, mypos);
            }
        }

        // ---- scan the union of the seeds (highest position first)
        {
            auto next_seed = [&]() {
                int mm = -1;
#pragma unroll
                for (int f = 0; f < TNN_GMAX_F; ++f)
                    mm = max(mm, bp[f]);
                return __reduce_max_sync(FULLMASK, mm);
            };
            int pos = next_seed();
            SegPoints cur, nxt;
            if (pos >= 0)
                seg_points_load(cur, pts, __ldg(seg + 4 * (size_t)pos + 3), lane);
            while (pos >= 0 && nu < TNN_UCAP) {
#pragma unroll
                for (int f = 0; f < TNN_GMAX_F; ++f)
                    if (bp[f] == pos)
                        bp[f] = -1;
                if (lane == 0)
                    ulist[nu] = pos;
                ++nu;
                const int npos = nu < TNN_UCAP ? next_seed() : -1;
                if (npos >= 0)
                    seg_points_load(nxt, pts, __ldg(seg + 4 * (size_t)npos + 3), lane);
                __syncwarp();
                seg_points_store(cur, pbuf, lane);
                __syncwarp();
                scan_pbuf(cur.first, cur.cnt, active);
                cur = nxt;
                pos = npos;
            }
        }
        __syncwarp();

        // ---- a lane whose key is still above the deferral threshold (far
        // neighbours, or a list not yet full) would make the whole tile visit
        // a wide region: it is handed to the warp-per-query kernel instead
        const bool deferred = active && !(tau <= W->tau_defer);
        if (deferred) {
            const unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
            if (slot < (unsigned long long)L.fb_cap) {
                L.fb_list[slot] = make_int2(window_id(L, W), (int)qrow);
                L.fb_tau[slot] = tau;
            } else
                atomicOr(&L.scr->status, 1u);
        }

        // ---- main: buckets backwards, cells within reach, keys by bound
        for (int b = bhi; b >= 0; --b) {
            done = !active || deferred || !(time_lb(c, s3, __ldg(G.bpm + b)) <= tau);
            if (__all_sync(FULLMASK, done))
                break;
            const float tmx = warp_maxf(done ? 0.0f : tau);
            int cx0 = 0, cx1 = G.nx - 1, cy0 = 0, cy1 = G.ny - 1;
            if (tmx < INFINITY) {
                // any key outside this reach has a bound above every key
                const float R = sqrtf(tmx) * (1.0f + 0x1p-18f) + ext_max + dmax;
                reach_cells(bx0, bx1, R, G.x0, G.inv_cell, G.nx, cx0, cx1);
                reach_cells(by0, by1, R, G.y0, G.inv_cell, G.ny, cy0, cy1);
            }
            const int kb = b * G.ncell;
            for (int cy = cy0; cy <= cy1; ++cy) {
                const float ry0 = G.y0 + (float)cy * G.cell, ry1 = ry0 + G.cell;
                for (int cxb = cx0; cxb <= cx1; cxb += 32) {
                    const int cx = cxb + lane;
                    int lo = 0, hi = 0;
                    float ex = 0.f, tk = 0.f;
                    if (cx <= cx1) {
                        const int key = kb + cy * G.nx + cx;
                        const int4 kr = __ldg(G.krec + key);
                        lo = kr.x;
                        hi = kr.y;
                        ex = __int_as_float(kr.z);
                        tk = __int_as_float(kr.w);
                    }
                    unsigned m = __ballot_sync(FULLMASK, hi > lo);
                    while (m) {
                        const int j = __ffs(m) - 1;
                        m &= m - 1;
                        const int jlo = __shfl_sync(FULLMASK, lo, j);
                        const int jhi = __shfl_sync(FULLMASK, hi, j);
                        const float jex = __shfl_sync(FULLMASK, ex, j);
                        const float jtk = __shfl_sync(FULLMASK, tk, j);
                        const float rx0 = G.x0 + (float)(cxb + j) * G.cell, rx1 = rx0 + G.cell;
                        const bool want = !done && cell_lb(c, s3, rx0, rx1, ry0, ry1, jex, jtk) <= tau;
                        if (__any_sync(FULLMASK, want))
                            visit(jlo, jhi);
                    }
                }
            }
        }

        // ---- settle and write
        __syncwarp();
        if (active)
            st.q++;
        if (active && !deferred) {
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st)) {
                const unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
                if (slot < (unsigned long long)L.fb_cap) // unsettled: -1 - window
                    L.fb_list[slot] = make_int2(-1 - window_id(L, W), (int)qrow);
                else
                    atomicOr(&L.scr->status, 1u);
            }
        }
        __syncwarp();
        if (MIRROR) {
            const int cnt = __popc(__ballot_sync(FULLMASK, active));
            if (cnt > 0)
                mirror_tile(L, W, __shfl_sync(FULLMASK, qrow, 0), cnt, lane);
        }
    }
    flush_stats(L.scr, st);
}
