// TNN search kernel (Sec. 3.5: Algorithm 1 bounds, Algorithm 2 search).
//
// One warp answers a tile of 32 queries, one per lane; segment records and
// member points are staged in shared memory and read by every lane as
// broadcasts.  Per tile:
//
//   pass 1  bounds only, walking the t_A order backwards from the warp's
//           causal end in chunks of 32: every lane keeps its F smallest
//           cylinder bounds; the pass ends when the temporal bound of every
//           remaining segment (running maximum of t_B) exceeds the F-th
//           smallest.  These are the F nearest segments Algorithm 2 fetches
//           first.  Every segment whose bound did not exceed RHO times the
//           lane's running F-th smallest is recorded (warp union, in order).
//   pass 2  the union of the warp's seeds is scanned by all lanes, which
//           fills every candidate list and tightens the pruning key.
//   pass 3  the exclusion criterion: a segment is scanned for a lane only if
//           its bound does not exceed that lane's pruning key (the largest
//           key of its full candidate list); seeds are skipped.  When every
//           lane's key is at most RHO times its final F-th smallest bound,
//           any segment pass 1 did not record is already excluded (its bound
//           exceeded RHO times a value that only decreased), so only the list is
//           visited; otherwise the table is walked again, backwards, until
//           the temporal bound of every remaining segment exceeds the key
//           (Algorithm 2's stop rule).
//
// Global loads are software-pipelined: the records of the next chunk and
// the points of the next segment are loaded into registers while the
// current ones are processed.
#pragma once
#include "tnn_device.cuh"

#define TNN_FMAX 6
// Pass 1 records every segment whose bound is at most TNN_RHO times the
// lane's running F-th smallest bound.
#define TNN_RHO 4.0f

#ifndef TNN_MINB
#define TNN_MINB 3 // resident CTAs per SM the register allocation targets
#endif

// MIRROR: also copy each finished tile's rows to KnnLaunch::mirror_idx /
// mirror_d2 (a separate instantiation, so that the plain search compiles
// without that code).
template <bool MIRROR>
__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32, TNN_MINB)
    k_tnn_search(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const size_t pw = smem_per_warp(L.L_max, L.kseg_max, SMEM_SWEEP);
    unsigned char *ws = smem + (threadIdx.x >> 5) * pw;
    unsigned long long *K = (unsigned long long *)ws + lane;
    unsigned char *rest = ws + (size_t)L.L_max * 256;
    float4 *segbuf = (float4 *)rest;                     // [32][4]
    float4 *pbuf = (float4 *)(rest + 2048);              // [kseg_max]
    int *ulist = (int *)(rest + 2048 + 16 * L.kseg_max); // [TNN_UCAP] seeds
    int *wlist = ulist + TNN_UCAP;                       // [TNN_WCAP] pass 1
    unsigned long long *cl_d = (unsigned long long *)rest + lane; // settlement
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
        const float *__restrict__ segPM = W->segPM;
        const int Lw = W->L, F = W->F;
        const int cap1 = W->W0 > 0 ? W->W0 : 0x7fffffff;

        float tmax = c.T32;
        for (int o = 16; o > 0; o >>= 1)
            tmax = fmaxf(tmax, __shfl_xor_sync(FULLMASK, tmax, o));
        const float *__restrict__ segTA = W->segTA;
        const int hi = warp_count_less([&](int p) { return __ldg(segTA + p); }, W->S, tmax, lane);

        for (int i = 0; i < Lw; ++i)
            K[i * 32] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY;

        float4 r0, r1, r2, r3; // this lane's record of the next chunk
        auto chunk_load = [&](int c0, int cnt) {
            if (lane < cnt) {
                const float4 *src = seg + 4 * (size_t)(c0 + lane);
                r0 = __ldg(src);
                r1 = __ldg(src + 1);
                r2 = __ldg(src + 2);
                r3 = __ldg(src + 3);
            }
        };
        auto chunk_load_list = [&](const int *lst, int c0, int cnt) {
            if (lane < cnt) {
                const float4 *src = seg + 4 * (size_t)lst[c0 + lane];
                r0 = __ldg(src);
                r1 = __ldg(src + 1);
                r2 = __ldg(src + 2);
                r3 = __ldg(src + 3);
            }
        };
        auto chunk_store = [&](int cnt) {
            if (lane < cnt) {
                segbuf[4 * lane] = r0;
                segbuf[4 * lane + 1] = r1;
                segbuf[4 * lane + 2] = r2;
                segbuf[4 * lane + 3] = r3;
            }
        };
        // Distances from this lane's query to the points staged in pbuf.
        auto scan_pbuf = [&](int first, int cnt, bool need) {
            if (!need)
                return;
            st.segs++;
            st.pairs += cnt;
            for (int j = 0; j < cnt; ++j) {
                const float4 p = pbuf[j];
                const float d = dist32(c, s0, s1, s2, s3, p);
                if (p.w < c.T32 && d <= tau) {
                    const unsigned long long key = pack_key(d, first + j);
                    if (key < tauk) {
                        tauk = lane_push(K, Lw, nv, key);
                        tau = key_d(tauk);
                    }
                }
            }
        };
        // Scan the segments of segbuf selected by the warp mask `any`
        // (highest slot first) for the lanes whose `need` bit is set.
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
        __syncwarp();

        // ---- pass 1: the F smallest bounds of every lane
        float bl[TNN_FMAX];
        int bp[TNN_FMAX];
#pragma unroll
        for (int f = 0; f < TNN_FMAX; ++f) {
            bl[f] = INFINITY;
            bp[f] = -1;
        }
        float wF = INFINITY;
        int nw = 0;          // segments recorded (may exceed TNN_WCAP)
        bool complete = true; // pass 1 was not cut by the seed window
        int p1_end = -1;      // this lane's bounds were taken down to here
        {
            int pos_hi = hi, seen = 0;
            if (pos_hi > 0)
                chunk_load(pos_hi > 32 ? pos_hi - 32 : 0, pos_hi > 32 ? 32 : pos_hi);
            while (pos_hi > 0) {
                if (seen >= cap1) {
                    complete = false;
                    break;
                }
                const int c0 = pos_hi > 32 ? pos_hi - 32 : 0;
                const int cnt = pos_hi - c0;
                const bool done = !active || !(time_lb(c, s3, __ldg(segPM + pos_hi - 1)) <= wF);
                if (done && p1_end < 0)
                    p1_end = pos_hi; // stays done: segPM only falls below
                if (__all_sync(FULLMASK, done))
                    break;
                __syncwarp();
                chunk_store(cnt);
                __syncwarp();
                if (c0 > 0)
                    chunk_load(c0 > 32 ? c0 - 32 : 0, c0 > 32 ? 32 : c0);
                // bounds of 4 segments at a time (independent chains), then
                // the bookkeeping in descending position order
                for (int i0 = cnt - 1; i0 >= 0; i0 -= 4) {
                    float lbv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 - u;
                        lbv[u] = (done || i < 0)
                                     ? __int_as_float(0x7fffffff)
                                     : seg_lb(c, s3, segbuf[4 * max(i, 0)], segbuf[4 * max(i, 0) + 1],
                                              segbuf[4 * max(i, 0) + 2]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 - u;
                        if (i < 0)
                            break;
                        const float lb = lbv[u];
                        const bool keep = lb <= TNN_RHO * wF;
                        if (__any_sync(FULLMASK, keep)) {
                            if (lane == 0 && nw < TNN_WCAP)
                                wlist[nw] = c0 + i;
                            ++nw;
                        }
                        if (lb < wF) {
                            float cur = lb;
                            int cp = c0 + i;
#pragma unroll
                            for (int f = 0; f < TNN_FMAX; ++f) {
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
                            for (int f = 0; f < TNN_FMAX; ++f)
                                if (f == F - 1)
                                    wF = bl[f];
                        }
                    }
                }
                if (!done)
                    st.lb += cnt;
                seen += cnt;
                pos_hi = c0;
            }
            if (p1_end < 0)
                p1_end = pos_hi;
        }

        // ---- pass 2: scan the union of the seeds, highest position first
        int nu = 0;
        {
            auto next_seed = [&]() {
                int mm = -1;
#pragma unroll
                for (int f = 0; f < TNN_FMAX; ++f)
                    mm = max(mm, bp[f]);
                return __reduce_max_sync(FULLMASK, mm);
            };
            int pos = next_seed();
            SegPoints cur, nxt;
            if (pos >= 0)
                seg_points_load(cur, pts, __ldg(seg + 4 * (size_t)pos + 3), lane);
            while (pos >= 0 && nu < TNN_UCAP) {
#pragma unroll
                for (int f = 0; f < TNN_FMAX; ++f)
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

        // ---- pass 3: exclusion criterion and stop rule
        // The list suffices when every segment it lacks is excluded for
        // every lane: those pass 1 bounded for the lane and did not record
        // have a bound above RHO times the lane's final F-th smallest (so
        // above its key when the key is at most that), and those below where
        // the lane's pass ended have a temporal bound at least that of the
        // running maximum of t_B there, which must then exceed the key as
        // well (the pass ended when it exceeded the F-th smallest bound,
        // which the key can pass when every bound shares a large temporal
        // part, e.g. under a long lag).
        const bool beyond = p1_end == 0 || !(time_lb(c, s3, __ldg(segPM + p1_end - 1)) <= tau);
        const bool list_mode = complete && nw <= TNN_WCAP &&
                               __all_sync(FULLMASK, !active || (tau <= TNN_RHO * wF && beyond));
        if (list_mode) {
            int up = 0;
            if (nw > 0)
                chunk_load_list(wlist, 0, nw > 32 ? 32 : nw);
            for (int b = 0; b < nw; b += 32) {
                const int cnt = nw - b > 32 ? 32 : nw - b;
                __syncwarp();
                chunk_store(cnt);
                __syncwarp();
                if (b + 32 < nw)
                    chunk_load_list(wlist, b + 32, nw - b - 32 > 32 ? 32 : nw - b - 32);
                // positions of this chunk are wlist[b .. b+cnt), descending
                unsigned smask = 0;
                for (int i = 0; i < cnt; ++i) {
                    const int pos = wlist[b + i];
                    while (up < nu && ulist[up] > pos)
                        ++up;
                    if (up < nu && ulist[up] == pos)
                        smask |= 1u << i;
                }
                unsigned need = 0;
                if (active) {
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
        } else {
            int pos_hi = hi, up = 0;
            if (pos_hi > 0)
                chunk_load(pos_hi > 32 ? pos_hi - 32 : 0, pos_hi > 32 ? 32 : pos_hi);
            while (pos_hi > 0) {
                const int c0 = pos_hi > 32 ? pos_hi - 32 : 0;
                const int cnt = pos_hi - c0;
                const bool done = !active || !(time_lb(c, s3, __ldg(segPM + pos_hi - 1)) <= tau);
                if (__all_sync(FULLMASK, done))
                    break;
                __syncwarp();
                chunk_store(cnt);
                __syncwarp();
                if (c0 > 0)
                    chunk_load(c0 > 32 ? c0 - 32 : 0, c0 > 32 ? 32 : c0);
                unsigned smask = 0;
                while (up < nu && ulist[up] >= c0) {
                    if (ulist[up] < pos_hi)
                        smask |= 1u << (ulist[up] - c0);
                    ++up;
                }
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
                pos_hi = c0;
            }
        }

        // ---- settle and write
        __syncwarp();
        if (active) {
            st.q++;
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st)) {
                const unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
                if (slot < (unsigned long long)L.fb_cap)
                    L.fb_list[slot] = make_int2(-1 - window_id(L, W), (int)qrow); // unsettled
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
