// TNN with the candidate distances on the tensor cores (TNN_FLAG_TC_TILES):
// Algorithm 2's search over the time-bucketed grid, with the point
// distances of the fetched segments formed as 128 x 128 tiles by tcgen05
// (TF32 operands, FP32 accumulation in TMEM) and screened with the certified
// margin of the linear search (tnn_linear_tc.cuh); only the points that pass
// are scored again with the exact FP32 distance, so keys, lists and the FP64
// settlement are those of the other kernels.
//
// A CTA answers 128 consecutive queries (thread t of warps 0-3 = query t =
// TMEM lane t).  The index keeps the points in grid-key order (every key's
// members contiguous, runs padded to a multiple of 4 points), so keys that
// follow each other in key order are one contiguous run of points.
//   seed    every query scans, on its own thread in FP32, the F segments of
//           smallest cylinder bound among the 3 x 3 cells around the CTA in
//           the two most recent buckets (Algorithm 2's first fetch); this
//           fills its list, so the screen has a finite threshold from the
//           first tile on.  A query whose key is still beyond the deferral
//           radius goes to the warp-per-query kernel, as in the tile kernel.
//   main    buckets from the causal end backwards while the temporal bound of
//           some query's bucket stays within its key (the stop rule); in each
//           bucket, the keys within reach of the CTA whose bound against the
//           CTA's box (cell rectangle, extent, largest t_B) does not exceed
//           the largest key of its queries are merged into runs of points and
//           streamed 128 points at a time (TMA bulk copies into a ring), one
//           tcgen05.mma per tile, and every query screens its accumulator row.
//           The threshold in each query's operand row is its key when the
//           row is written, never below the key used to accept a point.
// Points of a query's own seed segments are not inserted twice; padding
// points (index -1) and points not strictly before the query are skipped
// when scored again.
#pragma once
#include "tnn_device.cuh"
#include "tnn_grid.cuh"
#include "tnn_tc.cuh"

#define TT_Q 128
#define TT_P 128
#define TT_S 8         // ring slots
#define TT_THREADS 160 // 4 screening warps + 1 control warp
#define TT_RMAX 256    // runs of points per pass

#define TT_OFF_A 0                              // [2][128 x 8] TF32
#define TT_OFF_B (TT_OFF_A + 8192)              // [2][128 x 8] TF32
#define TT_OFF_RAW (TT_OFF_B + 8192)            // [TT_S][128] float4
#define TT_OFF_IDX (TT_OFF_RAW + TT_S * 2048)   // [TT_S][128] int32
#define TT_OFF_BAR (TT_OFF_IDX + TT_S * 512)    // barriers + CTA scalars (512 B)
#define TT_OFF_SEG (TT_OFF_BAR + 512)           // [128][4] float4 seed records
#define TT_OFF_TMP (TT_OFF_SEG + 8192)          // [32] int2 runs of one batch of keys
#define TT_OFF_ROWS (TT_OFF_TMP + 256)          // [TT_RMAX] int4 runs of points
#define TT_OFF_LIST (TT_OFF_ROWS + TT_RMAX * 16) // [L][128] keys

#define TT_BAR_RAW 0
#define TT_BAR_BFULL TT_S
#define TT_BAR_ACC (TT_S + 2)
#define TT_BAR_USED (TT_S + 4)
#define TT_BAR_END (TT_BAR_USED + TT_S)

__host__ __device__ inline size_t tt_smem_bytes(int L_max)
{
    return TT_OFF_LIST + (size_t)L_max * TT_Q * 8;
}

// Chunk i of the pass: its run of points [lo, hi) in key order.  `cur` is
// the caller's row cursor (chunk indices asked for never decrease).
__device__ __forceinline__ void tt_chunk(const int4 *rows, int nrows, int i, int &cur, int &lo, int &hi)
{
    while (cur + 1 < nrows && rows[cur + 1].z <= i)
        ++cur;
    const int4 r = rows[cur];
    lo = r.x + (i - r.z) * TT_P;
    hi = min(r.y, lo + TT_P);
}

__device__ __forceinline__ void tt_load_chunk(const float4 *pk, const int32_t *ik, int lo, int hi, uint32_t raw_s,
                                              uint32_t idx_s, uint32_t bar)
{
    // lo is a multiple of 4 (runs start on 4-point boundaries and advance by
    // 128); sizes are multiples of 16 B (idx_k holds 4 entries of padding)
    const uint32_t np = (uint32_t)(hi - lo);
    const uint32_t ni = (np + 3u) & ~3u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(np * 16u + ni * 4u)
                 : "memory");
    tma_copy_1d(raw_s, pk + lo, np * 16u, bar);
    tma_copy_1d(idx_s, ik + lo, ni * 4u, bar);
}

__global__ void __launch_bounds__(TT_THREADS, 1) k_tnn_tc(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool ctrl = warp == 4;
    const int tq = t & (TT_Q - 1);
    unsigned char *sA = smem + TT_OFF_A;
    unsigned char *sB = smem + TT_OFF_B;
    float4 *raw = (float4 *)(smem + TT_OFF_RAW);
    const int32_t *sidx = (const int32_t *)(smem + TT_OFF_IDX);
    const uint32_t bar0 = su32(smem + TT_OFF_BAR);
    unsigned char *sc = smem + TT_OFF_BAR + 8 * TT_BAR_END;
    uint32_t *tmem_slot = (uint32_t *)(sc + 0);
    volatile int *s_err = (volatile int *)(sc + 4);
    long long *s_tile = (long long *)(sc + 8);
    int *s_nrows = (int *)(sc + 16);
    int *s_nch = (int *)(sc + 20);
    float *s_red = (float *)(sc + 32); // [4 warps][16]
    float4 *sseg = (float4 *)(smem + TT_OFF_SEG);
    int *kst = (int *)(smem + TT_OFF_ROWS);      // seed keys: exclusive starts [32]
    int *klo = (int *)(smem + TT_OFF_ROWS) + 32; //            their first record [32]
    int2 *tmp = (int2 *)(smem + TT_OFF_TMP);
    int4 *rows = (int4 *)(smem + TT_OFF_ROWS);
    int *s_kc = (int *)(sc + 24); // key cursor of the bucket's rectangle
    unsigned long long *K = (unsigned long long *)(smem + TT_OFF_LIST) + tq;
    unsigned long long *cl_d = (unsigned long long *)(smem + TT_OFF_A + (warp & 3) * 3072) + lane;
    int *cl_i = (int *)(smem + TT_OFF_A + (warp & 3) * 3072 + CMAX * 32 * 8) + lane;
#define BAR(i) (bar0 + 8u * (uint32_t)(i))

    if (t == 0) {
        for (int b = 0; b < TT_S; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(BAR(TT_BAR_RAW + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(BAR(TT_BAR_USED + b)));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(BAR(TT_BAR_BFULL + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(BAR(TT_BAR_ACC + b)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
    }
    if (ctrl) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(2 * TT_P));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr_row = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TT_P >> 3) << 17) |
                           ((uint32_t)(TT_Q >> 4) << 24);
    LaneStats st = {0, 0, 0, 0, 0};
    const KnnWin *W = &L.w0;
    const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
    const float q0 = W->ssq[0], q1 = W->ssq[1], q2 = W->ssq[2], q3 = sqrtf(s3);
    const GridDesc &G = W->grid;
    const float4 *__restrict__ pk = W->pts_k;
    const int32_t *__restrict__ ik = W->idx_k;
    const int32_t *__restrict__ ks = W->kp_start;
    const int Lw = W->L, F = W->F;
    const float ext_max = __ldg(G.ext_max);
    long long g = 0;         // chunks this CTA has processed (same in every thread)
    long long issued = -1;   // control thread: last chunk copied
    long long mma_last = -1; // control thread: last chunk multiplied

    for (;;) {
        if (t == 0)
            *s_tile = (long long)atomicAdd(&L.scr->tile_counter, 1ull);
        __syncthreads();
        const long long tile = *s_tile;
        if (tile >= L.total_tiles || *s_err)
            break;
        const int64_t qrow = tile * TT_Q + tq;
        const bool inq = !ctrl && qrow < W->m;
        const float4 q = inq ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, inq);

        // ---- CTA extents: scaled x, y (reach), raw x, y, z, t (operand
        // centre), largest causal end and slack
        {
            // minima of each value and of its negation (the maxima); a lane
            // without a query contributes the neutral +inf to both
            float v[16];
            v[0] = inq ? c.sx : INFINITY;
            v[1] = inq ? -c.sx : INFINITY;
            v[2] = inq ? c.sy : INFINITY;
            v[3] = inq ? -c.sy : INFINITY;
            v[4] = inq ? q.x : INFINITY;
            v[5] = inq ? -q.x : INFINITY;
            v[6] = inq ? q.y : INFINITY;
            v[7] = inq ? -q.y : INFINITY;
            v[8] = inq ? q.z : INFINITY;
            v[9] = inq ? -q.z : INFINITY;
            v[10] = inq ? q.w : INFINITY;
            v[11] = inq ? -q.w : INFINITY;
            v[12] = inq ? -c.T32 : INFINITY; // -max T32
            v[13] = inq ? -c.delta : 0.0f;   // -max delta
            v[14] = 0.f;
            v[15] = 0.f;
            if (!ctrl) {
#pragma unroll
                for (int i = 0; i < 14; ++i)
                    for (int o = 16; o > 0; o >>= 1)
                        v[i] = fminf(v[i], __shfl_xor_sync(FULLMASK, v[i], o));
                if (lane == 0)
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        s_red[warp * 16 + i] = v[i];
            }
        }
        __syncthreads();
        float ex[14];
#pragma unroll
        for (int i = 0; i < 14; ++i)
            ex[i] = fminf(fminf(s_red[i], s_red[16 + i]), fminf(s_red[32 + i], s_red[48 + i]));
        const float bx0 = ex[0], bx1 = -ex[1], by0 = ex[2], by1 = -ex[3];
        const float cc[4] = {0.5f * ex[4] - 0.5f * ex[5], 0.5f * ex[6] - 0.5f * ex[7], 0.5f * ex[8] - 0.5f * ex[9],
                             0.5f * ex[10] - 0.5f * ex[11]};
        const float tmax = -ex[12], dmax = -ex[13], tqmin = ex[10];
        int bhi = -1;
        {
            const float fb = (tmax - G.t0) * G.inv_dt;
            if (fb >= 0.0f)
                bhi = (int)fminf(floorf(fb), (float)(G.nb - 1));
        }
        if (!ctrl)
            for (int i = 0; i < Lw; ++i)
                K[i * TT_Q] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY;

        // ---- seed: the F segments of smallest bound in the 3 x 3 cells
        // around the CTA, two most recent buckets, each scanned by its query
        float bl[TNN_GMAX_F];
        int bf[TNN_GMAX_F], bc[TNN_GMAX_F];
#pragma unroll
        for (int f = 0; f < TNN_GMAX_F; ++f) {
            bl[f] = INFINITY;
            bf[f] = 0;
            bc[f] = 0;
        }
        float wF = INFINITY; // the F-th smallest bound so far
        if (bhi >= 0) {
            if (warp == 0) {
                const int hx = min(max((int)floorf((0.5f * (bx0 + bx1) - G.x0) * G.inv_cell), 0), G.nx - 1);
                const int hy = min(max((int)floorf((0.5f * (by0 + by1) - G.y0) * G.inv_cell), 0), G.ny - 1);
                const int bq = bhi - lane / 9, cl = lane % 9;
                const int cx = hx + cl % 3 - 1, cy = hy + cl / 3 - 1;
                const bool ok = lane < 18 && bq >= 0 && cx >= 0 && cx < G.nx && cy >= 0 && cy < G.ny;
                int lo = 0, n = 0;
                if (ok) {
                    const int key = bq * G.ncell + cy * G.nx + cx;
                    lo = __ldg(G.off + key);
                    n = __ldg(G.off + key + 1) - lo;
                }
                int inc = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULLMASK, inc, o);
                    if (lane >= o)
                        inc += v;
                }
                kst[lane] = inc - n;
                klo[lane] = lo;
                if (lane == 31)
                    *s_nrows = inc; // number of seed records
            }
            __syncthreads();
            const int total = *s_nrows;
            for (int base = 0; base < total; base += TT_Q) {
                const int cnt = min(TT_Q, total - base);
                if (!ctrl && tq < cnt) {
                    const int gidx = base + tq;
                    int j = 0;
                    while (j + 1 < 18 && kst[j + 1] <= gidx)
                        ++j;
                    const float4 *r = G.gseg + 4 * (size_t)(klo[j] + (gidx - kst[j]));
                    sseg[4 * tq] = __ldg(r);
                    sseg[4 * tq + 1] = __ldg(r + 1);
                    sseg[4 * tq + 2] = __ldg(r + 2);
                    sseg[4 * tq + 3] = __ldg(r + 3);
                }
                __syncthreads();
                if (inq) {
                    for (int i = 0; i < cnt; ++i) {
                        const float lb = seg_lb(c, s3, sseg[4 * i], sseg[4 * i + 1], sseg[4 * i + 2]);
                        if (lb < wF) {
                            float cur = lb;
                            int cf = __float_as_int(sseg[4 * i + 3].x), cn = __float_as_int(sseg[4 * i + 3].y);
#pragma unroll
                            for (int f = 0; f < TNN_GMAX_F; ++f) {
                                if (f < F && cur < bl[f]) {
                                    const float tl = bl[f];
                                    bl[f] = cur;
                                    cur = tl;
                                    const int tf = bf[f];
                                    bf[f] = cf;
                                    cf = tf;
                                    const int tc = bc[f];
                                    bc[f] = cn;
                                    cn = tc;
                                }
                            }
#pragma unroll
                            for (int f = 0; f < TNN_GMAX_F; ++f)
                                if (f == F - 1)
                                    wF = bl[f];
                        }
                    }
                    st.lb += cnt;
                }
                __syncthreads();
            }
        }
        if (inq) {
#pragma unroll
            for (int f = 0; f < TNN_GMAX_F; ++f) {
                if (f >= F || bc[f] == 0)
                    continue;
                st.segs++;
                st.pairs += bc[f];
                for (int j = 0; j < bc[f]; ++j) {
                    const float4 p = __ldg(W->pts + bf[f] + j);
                    const float d = dist32(c, s0, s1, s2, s3, p);
                    if (p.w < c.T32 && d <= tau) {
                        const unsigned long long key = pack_key(d, bf[f] + j);
                        if (key < tauk) {
                            tauk = list_push<TT_Q>(K, Lw, nv, key);
                            tau = key_d(tauk);
                        }
                    }
                }
            }
        }
        // a query whose key is still far leaves the tile
        const bool deferred = inq && !(tau <= W->tau_defer);
        if (deferred) {
            const unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
            if (slot < (unsigned long long)L.fb_cap) {
                L.fb_list[slot] = make_int2(0, (int)qrow);
                L.fb_tau[slot] = tau;
            } else
                atomicOr(&L.scr->status, 1u);
        }
        const bool active = inq && !deferred;

        // the fixed part of the query's operand row
        float arow[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (active) {
            const float f[4] = {q0 * (q.x - cc[0]), q1 * (q.y - cc[1]), q2 * (q.z - cc[2]), q3 * (q.w - cc[3])};
            float n2 = 0.f;
#pragma unroll
            for (int d = 0; d < 4; ++d)
                n2 = fmaf(f[d], f[d], n2);
            arow[0] = tf32_rna(f[0]);
            arow[1] = tf32_rna(f[1]);
            arow[2] = tf32_rna(f[2]);
            arow[3] = tf32_rna(f[3]);
            arow[4] = tf32_rna((1.0f - TC_EPS) * n2);
            arow[5] = 1.0f;
            arow[6] = tf32_rna(TC_EPS * sqrtf(n2));
        }

        // ---- main: buckets backwards, rows of cells within reach
        for (int b = bhi; b >= 0; --b) {
            const bool want = active && time_lb(c, s3, __ldg(G.bpm + b)) <= tau;
            if (!__syncthreads_or(want) || *s_err)
                break;
            // the largest key among the queries still searching
            float tm = active ? tau : 0.0f;
            if (!ctrl) {
                for (int o = 16; o > 0; o >>= 1)
                    tm = fmaxf(tm, __shfl_xor_sync(FULLMASK, tm, o));
                if (lane == 0)
                    s_red[warp * 16 + 14] = tm;
            }
            __syncthreads();
            tm = fmaxf(fmaxf(s_red[14], s_red[30]), fmaxf(s_red[46], s_red[62]));
            int cx0 = 0, cx1 = G.nx - 1, cy0 = 0, cy1 = G.ny - 1;
            if (tm < INFINITY) {
                const float R = sqrtf(tm) * (1.0f + 0x1p-18f) + ext_max + dmax;
                reach_cells(bx0, bx1, R, G.x0, G.inv_cell, G.nx, cx0, cx1);
                reach_cells(by0, by1, R, G.y0, G.inv_cell, G.ny, cy0, cy1);
            }
            if (cx0 > cx1 || cy0 > cy1) // the reach misses the grid (queries far outside it)
                continue;
            const int wx = cx1 - cx0 + 1, nkr = (cy1 - cy0 + 1) * wx;
            if (t == 0)
                *s_kc = 0;
            __syncthreads();
            for (;;) {
                // runs of the needed keys from the cursor on, at most TT_RMAX
                if (warp == 0) {
                    int kc = *s_kc, nr = 0, nc = 0;
                    int olo = -1, ohi = -1; // lane 0: the open run
                    while (kc < nkr && nr < TT_RMAX - 32) {
                        const int tk = kc + lane;
                        bool need = false;
                        int p0 = 0, p1 = 0;
                        if (tk < nkr) {
                            const int cy = cy0 + tk / wx, cx = cx0 + tk % wx;
                            const int key = b * G.ncell + cy * G.nx + cx;
                            const int4 kr = __ldg(G.krec + key);
                            if (kr.y > kr.x) {
                                // bound of the key against the CTA's box
                                const float rx0 = G.x0 + (float)cx * G.cell, ry0 = G.y0 + (float)cy * G.cell;
                                const float ddx = fmaxf(fmaxf(rx0 - bx1, bx0 - (rx0 + G.cell)), 0.0f);
                                const float ddy = fmaxf(fmaxf(ry0 - by1, by0 - (ry0 + G.cell)), 0.0f);
                                const float a2 = fmaf(ddy, ddy, ddx * ddx);
                                const float dist = a2 * rsqrtf(fmaxf(a2, 1e-37f));
                                const float sp = fmaxf(fmaf(dist, 1.0f - 0x1p-20f, -(__int_as_float(kr.z) + dmax)), 0.0f);
                                const float et = fmaxf(__fsub_rd(tqmin, fminf(__int_as_float(kr.w), tmax)), 0.0f);
                                const float lb = fmaf(sp, sp, (s3 * et) * et) * (1.0f - 0x1p-19f);
                                if (lb <= tm) {
                                    need = true;
                                    p0 = __ldg(ks + key);
                                    p1 = __ldg(ks + key + 1);
                                }
                            }
                        }
                        const unsigned m = __ballot_sync(FULLMASK, need && p1 > p0);
                        if (need && p1 > p0)
                            tmp[__popc(m & ((1u << lane) - 1u))] = make_int2(p0, p1);
                        __syncwarp();
                        if (lane == 0) {
                            // consecutive keys are contiguous runs: merge them
                            const int cnt = __popc(m);
                            for (int u = 0; u < cnt; ++u) {
                                const int2 r = tmp[u];
                                if (r.x == ohi) {
                                    ohi = r.y;
                                } else {
                                    if (olo >= 0) {
                                        const int nchr = (ohi - olo + TT_P - 1) / TT_P;
                                        rows[nr++] = make_int4(olo, ohi, nc, 0);
                                        nc += nchr;
                                    }
                                    olo = r.x;
                                    ohi = r.y;
                                }
                            }
                        }
                        __syncwarp();
                        nr = __shfl_sync(FULLMASK, nr, 0);
                        nc = __shfl_sync(FULLMASK, nc, 0);
                        kc += 32;
                    }
                    if (lane == 0) {
                        if (olo >= 0) {
                            rows[nr++] = make_int4(olo, ohi, nc, 0);
                            nc += (ohi - olo + TT_P - 1) / TT_P;
                        }
                        *s_nrows = nr;
                        *s_nch = nc;
                        *s_kc = min(kc, nkr);
                    }
                }
                __syncthreads();
                const int nrows = *s_nrows, nch = *s_nch, kdone = *s_kc;
                // every thread has read the counts before warp 0 may write
                // the next pass's
                __syncthreads();
                if (nch > 0) {
                    if (ctrl) {
                        // ---- control thread: copies and MMAs
                        if (lane == 0) {
                            int curp = 0;
                            const int pre = min(nch, TT_S - 2);
                            for (int j = 0; j < pre; ++j) {
                                const long long gj = g + j;
                                int lo, hi;
                                tt_chunk(rows, nrows, j, curp, lo, hi);
                                tt_load_chunk(pk, ik, lo, hi, su32(raw + (gj % TT_S) * TT_P),
                                              su32(sidx + (gj % TT_S) * TT_P), BAR(TT_BAR_RAW + gj % TT_S));
                                issued = gj;
                            }
                            for (int i = 0; i < nch; ++i) {
                                const long long gi = g + i;
                                const int bb = (int)(gi & 1);
                                if (!mbar_wait(BAR(TT_BAR_BFULL + bb), (uint32_t)((gi >> 1) & 1), s_err))
                                    break;
                                if (gi >= 2 && !mbar_wait(BAR(TT_BAR_USED + (gi - 2) % TT_S),
                                                          (uint32_t)(((gi - 2) / TT_S) & 1), s_err))
                                    break;
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                                const uint64_t da = umma_desc(su32(sA + bb * 4096));
                                const uint64_t db = umma_desc(su32(sB + bb * 4096));
                                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                             ::"r"(tmem + (uint32_t)(bb * TT_P)), "l"(da), "l"(db), "r"(idesc),
                                             "r"(0));
                                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                             ::"r"(BAR(TT_BAR_ACC + bb))
                                             : "memory");
                                mma_last = gi;
                                const int j = i + TT_S - 2;
                                if (j < nch) {
                                    const long long gj = g + j;
                                    int lo, hi;
                                    tt_chunk(rows, nrows, j, curp, lo, hi);
                                    tt_load_chunk(pk, ik, lo, hi, su32(raw + (gj % TT_S) * TT_P),
                                                  su32(sidx + (gj % TT_S) * TT_P), BAR(TT_BAR_RAW + gj % TT_S));
                                    issued = gj;
                                }
                            }
                        }
                    } else {
                        // ---- screening warps
                        int curb = 0, curs = 0;
                        auto build = [&](long long gi, int i) -> bool {
                            const int s = (int)(gi % TT_S), bb = (int)(gi & 1);
                            const bool okw = mbar_wait(BAR(TT_BAR_RAW + s), (uint32_t)((gi / TT_S) & 1), s_err);
                            if (!__all_sync(FULLMASK, okw))
                                return false;
                            int lo, hi;
                            tt_chunk(rows, nrows, i, curb, lo, hi);
                            float bv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                            if (tq < hi - lo) {
                                const float4 p = raw[s * TT_P + tq];
                                if (p.w < tmax) { // a point no query of the CTA may take keeps a zero row
                                    const float e[4] = {q0 * (p.x - cc[0]), q1 * (p.y - cc[1]), q2 * (p.z - cc[2]),
                                                        q3 * (p.w - cc[3])};
                                    float m2 = 0.f;
    #pragma unroll
                                    for (int d = 0; d < 4; ++d)
                                        m2 = fmaf(e[d], e[d], m2);
                                    bv[0] = tf32_rna(-2.0f * e[0]);
                                    bv[1] = tf32_rna(-2.0f * e[1]);
                                    bv[2] = tf32_rna(-2.0f * e[2]);
                                    bv[3] = tf32_rna(-2.0f * e[3]);
                                    bv[4] = 1.0f;
                                    bv[5] = tf32_rna((1.0f - TC_EPS) * m2);
                                    bv[6] = tf32_rna(-2.0f * sqrtf(m2));
                                    bv[7] = 1.0f;
                                }
                            }
                            store_row(sB + bb * 4096, tq, bv);
                            arow[7] = active ? tc_neg_T(tau) : 0.0f;
                            store_row(sA + bb * 4096, tq, arow);
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            __syncwarp();
                            if (lane == 0)
                                mbar_arrive(BAR(TT_BAR_BFULL + bb));
                            return true;
                        };
                        bool ok = build(g, 0);
                        for (int i = 0; ok && i < nch; ++i) {
                            const long long gi = g + i;
                            const int s = (int)(gi % TT_S), bb = (int)(gi & 1);
                            if (i + 1 < nch && !build(gi + 1, i + 1))
                                break;
                            const bool okw = mbar_wait(BAR(TT_BAR_ACC + bb), (uint32_t)((gi >> 1) & 1), s_err);
                            if (!__all_sync(FULLMASK, okw))
                                break;
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            int lo, hi;
                            tt_chunk(rows, nrows, i, curs, lo, hi);
                            const int ncol = hi - lo;
                            if (active)
                                st.pairs += ncol;
                            if (t == 0)
                                st.segs++; // 128 x 128 tiles multiplied
    #pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                uint32_t v[64];
                                tmem_ld32_nowait(taddr_row + (uint32_t)(bb * TT_P + h * 64), v);
                                tmem_ld32_nowait(taddr_row + (uint32_t)(bb * TT_P + h * 64 + 32), v + 32);
                                tmem_wait_ld();
                                uint32_t any = 0u;
    #pragma unroll
                                for (int j = 0; j < 64; ++j)
                                    any |= v[j];
                                const int lim = ncol - h * 64;
                                if ((int)any < 0 && lim > 0) {
                                    uint32_t m0 = 0u, m1 = 0u;
    #pragma unroll
                                    for (int j = 0; j < 32; ++j) {
                                        m0 |= (v[j] >> 31) << j;
                                        m1 |= (v[32 + j] >> 31) << j;
                                    }
                                    if (lim <= 32) {
                                        m1 = 0u;
                                        if (lim < 32)
                                            m0 &= (1u << lim) - 1u;
                                    } else if (lim < 64) {
                                        m1 &= (1u << (lim - 32)) - 1u;
                                    }
    #pragma unroll
                                    for (int part = 0; part < 2; ++part) {
                                        uint32_t msk = part ? m1 : m0;
                                        while (msk) {
                                            const int col = h * 64 + part * 32 + __ffs(msk) - 1;
                                            msk &= msk - 1u;
                                            const int j = sidx[s * TT_P + col];
                                            if (j < 0)
                                                continue; // padding
                                            bool seed = false;
    #pragma unroll
                                            for (int f = 0; f < TNN_GMAX_F; ++f)
                                                seed |= f < F && j >= bf[f] && j < bf[f] + bc[f];
                                            if (seed)
                                                continue; // scanned in the seed phase
                                            const float4 p = raw[s * TT_P + col];
                                            const float d = dist32(c, s0, s1, s2, s3, p);
                                            st.lb++; // screened points scored again in FP32
                                            if (p.w < c.T32 && d <= tau) {
                                                const unsigned long long key = pack_key(d, j);
                                                if (key < tauk) {
                                                    tauk = list_push<TT_Q>(K, Lw, nv, key);
                                                    tau = key_d(tauk);
                                                }
                                            }
                                        }
                                    }
                                }
                            }
                            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                            __syncwarp();
                            if (lane == 0)
                                mbar_arrive(BAR(TT_BAR_USED + s));
                        }
                    }
                    g += nch;
                }
                __syncthreads();
                if (kdone >= nkr || *s_err)
                    break;
            }
        }
        __syncthreads();
        if (*s_err)
            break;
        if (inq)
            st.q++;
        if (active) {
            list_sort<TT_Q>(K, nv);
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st, TT_Q)) {
                const unsigned fslot = atomicAdd(&L.scr->n_fallback, 1u);
                if (fslot < (unsigned long long)L.fb_cap)
                    L.fb_list[fslot] = make_int2(-1, (int)qrow); // unsettled, window 0
                else
                    atomicOr(&L.scr->status, 1u);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); // A, B, raw are refilled async
        __syncthreads();
    }
    if (*s_err && ctrl && lane == 0) {
        // a wait timed out: let the copies and the MMA still in flight land
        // (each wait bounded) before the memory they write is released
        atomicOr(&L.scr->status, 4u);
        for (long long gj = issued; gj >= 0 && gj > issued - TT_S; --gj)
            mbar_wait(BAR(TT_BAR_RAW + gj % TT_S), (uint32_t)((gj / TT_S) & 1), nullptr);
        if (mma_last >= 0)
            mbar_wait(BAR(TT_BAR_ACC + (mma_last & 1)), (uint32_t)((mma_last >> 1) & 1), nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (ctrl)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TT_P));
    else
        flush_stats(L.scr, st);
#undef BAR
}
