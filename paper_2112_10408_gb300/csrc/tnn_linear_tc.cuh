// Linear search on the tensor cores (Sec. 3.6: the linear search computes
// the distance matrix with the classic expansion |q|^2 + |p|^2 - 2 q.p,
// Table 1 "Distance Matrix").
//
// A CTA answers 128 queries (thread t of warps 0-3 = query t = TMEM lane t)
// over the time-ordered copy of the points, most recent first, 128 points per
// chunk.  The queries are taken in a space-time order (sorted key of x, y,
// t), so the 128 of a CTA are close together and share a short causal prefix.
// With c the centre of the CTA's queries, f = sqrt(sigma) (q - c) and
// e = sqrt(sigma) (p - c), the TF32 operand rows are
//     a = [f, (1 - 2 eps) |f|^2, 1, -T, 0]
//     b = [-2 e, 1, (1 - 2 eps) |e|^2, 1, 0]
// so that a . b = |f - e|^2 - 2 eps (|f|^2 + |e|^2) - T: the scaled squared
// distance, minus an error allowance that scales with the magnitudes that
// cancel, minus the query's current pruning threshold T.  A point can enter
// the query's list only where that value is negative.  The fixed part of a
// is written once per CTA tile; per chunk only its -T entry changes.
//
// Roles (warp specialisation, chained by mbarriers):
//   warp 4, one thread: TMA (cp.async.bulk) of raw 128-point chunks and
//     their input indices into a ring of TC_S slots, TC_S - 2 chunks ahead; one tcgen05.mma kind::tf32
//     (M = N = 128, K = 8) per chunk into one of two TMEM accumulators,
//     committed to an mbarrier;
//   warps 0-3: before the first chunk, score the 1,024 points nearest the
//     CTA's queries in space-time order (the index's Morton-ordered copy,
//     around the key of the CTA's middle query) on the CUDA cores; the L-th
//     smallest of those keys is an upper bound on the query's final L-th key,
//     so it becomes the admission bound of the list, which starts empty again
//     (those points come again in the scan).  The screen then works with a
//     threshold near the final one from the newest chunk on, instead of
//     letting through most points of the first chunks while the lists fill.
//   warps 0-3: write the B row and the -T entry of the A row of chunk i + 1
//     (one row each), then read their accumulator rows of chunk i
//     (tcgen05.ld), OR the bit patterns of the values in groups of 8 to find
//     the groups holding a negative one, and score only those points again
//     with the exact FP32 distance of the other kernels -- so candidate keys,
//     lists and the FP64 settlement are the same.  The MMA of chunk i + 1
//     runs while chunk i is screened.
// Soundness of the screen (a point whose FP32 distance is at most the k-th
// key must give a negative value): rounding every operand to TF32 (nearest)
// changes each product by at most 2^-10 |a_k b_k| and the FP32 sum of the 8
// exact products adds ~2^-20 of sum |a_k b_k| <= 2 (|f|^2 + |e|^2) + T;
// centring and scaling in FP32 move |f - e|^2 by < 2^-20 (|f|^2 + |e|^2) and
// the FP32 distance is within 2^-21 of the exact one.  The allowance
// 2 eps (|f|^2 + |e|^2) with eps = 2^-9 covers the distance terms twice over
// (it is at least eps (|f| + |e|)^2), and T = RNA_tf32(thr (1 + 2^-8) + 2^-100)
// exceeds the threshold by more than the error of its own term.
#pragma once
#include "tnn_device.cuh"
#include "tnn_tc.cuh"

#define TC_Q 128        // queries per CTA (TMEM lanes)
#define TC_P 128        // points per chunk (accumulator columns)
#define TC_S 16         // raw-point ring slots
#define TC_THREADS 160  // 4 screening warps + 1 control warp
#define TC_EPS 0x1p-9f
#ifndef TC_SEED_BATCHES
#define TC_SEED_BATCHES 8 // threshold seeds per CTA, in batches of 128 points
#endif

#define TC_OFF_A 0                            // [2][128 rows x 8] TF32, K-major
#define TC_OFF_B (TC_OFF_A + 8192)            // [2][128 rows x 8]
#define TC_OFF_RAW (TC_OFF_B + 8192)          // [TC_S][128] float4
#define TC_OFF_IDX (TC_OFF_RAW + TC_S * 2048) // [TC_S][128] int32 input index
#define TC_OFF_BAR (TC_OFF_IDX + TC_S * 512)  // mbarriers and CTA scalars (512 B)
#define TC_OFF_SEED (TC_OFF_BAR + 512)        // [128] float4 + [128] int32 threshold seeds
#define TC_OFF_LIST (TC_OFF_SEED + TC_P * 20) // [L][128] candidate keys
// the settlement scratch of the 4 warps (4 x 3 KB) reuses A and B once the
// tile's last MMA has completed

// mbarrier slots (8 B each) at TC_OFF_BAR
#define TC_BAR_RAW 0    // [TC_S] raw chunk landed (TMA transaction count)
#define TC_BAR_BFULL 16 // [2] A/B rows written (one arrival per warp)
#define TC_BAR_ACC 18   // [2] accumulator ready (tcgen05.commit)
#define TC_BAR_USED 20  // [TC_S] chunk screened (one arrival per warp)
#define TC_BAR_END (TC_BAR_USED + TC_S)

__host__ __device__ inline size_t tc_smem_bytes(int L_max)
{
    return TC_OFF_LIST + (size_t)L_max * TC_Q * 8;
}


// Byte offset of (row r, k) inside one 128-row x 8 TF32 operand: core
// matrices of 8 rows x 16 B, K-adjacent ones 128 B apart, row-group adjacent
// ones 256 B apart.
__device__ __forceinline__ uint32_t kmaj_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}








// Chunk i (0 = newest) of the causal prefix [0, hi): the 128-aligned block
// [c_lo, c_lo + 128) clipped to hi, so every copy starts on a 16-byte boundary.
__device__ __forceinline__ void tc_chunk(int hi, int i, int &c_lo, int &c_hi)
{
    c_lo = ((hi - 1) / TC_P - i) * TC_P;
    c_hi = min(hi, c_lo + TC_P);
}


// Chunk [c_lo, c_hi) of the time-ordered points and of their input indices
// into ring slot s; both copies complete on the slot's barrier.  c_lo is a
// multiple of 128 and sizes are multiples of 16 B: the index copy rounds up
// to 4 entries (idx_t holds 4 entries of padding).
__device__ __forceinline__ void tc_load_chunk(const float4 *pts_t, const int32_t *idx_t, int c_lo, int c_hi,
                                              uint32_t raw_s, uint32_t idx_s, uint32_t bar)
{
    const uint32_t np = (uint32_t)(c_hi - c_lo);
    const uint32_t ni = (np + 3u) & ~3u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(np * 16u + ni * 4u)
                 : "memory");
    tma_copy_1d(raw_s, pts_t + c_lo, np * 16u, bar);
    tma_copy_1d(idx_s, idx_t + c_lo, ni * 4u, bar);
}



// One operand row (8 TF32 values, already rounded) as two 16-byte stores.
__device__ __forceinline__ void store_row(unsigned char *base, int row, const float (&v)[8])
{
    *(float4 *)(base + kmaj_off(row, 0)) = make_float4(v[0], v[1], v[2], v[3]);
    *(float4 *)(base + kmaj_off(row, 4)) = make_float4(v[4], v[5], v[6], v[7]);
}

// -T for a pruning threshold thr (see the soundness note above).
__device__ __forceinline__ float tc_neg_T(float thr)
{
    return -tf32_rna(fmaf(thr, 0x1p-8f, thr) + 0x1p-100f);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_linear_tc(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[]; // no-swizzle operands need 16 B
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const bool ctrl = warp == 4;
    const int tq = t & (TC_Q - 1);
    unsigned char *sA = smem + TC_OFF_A;
    unsigned char *sB = smem + TC_OFF_B;
    float4 *raw = (float4 *)(smem + TC_OFF_RAW);
    const int32_t *sidx = (const int32_t *)(smem + TC_OFF_IDX);
    const uint32_t bar0 = su32(smem + TC_OFF_BAR);
    unsigned char *sc = smem + TC_OFF_BAR + 8 * TC_BAR_END;
    uint32_t *tmem_slot = (uint32_t *)(sc + 0);
    volatile int *s_err = (volatile int *)(sc + 4);
    long long *s_tile = (long long *)(sc + 8);
    int *s_hi = (int *)(sc + 16);
    float *s_wmax = (float *)(sc + 32); // [4]
    float *s_bb = (float *)(sc + 48);   // [4 warps][8]: min, max per axis
    int *s_seed = (int *)(sc + 176);    // first seed point (space order), -1: none
    float4 *seedp = (float4 *)(smem + TC_OFF_SEED);
    int32_t *seedi = (int32_t *)(smem + TC_OFF_SEED + TC_P * 16);
    unsigned long long *K = (unsigned long long *)(smem + TC_OFF_LIST) + tq;
    unsigned long long *cl_d = (unsigned long long *)(smem + TC_OFF_A + (warp & 3) * 3072) + lane;
    int *cl_i = (int *)(smem + TC_OFF_A + (warp & 3) * 3072 + CMAX * 32 * 8) + lane;
#define BAR(i) (bar0 + 8u * (uint32_t)(i))

    if (t == 0) {
        for (int b = 0; b < TC_S; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(BAR(TC_BAR_RAW + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(BAR(TC_BAR_USED + b)));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(BAR(TC_BAR_BFULL + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(BAR(TC_BAR_ACC + b)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
    }
    if (ctrl) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(2 * TC_P));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr_row = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // F32 accumulate, A = B = TF32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_P >> 3) << 17) |
                           ((uint32_t)(TC_Q >> 4) << 24);
    LaneStats st = {0, 0, 0, 0, 0};
    const KnnWin *W = &L.w0;
    const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
    const float q0 = W->ssq[0], q1 = W->ssq[1], q2 = W->ssq[2], q3 = sqrtf(s3);
    const float4 *__restrict__ pts_t = W->pts_t;
    const int32_t *__restrict__ idx_t = W->idx_t;
    const int Lw = W->L;
    long long g = 0;        // chunks this CTA has processed (same in every thread)
    long long issued = -1;  // control thread: last chunk copied
    long long mma_last = -1; // control thread: last chunk multiplied

    for (;;) {
        if (t == 0)
            *s_tile = (long long)atomicAdd(&L.scr->tile_counter, 1ull);
        __syncthreads();
        const long long tile = *s_tile;
        if (tile >= L.total_tiles || *s_err)
            break;
        const int64_t slot = tile * TC_Q + tq;
        const bool active = !ctrl && slot < W->m;
        const int64_t qrow = !active ? 0 : L.qorder ? (int64_t)(L.qorder[slot] & 0xffffffffull) : slot;
        const float4 q = active ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, active);

        // causal prefix of the CTA (points with t < max T32) and the bounding
        // box of its queries
        if (!ctrl) {
            float wm = c.T32;
            float bb[8] = {q.x, q.x, q.y, q.y, q.z, q.z, q.w, q.w};
            if (!active)
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    bb[2 * d] = INFINITY;
                    bb[2 * d + 1] = -INFINITY;
                }
            for (int o = 16; o > 0; o >>= 1) {
                wm = fmaxf(wm, __shfl_xor_sync(FULLMASK, wm, o));
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    bb[2 * d] = fminf(bb[2 * d], __shfl_xor_sync(FULLMASK, bb[2 * d], o));
                    bb[2 * d + 1] = fmaxf(bb[2 * d + 1], __shfl_xor_sync(FULLMASK, bb[2 * d + 1], o));
                }
            }
            if (lane == 0) {
                s_wmax[warp] = wm;
#pragma unroll
                for (int d = 0; d < 8; ++d)
                    s_bb[warp * 8 + d] = bb[d];
            }
        }
        __syncthreads();
        float cc[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            float lo = s_bb[2 * d], hi = s_bb[2 * d + 1];
            for (int w = 1; w < 4; ++w) {
                lo = fminf(lo, s_bb[w * 8 + 2 * d]);
                hi = fmaxf(hi, s_bb[w * 8 + 2 * d + 1]);
            }
            cc[d] = 0.5f * lo + 0.5f * hi; // a tile holds at least one query
        }
        if (t == 0) {
            const float tm = fmaxf(fmaxf(s_wmax[0], s_wmax[1]), fmaxf(s_wmax[2], s_wmax[3]));
            int lo = 0, hi = W->n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (pts_t[mid].w < tm)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            *s_hi = lo;
        }
        if (t == 32) { // warp 1: the seed window, beside thread 0's search
            int sl = -1;
            if (L.seed_code && L.qorder) {
                const int64_t mid = min((int64_t)(tile * TC_Q + TC_Q / 2), (int64_t)(W->m - 1));
                const uint32_t code = (uint32_t)(L.qorder[mid] >> 32);
                int lo = 0, hi = W->n;
                while (lo < hi) {
                    const int md = (lo + hi) >> 1;
                    if (L.seed_code[md] < code)
                        lo = md + 1;
                    else
                        hi = md;
                }
                sl = min(max(lo - TC_SEED_BATCHES * TC_P / 2, 0), max(W->n - TC_SEED_BATCHES * TC_P, 0));
            }
            *s_seed = sl;
        }
        // causal end of this query: the time-ordered points [0, hq) are the
        // ones with t < T32
        int hq = 0;
        if (active) {
            int hi2 = W->n;
            while (hq < hi2) {
                const int mid = (hq + hi2) >> 1;
                if (pts_t[mid].w < c.T32)
                    hq = mid + 1;
                else
                    hi2 = mid;
            }
        }
        // the fixed part of the query row (entry 6, -T, is written per chunk)
        float arow[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (active) {
            const float f[4] = {q0 * (q.x - cc[0]), q1 * (q.y - cc[1]), q2 * (q.z - cc[2]),
                                q3 * (q.w - cc[3])};
            float n2 = 0.f;
#pragma unroll
            for (int d = 0; d < 4; ++d)
                n2 = fmaf(f[d], f[d], n2);
            arow[0] = tf32_rna(f[0]);
            arow[1] = tf32_rna(f[1]);
            arow[2] = tf32_rna(f[2]);
            arow[3] = tf32_rna(f[3]);
            arow[4] = tf32_rna((1.0f - 2.0f * TC_EPS) * n2);
            arow[5] = 1.0f;
        }
        if (!ctrl)
            for (int i = 0; i < Lw; ++i)
                K[i * TC_Q] = SENT;
        __syncthreads();
        const int hi = *s_hi;
        const int nch = (hi + TC_P - 1) / TC_P;
        int nv = 0;
        unsigned long long tauk = SENT;
        unsigned long long bound0 = SENT; // no key at or above it can enter the list
        float tau = INFINITY;

        if (ctrl) {
            // ---- control thread: copies and MMAs
            if (lane == 0 && nch > 0) {
                const int pre = min(nch, TC_S - 2);
                for (int j = 0; j < pre; ++j) {
                    // the slot's previous chunk belongs to an earlier tile and
                    // was screened before the tile barrier
                    const long long gj = g + j;
                    int c_lo, c_hi;
                    tc_chunk(hi, j, c_lo, c_hi);
                    tc_load_chunk(pts_t, idx_t, c_lo, c_hi, su32(raw + (gj % TC_S) * TC_P),
                                  su32(sidx + (gj % TC_S) * TC_P), BAR(TC_BAR_RAW + gj % TC_S));
                    issued = gj;
                }
                for (int i = 0; i < nch; ++i) {
                    const long long gi = g + i;
                    const int b = (int)(gi & 1);
                    if (!mbar_wait(BAR(TC_BAR_BFULL + b), (uint32_t)((gi >> 1) & 1), s_err))
                        break;
                    // accumulator b and the raw slot of chunk gi - 2 are free
                    // once that chunk is screened
                    if (gi >= 2 && !mbar_wait(BAR(TC_BAR_USED + (gi - 2) % TC_S),
                                              (uint32_t)(((gi - 2) / TC_S) & 1), s_err))
                        break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = umma_desc(su32(sA + b * 4096));
                    const uint64_t db = umma_desc(su32(sB + b * 4096));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(tmem + (uint32_t)(b * TC_P)), "l"(da), "l"(db), "r"(idesc), "r"(0));
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(BAR(TC_BAR_ACC + b))
                                 : "memory");
                    mma_last = gi;
                    const int j = i + TC_S - 2;
                    if (j < nch) {
                        const long long gj = g + j; // slot of chunk gi - 2
                        int c_lo, c_hi;
                        tc_chunk(hi, j, c_lo, c_hi);
                        tc_load_chunk(pts_t, idx_t, c_lo, c_hi, su32(raw + (gj % TC_S) * TC_P),
                                      su32(sidx + (gj % TC_S) * TC_P), BAR(TC_BAR_RAW + gj % TC_S));
                        issued = gj;
                    }
                }
            }
        } else if (nch > 0) {
            // ---- screening warps.  Every wait outcome is made warp-uniform
            // before the warp-collective steps that follow it.
            // Rows of chunk gi: B from its raw points, A with the current -T.
            auto build = [&](long long gi, int i) -> bool {
                const int s = (int)(gi % TC_S), b = (int)(gi & 1);
                const bool okw = mbar_wait(BAR(TC_BAR_RAW + s), (uint32_t)((gi / TC_S) & 1), s_err);
                if (!__all_sync(FULLMASK, okw))
                    return false;
                int c_lo, c_hi;
                tc_chunk(hi, i, c_lo, c_hi);
                float bv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (tq < c_hi - c_lo) {
                    const float4 p = raw[s * TC_P + tq];
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
                    bv[5] = tf32_rna((1.0f - 2.0f * TC_EPS) * m2);
                    bv[6] = 1.0f;
                }
                store_row(sB + b * 4096, tq, bv);
                *(float *)(sA + b * 4096 + kmaj_off(tq, 6)) = active ? tc_neg_T(tau) : 0.0f;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(BAR(TC_BAR_BFULL + b));
                return true;
            };
            // threshold seeds (see the header): scored on the CUDA cores
            const int sl = *s_seed;
            if (sl >= 0) {
                const int nseed = min(TC_SEED_BATCHES * TC_P, W->n);
                for (int b0 = 0; b0 < nseed; b0 += TC_P) {
                    const int ns = min(TC_P, nseed - b0);
                    if (b0 > 0) // the previous batch has been read
                        asm volatile("bar.sync 1, %0;" ::"r"(TC_Q) : "memory");
                    if (tq < ns) {
                        seedp[tq] = __ldg(L.seed_pts + sl + b0 + tq);
                        seedi[tq] = __ldg(L.seed_idx + sl + b0 + tq);
                    }
                    asm volatile("bar.sync 1, %0;" ::"r"(TC_Q) : "memory"); // the 4 screening warps
                    if (!active)
                        continue;
                    for (int j = 0; j < ns; ++j) {
                        const float4 p = seedp[j];
                        if (!(p.w < c.T32))
                            continue;
                        const float d = dist32(c, s0, s1, s2, s3, p);
                        st.lb++;
                        if (d <= tau) {
                            const unsigned long long key = pack_key(d, seedi[j]);
                            if (key < tauk) {
                                tauk = list_push<TC_Q>(K, Lw, nv, key);
                                tau = key_d(tauk);
                            }
                        }
                    }
                }
                if (active) {
                    // keys up to the L-th seed key stay admissible (+1: the
                    // test is strict and keys are unique)
                    bound0 = nv == Lw ? tauk + 1ull : SENT;
                    for (int i = 0; i < nv; ++i)
                        K[i * TC_Q] = SENT;
                    nv = 0;
                    tauk = bound0;
                    tau = key_d(bound0);
                }
            }
            // the fixed part of both A buffers (the settlement scratch of
            // the previous tile overlaps them)
            store_row(sA, tq, arow);
            store_row(sA + 4096, tq, arow);
            bool ok = build(g, 0);
            for (int i = 0; ok && i < nch; ++i) {
                const long long gi = g + i;
                const int s = (int)(gi % TC_S), b = (int)(gi & 1);
                if (i + 1 < nch && !build(gi + 1, i + 1))
                    break;
                const bool okw = mbar_wait(BAR(TC_BAR_ACC + b), (uint32_t)((gi >> 1) & 1), s_err);
                if (!__all_sync(FULLMASK, okw))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                int c_lo, c_hi;
                tc_chunk(hi, i, c_lo, c_hi);
                const int ncaus = max(0, min(c_hi - c_lo, hq - c_lo)); // causal columns of this lane
                st.pairs += ncaus;
                if (t == 0)
                    st.segs++; // 128 x 128 tiles multiplied
                if (__any_sync(FULLMASK, ncaus > 0)) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t v[64];
                        tmem_ld32_nowait(taddr_row + (uint32_t)(b * TC_P + h * 64), v);
                        tmem_ld32_nowait(taddr_row + (uint32_t)(b * TC_P + h * 64 + 32), v + 32);
                        tmem_wait_ld();
                        // OR of each group of 8 values: its sign bit says
                        // whether the group holds a negative one
                        uint32_t gor[8];
#pragma unroll
                        for (int q8 = 0; q8 < 8; ++q8) {
                            gor[q8] = v[8 * q8];
#pragma unroll
                            for (int j = 1; j < 8; ++j)
                                gor[q8] |= v[8 * q8 + j];
                        }
                        uint32_t any = 0u;
#pragma unroll
                        for (int q8 = 0; q8 < 8; ++q8)
                            any |= gor[q8];
                        const int lim = ncaus - h * 64; // causal columns in this half
                        if ((int)any < 0 && lim > 0) {
                            // sign bits of the groups that hold a negative value
                            uint32_t m0 = 0u, m1 = 0u;
#pragma unroll
                            for (int q8 = 0; q8 < 8; ++q8) {
                                if ((int)gor[q8] < 0) {
                                    uint32_t gm = 0u;
#pragma unroll
                                    for (int j = 0; j < 8; ++j)
                                        gm |= (v[8 * q8 + j] >> 31) << j;
                                    if (q8 < 4)
                                        m0 |= gm << (8 * q8);
                                    else
                                        m1 |= gm << (8 * (q8 - 4));
                                }
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
                                    const float4 p = raw[s * TC_P + col];
                                    const float d = dist32(c, s0, s1, s2, s3, p);
                                    st.lb++; // screened points scored again in FP32
                                    if (p.w < c.T32 && d <= tau) {
                                        const unsigned long long key = pack_key(d, sidx[s * TC_P + col]);
                                        if (key < tauk) {
                                            const unsigned long long r = list_push<TC_Q>(K, Lw, nv, key);
                                            tauk = r < bound0 ? r : bound0;
                                            tau = key_d(tauk);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                // the TMEM reads and raw[s] are finished: release the
                // accumulator and the slot
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(BAR(TC_BAR_USED + s));
            }
        }
        g += nch;
        __syncthreads();
        if (*s_err)
            break;
        if (active) {
            st.q++;
            list_sort<TC_Q>(K, nv);
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st, TC_Q)) {
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
        for (long long gj = issued; gj >= 0 && gj > issued - TC_S; --gj)
            mbar_wait(BAR(TC_BAR_RAW + gj % TC_S), (uint32_t)((gj / TC_S) & 1), nullptr);
        if (mma_last >= 0)
            mbar_wait(BAR(TC_BAR_ACC + (mma_last & 1)), (uint32_t)((mma_last >> 1) & 1), nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (ctrl)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_P));
    else
        flush_stats(L.scr, st);
#undef BAR
}
