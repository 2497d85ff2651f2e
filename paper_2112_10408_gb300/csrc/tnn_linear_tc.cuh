// Linear search on the tensor cores (Sec. 3.6: the linear search computes
// the distance matrix with the classic expansion |q|^2 + |p|^2 - 2 q.p,
// Table 1 "Distance Matrix").
//
// A CTA of 128 threads answers 128 queries (thread t = query t = TMEM lane t)
// over the time-ordered copy of the points, most recent first, 128 points per
// tile.  Each tile:
//   1. its raw points arrive by TMA (cp.async.bulk, completion on an
//      mbarrier), one tile ahead;
//   2. every thread turns one point into a row of the B operand in shared
//      memory (K-major, no swizzle): with e = sqrt(sigma) (p - c) for a
//      fixed centre c, b = [-2 e, 1, |e|^2, 0, 0]; the query rows are
//      a = [f, |f|^2, 1, 0, 0] with f = sqrt(sigma) (q - c), so a . b =
//      |f - e|^2, the scaled squared distance;
//   3. one thread issues tcgen05.mma kind::tf32 (M = 128, N = 128, K = 24):
//      the 3-term TF32 split [a_hi | a_lo | a_hi] x [b_hi | b_hi | b_lo]
//      keeps about 21 bits, the FP32 accumulator lives in TMEM;
//   4. each thread reads its row of the accumulator (tcgen05.ld) and keeps
//      only the points whose value is at most its pruning key plus a
//      certified margin; those are scored again with the exact FP32
//      distance of the other kernels, so candidate keys, lists and the FP64
//      settlement are the same.
// Margin: with R4 a bound on |e| over the points and |f| the query's, every
// product a_k b_k is off by at most ~3 * 2^-22 |a_k||b_k| and the 18-term
// FP32 accumulation by ~18 * 2^-24 of the sum of |a_k b_k| <= (|f| + R4)^2,
// so 2^-16 (|f| + R4)^2 covers both with room; the FP32 centring of q and p
// adds far less.  A point passing the FP32 test (d32 <= key) therefore
// always passes the screen.
#pragma once
#include "tnn_device.cuh"

#define TC_Q 128
#define TC_P 128
#define TC_KS 3
#define TC_WAIT_NS 1000000000ull // 1 s: a copy or an MMA that takes longer is an error

#define TC_OFF_A 0                       // [3 K-steps][128 rows x 8] TF32
#define TC_OFF_B (TC_OFF_A + 12288)      // same for the points
#define TC_OFF_RAW (TC_OFF_B + 12288)    // [2][128] float4 raw points
#define TC_OFF_BAR (TC_OFF_RAW + 4096)   // mbarriers, TMEM slot, CTA scalars
#define TC_OFF_LIST (TC_OFF_BAR + 128)   // [L][128] candidate keys
// after the last tile the settlement scratch of the 4 warps (4 x 3 KB)
// reuses the B operand and raw tiles (16 KB)

__host__ __device__ inline size_t tc_smem_bytes(int L_max)
{
    return TC_OFF_LIST + (size_t)L_max * TC_Q * 8;
}

__device__ __forceinline__ uint32_t su32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of (row r, k) inside one K-step block (128 rows x 8 TF32):
// core matrices of 8 rows x 16 B, K-adjacent ones 128 B apart, row-group
// adjacent ones 256 B apart.
__device__ __forceinline__ uint32_t kmaj_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor: start, leading (K) byte offset 128,
// stride (row-group) byte offset 256, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for an mbarrier phase for at most TC_WAIT_NS; false if it timed out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity)
{
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (ok)
            return true;
        if (it == 0)
            t0 = globaltimer_ns();
        else if (globaltimer_ns() - t0 > TC_WAIT_NS)
            return false;
    }
}

__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Write the 3 K-step rows of one operand row: steps (s0, s1, s2) take the
// high or low TF32 part of the 8 values v.
__device__ __forceinline__ void write_split_row(unsigned char *base, int row, const float (&v)[8],
                                                bool lo0, bool lo1, bool lo2)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float hi = tf32_rna(v[k]);
        const float lo = tf32_rna(v[k] - hi);
        const uint32_t off = kmaj_off(row, k);
        *(float *)(base + 0 * 4096 + off) = lo0 ? lo : hi;
        *(float *)(base + 1 * 4096 + off) = lo1 ? lo : hi;
        *(float *)(base + 2 * 4096 + off) = lo2 ? lo : hi;
    }
}

__global__ void __launch_bounds__(TC_Q, 1) k_linear_tc(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[]; // no-swizzle operands need 16 B
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned char *sA = smem + TC_OFF_A;
    unsigned char *sB = smem + TC_OFF_B;
    float4 *raw = (float4 *)(smem + TC_OFF_RAW);
    unsigned long long *bar = (unsigned long long *)(smem + TC_OFF_BAR); // [3]
    uint32_t *tmem_slot = (uint32_t *)(smem + TC_OFF_BAR + 24);
    long long *s_tile = (long long *)(smem + TC_OFF_BAR + 32);
    int *s_hi = (int *)(smem + TC_OFF_BAR + 40);
    float *s_wmax = (float *)(smem + TC_OFF_BAR + 48); // [4]
    unsigned long long *K = (unsigned long long *)(smem + TC_OFF_LIST) + t;
    unsigned long long *cl_d = (unsigned long long *)(sB + warp * 3072) + lane;
    int *cl_i = (int *)(sB + warp * 3072 + CMAX * 32 * 8) + lane;

    if (t == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar + b)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(TC_P));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t taddr_row = tmem + ((uint32_t)(warp * 32) << 16);
    // F32 accumulate, A = B = TF32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_P >> 3) << 17) |
                           ((uint32_t)(TC_Q >> 4) << 24);
    uint32_t ph[2] = {0u, 0u}, phm = 0u;
    LaneStats st = {0, 0, 0, 0, 0};
    const KnnWin *W = &L.w0;
    const float s0 = W->sig[0], s1 = W->sig[1], s2 = W->sig[2], s3 = W->sig[3];
    const float q0 = W->ssq[0], q1 = W->ssq[1], q2 = W->ssq[2], q3 = sqrtf(s3);
    const float c0 = W->center[0], c1 = W->center[1], c2 = W->center[2], c3 = W->center[3];
    const float4 *__restrict__ pts_t = W->pts_t;
    const int32_t *__restrict__ idx_t = W->idx_t;
    const int Lw = W->L;

    int err = 0; // the same in every thread: set only from __syncthreads_or results
    for (;;) {
        if (t == 0)
            *s_tile = (long long)atomicAdd(&L.scr->tile_counter, 1ull);
        __syncthreads();
        const long long tile = *s_tile;
        if (tile >= L.total_tiles)
            break;
        const int64_t qrow = tile * TC_Q + t;
        const bool active = qrow < W->m;
        const float4 q = active ? W->q[qrow] : make_float4(0.f, 0.f, 0.f, 0.f);
        const QCtx c = make_qctx(W, q, active);

        // causal prefix of the CTA: points with t < max T32
        float wm = c.T32;
        for (int o = 16; o > 0; o >>= 1)
            wm = fmaxf(wm, __shfl_xor_sync(FULLMASK, wm, o));
        if (lane == 0)
            s_wmax[warp] = wm;
        // query rows of A and the candidate lists
        float marg;
        {
            float f[4] = {q0 * (q.x - c0), q1 * (q.y - c1), q2 * (q.z - c2), q3 * (q.w - c3)};
            float n2 = 0.f;
#pragma unroll
            for (int d = 0; d < 4; ++d)
                n2 = fmaf(f[d], f[d], n2);
            float a[8] = {f[0], f[1], f[2], f[3], n2, 1.0f, 0.0f, 0.0f};
            if (!active)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    a[k] = 0.0f;
            write_split_row(sA, t, a, false, true, false);
            const float rr = sqrtf(n2) + W->R4;
            marg = 0x1p-16f * rr * rr;
        }
        for (int i = 0; i < Lw; ++i)
            K[i * TC_Q] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY, thr = INFINITY;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
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
            if (lo > 0) {
                const int cl = lo > TC_P ? lo - TC_P : 0;
                tma_load_1d(su32(raw), pts_t + cl, (uint32_t)(lo - cl) * 16u, su32(bar + 0));
            }
        }
        __syncthreads();
        const int hi = *s_hi;
        const int nch = (hi + TC_P - 1) / TC_P;
        // Chunk i's copy is issued (one ahead) only once chunk i - 1's copy
        // was waited for; a loop exit waits for the copy still in flight.
        for (int i = 0; i < nch; ++i) {
            const int b = i & 1;
            const int c_hi = hi - TC_P * i, c_lo = c_hi > TC_P ? c_hi - TC_P : 0;
            const int cnt = c_hi - c_lo;
            const bool bad_copy = !mbar_wait_bounded(su32(bar + b), ph[b]);
            ph[b] ^= 1u;
            // point row t of B
            {
                float bv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (t < cnt) {
                    const float4 p = raw[b * TC_P + t];
                    const float e[4] = {q0 * (p.x - c0), q1 * (p.y - c1), q2 * (p.z - c2), q3 * (p.w - c3)};
                    float m2 = 0.f;
#pragma unroll
                    for (int d = 0; d < 4; ++d)
                        m2 = fmaf(e[d], e[d], m2);
                    bv[0] = -2.0f * e[0];
                    bv[1] = -2.0f * e[1];
                    bv[2] = -2.0f * e[2];
                    bv[3] = -2.0f * e[3];
                    bv[4] = 1.0f;
                    bv[5] = m2;
                }
                write_split_row(sB, t, bv, false, false, true);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (__syncthreads_or(bad_copy)) {
                err = 1;
                break;
            }
            if (t == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int s = 0; s < TC_KS; ++s) {
                    const uint64_t da = umma_desc(su32(sA + s * 4096));
                    const uint64_t db = umma_desc(su32(sB + s * 4096));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(s));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(su32(bar + 2))
                             : "memory");
                if (i + 1 < nch) {
                    const int nh = c_lo, nl = nh > TC_P ? nh - TC_P : 0;
                    tma_load_1d(su32(raw + (b ^ 1) * TC_P), pts_t + nl, (uint32_t)(nh - nl) * 16u,
                                su32(bar + (b ^ 1)));
                }
            }
            const bool bad_mma = !mbar_wait_bounded(su32(bar + 2), phm);
            phm ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (__syncthreads_or(bad_mma)) {
                err = 2;
                if (i + 1 < nch) // the copy of chunk i + 1 is in flight
                    mbar_wait_bounded(su32(bar + (b ^ 1)), ph[b ^ 1]);
                break;
            }
            // screen the row, score the survivors exactly
            for (int col0 = 0; col0 < cnt; col0 += 32) {
                uint32_t v[32];
                tmem_ld32(taddr_row + (uint32_t)col0, v);
                if (active) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = col0 + j;
                        if (col < cnt && __uint_as_float(v[j]) <= thr) {
                            const float4 p = raw[b * TC_P + col];
                            const float d = dist32(c, s0, s1, s2, s3, p);
                            st.lb++; // screened points scored again in FP32
                            if (p.w < c.T32 && d <= tau) {
                                const unsigned long long key = pack_key(d, __ldg(idx_t + c_lo + col));
                                if (key < tauk) {
                                    tauk = lane_push_s(K, Lw, nv, key, TC_Q);
                                    tau = key_d(tauk);
                                    thr = fmaf(tau, 0x1p-18f, tau) + marg;
                                }
                            }
                        }
                    }
                }
            }
            if (active)
                st.pairs += cnt;
            // The next chunk's barrier orders these reads of TMEM and of
            // raw[b] before the MMA and the copy that overwrite them.
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        if (err)
            break;
        if (active) {
            st.q++;
            if (!finalize_query(W, q, K, Lw, cl_d, cl_i, qrow, st, TC_Q)) {
                const unsigned slot = atomicAdd(&L.scr->n_fallback, 1u);
                if (slot < (unsigned long long)L.fb_cap)
                    L.fb_list[slot] = make_int2(-1, (int)qrow); // unsettled, window 0
                else
                    atomicOr(&L.scr->status, 1u);
            }
        }
        __syncthreads();
    }
    if (t == 0 && err)
        atomicOr(&L.scr->status, 4u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_P));
    flush_stats(L.scr, st);
}
