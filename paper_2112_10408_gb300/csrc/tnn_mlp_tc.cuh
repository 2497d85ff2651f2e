// The MLP of the learned nowcaster on the tensor cores (tcgen05, kind::f16
// with BF16 operands, FP32 accumulation in TMEM).
//
// k_mlp_fwd_tc — one CTA of 128 threads per 128 rows of the batch:
//   Z = X W1 + b1 with X [B, d_in] (A operand, rows of the batch) and W1
//   kept transposed in the UMMA core-matrix order (B operand, one 16-column
//   K step = dh rows x 32 B, moved by one bulk copy).  The K loop is double
//   buffered: the threads write the next X slice while the previous MMA
//   runs.  Epilogue, thread = row = TMEM lane: H = bf16(GELU(Z)), the
//   256 -> 2 head Y = H W2 + b2; with targets also the MSE gradient dY,
//   dZ = (dY W2^T) * GELU'(Z) (written transposed for the dW1 product, as is
//   X), the squared error, and the per-CTA column sums that give db1, dW2 and
//   db2 (warp reduce-scatter, then the 4 warps' rows summed in a fixed order,
//   so that training is deterministic).
// k_mlp_dw1_tc — dW1^T = dZ^T X over the batch: one CTA per (128 hidden
//   units, up to 256 inputs, batch slice); both operands are read K-major
//   from the transposed copies; the partial products of the batch slices are
//   summed by the AdamW kernel.
#pragma once
#include "tnn_tc.cuh"

#define MLP_ROWS 128

// Two floats rounded to BF16 (round to nearest even) in one 32-bit word:
// a in the low half, b in the high half.
__device__ __forceinline__ uint32_t bf2_pack(float a, float b)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// Byte offset of (row r, k) inside one 16-column BF16 K step of a K-major
// operand: core matrices of 8 rows x 16 B, the two K halves 128 B apart,
// row groups 256 B apart.
__device__ __forceinline__ uint32_t kmaj_off_bf16(int r, int k)
{
    return (uint32_t)((r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Instruction descriptor: F32 accumulate, A = B = BF16, both K-major.
__host__ __device__ inline uint32_t mlp_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ inline uint32_t tmem_cols_for(int n)
{
    uint32_t c = 32;
    while (c < (uint32_t)n)
        c <<= 1;
    return c;
}

struct MlpFwdArgs {
    const uint16_t *X; // [B][d_in]
    long long B;
    int d_in, dh;
    const uint16_t *w1t; // W1^T, K steps of [dh][16] in core-matrix order
    const float *b1;     // [dh]
    const float *W2;     // [dh][2]
    const float *b2;     // [2]
    float *Y;            // [B][2] or NULL
    const float *T;      // targets [B][2]; NULL = inference
    float *dY;           // [B][2]
    uint16_t *dZt;       // [dh][ldt]
    uint16_t *Xt;        // [d_in][ldt]
    long long ldt;       // >= B rounded up to 16
    float *pCol;         // [gridDim.x][3 dh + 2]: db1 | dW2 | db2 per CTA
    float *sse;          // squared error, summed
    float inv_B;
    uint32_t tmem_cols;
    int *err;            // set when a device wait timed out
    int resident;        // 1: all K steps of X and W1^T staged at once (mlp_fwd_smem_res)
};

#define MLP_FWD_THREADS 256 // two warps per TMEM lane quadrant, one per half of the hidden units

// Shared memory with every K step staged at once (resident = 1): the same
// layout with nk stages instead of 4.
__host__ __device__ inline size_t mlp_fwd_smem_res(int d_in, int dh)
{
    const size_t nk = (size_t)d_in / 16;
    return nk * (4096 + (size_t)dh * 32) + (size_t)dh * 12 + 4 * ((size_t)dh * 3 + 2) * 4 + 2048 + 128;
}

__host__ __device__ inline size_t mlp_fwd_smem(int dh)
{
    // 4 stages x (A 4 KB + B dh x 32 B) + b1, W2 (3 dh floats) + column sums
    // of the 4 lane quadrants (4 x (3 dh + 2) floats) + head partials
    // (2 x 128 x 2 floats) + barriers
    return 4 * (4096 + (size_t)dh * 32) + (size_t)dh * 12 + 4 * ((size_t)dh * 3 + 2) * 4 + 2048 + 128;
}

// Sum over the 32 lanes of v[i] for 16 columns i: on return lanes l and
// l ^ 16 hold the sum of column l & 15.
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16], int lane)
{
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

__global__ void __launch_bounds__(MLP_FWD_THREADS, 2) k_mlp_fwd_tc(const __grid_constant__ MlpFwdArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int quad = warp & 3, half = warp >> 2; // TMEM lane quadrant, hidden-unit half
    const int rr = t & (MLP_ROWS - 1);           // row of the tile (= TMEM lane)
    const int dh = a.dh, nk = a.d_in / 16, hh = dh / 2;
    const size_t bstage = (size_t)dh * 32;
    const int nst = a.resident ? nk : 4;        // K-step stages in shared memory
    unsigned char *sA = smem;                   // [nst][4096]
    unsigned char *sB = smem + (size_t)nst * 4096; // [nst][bstage]
    float *s_b1 = (float *)(sB + nst * bstage); // [dh]
    float *s_W2 = s_b1 + dh;                  // [dh][2]
    const int ncol = 3 * dh + 2;
    float *s_col = s_W2 + 2 * dh;             // [4 quadrants][3 dh + 2]
    float *s_y = s_col + 4 * ncol;            // [2 halves][128][2]
    unsigned long long *bars = (unsigned long long *)(s_y + 2 * MLP_ROWS * 2);
    uint32_t *tmem_slot = (uint32_t *)(bars + 8);
    const uint32_t bar_full0 = su32(bars), bar_mma0 = su32(bars + 4); // [4] each
    volatile int *s_err = (volatile int *)(tmem_slot + 1);
    const long long row0 = (long long)blockIdx.x * MLP_ROWS;
    const long long r = row0 + rr;
    const long long Bp = (a.B + 15) & ~15ll;
    const bool valid = r < a.B;
    const bool train = a.T != nullptr;

    if (t == 0) {
        for (int i = 0; i < 8; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bars + i)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
        if (a.resident) {
            // every W1^T slice, on one barrier
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(bar_full0), "r"((uint32_t)(bstage * nk))
                         : "memory");
            for (int s = 0; s < nk; ++s)
                tma_copy_1d(su32(sB + s * bstage), a.w1t + (size_t)s * dh * 16, (uint32_t)bstage, bar_full0);
        } else {
            // W1^T slices of the first two K steps
            for (int s = 0; s < 2 && s < nk; ++s) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(bar_full0 + 8u * s), "r"((uint32_t)bstage)
                             : "memory");
                tma_copy_1d(su32(sB + s * bstage), a.w1t + (size_t)s * dh * 16, (uint32_t)bstage,
                            bar_full0 + 8u * s);
            }
        }
    }
    for (int i = t; i < dh; i += MLP_FWD_THREADS) {
        s_b1[i] = a.b1[i];
        s_W2[2 * i] = a.W2[2 * i];
        s_W2[2 * i + 1] = a.W2[2 * i + 1];
    }
    for (int i = t; i < 4 * ncol; i += MLP_FWD_THREADS)
        s_col[i] = 0.0f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (a.resident) {
        // ---- Z = X W1 with every K step staged at once: the threads write
        // all of X (and X^T when training), then one thread issues every MMA
#pragma unroll 4
        for (int s = 0; s < nk; ++s) {
            const uint4 x = valid ? __ldg((const uint4 *)(a.X + r * a.d_in + s * 16 + half * 8))
                                  : make_uint4(0, 0, 0, 0);
            *(uint4 *)(sA + (size_t)s * 4096 + kmaj_off_bf16(rr, half * 8)) = x;
            if (train && r < Bp) {
                const uint16_t *xs = (const uint16_t *)&x;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    a.Xt[(long long)(s * 16 + half * 8 + j) * a.ldt + r] = xs[j];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            if (!mbar_wait(bar_full0, 0u, s_err)) {
                ok = false;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int s = 0; s < nk; ++s) {
                    const uint64_t da = umma_desc(su32(sA + (size_t)s * 4096));
                    for (int n0 = 0; n0 < dh; n0 += 256) {
                        const int nn = min(256, dh - n0);
                        const uint64_t db = umma_desc(su32(sB + s * bstage + (size_t)n0 * 32));
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     ::"r"(tmem + (uint32_t)n0), "l"(da), "l"(db), "r"(mlp_idesc(128, nn)),
                                     "r"(s));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(bar_mma0)
                             : "memory");
            }
        }
        const bool w = __syncthreads_and(ok) && mbar_wait(bar_mma0, 0u, s_err);
        ok = !__syncthreads_or(!w);
    } else {
        // ---- Z = X W1: K steps of 16 inputs, four stages; the W1^T slice of
        // step s + 2 is copied while step s is prepared; thread (row rr, half)
        // moves 8 of the 16 values of its row
        uint4 xq[8]; // this thread's X values of the next 8 K steps, loaded together
        for (int s = 0; s < nk; ++s) {
            const int st = s & 3;
            if ((s & 7) == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    xq[i] = (valid && s + i < nk) ? __ldg((const uint4 *)(a.X + r * a.d_in + (s + i) * 16 + half * 8))
                                                  : make_uint4(0, 0, 0, 0);
            }
            if (s >= 2) {
                // the MMA of step s - 2 (and every one before it) has completed:
                // stage (s + 2) & 3 and stage s & 3 are free
                const bool w = mbar_wait(bar_mma0 + 8u * ((s - 2) & 3), (uint32_t)(((s - 2) >> 2) & 1), s_err);
                if (__syncthreads_or(!w)) {
                    ok = false;
                    break;
                }
            }
            if (t == 0 && s + 2 < nk) {
                const int s2 = s + 2, st2 = s2 & 3;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(bar_full0 + 8u * st2), "r"((uint32_t)bstage)
                             : "memory");
                tma_copy_1d(su32(sB + st2 * bstage), a.w1t + (size_t)s2 * dh * 16, (uint32_t)bstage,
                            bar_full0 + 8u * st2);
            }
            uint4 x = xq[0];
#pragma unroll
            for (int i = 1; i < 8; ++i)
                if ((s & 7) == i)
                    x = xq[i];
            *(uint4 *)(sA + st * 4096 + kmaj_off_bf16(rr, half * 8)) = x;
            if (train && r < Bp) {
                // X^T for the dW1 product (zeros pad the batch to 16)
                const uint16_t *xs = (const uint16_t *)&x;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    a.Xt[(long long)(s * 16 + half * 8 + j) * a.ldt + r] = xs[j];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (t == 0) {
                if (!mbar_wait(bar_full0 + 8u * st, (uint32_t)((s >> 2) & 1), s_err)) {
                    ok = false;
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = umma_desc(su32(sA + st * 4096));
                    for (int n0 = 0; n0 < dh; n0 += 256) {
                        const int nn = min(256, dh - n0);
                        const uint64_t db = umma_desc(su32(sB + st * bstage + (size_t)n0 * 32));
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     ::"r"(tmem + (uint32_t)n0), "l"(da), "l"(db), "r"(mlp_idesc(128, nn)),
                                     "r"(s));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(bar_mma0 + 8u * st)
                                 : "memory");
                }
            }
        }
        // the last MMA's barrier covers every MMA before it
        {
            const int sl = nk - 1;
            const bool w = ok && mbar_wait(bar_mma0 + 8u * (sl & 3), (uint32_t)((sl >> 2) & 1), s_err);
            ok = !__syncthreads_or(!w);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
        const int c0 = half * hh, c1 = c0 + hh;
        // ---- pass 1: H = bf16(GELU(Z + b1)), partial head over this half
        float y0 = 0.f, y1 = 0.f;
        for (int c = c0; c < c1; c += 32) {
            uint32_t v[32];
            tmem_ld32_nowait(trow + (uint32_t)c, v);
            tmem_wait_ld();
            const float4 *b1v = (const float4 *)(s_b1 + c);
            const float4 *w2v = (const float4 *)(s_W2 + 2 * c);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 bb = b1v[j >> 2], wa = w2v[j >> 1], wb = w2v[(j >> 1) + 1];
                const uint32_t p01 = bf2_pack(gelu_f(__uint_as_float(v[j]) + bb.x),
                                              gelu_f(__uint_as_float(v[j + 1]) + bb.y));
                const uint32_t p23 = bf2_pack(gelu_f(__uint_as_float(v[j + 2]) + bb.z),
                                              gelu_f(__uint_as_float(v[j + 3]) + bb.w));
                const float h0 = __uint_as_float(p01 << 16), h1 = __uint_as_float(p01 & 0xffff0000u);
                const float h2 = __uint_as_float(p23 << 16), h3 = __uint_as_float(p23 & 0xffff0000u);
                y0 = fmaf(h0, wa.x, y0);
                y1 = fmaf(h0, wa.y, y1);
                y0 = fmaf(h1, wa.z, y0);
                y1 = fmaf(h1, wa.w, y1);
                y0 = fmaf(h2, wb.x, y0);
                y1 = fmaf(h2, wb.y, y1);
                y0 = fmaf(h3, wb.z, y0);
                y1 = fmaf(h3, wb.w, y1);
            }
        }
        s_y[(half * MLP_ROWS + rr) * 2] = y0;
        s_y[(half * MLP_ROWS + rr) * 2 + 1] = y1;
        __syncthreads();
        y0 = s_y[rr * 2] + s_y[(MLP_ROWS + rr) * 2] + a.b2[0];
        y1 = s_y[rr * 2 + 1] + s_y[(MLP_ROWS + rr) * 2 + 1] + a.b2[1];
        if (valid && a.Y && half == 0) {
            a.Y[2 * r] = y0;
            a.Y[2 * r + 1] = y1;
        }
        if (train) {
            // ---- pass 2: dY, dZ = (dY W2^T) GELU'(Z), column sums
            const float e0 = valid ? y0 - a.T[2 * r] : 0.f, e1 = valid ? y1 - a.T[2 * r + 1] : 0.f;
            const float g0 = e0 * a.inv_B, g1 = e1 * a.inv_B; // d mean over 2B of e^2
            float *wcol = s_col + quad * ncol;
            if (half == 0) {
                if (valid) {
                    a.dY[2 * r] = g0;
                    a.dY[2 * r + 1] = g1;
                }
                float se = e0 * e0 + e1 * e1, gs0 = g0, gs1 = g1;
                for (int o = 16; o > 0; o >>= 1) {
                    se += __shfl_xor_sync(FULLMASK, se, o);
                    gs0 += __shfl_xor_sync(FULLMASK, gs0, o);
                    gs1 += __shfl_xor_sync(FULLMASK, gs1, o);
                }
                if (lane == 0) {
                    atomicAdd(a.sse, se);
                    wcol[3 * dh] = gs0;
                    wcol[3 * dh + 1] = gs1;
                }
            }
            const bool padrow = !valid && r < Bp;
            for (int c = c0; c < c1; c += 16) {
                uint32_t v[16];
                tmem_ld16_nowait(trow + (uint32_t)c, v);
                tmem_wait_ld();
                float db[16], w0[16], w1[16];
                const float4 *b1v = (const float4 *)(s_b1 + c);
                const float4 *w2v = (const float4 *)(s_W2 + 2 * c);
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    const float4 w = w2v[j >> 1];
                    const float2 bb = (j & 2) ? make_float2(b1v[j >> 2].z, b1v[j >> 2].w)
                                              : make_float2(b1v[j >> 2].x, b1v[j >> 2].y);
                    const float za = __uint_as_float(v[j]) + bb.x, zb = __uint_as_float(v[j + 1]) + bb.y;
                    const float2 pa = normal_cdf_and_gauss(za), pb = normal_cdf_and_gauss(zb);
                    const uint32_t hp = bf2_pack(za * pa.x, zb * pb.x);
                    const float ha = valid ? __uint_as_float(hp << 16) : 0.f;
                    const float hb = valid ? __uint_as_float(hp & 0xffff0000u) : 0.f;
                    const float dha = fmaf(g0, w.x, g1 * w.y), dhb = fmaf(g0, w.z, g1 * w.w);
                    const float gpa = fmaf(za * 0.39894228040143268f, pa.y, pa.x);
                    const float gpb = fmaf(zb * 0.39894228040143268f, pb.y, pb.x);
                    const uint32_t dp = valid ? bf2_pack(dha * gpa, dhb * gpb) : 0u;
                    if (valid || padrow) {
                        a.dZt[(long long)(c + j) * a.ldt + r] = (uint16_t)(dp & 0xffffu);
                        a.dZt[(long long)(c + j + 1) * a.ldt + r] = (uint16_t)(dp >> 16);
                    }
                    db[j] = __uint_as_float(dp << 16);
                    db[j + 1] = __uint_as_float(dp & 0xffff0000u);
                    w0[j] = ha * g0;
                    w1[j] = ha * g1;
                    w0[j + 1] = hb * g0;
                    w1[j + 1] = hb * g1;
                }
                const float sdb = warp_reduce_scatter16(db, lane);
                const float sw0 = warp_reduce_scatter16(w0, lane);
                const float sw1 = warp_reduce_scatter16(w1, lane);
                if (lane < 16) {
                    wcol[c + lane] = sdb;
                    wcol[dh + 2 * (c + lane)] = sw0;
                    wcol[dh + 2 * (c + lane) + 1] = sw1;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    if (!ok) {
        if (t == 0)
            atomicOr(a.err, 1);
        return;
    }
    if (train)
        for (int i = t; i < ncol; i += MLP_FWD_THREADS)
            a.pCol[(long long)blockIdx.x * ncol + i] =
                ((s_col[i] + s_col[ncol + i]) + s_col[2 * ncol + i]) + s_col[3 * ncol + i];
}

struct MlpDw1Args {
    const uint16_t *dZt; // [dh][ldt]
    const uint16_t *Xt;  // [d_in][ldt]
    long long ldt;
    long long Bp;        // batch rounded up to 16 (rows beyond B are zeros)
    int d_in, dh;
    long long rows_per;  // batch rows per split (multiple of 16)
    float *pW1;          // [splits][d_in][dh]
    uint32_t tmem_cols;
    int *err;
    long long *step_inc; // AdamW step count to advance (NULL: gradients only)
};

#define DW1_KSTEPS 8 // 128 batch rows per pass

__host__ __device__ inline size_t mlp_dw1_smem()
{
    // A: 8 K steps x 4 KB; B: 8 K steps x 256 rows x 32 B; barrier
    return (size_t)DW1_KSTEPS * 4096 + (size_t)DW1_KSTEPS * 256 * 32 + 64;
}

// grid: (ceil(dh / 128), ceil(d_in / 256), splits)
__global__ void __launch_bounds__(MLP_ROWS, 1) k_mlp_dw1_tc(const __grid_constant__ MlpDw1Args a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x, warp = t >> 5;
    const int h0 = blockIdx.x * 128, f0 = blockIdx.y * 256;
    const int nn = min(256, a.d_in - f0);
    const long long k0 = (long long)blockIdx.z * a.rows_per;
    const long long k1 = a.Bp < k0 + a.rows_per ? a.Bp : k0 + a.rows_per;
    unsigned char *sA = smem;                       // [8][4096]
    unsigned char *sB = smem + DW1_KSTEPS * 4096;   // [8][nn x 32]
    unsigned long long *bar = (unsigned long long *)(sB + (size_t)DW1_KSTEPS * 256 * 32);
    uint32_t *tmem_slot = (uint32_t *)(bar + 1);
    volatile int *s_err = (volatile int *)(tmem_slot + 1);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
        // the AdamW kernel that follows on the stream reads the new count
        if (a.step_inc && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            *a.step_inc += 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = mlp_idesc(128, nn);
    const int h = h0 + t;
    bool ok = true;
    int pass = 0;
    for (long long kb = k0; kb < k1; kb += 16 * DW1_KSTEPS, ++pass) {
        const long long left = (k1 - kb) / 16;
        const int ks = left < DW1_KSTEPS ? (int)left : DW1_KSTEPS;
        if (pass > 0) {
            // the previous pass's MMAs have read the operands
            const bool w = mbar_wait(su32(bar), (uint32_t)((pass - 1) & 1), s_err);
            if (__syncthreads_or(!w)) {
                ok = false;
                break;
            }
        }
        // A: row t = hidden unit h, 16 batch values per K step
        for (int s = 0; s < ks; ++s) {
            uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
            if (h < a.dh) {
                const uint4 *src = (const uint4 *)(a.dZt + (long long)h * a.ldt + kb + s * 16);
                v0 = __ldg(src);
                v1 = __ldg(src + 1);
            }
            *(uint4 *)(sA + s * 4096 + kmaj_off_bf16(t, 0)) = v0;
            *(uint4 *)(sA + s * 4096 + kmaj_off_bf16(t, 8)) = v1;
        }
        // B: row n = input f0 + n
        for (int n = t; n < nn; n += MLP_ROWS) {
            for (int s = 0; s < ks; ++s) {
                const uint4 *src = (const uint4 *)(a.Xt + (long long)(f0 + n) * a.ldt + kb + s * 16);
                *(uint4 *)(sB + (size_t)s * nn * 32 + kmaj_off_bf16(n, 0)) = __ldg(src);
                *(uint4 *)(sB + (size_t)s * nn * 32 + kmaj_off_bf16(n, 8)) = __ldg(src + 1);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int s = 0; s < ks; ++s) {
                const uint64_t da = umma_desc(su32(sA + s * 4096));
                const uint64_t db = umma_desc(su32(sB + (size_t)s * nn * 32));
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                             ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"((int)(pass > 0 || s > 0)));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(su32(bar))
                         : "memory");
        }
    }
    if (ok && pass > 0) {
        const bool w = mbar_wait(su32(bar), (uint32_t)((pass - 1) & 1), s_err);
        ok = !__syncthreads_or(!w);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // D[h][f] for this batch slice -> pW1[split][f][h]
        const long long nW1 = (long long)a.d_in * a.dh;
        float *dst = a.pW1 + (long long)blockIdx.z * nW1;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < nn; c += 32) {
            uint32_t v[32];
            tmem_ld32_nowait(trow + (uint32_t)c, v);
            tmem_wait_ld();
            if (h < a.dh) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c + j < nn)
                        dst[(long long)(f0 + c + j) * a.dh + h] = pass > 0 ? __uint_as_float(v[j]) : 0.f;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    if (!ok && t == 0)
        atomicOr(a.err, 1);
}

// k_mlp_infer_tc — inference (no targets), one persistent CTA per SM over
// 128-row tiles, warp-specialised so that loading, the tensor cores and the
// epilogue of different tiles overlap:
//   warps 0-1   load the X tile of the next row block (two rows per thread,
//               written in the core-matrix order) into one of two buffers;
//   warp 18     (one thread) issues the MMAs of a tile, all K steps at once
//               (W1^T stays in shared memory for the whole kernel), into one
//               of two TMEM accumulators;
//   warps 2-17  (four per TMEM lane quadrant, a quarter of the hidden units
//               each) read an accumulator, H = bf16(GELU(Z + b1)), the head.
// 19 warps: at most 5 per SM sub-partition, so 96 registers per thread.
// (X moved by TMA tensor copies of 16-byte-wide boxes measured slower.)
// Barriers: x_full / x_empty per X buffer, acc_full / acc_empty per
// accumulator; every wait is bounded (TC_WAIT_NS) and a failed wait ends the
// kernel with a.err set.
#define MLP_INF_LOADERS 64
#define MLP_INF_MMA_WARP ((MLP_INF_LOADERS + MLP_INF_EPI) / 32)
#define MLP_INF_EPI 512
#define MLP_INF_THREADS (MLP_INF_LOADERS + MLP_INF_EPI + 32)

__host__ __device__ inline size_t mlp_infer_smem(int d_in, int dh)
{
    const size_t nk = (size_t)d_in / 16;
    // W1^T + 2 X buffers + b1, W2 + head partials [2][4][128][2] + barriers
    return nk * (size_t)dh * 32 + 2 * nk * 4096 + (size_t)dh * 12 + 2 * 4 * 128 * 2 * 4 + 256;
}

__device__ __forceinline__ bool epi_any(bool v)
{
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "n"(MLP_INF_EPI)
                 : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(MLP_INF_THREADS, 1) k_mlp_infer_tc(const __grid_constant__ MlpFwdArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int dh = a.dh, nk = a.d_in / 16;
    const size_t wbytes = (size_t)nk * dh * 32, xbytes = (size_t)nk * 4096;
    unsigned char *sW = smem;
    unsigned char *sX = smem + wbytes; // [2][xbytes]
    float *s_b1 = (float *)(sX + 2 * xbytes);
    float *s_W2 = s_b1 + dh;
    float2 *s_y = (float2 *)(s_W2 + 2 * dh); // [2 buffers][4 quarters][128 rows]
    unsigned long long *bars = (unsigned long long *)(s_y + 2 * 4 * 128);
    uint32_t *tmem_slot = (uint32_t *)(bars + 10);
    volatile int *s_err = (volatile int *)(tmem_slot + 1);
    const uint32_t b_w = su32(bars), b_xf = su32(bars + 1), b_xe = su32(bars + 3);
    const uint32_t b_af = su32(bars + 5), b_ae = su32(bars + 7);
    const long long ntiles = (a.B + MLP_ROWS - 1) / MLP_ROWS;

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_w));
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_xf + 8u * b), "n"(MLP_INF_LOADERS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_xe + 8u * b));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_af + 8u * b));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_ae + 8u * b), "n"(MLP_INF_EPI));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_err = 0;
        // W1^T, one bulk copy per K step, all on one barrier
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_w), "r"((uint32_t)wbytes)
                     : "memory");
        for (int s = 0; s < nk; ++s)
            tma_copy_1d(su32(sW + (size_t)s * dh * 32), a.w1t + (size_t)s * dh * 16, (uint32_t)dh * 32, b_w);
    }
    for (int i = t; i < dh; i += MLP_INF_THREADS) {
        s_b1[i] = a.b1[i];
        s_W2[2 * i] = a.W2[2 * i];
        s_W2[2 * i + 1] = a.W2[2 * i + 1];
    }
    const uint32_t cols = a.tmem_cols; // >= 2 dh
    if (warp == MLP_INF_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(tmem_slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool w_seen = false;

    if (t < MLP_INF_LOADERS) {
        // ---- loaders: rows t and t + 64 of each tile
        for (long long j = 0;; ++j) {
            const long long T = blockIdx.x + j * gridDim.x;
            if (T >= ntiles)
                break;
            const int b = (int)(j & 1);
            if (j >= 2 && !mbar_wait(b_xe + 8u * b, (uint32_t)(((j >> 1) + 1) & 1), s_err))
                break;
            unsigned char *dst = sX + (size_t)b * xbytes;
            for (int h = 0; h < 2; ++h) {
                const int row = t + h * MLP_INF_LOADERS;
                const long long r = T * MLP_ROWS + row;
                const bool valid = r < a.B;
                const uint4 *src = (const uint4 *)(a.X + r * a.d_in);
                for (int s0 = 0; s0 < nk; s0 += 8) {
                    uint4 q[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        q[i] = (valid && s0 + (i >> 1) < nk) ? __ldg(src + 2 * s0 + i) : make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (s0 + (i >> 1) < nk)
                            *(uint4 *)(dst + (size_t)(s0 + (i >> 1)) * 4096 + kmaj_off_bf16(row, (i & 1) * 8)) = q[i];
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(b_xf + 8u * b);
        }
    } else if (t < MLP_INF_LOADERS + MLP_INF_EPI) {
        // ---- epilogue: warp e of 16; TMEM lane quadrant warp % 4, quarter
        // (e / 4) of the hidden units
        const int quad = warp & 3, quarter = (warp - MLP_INF_LOADERS / 32) >> 2;
        const int rr = quad * 32 + lane;
        const int qc = dh / 4, c0 = quarter * qc, c1 = c0 + qc;
        for (long long j = 0;; ++j) {
            const long long T = blockIdx.x + j * gridDim.x;
            if (T >= ntiles)
                break;
            const int b = (int)(j & 1);
            const bool ok = mbar_wait(b_af + 8u * b, (uint32_t)((j >> 1) & 1), s_err);
            if (epi_any(!ok))
                break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t trow = tmem + (uint32_t)(b * dh) + ((uint32_t)(quad * 32) << 16);
            float y0 = 0.f, y1 = 0.f;
            // 32 columns at a time; the load of the next 32 is in flight
            // while these are evaluated
            uint32_t va[32], vb[32];
            auto head32 = [&](const uint32_t (&v)[32], int c) {
                const float4 *b1v = (const float4 *)(s_b1 + c);
                const float4 *w2v = (const float4 *)(s_W2 + 2 * c);
#pragma unroll
                for (int jj = 0; jj < 32; jj += 4) {
                    const float4 bb = b1v[jj >> 2], wa = w2v[jj >> 1], wb = w2v[(jj >> 1) + 1];
                    const uint32_t p01 = bf2_pack(gelu_f(__uint_as_float(v[jj]) + bb.x),
                                                  gelu_f(__uint_as_float(v[jj + 1]) + bb.y));
                    const uint32_t p23 = bf2_pack(gelu_f(__uint_as_float(v[jj + 2]) + bb.z),
                                                  gelu_f(__uint_as_float(v[jj + 3]) + bb.w));
                    const float h0 = __uint_as_float(p01 << 16), h1 = __uint_as_float(p01 & 0xffff0000u);
                    const float h2 = __uint_as_float(p23 << 16), h3 = __uint_as_float(p23 & 0xffff0000u);
                    y0 = fmaf(h0, wa.x, y0);
                    y1 = fmaf(h0, wa.y, y1);
                    y0 = fmaf(h1, wa.z, y0);
                    y1 = fmaf(h1, wa.w, y1);
                    y0 = fmaf(h2, wb.x, y0);
                    y1 = fmaf(h2, wb.y, y1);
                    y0 = fmaf(h3, wb.z, y0);
                    y1 = fmaf(h3, wb.w, y1);
                }
            };
            tmem_ld32_nowait(trow + (uint32_t)c0, va);
            for (int c = c0; c < c1; c += 64) {
                tmem_wait_ld();
                if (c + 32 < c1)
                    tmem_ld32_nowait(trow + (uint32_t)(c + 32), vb);
                head32(va, c);
                if (c + 32 >= c1)
                    break;
                tmem_wait_ld();
                if (c + 64 < c1)
                    tmem_ld32_nowait(trow + (uint32_t)(c + 64), va);
                head32(vb, c + 32);
            }
            tmem_wait_ld();
            // the accumulator is free once this thread's loads have completed
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(b_ae + 8u * b);
            s_y[(b * 4 + quarter) * 128 + rr] = make_float2(y0, y1);
            asm volatile("bar.sync 1, %0;" ::"n"(MLP_INF_EPI) : "memory");
            const long long r = T * MLP_ROWS + rr;
            if (quarter == 0 && r < a.B) {
                const float2 p0 = s_y[(b * 4) * 128 + rr], p1 = s_y[(b * 4 + 1) * 128 + rr];
                const float2 p2 = s_y[(b * 4 + 2) * 128 + rr], p3 = s_y[(b * 4 + 3) * 128 + rr];
                a.Y[2 * r] = ((p0.x + p1.x) + (p2.x + p3.x)) + a.b2[0];
                a.Y[2 * r + 1] = ((p0.y + p1.y) + (p2.y + p3.y)) + a.b2[1];
            }
        }
    } else if (lane == 0) {
        // ---- MMA issuer
        long long last = -1;
        if (mbar_wait(b_w, 0, s_err)) {
            w_seen = true;
            const uint32_t idesc = mlp_idesc(128, dh);
            for (long long j = 0;; ++j) {
                const long long T = blockIdx.x + j * gridDim.x;
                if (T >= ntiles)
                    break;
                const int b = (int)(j & 1);
                if (!mbar_wait(b_xf + 8u * b, (uint32_t)((j >> 1) & 1), s_err))
                    break;
                if (j >= 2 && !mbar_wait(b_ae + 8u * b, (uint32_t)(((j >> 1) + 1) & 1), s_err))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t xa = su32(sX + (size_t)b * xbytes), wa = su32(sW);
                for (int s = 0; s < nk; ++s) {
                    const uint64_t da = umma_desc(xa + (uint32_t)s * 4096u);
                    const uint64_t db = umma_desc(wa + (uint32_t)(s * dh * 32));
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 ::"r"(tmem + (uint32_t)(b * dh)), "l"(da), "l"(db), "r"(idesc), "r"(s));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(b_xe + 8u * b)
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(b_af + 8u * b)
                             : "memory");
                last = j;
            }
        }
        // no MMA of this CTA may still run, and no commit still arrive, when
        // its TMEM and shared memory are released
        if (last >= 0) {
            mbar_wait(b_af + 8u * (int)(last & 1), (uint32_t)((last >> 1) & 1), nullptr);
            mbar_wait(b_xe + 8u * (int)(last & 1), (uint32_t)((last >> 1) & 1), nullptr);
        }
        // nor a copy into its shared memory
        if (!w_seen)
            mbar_wait(b_w, 0, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == MLP_INF_MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
    if (t == 0 && *s_err)
        atomicOr(a.err, 1);
}
