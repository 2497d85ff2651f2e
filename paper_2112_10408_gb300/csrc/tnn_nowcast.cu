// Nowcasting on top of the TNN context (Sec. 3.1-3.2): context features,
// the inverse-distance-weighted average, and a two-layer GELU MLP trained
// with AdamW (Sec. 4.1 trains its models with Adam over the whole training
// set, each sample with its own TNN context).
//
// MLP layout (flat FP32 master parameters, row-major):
//   W1 [d_in][d_h] | b1 [d_h] | W2 [d_h][2] | b2 [2]
// Forward  Z = X W1 + b1 (X, W1 in BF16, FP32 accumulation on the tensor
//          cores), H = GELU(Z) (rounded to BF16), Y = H W2 + b2 (FP32).
// Backward of mean((Y - T)^2) over B x 2:
//          dY = (Y - T) / B, dW2 = H^T dY, db2 = sum dY,
//          dZ = (dY W2^T) * GELU'(Z) (BF16), dW1 = X^T dZ, db1 = sum dZ.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "tnn_internal.cuh"

#define FULLMASK 0xffffffffu

__device__ __forceinline__ float bf2f(uint16_t h)
{
    return __uint_as_float(((unsigned)h) << 16);
}
__device__ __forceinline__ uint16_t f2bf(float f)
{
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&b);
}

// ---------------------------------------------------------------- features

struct FeatNorm {
    float mean[TNN_N_FEAT];
    float inv_std[TNN_N_FEAT];
    float ssq[4];
};

// One warp per query; lane r handles neighbour ranks r, r + 32.
__global__ void k_context_features(const float4 *__restrict__ pts,
                                   const float2 *__restrict__ wind,
                                   const float4 *__restrict__ q, int64_t m,
                                   const int32_t *__restrict__ idx,
                                   const float *__restrict__ d2, int k,
                                   const __grid_constant__ FeatNorm nrm, float eps,
                                   uint16_t *__restrict__ feat, float *__restrict__ idw)
{
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (qi >= m)
        return;
    const float4 qq = q[qi];
    float nu = 0.f, nv = 0.f, den = 0.f;
    for (int r = lane; r < k; r += 32) {
        const int j = idx[qi * k + r];
        float f[TNN_N_FEAT];
        if (j >= 0) {
            const float4 p = pts[j];
            const float2 w = wind[j];
            const float wt = 1.0f / (d2[qi * k + r] + eps);
            nu = fmaf(wt, w.x, nu);
            nv = fmaf(wt, w.y, nv);
            den += wt;
            f[0] = nrm.ssq[0] * (p.x - qq.x);
            f[1] = nrm.ssq[1] * (p.y - qq.y);
            f[2] = nrm.ssq[2] * (p.z - qq.z);
            f[3] = nrm.ssq[3] * (p.w - qq.w);
            f[4] = w.x;
            f[5] = w.y;
#pragma unroll
            for (int c = 0; c < TNN_N_FEAT; ++c)
                f[c] = (f[c] - nrm.mean[c]) * nrm.inv_std[c];
        } else {
#pragma unroll
            for (int c = 0; c < TNN_N_FEAT; ++c)
                f[c] = 0.f;
        }
        if (feat) {
            uint32_t *o = reinterpret_cast<uint32_t *>(feat + (qi * k + r) * TNN_N_FEAT);
#pragma unroll
            for (int c = 0; c < TNN_N_FEAT; c += 2)
                o[c / 2] = (uint32_t)f2bf(f[c]) | ((uint32_t)f2bf(f[c + 1]) << 16);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nu += __shfl_xor_sync(FULLMASK, nu, o);
        nv += __shfl_xor_sync(FULLMASK, nv, o);
        den += __shfl_xor_sync(FULLMASK, den, o);
    }
    if (lane == 0 && idw) {
        idw[2 * qi] = den > 0.f ? nu / den : __int_as_float(0x7fffffff);
        idw[2 * qi + 1] = den > 0.f ? nv / den : __int_as_float(0x7fffffff);
    }
}

extern "C" tnn_status tnn_context_features(const tnn_index *ix, const float *d_wind,
                                           const float *d_q, int64_t m,
                                           const int32_t *d_idx, const float *d_d2,
                                           int32_t k, const float *h_mean,
                                           const float *h_std, float idw_eps,
                                           uint16_t *d_feat, float *d_idw,
                                           tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && d_wind, "NULL argument");
    TNN_ARG_CHECK(k >= 1 && k <= 64, "k must be in [1, 64]");
    TNN_ARG_CHECK(m >= 0, "m must be >= 0");
    TNN_ARG_CHECK(d_q != nullptr || m == ix->n, "self-query needs m == n_points");
    TNN_ARG_CHECK(isfinite(idw_eps) && idw_eps >= 0.f, "idw_eps must be finite, >= 0");
    TNN_ARG_CHECK(((uintptr_t)d_wind & 7) == 0, "d_wind must be 8-byte aligned");
    if (m == 0)
        return TNN_OK;
    TNN_ARG_CHECK(d_idx && d_d2, "NULL neighbour lists");
    FeatNorm nrm;
    for (int c = 0; c < TNN_N_FEAT; ++c) {
        nrm.mean[c] = h_mean ? h_mean[c] : 0.f;
        float sd = h_std ? h_std[c] : 1.f;
        TNN_ARG_CHECK(isfinite(sd) && sd > 0.f, "std[%d] must be finite and > 0", c);
        nrm.inv_std[c] = 1.0f / sd;
    }
    for (int i = 0; i < 4; ++i)
        nrm.ssq[i] = (float)sqrt(ix->sigma[i]);
    const float4 *q = d_q ? (const float4 *)d_q : ix->pts;
    const int64_t threads = m * 32;
    k_context_features<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        ix->pts, (const float2 *)d_wind, q, m, d_idx, d_d2, k, nrm, idw_eps, d_feat, d_idw);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

// ------------------------------------------------------------------- MLP

// GELU(z) = z Phi(z) and GELU'(z) = Phi(z) + z phi(z), with the normal CDF
// Phi(z) = (1 + erf(z / sqrt 2)) / 2 and density phi(z) = exp(-z^2 / 2) /
// sqrt(2 pi).  erf by Abramowitz & Stegun, Handbook of Mathematical
// Functions, formula 7.1.26: erf(x) = 1 - (a1 t + ... + a5 t^5) exp(-x^2),
// t = 1 / (1 + p x) for x >= 0, absolute error <= 1.5e-7 -- far below the
// BF16 rounding that H and dZ receive.  The same exp(-x^2) = exp(-z^2 / 2)
// serves phi.  Returns (Phi(z), exp(-z^2 / 2)).
__device__ __forceinline__ float2 normal_cdf_and_gauss(float z)
{
    const float x = z * 0.70710678118654752f;
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    float poly = fmaf(t, 1.061405429f, -1.453152027f);
    poly = fmaf(t, poly, 1.421413741f);
    poly = fmaf(t, poly, -0.284496736f);
    poly = fmaf(t, poly, 0.254829592f);
    poly *= t;
    const float g = __expf(-ax * ax);
    const float erf_ax = fmaf(-poly, g, 1.0f);
    const float erf_x = copysignf(erf_ax, x);
    return make_float2(fmaf(0.5f, erf_x, 0.5f), g);
}
// z Phi(z) by the same approximation, with the scalings by 1/sqrt(2) and 1/2
// folded into its constants: for z >= 0, z Phi(z) = z - q and for z < 0 it is
// q, where q = z t P(t) exp(-z^2 / 2) / 2 and t = 1 / (1 + p |z| / sqrt(2)).
__device__ __forceinline__ float gelu_f(float z)
{
    const float t = __fdividef(1.0f, fmaf(0.3275911f * 0.70710678118654752f, fabsf(z), 1.0f));
    float poly = fmaf(t, 0.5f * 1.061405429f, 0.5f * -1.453152027f);
    poly = fmaf(t, poly, 0.5f * 1.421413741f);
    poly = fmaf(t, poly, 0.5f * -0.284496736f);
    poly = fmaf(t, poly, 0.5f * 0.254829592f);
    poly *= t;
    float g; // 2^(-z^2 log2(e) / 2)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(z * (z * -0.72134752044448170f)));
    const float q = (poly * g) * z;
    return z >= 0.0f ? z - q : q;
}
__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float2 pg = normal_cdf_and_gauss(z);
    return fmaf(z * 0.39894228040143268f, pg.y, pg.x);
}

#include "tnn_mlp_tc.cuh"

// Position of W1[f][h] in the BF16 W1^T operand: K step f / 16 holds
// [dh rows][16] in core-matrix order.
__device__ __forceinline__ long long w1t_index(int f, int h, int dh)
{
    return (long long)(f >> 4) * dh * 16 + (kmaj_off_bf16(h, f & 15) >> 1);
}

struct AdamArgs {
    float *w, *m, *v;
    uint16_t *w1t;    // BF16 W1^T operand, refreshed after the update
    float *grad_out; // if non-null: write the reduced gradient, no update
    const float *pW1; // [splits1][d_in*dh]
    int splits1;
    const float *pCol; // [splits2][dh*3+2]
    int splits2;
    int d_in, dh;
    long long P;
    float lr, b1, b2, eps, wd;
    const long long *step; // already advanced for this update
    const float *sse;
    float *loss_out;
    float inv_count;
};

// Reduce the gradient partials and apply AdamW (decoupled weight decay),
// refreshing the BF16 W1^T operand.
__global__ void k_adamw(const __grid_constant__ AdamArgs a)
{
    __shared__ float s_bc[2];
    if (threadIdx.x == 0 && !a.grad_out) {
        // 1 - beta^t = -expm1(t log1p(beta - 1)): beta - 1 is exact in FP32
        // and neither step cancels, so no FP64 is needed
        const float t = (float)*a.step;
        s_bc[0] = -expm1f(t * log1pf(a.b1 - 1.0f));
        s_bc[1] = -expm1f(t * log1pf(a.b2 - 1.0f));
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && a.loss_out)
        *a.loss_out = *a.sse * a.inv_count;
    if (p >= a.P)
        return;
    const long long nW1 = (long long)a.d_in * a.dh;
    const int stride = a.dh * 3 + 2;
    // partial sums over the batch slices: four independent chains so that
    // the loads overlap (the order is fixed, so the result is deterministic)
    const float *src;
    long long ld;
    int ns;
    if (p < nW1) {
        src = a.pW1 + p;
        ld = nW1;
        ns = a.splits1;
    } else {
        src = a.pCol + (p - nW1); // b1 | W2 | b2 in the same order as pCol
        ld = stride;
        ns = a.splits2;
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
    int s = 0;
    for (; s + 4 <= ns; s += 4) {
        g0 += src[(long long)s * ld];
        g1 += src[(long long)(s + 1) * ld];
        g2 += src[(long long)(s + 2) * ld];
        g3 += src[(long long)(s + 3) * ld];
    }
    for (; s < ns; ++s)
        g0 += src[(long long)s * ld];
    const float g = (g0 + g1) + (g2 + g3);
    if (a.grad_out) {
        a.grad_out[p] = g;
        return;
    }
    const float m = a.b1 * a.m[p] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[p] + (1.f - a.b2) * g * g;
    a.m[p] = m;
    a.v[p] = v;
    const float mh = m / s_bc[0], vh = v / s_bc[1];
    const float w = a.w[p] - a.lr * (mh / (sqrtf(vh) + a.eps) + a.wd * a.w[p]);
    a.w[p] = w;
    if (p < nW1)
        a.w1t[w1t_index((int)(p / a.dh), (int)(p % a.dh), a.dh)] = f2bf(w);
}

// The BF16 W1^T operand from the FP32 master W1 [d_in][dh].
__global__ void k_to_w1t(const float *__restrict__ w, uint16_t *__restrict__ w1t, int d_in, int dh)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < (long long)d_in * dh)
        w1t[w1t_index((int)(p / dh), (int)(p % dh), dh)] = f2bf(w[p]);
}

// ---------------------------------------------------------------- objects

struct tnn_mlp {
    int device;
    int d_in, dh;
    long long P;
    float *w, *m, *v;
    uint16_t *w1t; // BF16 W1^T in the tensor-core operand order
    float *acc;    // [0] squared error, [1] loss
    int *err;      // set by a kernel whose device wait timed out
    long long *step; // AdamW step count, on the device (CUDA-graph replays advance it)
    // training workspace, grown on demand
    long long cap_B, ldt;
    float *dY, *Y, *pW1, *pCol, *grad;
    uint16_t *Xt, *dZt;
};

static void mlp_free_ws(tnn_mlp *n)
{
    cudaFree(n->dY);
    cudaFree(n->Y);
    cudaFree(n->pW1);
    cudaFree(n->pCol);
    cudaFree(n->grad);
    cudaFree(n->Xt);
    cudaFree(n->dZt);
    n->dY = n->Y = n->pW1 = n->pCol = n->grad = nullptr;
    n->Xt = n->dZt = nullptr;
    n->cap_B = n->ldt = 0;
}

extern "C" void tnn_mlp_destroy(tnn_mlp *n)
{
    if (!n)
        return;
    mlp_free_ws(n);
    cudaFree(n->w);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->w1t);
    cudaFree(n->acc);
    cudaFree(n->err);
    cudaFree(n->step);
    delete n;
}

#define MLP_MAX_SPLITS 64

// Batch slices of the dW1 product: at most MLP_MAX_SPLITS, each a multiple
// of 16 rows.
static long long mlp_rows_per_split(long long B)
{
    const long long Bp = (B + 15) / 16 * 16;
    long long rows = (Bp + MLP_MAX_SPLITS - 1) / MLP_MAX_SPLITS;
    rows = std::max<long long>(128, (rows + 15) / 16 * 16);
    return rows;
}

// Training workspace for batches of up to B rows (inference needs none).
static tnn_status mlp_reserve(tnn_mlp *n, long long B)
{
    if (B <= n->cap_B)
        return TNN_OK;
    mlp_free_ws(n);
    const long long cap = std::max<long long>(B, 256);
    const long long ldt = (cap + 15) / 16 * 16;
    const long long nW1 = (long long)n->d_in * n->dh;
    cudaError_t e = cudaSuccess;
#define A_(p, bytes)                                                          \
    if (e == cudaSuccess)                                                     \
        e = cudaMalloc((void **)&(p), (bytes));
    A_(n->dY, sizeof(float) * cap * 2);
    A_(n->Y, sizeof(float) * cap * 2);
    A_(n->pW1, sizeof(float) * MLP_MAX_SPLITS * nW1);
    A_(n->pCol, sizeof(float) * ((cap + MLP_ROWS - 1) / MLP_ROWS) * (3LL * n->dh + 2));
    A_(n->grad, sizeof(float) * n->P);
    A_(n->Xt, sizeof(uint16_t) * n->d_in * ldt);
    A_(n->dZt, sizeof(uint16_t) * n->dh * ldt);
#undef A_
    if (e != cudaSuccess) {
        mlp_free_ws(n);
        tnn_set_error("MLP workspace allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    n->cap_B = cap;
    n->ldt = ldt;
    return TNN_OK;
}

static uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" tnn_status tnn_mlp_create(int32_t d_in, int32_t d_hidden, uint64_t seed,
                                     tnn_mlp **out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    TNN_ARG_CHECK(d_in >= 16 && d_in <= 1024 && d_in % 16 == 0,
                  "d_in must be a multiple of 16 in [16, 1024]");
    TNN_ARG_CHECK(d_hidden >= 64 && d_hidden <= 512 && d_hidden % 64 == 0,
                  "d_hidden must be a multiple of 64 in [64, 512]");
    tnn_mlp *n = new tnn_mlp();
    memset(n, 0, sizeof(*n));
    cudaGetDevice(&n->device);
    n->d_in = d_in;
    n->dh = d_hidden;
    n->P = (long long)d_in * d_hidden + d_hidden + 2LL * d_hidden + 2;
    // Kaiming-uniform: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases.
    std::vector<float> h(n->P);
    uint64_t s = seed;
    const float b1 = 1.0f / sqrtf((float)d_in), b2 = 1.0f / sqrtf((float)d_hidden);
    const long long nW1 = (long long)d_in * d_hidden;
    for (long long i = 0; i < n->P; ++i) {
        const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
        const float bound = i < nW1 + d_hidden ? b1 : b2;
        h[i] = (float)((2.0 * u - 1.0) * bound);
    }
    cudaError_t e = cudaMalloc(&n->w, sizeof(float) * n->P);
    if (e == cudaSuccess)
        e = cudaMalloc(&n->m, sizeof(float) * n->P);
    if (e == cudaSuccess)
        e = cudaMalloc(&n->v, sizeof(float) * n->P);
    if (e == cudaSuccess)
        e = cudaMalloc(&n->w1t, sizeof(uint16_t) * nW1);
    if (e == cudaSuccess)
        e = cudaMalloc(&n->acc, sizeof(float) * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(&n->err, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(&n->step, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemset(n->step, 0, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemset(n->err, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(n->w, h.data(), sizeof(float) * n->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(n->m, 0, sizeof(float) * n->P);
    if (e == cudaSuccess)
        e = cudaMemset(n->v, 0, sizeof(float) * n->P);
    if (e == cudaSuccess) {
        k_to_w1t<<<(unsigned)((nW1 + 255) / 256), 256>>>(n->w, n->w1t, d_in, d_hidden);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        tnn_mlp_destroy(n);
        tnn_set_error("MLP allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    *out = n;
    return TNN_OK;
}

extern "C" int64_t tnn_mlp_num_params(const tnn_mlp *n) { return n ? n->P : 0; }

extern "C" tnn_status tnn_mlp_get_params(const tnn_mlp *n, float *h_params, float *h_m,
                                         float *h_v, int64_t *h_step)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n != nullptr, "mlp is NULL");
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    int derr = 0;
    TNN_CUDA_TRY(cudaMemcpy(&derr, n->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (derr) {
        tnn_set_error("a device wait of the MLP kernels timed out");
        return TNN_ERR_TIMEOUT;
    }
    if (h_params)
        TNN_CUDA_TRY(cudaMemcpy(h_params, n->w, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_m)
        TNN_CUDA_TRY(cudaMemcpy(h_m, n->m, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_v)
        TNN_CUDA_TRY(cudaMemcpy(h_v, n->v, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_step)
        TNN_CUDA_TRY(cudaMemcpy(h_step, n->step, sizeof(long long), cudaMemcpyDeviceToHost));
    return TNN_OK;
}

extern "C" tnn_status tnn_mlp_set_params(tnn_mlp *n, const float *h_params, const float *h_m,
                                         const float *h_v, int64_t step)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n != nullptr && h_params != nullptr, "NULL argument");
    TNN_ARG_CHECK(step >= 0, "step must be >= 0");
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    TNN_CUDA_TRY(cudaMemcpy(n->w, h_params, sizeof(float) * n->P, cudaMemcpyHostToDevice));
    if (h_m)
        TNN_CUDA_TRY(cudaMemcpy(n->m, h_m, sizeof(float) * n->P, cudaMemcpyHostToDevice));
    else
        TNN_CUDA_TRY(cudaMemset(n->m, 0, sizeof(float) * n->P));
    if (h_v)
        TNN_CUDA_TRY(cudaMemcpy(n->v, h_v, sizeof(float) * n->P, cudaMemcpyHostToDevice));
    else
        TNN_CUDA_TRY(cudaMemset(n->v, 0, sizeof(float) * n->P));
    {
        const long long hs = step;
        TNN_CUDA_TRY(cudaMemcpy(n->step, &hs, sizeof(long long), cudaMemcpyHostToDevice));
    }
    const long long nW1 = (long long)n->d_in * n->dh;
    k_to_w1t<<<(unsigned)((nW1 + 255) / 256), 256>>>(n->w, n->w1t, n->d_in, n->dh);
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    return TNN_OK;
}

// ------------------------------------------------------------- checkpoint

// File layout (little-endian whatever the host): five int64 -- magic
// "TNNM" (0x544E4E4D), version 1, d_in, d_hidden, AdamW step -- then the
// flat parameters, the first and the second AdamW moments, P float32 each.
#define TNN_MLP_MAGIC 0x544E4E4Dll
#define TNN_MLP_VERSION 1

static void put_le64(unsigned char *b, long long v)
{
    const unsigned long long u = (unsigned long long)v;
    for (int i = 0; i < 8; ++i)
        b[i] = (unsigned char)(u >> (8 * i));
}
static long long get_le64(const unsigned char *b)
{
    unsigned long long u = 0;
    for (int i = 0; i < 8; ++i)
        u |= (unsigned long long)b[i] << (8 * i);
    return (long long)u;
}
static void f32_to_le(const float *x, long long n, unsigned char *b)
{
    for (long long i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, x + i, 4);
        for (int j = 0; j < 4; ++j)
            b[4 * i + j] = (unsigned char)(u >> (8 * j));
    }
}
static void le_to_f32(const unsigned char *b, long long n, float *x)
{
    for (long long i = 0; i < n; ++i) {
        uint32_t u = 0;
        for (int j = 0; j < 4; ++j)
            u |= (uint32_t)b[4 * i + j] << (8 * j);
        memcpy(x + i, &u, 4);
    }
}

extern "C" tnn_status tnn_mlp_save(const tnn_mlp *n, const char *path)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n != nullptr && path != nullptr, "NULL argument");
    std::vector<float> h(3 * (size_t)n->P);
    int64_t step = 0;
    tnn_status s = tnn_mlp_get_params(n, h.data(), h.data() + n->P, h.data() + 2 * n->P, &step);
    if (s != TNN_OK)
        return s;
    std::vector<unsigned char> buf(40 + 4 * h.size());
    put_le64(&buf[0], TNN_MLP_MAGIC);
    put_le64(&buf[8], TNN_MLP_VERSION);
    put_le64(&buf[16], n->d_in);
    put_le64(&buf[24], n->dh);
    put_le64(&buf[32], step);
    f32_to_le(h.data(), (long long)h.size(), &buf[40]);
    FILE *f = fopen(path, "wb");
    TNN_ARG_CHECK(f != nullptr, "cannot open %s for writing", path);
    const size_t wr = fwrite(buf.data(), 1, buf.size(), f);
    const int cl = fclose(f);
    TNN_ARG_CHECK(wr == buf.size() && cl == 0, "writing %s failed", path);
    return TNN_OK;
}

extern "C" tnn_status tnn_mlp_load(tnn_mlp *n, const char *path)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n != nullptr && path != nullptr, "NULL argument");
    FILE *f = fopen(path, "rb");
    TNN_ARG_CHECK(f != nullptr, "cannot open %s", path);
    unsigned char hdr[40];
    const size_t got = fread(hdr, 1, sizeof(hdr), f);
    if (got != sizeof(hdr) || get_le64(hdr) != TNN_MLP_MAGIC || get_le64(hdr + 8) != TNN_MLP_VERSION ||
        get_le64(hdr + 16) != n->d_in || get_le64(hdr + 24) != n->dh || get_le64(hdr + 32) < 0) {
        fclose(f);
        tnn_set_error("%s is not a checkpoint of a %d -> %d MLP", path, n->d_in, n->dh);
        return TNN_ERR_INVALID_ARG;
    }
    std::vector<unsigned char> buf(12 * (size_t)n->P);
    const size_t body = fread(buf.data(), 1, buf.size(), f);
    fclose(f);
    TNN_ARG_CHECK(body == buf.size(), "%s is truncated", path);
    std::vector<float> h(3 * (size_t)n->P);
    le_to_f32(buf.data(), (long long)h.size(), h.data());
    return tnn_mlp_set_params(n, h.data(), h.data() + n->P, h.data() + 2 * n->P, get_le64(hdr + 32));
}

// Dynamic shared memory of a tensor-core kernel, raised so that no more CTAs
// share an SM than its TMEM (512 columns) holds at once.
static size_t tc_smem_request(size_t need, uint32_t cols)
{
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int max_ctas = (int)(512 / cols);
    const size_t floor_ = (size_t)per_sm / (size_t)(max_ctas + 1); // (max_ctas + 1) x (smem + 1 KB) > per SM
    return std::max(need, floor_);
}

static tnn_status mlp_setup()
{
    static bool done = false;
    if (!done) {
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_mlp_dw1_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        TNN_CUDA_TRY(cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        done = true;
    }
    return TNN_OK;
}

static tnn_status mlp_forward_impl(const tnn_mlp *n, const uint16_t *d_x, long long B,
                                   float *d_y, const float *d_t, cudaStream_t st)
{
    TNN_ARG_CHECK(((uintptr_t)d_x & 15) == 0, "X must be 16-byte aligned");
    tnn_status s = mlp_setup();
    if (s != TNN_OK)
        return s;
    const long long nW1 = (long long)n->d_in * n->dh;
    MlpFwdArgs a;
    memset(&a, 0, sizeof(a));
    a.X = d_x;
    a.B = B;
    a.d_in = n->d_in;
    a.dh = n->dh;
    a.w1t = n->w1t;
    a.b1 = n->w + nW1;
    a.W2 = a.b1 + n->dh;
    a.b2 = a.W2 + 2 * n->dh;
    a.Y = d_y;
    a.T = d_t;
    a.dY = n->dY;
    a.dZt = n->dZt;
    a.Xt = n->Xt;
    a.ldt = n->ldt;
    a.pCol = n->pCol;
    a.sse = n->acc;
    a.inv_B = 1.0f / (float)B;
    a.tmem_cols = tmem_cols_for(n->dh);
    a.err = n->err;
    if (d_t)
        TNN_CUDA_TRY(cudaMemsetAsync(n->acc, 0, sizeof(float) * 4, st));
    if (!d_t && n->dh % 128 == 0 && n->dh <= 256 &&
        mlp_infer_smem(n->d_in, n->dh) <= (size_t)227 * 1024) {
        // inference: persistent warp-specialised kernel, one CTA per SM
        int dev = 0, nsm = 0;
        TNN_CUDA_TRY(cudaGetDevice(&dev));
        TNN_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        a.tmem_cols = tmem_cols_for(2 * n->dh);
        const long long tiles = (B + MLP_ROWS - 1) / MLP_ROWS;
        k_mlp_infer_tc<<<(unsigned)std::min<long long>(tiles, nsm), MLP_INF_THREADS,
                         mlp_infer_smem(n->d_in, n->dh), st>>>(a);
        TNN_CUDA_TRY(cudaGetLastError());
        return TNN_OK;
    }
    // every K step staged at once when it fits (no per-step synchronisation)
    a.resident = mlp_fwd_smem_res(n->d_in, n->dh) <= (size_t)227 * 1024;
    const size_t smem = tc_smem_request(a.resident ? mlp_fwd_smem_res(n->d_in, n->dh) : mlp_fwd_smem(n->dh),
                                        a.tmem_cols);
    k_mlp_fwd_tc<<<(unsigned)((B + MLP_ROWS - 1) / MLP_ROWS), MLP_FWD_THREADS, smem, st>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

extern "C" tnn_status tnn_mlp_forward(const tnn_mlp *n, const uint16_t *d_x, int64_t B,
                                      float *d_y, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n && d_x && d_y, "NULL argument");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31) / 512, "B out of range");
    return mlp_forward_impl(n, d_x, B, d_y, nullptr, (cudaStream_t)stream);
}

static tnn_status mlp_backward_impl(tnn_mlp *n, const uint16_t *d_x, long long B,
                                    const float *d_t, const tnn_adamw_params *opt,
                                    float *d_loss, float *d_grad, cudaStream_t st)
{
    tnn_status s = mlp_forward_impl(n, d_x, B, n->Y, d_t, st);
    if (s != TNN_OK)
        return s;
    // dW1^T = dZ^T X over batch slices
    const long long rows_per = mlp_rows_per_split(B);
    const long long Bp = (B + 15) / 16 * 16;
    const int splits1 = (int)((Bp + rows_per - 1) / rows_per);
    MlpDw1Args d;
    memset(&d, 0, sizeof(d));
    d.dZt = n->dZt;
    d.Xt = n->Xt;
    d.ldt = n->ldt;
    d.Bp = Bp;
    d.d_in = n->d_in;
    d.dh = n->dh;
    d.rows_per = rows_per;
    d.pW1 = n->pW1;
    d.tmem_cols = tmem_cols_for(std::min(256, n->d_in));
    d.err = n->err;
    d.step_inc = opt ? n->step : nullptr;
    dim3 grid((unsigned)((n->dh + 127) / 128), (unsigned)((n->d_in + 255) / 256), (unsigned)splits1);
    k_mlp_dw1_tc<<<grid, MLP_ROWS, tc_smem_request(mlp_dw1_smem(), d.tmem_cols), st>>>(d);
    TNN_CUDA_TRY(cudaGetLastError());
    AdamArgs a;
    memset(&a, 0, sizeof(a));
    a.w = n->w;
    a.m = n->m;
    a.v = n->v;
    a.w1t = n->w1t;
    a.grad_out = d_grad;
    a.pW1 = n->pW1;
    a.splits1 = splits1;
    a.pCol = n->pCol;
    a.splits2 = (int)((B + MLP_ROWS - 1) / MLP_ROWS);
    a.d_in = n->d_in;
    a.dh = n->dh;
    a.P = n->P;
    a.sse = n->acc;
    a.loss_out = d_loss;
    a.inv_count = 1.0f / (2.0f * (float)B);
    if (opt) {
        a.lr = opt->lr;
        a.b1 = opt->beta1;
        a.b2 = opt->beta2;
        a.eps = opt->eps;
        a.wd = opt->weight_decay;
        a.step = n->step;
    }
    k_adamw<<<(unsigned)((n->P + 255) / 256), 256, 0, st>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

extern "C" tnn_status tnn_mlp_gradients(tnn_mlp *n, const uint16_t *d_x,
                                        const float *d_target, int64_t B, float *d_loss,
                                        float *d_grad, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n && d_x && d_target && d_grad, "NULL argument");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31) / 512, "B out of range");
    tnn_status s = mlp_reserve(n, B);
    if (s != TNN_OK)
        return s;
    return mlp_backward_impl(n, d_x, B, d_target, nullptr, d_loss, d_grad,
                             (cudaStream_t)stream);
}

extern "C" tnn_status tnn_mlp_train_step(tnn_mlp *n, const uint16_t *d_x,
                                         const float *d_target, int64_t B,
                                         const tnn_adamw_params *opt, float *d_loss,
                                         tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n && d_x && d_target && opt, "NULL argument");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31) / 512, "B out of range");
    TNN_ARG_CHECK(opt->lr >= 0.f && opt->beta1 >= 0.f && opt->beta1 < 1.f &&
                      opt->beta2 >= 0.f && opt->beta2 < 1.f && opt->eps > 0.f &&
                      opt->weight_decay >= 0.f,
                  "invalid AdamW parameters");
    tnn_status s = mlp_reserve(n, B);
    if (s != TNN_OK)
        return s;
    return mlp_backward_impl(n, d_x, B, d_target, opt, d_loss, nullptr,
                             (cudaStream_t)stream);
}

// ----------------------------------------------------------------- nowcast

extern "C" tnn_status tnn_nowcast(const tnn_index *ix, const float *d_wind,
                                  const float *d_q, int64_t m,
                                  const tnn_knn_params *params, const tnn_mlp *mlp,
                                  const float *h_mean, const float *h_std, float idw_eps,
                                  float *d_uv, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(ix && d_wind && params && d_uv, "NULL argument");
    if (m == 0)
        return TNN_OK;
    const int k = params->k;
    if (mlp)
        TNN_ARG_CHECK(mlp->d_in == k * TNN_N_FEAT, "MLP input width %d != k * 6 = %d",
                      mlp->d_in, k * TNN_N_FEAT);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *idx = nullptr;
    float *d2 = nullptr;
    uint16_t *feat = nullptr;
    TNN_CUDA_TRY(tnn_alloc((void **)&idx, sizeof(int32_t) * m * k, st));
    cudaError_t e = tnn_alloc((void **)&d2, sizeof(float) * m * k, st);
    if (e == cudaSuccess && mlp)
        e = tnn_alloc((void **)&feat, sizeof(uint16_t) * m * k * TNN_N_FEAT, st);
    tnn_status s = TNN_OK;
    if (e != cudaSuccess) {
        tnn_set_error("nowcast allocation failed: %s", cudaGetErrorString(e));
        s = TNN_ERR_OOM;
    }
    if (s == TNN_OK)
        s = tnn_knn(ix, d_q, m, params, idx, d2, nullptr, stream);
    if (s == TNN_OK)
        s = tnn_context_features(ix, d_wind, d_q, m, idx, d2, k, h_mean, h_std, idw_eps,
                                 feat, mlp ? nullptr : d_uv, stream);
    if (s == TNN_OK && mlp)
        s = tnn_mlp_forward(mlp, feat, m, d_uv, stream);
    tnn_free(idx, st);
    if (d2)
        tnn_free(d2, st);
    if (feat)
        tnn_free(feat, st);
    return s;
}
