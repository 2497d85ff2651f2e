// Nowcasting on top of the TNN context (Sec. 3.1-3.2): context features,
// the inverse-distance-weighted average, and a two-layer GELU MLP trained
// with AdamW (Sec. 4.1 trains its models with Adam over the whole training
// set, each sample with its own TNN context).
//
// MLP layout (flat FP32 master parameters, row-major):
//   W1 [d_in][d_h] | b1 [d_h] | W2 [d_h][2] | b2 [2]
// Forward  Z = X W1 + b1 (X, W1 in BF16, FP32 accumulation), H = GELU(Z)
//          (kept in BF16), Y = H W2 + b2 (FP32).
// Backward of mean((Y - T)^2) over B x 2:
//          dY = (Y - T) / B, dW2 = H^T dY, db2 = sum dY,
//          dZ = (dY W2^T) * GELU'(Z) (BF16), dW1 = X^T dZ, db1 = sum dZ.
#include <math.h>
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

// --------------------------------------------------------------- SIMT GEMM

// C(m, n) = sum_k A(m, k) B(k, n) with A, B in BF16 (strided), FP32
// accumulation.  64 x 64 output tile per block of 256 threads (4 x 4 per
// thread), K staged 16 at a time through shared memory.  blockIdx.z splits K.
enum { EPI_FWD = 0, EPI_PARTIAL = 1 };

struct GemmArgs {
    const uint16_t *A;
    long long lda_m, lda_k;
    const uint16_t *B;
    long long ldb_k, ldb_n;
    int M, N, K;
    int k_per_split;
    // EPI_FWD: Z = acc + bias[n] (FP32), H = bf16(GELU(Z))
    const float *bias;
    float *Z;
    uint16_t *H;
    // EPI_PARTIAL: P[split][m][n] = acc
    float *P;
};

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

template <int EPI>
__global__ void __launch_bounds__(256) k_gemm_bf16(const __grid_constant__ GemmArgs g)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * g.k_per_split;
    const int ke = min(g.K, kb + g.k_per_split);
    const int tm = (tid >> 4) * 4, tn = (tid & 15) * 4;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e >> 6, mm = e & 63;
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < g.M && gk < ke) ? bf2f(g.A[gm * g.lda_m + gk * g.lda_k]) : 0.f;
            const int gn = n0 + mm;
            Bs[kk][mm] = (gn < g.N && gk < ke) ? bf2f(g.B[gk * g.ldb_k + gn * g.ldb_n]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][tm + i];
                b[i] = Bs[kk][tn + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tm + i;
        if (gm >= g.M)
            continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tn + j;
            if (gn >= g.N)
                continue;
            if (EPI == EPI_FWD) {
                const float z = acc[i][j] + g.bias[gn];
                g.Z[(long long)gm * g.N + gn] = z;
                g.H[(long long)gm * g.N + gn] = f2bf(gelu_f(z));
            } else {
                g.P[((long long)blockIdx.z * g.M + gm) * g.N + gn] = acc[i][j];
            }
        }
    }
}

// Output head and its backward, one warp per row: Y = H W2 + b2; with a
// target, dY = (Y - T)/B, dZ = (dY W2^T) * GELU'(Z) (BF16) and the squared
// error summed into *sse.
__global__ void k_head(const uint16_t *__restrict__ H, const float *__restrict__ Z,
                       const float *__restrict__ W2, const float *__restrict__ b2,
                       int B, int dh, float *__restrict__ Y,
                       const float *__restrict__ T, float *__restrict__ dY,
                       uint16_t *__restrict__ dZ, float *sse)
{
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= B)
        return;
    float y0 = 0.f, y1 = 0.f;
    for (int h = lane; h < dh; h += 32) {
        const float hv = bf2f(H[(long long)r * dh + h]);
        y0 = fmaf(hv, W2[2 * h], y0);
        y1 = fmaf(hv, W2[2 * h + 1], y1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(FULLMASK, y0, o);
        y1 += __shfl_xor_sync(FULLMASK, y1, o);
    }
    y0 += b2[0];
    y1 += b2[1];
    if (lane == 0 && Y) {
        Y[2 * r] = y0;
        Y[2 * r + 1] = y1;
    }
    if (!T)
        return;
    const float e0 = y0 - T[2 * r], e1 = y1 - T[2 * r + 1];
    const float g0 = e0 / (float)B, g1 = e1 / (float)B; // d mean over 2B of e^2
    if (lane == 0) {
        dY[2 * r] = g0;
        dY[2 * r + 1] = g1;
        atomicAdd(sse, e0 * e0 + e1 * e1);
    }
    for (int h = lane; h < dh; h += 32) {
        const float dh_ = fmaf(g0, W2[2 * h], g1 * W2[2 * h + 1]);
        dZ[(long long)r * dh + h] = f2bf(dh_ * gelu_grad_f(Z[(long long)r * dh + h]));
    }
}

// Column sums over row slices: partials of db1 [dh], dW2 [dh][2], db2 [2].
__global__ void k_colsums(const uint16_t *__restrict__ H, const uint16_t *__restrict__ dZ,
                          const float *__restrict__ dY, int B, int dh, int rows_per,
                          float *__restrict__ part) // [splits][dh*3 + 2]
{
    const int s = blockIdx.x;
    const int r0 = s * rows_per, r1 = min(B, r0 + rows_per);
    const int stride = dh * 3 + 2;
    for (int h = threadIdx.x; h < dh; h += blockDim.x) {
        float db1 = 0.f, w0 = 0.f, w1 = 0.f;
        for (int r = r0; r < r1; ++r) {
            db1 += bf2f(dZ[(long long)r * dh + h]);
            const float hv = bf2f(H[(long long)r * dh + h]);
            w0 = fmaf(hv, dY[2 * r], w0);
            w1 = fmaf(hv, dY[2 * r + 1], w1);
        }
        part[(long long)s * stride + h] = db1;
        part[(long long)s * stride + dh + 2 * h] = w0;
        part[(long long)s * stride + dh + 2 * h + 1] = w1;
    }
    if (threadIdx.x < 2) {
        float g = 0.f;
        for (int r = r0; r < r1; ++r)
            g += dY[2 * r + threadIdx.x];
        part[(long long)s * stride + 3 * dh + threadIdx.x] = g;
    }
}

struct AdamArgs {
    float *w, *m, *v;
    uint16_t *w1_bf16;
    float *grad_out; // if non-null: write the reduced gradient, no update
    const float *pW1; // [splits1][d_in*dh]
    int splits1;
    const float *pCol; // [splits2][dh*3+2]
    int splits2;
    int d_in, dh;
    long long P;
    float lr, b1, b2, eps, wd, bc1, bc2;
    const float *sse;
    float *loss_out;
    float inv_count;
};

// Reduce the gradient partials and apply AdamW (decoupled weight decay),
// refreshing the BF16 copy of W1.
__global__ void k_adamw(const __grid_constant__ AdamArgs a)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && a.loss_out)
        *a.loss_out = *a.sse * a.inv_count;
    if (p >= a.P)
        return;
    const long long nW1 = (long long)a.d_in * a.dh;
    const int stride = a.dh * 3 + 2;
    float g = 0.f;
    if (p < nW1) {
        for (int s = 0; s < a.splits1; ++s)
            g += a.pW1[(long long)s * nW1 + p];
    } else {
        const long long q = p - nW1; // b1 | W2 | b2 in the same order as pCol
        for (int s = 0; s < a.splits2; ++s)
            g += a.pCol[(long long)s * stride + q];
    }
    if (a.grad_out) {
        a.grad_out[p] = g;
        return;
    }
    const float m = a.b1 * a.m[p] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[p] + (1.f - a.b2) * g * g;
    a.m[p] = m;
    a.v[p] = v;
    const float mh = m / a.bc1, vh = v / a.bc2;
    const float w = a.w[p] - a.lr * (mh / (sqrtf(vh) + a.eps) + a.wd * a.w[p]);
    a.w[p] = w;
    if (p < nW1)
        a.w1_bf16[p] = f2bf(w);
}

__global__ void k_to_bf16(const float *__restrict__ x, uint16_t *__restrict__ y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        y[i] = f2bf(x[i]);
}

// ---------------------------------------------------------------- objects

struct tnn_mlp {
    int device;
    int d_in, dh;
    long long P;
    float *w, *m, *v;
    uint16_t *w1b;
    long long step;
    // workspace, grown on demand
    long long cap_B;
    float *Z, *dY, *Y, *pW1, *pCol, *grad, *acc; // acc: [0] sse, [1] loss
    uint16_t *H, *dZ;
    int splits1, splits2;
};

static void mlp_free_ws(tnn_mlp *n)
{
    cudaFree(n->Z);
    cudaFree(n->dY);
    cudaFree(n->Y);
    cudaFree(n->pW1);
    cudaFree(n->pCol);
    cudaFree(n->grad);
    cudaFree(n->acc);
    cudaFree(n->H);
    cudaFree(n->dZ);
    n->Z = n->dY = n->Y = n->pW1 = n->pCol = n->grad = n->acc = nullptr;
    n->H = n->dZ = nullptr;
    n->cap_B = 0;
}

extern "C" void tnn_mlp_destroy(tnn_mlp *n)
{
    if (!n)
        return;
    mlp_free_ws(n);
    cudaFree(n->w);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->w1b);
    delete n;
}

static tnn_status mlp_reserve(tnn_mlp *n, long long B)
{
    if (B <= n->cap_B)
        return TNN_OK;
    mlp_free_ws(n);
    const long long cap = std::max<long long>(B, 256);
    n->splits1 = (int)std::min<long long>(32, (cap + 127) / 128);
    n->splits2 = (int)std::min<long long>(64, (cap + 63) / 64);
    cudaError_t e = cudaSuccess;
#define A_(p, bytes)                                                          \
    if (e == cudaSuccess)                                                     \
        e = cudaMalloc((void **)&(p), (bytes));
    A_(n->Z, sizeof(float) * cap * n->dh);
    A_(n->H, sizeof(uint16_t) * cap * n->dh);
    A_(n->dZ, sizeof(uint16_t) * cap * n->dh);
    A_(n->dY, sizeof(float) * cap * 2);
    A_(n->Y, sizeof(float) * cap * 2);
    A_(n->pW1, sizeof(float) * n->splits1 * (long long)n->d_in * n->dh);
    A_(n->pCol, sizeof(float) * n->splits2 * (long long)(3 * n->dh + 2));
    A_(n->grad, sizeof(float) * n->P);
    A_(n->acc, sizeof(float) * 4);
#undef A_
    if (e != cudaSuccess) {
        mlp_free_ws(n);
        tnn_set_error("MLP workspace allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    n->cap_B = cap;
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
        e = cudaMalloc(&n->w1b, sizeof(uint16_t) * nW1);
    if (e == cudaSuccess)
        e = cudaMemcpy(n->w, h.data(), sizeof(float) * n->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(n->m, 0, sizeof(float) * n->P);
    if (e == cudaSuccess)
        e = cudaMemset(n->v, 0, sizeof(float) * n->P);
    if (e == cudaSuccess) {
        k_to_bf16<<<(unsigned)((nW1 + 255) / 256), 256>>>(n->w, n->w1b, nW1);
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
    if (h_params)
        TNN_CUDA_TRY(cudaMemcpy(h_params, n->w, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_m)
        TNN_CUDA_TRY(cudaMemcpy(h_m, n->m, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_v)
        TNN_CUDA_TRY(cudaMemcpy(h_v, n->v, sizeof(float) * n->P, cudaMemcpyDeviceToHost));
    if (h_step)
        *h_step = n->step;
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
    n->step = step;
    const long long nW1 = (long long)n->d_in * n->dh;
    k_to_bf16<<<(unsigned)((nW1 + 255) / 256), 256>>>(n->w, n->w1b, nW1);
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    return TNN_OK;
}

static tnn_status mlp_forward_impl(const tnn_mlp *n, const uint16_t *d_x, long long B,
                                   float *d_y, const float *d_t, cudaStream_t st)
{
    const long long nW1 = (long long)n->d_in * n->dh;
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = d_x;
    g.lda_m = n->d_in;
    g.lda_k = 1;
    g.B = n->w1b;
    g.ldb_k = n->dh;
    g.ldb_n = 1;
    g.M = (int)B;
    g.N = n->dh;
    g.K = n->d_in;
    g.k_per_split = n->d_in;
    g.bias = n->w + nW1;
    g.Z = n->Z;
    g.H = n->H;
    dim3 grid((n->dh + 63) / 64, (unsigned)((B + 63) / 64), 1);
    k_gemm_bf16<EPI_FWD><<<grid, 256, 0, st>>>(g);
    const float *W2 = n->w + nW1 + n->dh;
    const float *b2 = W2 + 2 * n->dh;
    if (d_t)
        TNN_CUDA_TRY(cudaMemsetAsync(n->acc, 0, sizeof(float) * 4, st));
    k_head<<<(unsigned)((B * 32 + 255) / 256), 256, 0, st>>>(
        n->H, n->Z, W2, b2, (int)B, n->dh, d_y, d_t, n->dY, n->dZ, n->acc);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

extern "C" tnn_status tnn_mlp_forward(const tnn_mlp *n, const uint16_t *d_x, int64_t B,
                                      float *d_y, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(n && d_x && d_y, "NULL argument");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31) / 512, "B out of range");
    tnn_status s = mlp_reserve(const_cast<tnn_mlp *>(n), B);
    if (s != TNN_OK)
        return s;
    return mlp_forward_impl(n, d_x, B, d_y, nullptr, (cudaStream_t)stream);
}

static tnn_status mlp_backward_impl(tnn_mlp *n, const uint16_t *d_x, long long B,
                                    const float *d_t, const tnn_adamw_params *opt,
                                    float *d_loss, float *d_grad, cudaStream_t st)
{
    tnn_status s = mlp_forward_impl(n, d_x, B, n->Y, d_t, st);
    if (s != TNN_OK)
        return s;
    // dW1 partials: X^T dZ, split over the batch.
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = d_x;
    g.lda_m = 1;
    g.lda_k = n->d_in;
    g.B = n->dZ;
    g.ldb_k = n->dh;
    g.ldb_n = 1;
    g.M = n->d_in;
    g.N = n->dh;
    g.K = (int)B;
    g.k_per_split = (int)((B + n->splits1 - 1) / n->splits1);
    g.k_per_split = (g.k_per_split + 15) / 16 * 16;
    g.P = n->pW1;
    const int used1 = (int)((B + g.k_per_split - 1) / g.k_per_split);
    dim3 grid((n->dh + 63) / 64, (n->d_in + 63) / 64, used1);
    k_gemm_bf16<EPI_PARTIAL><<<grid, 256, 0, st>>>(g);
    const int rows_per = (int)((B + n->splits2 - 1) / n->splits2);
    const int used2 = (int)((B + rows_per - 1) / rows_per);
    k_colsums<<<used2, 256, 0, st>>>(n->H, n->dZ, n->dY, (int)B, n->dh, rows_per, n->pCol);
    AdamArgs a;
    memset(&a, 0, sizeof(a));
    a.w = n->w;
    a.m = n->m;
    a.v = n->v;
    a.w1_bf16 = n->w1b;
    a.grad_out = d_grad;
    a.pW1 = n->pW1;
    a.splits1 = used1;
    a.pCol = n->pCol;
    a.splits2 = used2;
    a.d_in = n->d_in;
    a.dh = n->dh;
    a.P = n->P;
    a.sse = n->acc;
    a.loss_out = d_loss;
    a.inv_count = 1.0f / (2.0f * (float)B);
    if (opt) {
        n->step += 1;
        a.lr = opt->lr;
        a.b1 = opt->beta1;
        a.b2 = opt->beta2;
        a.eps = opt->eps;
        a.wd = opt->weight_decay;
        a.bc1 = (float)(1.0 - pow((double)opt->beta1, (double)n->step));
        a.bc2 = (float)(1.0 - pow((double)opt->beta2, (double)n->step));
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
    TNN_CUDA_TRY(cudaMallocAsync((void **)&idx, sizeof(int32_t) * m * k, st));
    cudaError_t e = cudaMallocAsync((void **)&d2, sizeof(float) * m * k, st);
    if (e == cudaSuccess && mlp)
        e = cudaMallocAsync((void **)&feat, sizeof(uint16_t) * m * k * TNN_N_FEAT, st);
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
    cudaFreeAsync(idx, st);
    if (d2)
        cudaFreeAsync(d2, st);
    if (feat)
        cudaFreeAsync(feat, st);
    return s;
}
