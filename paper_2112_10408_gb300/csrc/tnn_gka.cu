// Gaussian kernel averaging over the TNN context (Sec. 3.2, Eq. GKA):
//   s_hat(q) = sum_k w_k s_k / sum_k w_k,
//   w_k = exp(-(s_xy ((x - x_k)^2 + (y - y_k)^2) + s_z (z - z_k)^2 + s_t (t - t_k)^2)),
// with the parameters kept as theta = log(s) and trained with Adam on the mean
// squared error of the nowcast (GKA-TNN, Sec. 4.1).
//
// k_gka: one warp per query, lane = neighbour (k <= 64, two per lane).  The
// exponent is taken relative to its warp minimum (the factor cancels), the
// sums are warp reductions; for training the same warp forms the gradient
//   d s_hat / d s_f = -sum_k w_k D_kf (s_k - s_hat) / W
// (D_kf the squared offsets of group f) and the block sums its warps in a
// fixed order into one partial per block.  k_gka_adam sums the partials in a
// fixed order and applies Adam to theta with the step count on the device.
#include <math.h>
#include <string.h>

#include <vector>

#include "tnn_internal.cuh"

#define FULLMASK 0xffffffffu
#define GKA_WARPS 8

struct tnn_gka {
    int device;
    float *theta; // [3] log s_xy, log s_z, log s_t
    float *m, *v; // Adam moments [3]
    long long *step;
    float *part;  // [cap][4]: gradient (3) and squared error per block
    float *acc;   // [4] reduced gradient and loss
    long long cap;
};

struct GkaArgs {
    const float4 *pts;
    const float2 *wind;
    const float4 *q;     // queries (forward), NULL = the indexed points
    const int32_t *rows; // training: dataset rows of the batch (query = point)
    long long m;
    const int32_t *idx;  // [.. ][k] neighbours (row-indexed when training)
    int k;
    const float *theta;
    float2 *out;         // forward: [m] estimate (NaN for an empty context)
    float *part;         // training: [blocks][4]
    float inv_B;
};

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

__global__ void __launch_bounds__(GKA_WARPS * 32) k_gka(const __grid_constant__ GkaArgs a)
{
    __shared__ float s_part[GKA_WARPS][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long r = (long long)blockIdx.x * GKA_WARPS + warp;
    const bool train = a.rows != nullptr;
    const float sxy = __expf(a.theta[0]), sz = __expf(a.theta[1]), st = __expf(a.theta[2]);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, se = 0.f;
    if (r < a.m) {
        const long long row = train ? (long long)a.rows[r] : r;
        const float4 q = train ? a.pts[row] : (a.q ? a.q[r] : a.pts[r]);
        float e[2], du[2][3], su[2], sv[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            const int id = j < a.k ? a.idx[row * a.k + j] : -1;
            ok[h] = id >= 0;
            e[h] = INFINITY;
            su[h] = sv[h] = 0.f;
            du[h][0] = du[h][1] = du[h][2] = 0.f;
            if (ok[h]) {
                const float4 p = a.pts[id];
                const float2 s = a.wind[id];
                const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z, dt = p.w - q.w;
                du[h][0] = fmaf(dx, dx, dy * dy);
                du[h][1] = dz * dz;
                du[h][2] = dt * dt;
                e[h] = fmaf(sxy, du[h][0], fmaf(sz, du[h][1], st * du[h][2]));
                su[h] = s.x;
                sv[h] = s.y;
            }
        }
        float emin = fminf(e[0], e[1]);
        for (int o = 16; o > 0; o >>= 1)
            emin = fminf(emin, __shfl_xor_sync(FULLMASK, emin, o));
        float w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            w[h] = ok[h] ? expf(emin - e[h]) : 0.f;
        const float W = warp_sum(w[0] + w[1]);
        const float U = warp_sum(fmaf(w[0], su[0], w[1] * su[1]));
        const float V = warp_sum(fmaf(w[0], sv[0], w[1] * sv[1]));
        const float pu = U / W, pv = V / W; // NaN for an empty context
        if (!train) {
            if (lane == 0)
                a.out[r] = make_float2(pu, pv);
        } else if (W > 0.f) {
            const float2 t = a.wind[row];
            const float eu = pu - t.x, ev = pv - t.y;
            se = eu * eu + ev * ev;
            // sum_k w_k D_kf ((s_k - s_hat) . err)
            float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float proj = w[h] * fmaf(su[h] - pu, eu, (sv[h] - pv) * ev);
                c0 = fmaf(proj, du[h][0], c0);
                c1 = fmaf(proj, du[h][1], c1);
                c2 = fmaf(proj, du[h][2], c2);
            }
            c0 = warp_sum(c0);
            c1 = warp_sum(c1);
            c2 = warp_sum(c2);
            // d loss / d theta_f = s_f (1/B) sum err . d s_hat / d s_f
            const float f = -a.inv_B / W;
            g0 = sxy * f * c0;
            g1 = sz * f * c1;
            g2 = st * f * c2;
        }
    }
    if (!train)
        return;
    if (lane == 0) {
        s_part[warp][0] = g0;
        s_part[warp][1] = g1;
        s_part[warp][2] = g2;
        s_part[warp][3] = se;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float acc = 0.f;
        for (int w = 0; w < GKA_WARPS; ++w)
            acc += s_part[w][threadIdx.x];
        a.part[(long long)blockIdx.x * 4 + threadIdx.x] = acc;
    }
}

// Forward for k <= 32: two queries per warp, lane = neighbour, so that the
// index loads and the neighbour gathers of both queries are in flight
// together.  The arithmetic is k_gka's, operation for operation.
__global__ void __launch_bounds__(GKA_WARPS * 32) k_gka_fwd_pair(const __grid_constant__ GkaArgs a)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long r0 = ((long long)blockIdx.x * GKA_WARPS + warp) * 2;
    const float sxy = __expf(a.theta[0]), sz = __expf(a.theta[1]), st = __expf(a.theta[2]);
    int id[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long r = r0 + h;
        id[h] = (r < a.m && lane < a.k) ? a.idx[r * a.k + lane] : -1;
    }
    float4 q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long r = r0 + h < a.m ? r0 + h : 0;
        q[h] = a.q ? a.q[r] : a.pts[r];
    }
    float e[2], su[2], sv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        e[h] = INFINITY;
        su[h] = sv[h] = 0.f;
        if (id[h] >= 0) {
            const float4 p = a.pts[id[h]];
            const float2 s = a.wind[id[h]];
            const float dx = p.x - q[h].x, dy = p.y - q[h].y, dz = p.z - q[h].z, dt = p.w - q[h].w;
            e[h] = fmaf(sxy, fmaf(dx, dx, dy * dy), fmaf(sz, dz * dz, st * (dt * dt)));
            su[h] = s.x;
            sv[h] = s.y;
        }
    }
    float emin[2] = {e[0], e[1]};
    for (int o = 16; o > 0; o >>= 1) {
        emin[0] = fminf(emin[0], __shfl_xor_sync(FULLMASK, emin[0], o));
        emin[1] = fminf(emin[1], __shfl_xor_sync(FULLMASK, emin[1], o));
    }
    float W[2], U[2], V[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float w = id[h] >= 0 ? expf(emin[h] - e[h]) : 0.f;
        W[h] = w;
        U[h] = fmaf(w, su[h], 0.f);
        V[h] = fmaf(w, sv[h], 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            W[h] += __shfl_xor_sync(FULLMASK, W[h], o);
            U[h] += __shfl_xor_sync(FULLMASK, U[h], o);
            V[h] += __shfl_xor_sync(FULLMASK, V[h], o);
        }
    }
    if (lane < 2 && r0 + lane < a.m) {
        const int h = lane;
        a.out[r0 + h] = make_float2(U[h] / W[h], V[h] / W[h]); // NaN for an empty context
    }
}

struct GkaAdamArgs {
    const float *part;
    long long nblocks;
    float *theta, *m, *v;
    long long *step;
    float *acc;      // [4] reduced gradient, loss
    float *grad_out; // optional [3]
    float *loss_out; // optional
    float inv_2B;
    int update;
    float lr, b1, b2, eps, wd;
};

// One block of 128 threads: fixed-order reduction of the partials, then
// Adam on theta.
__global__ void k_gka_adam(const __grid_constant__ GkaAdamArgs a)
{
    __shared__ float s[4][32];
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31; // warp c sums component c
    float v = 0.f;
    for (long long b = lane; b < a.nblocks; b += 32)
        v += a.part[b * 4 + c];
    s[c][lane] = v;
    __syncthreads();
    if (threadIdx.x < 4) {
        float t = 0.f;
        for (int i = 0; i < 32; ++i)
            t += s[threadIdx.x][i];
        a.acc[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.loss_out)
            *a.loss_out = a.acc[3] * a.inv_2B;
        if (a.grad_out)
            for (int i = 0; i < 3; ++i)
                a.grad_out[i] = a.acc[i];
        if (a.update) {
            const long long st = *a.step + 1;
            *a.step = st;
            const float bc1 = -expm1f((float)st * log1pf(a.b1 - 1.0f));
            const float bc2 = -expm1f((float)st * log1pf(a.b2 - 1.0f));
            for (int i = 0; i < 3; ++i) {
                const float g = a.acc[i];
                const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
                const float vv = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
                a.m[i] = m;
                a.v[i] = vv;
                const float th = a.theta[i];
                a.theta[i] = th - a.lr * ((m / bc1) / (sqrtf(vv / bc2) + a.eps) + a.wd * th);
            }
        }
    }
}

extern "C" tnn_status tnn_gka_create(const float *h_sigma, tnn_gka **out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(out != nullptr && h_sigma != nullptr, "NULL argument");
    *out = nullptr;
    for (int i = 0; i < 3; ++i)
        TNN_ARG_CHECK(h_sigma[i] > 0.f && isfinite(h_sigma[i]), "sigma[%d] must be finite and > 0", i);
    tnn_gka *g = new tnn_gka();
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    float th[3] = {logf(h_sigma[0]), logf(h_sigma[1]), logf(h_sigma[2])};
    cudaError_t e = cudaMalloc(&g->theta, 3 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->m, 3 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->v, 3 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->step, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->acc, 4 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->theta, th, sizeof(th), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(g->m, 0, 3 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(g->v, 0, 3 * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(g->step, 0, sizeof(long long));
    if (e != cudaSuccess) {
        tnn_gka_destroy(g);
        tnn_set_error("GKA allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    *out = g;
    return TNN_OK;
}

extern "C" void tnn_gka_destroy(tnn_gka *g)
{
    if (!g)
        return;
    cudaFree(g->theta);
    cudaFree(g->m);
    cudaFree(g->v);
    cudaFree(g->step);
    cudaFree(g->part);
    cudaFree(g->acc);
    delete g;
}

extern "C" tnn_status tnn_gka_get_params(const tnn_gka *g, float *h_sigma, int64_t *h_step)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g != nullptr && h_sigma != nullptr, "NULL argument");
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    float th[3];
    TNN_CUDA_TRY(cudaMemcpy(th, g->theta, sizeof(th), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 3; ++i)
        h_sigma[i] = expf(th[i]);
    if (h_step) {
        long long s = 0;
        TNN_CUDA_TRY(cudaMemcpy(&s, g->step, sizeof(s), cudaMemcpyDeviceToHost));
        *h_step = s;
    }
    return TNN_OK;
}

extern "C" tnn_status tnn_gka_set_params(tnn_gka *g, const float *h_sigma)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g != nullptr && h_sigma != nullptr, "NULL argument");
    for (int i = 0; i < 3; ++i)
        TNN_ARG_CHECK(h_sigma[i] > 0.f && isfinite(h_sigma[i]), "sigma[%d] must be finite and > 0", i);
    float th[3] = {logf(h_sigma[0]), logf(h_sigma[1]), logf(h_sigma[2])};
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    TNN_CUDA_TRY(cudaMemcpy(g->theta, th, sizeof(th), cudaMemcpyHostToDevice));
    TNN_CUDA_TRY(cudaMemset(g->m, 0, 3 * sizeof(float)));
    TNN_CUDA_TRY(cudaMemset(g->v, 0, 3 * sizeof(float)));
    TNN_CUDA_TRY(cudaMemset(g->step, 0, sizeof(long long)));
    return TNN_OK;
}

static tnn_status gka_check(const tnn_gka *g, const tnn_index *ix, const float *d_wind,
                            const int32_t *d_idx, int32_t k)
{
    TNN_ARG_CHECK(g && ix && d_wind && d_idx, "NULL argument");
    TNN_ARG_CHECK(k >= 1 && k <= 64, "k must be in [1, 64]");
    int dev = -1;
    cudaGetDevice(&dev);
    TNN_ARG_CHECK(dev == g->device && dev == ix->device, "GKA, index and current device differ");
    return TNN_OK;
}

extern "C" tnn_status tnn_gka_forward(const tnn_gka *g, const tnn_index *ix, const float *d_wind,
                                      const float *d_q, int64_t m, const int32_t *d_idx, int32_t k,
                                      float *d_uv, tnn_stream_t stream)
{
    tnn_clear_error();
    tnn_status s = gka_check(g, ix, d_wind, d_idx, k);
    if (s != TNN_OK)
        return s;
    TNN_ARG_CHECK(d_uv != nullptr, "d_uv is NULL");
    TNN_ARG_CHECK(m >= 0 && m < (1ll << 31), "m out of range");
    TNN_ARG_CHECK(d_q != nullptr || m == ix->n, "self-query needs m == n_points");
    if (m == 0)
        return TNN_OK;
    GkaArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = ix->pts;
    a.wind = (const float2 *)d_wind;
    a.q = (const float4 *)d_q;
    a.m = m;
    a.idx = d_idx;
    a.k = k;
    a.theta = g->theta;
    a.out = (float2 *)d_uv;
    if (k <= 32)
        k_gka_fwd_pair<<<(unsigned)((m + 2 * GKA_WARPS - 1) / (2 * GKA_WARPS)), GKA_WARPS * 32, 0,
                         (cudaStream_t)stream>>>(a);
    else
        k_gka<<<(unsigned)((m + GKA_WARPS - 1) / GKA_WARPS), GKA_WARPS * 32, 0, (cudaStream_t)stream>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

extern "C" tnn_status tnn_gka_train_step(tnn_gka *g, const tnn_index *ix, const float *d_wind,
                                         const int32_t *d_rows, int64_t B, const int32_t *d_idx,
                                         int32_t k, const tnn_adamw_params *opt, float *d_loss,
                                         float *d_grad, tnn_stream_t stream)
{
    tnn_clear_error();
    tnn_status s = gka_check(g, ix, d_wind, d_idx, k);
    if (s != TNN_OK)
        return s;
    TNN_ARG_CHECK(d_rows != nullptr, "d_rows is NULL");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31), "B out of range");
    if (opt)
        TNN_ARG_CHECK(opt->lr >= 0.f && opt->beta1 >= 0.f && opt->beta1 < 1.f && opt->beta2 >= 0.f &&
                          opt->beta2 < 1.f && opt->eps > 0.f && opt->weight_decay >= 0.f,
                      "invalid Adam parameters");
    TNN_ARG_CHECK(opt != nullptr || d_grad != nullptr, "nothing to do: no optimiser and no gradient output");
    const long long nb = (B + GKA_WARPS - 1) / GKA_WARPS;
    if (nb > g->cap) {
        cudaFree(g->part);
        g->part = nullptr;
        g->cap = 0;
        TNN_CUDA_TRY(cudaMalloc(&g->part, (size_t)nb * 4 * sizeof(float)));
        g->cap = nb;
    }
    cudaStream_t st = (cudaStream_t)stream;
    GkaArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = ix->pts;
    a.wind = (const float2 *)d_wind;
    a.rows = d_rows;
    a.m = B;
    a.idx = d_idx;
    a.k = k;
    a.theta = g->theta;
    a.part = g->part;
    a.inv_B = 1.0f / (float)B;
    k_gka<<<(unsigned)nb, GKA_WARPS * 32, 0, st>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    GkaAdamArgs d;
    memset(&d, 0, sizeof(d));
    d.part = g->part;
    d.nblocks = nb;
    d.theta = g->theta;
    d.m = g->m;
    d.v = g->v;
    d.step = g->step;
    d.acc = g->acc;
    d.grad_out = d_grad;
    d.loss_out = d_loss;
    d.inv_2B = 1.0f / (2.0f * (float)B);
    d.update = opt != nullptr;
    if (opt) {
        d.lr = opt->lr;
        d.b1 = opt->beta1;
        d.b2 = opt->beta2;
        d.eps = opt->eps;
        d.wd = opt->weight_decay;
    }
    k_gka_adam<<<1, 128, 0, st>>>(d);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

// ------------------------------------------------------------------ GKA-MLP
//
// The scales as a function of the location (Sec. 3.2): per query
//   theta(q) = tanh(u W1 + b1) W2 + b2,  u = (q_xyz - lo) / (hi - lo)
// (u: location normalised by the points' bounding box), then GKA with
// s = exp(theta(q)).  Flat parameters W1 [3][H] | b1 [H] | W2 [H][3] | b2 [3],
// H <= 32.  k_gkamlp: one warp per query; lane j is hidden unit j for the
// MLP and neighbour j for GKA.  For training the per-query gradient in theta
// (as in k_gka) is carried back through the MLP in the same warp and summed
// per block in a fixed order; k_gkamlp_adam reduces the partials and steps
// Adam.

#define GKAMLP_HMAX 32

struct tnn_gkamlp {
    int device;
    int H;
    int P;
    float *w, *m, *v; // [P]
    long long *step;
    float *part;      // [cap][P + 1]: gradient and squared error per block
    long long cap;
};

struct GkaMlpArgs {
    const float4 *pts;
    const float2 *wind;
    const float4 *q;
    const int32_t *rows;
    long long m;
    const int32_t *idx;
    int k;
    int H, P;
    const float *w;
    float lo[3], inv_ext[3];
    float2 *out;
    float *part;
    float inv_B;
};

// Forward for k <= 32: two queries per warp (lane = neighbour, lane =
// hidden unit), the arithmetic of k_gkamlp operation for operation.
__global__ void __launch_bounds__(GKA_WARPS * 32) k_gkamlp_fwd_pair(const __grid_constant__ GkaMlpArgs a)
{
    extern __shared__ float s_w[]; // [P] parameters
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int H = a.H, P = a.P;
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        s_w[i] = a.w[i];
    __syncthreads();
    const float *W1 = s_w, *b1 = s_w + 3 * H, *W2 = s_w + 4 * H, *b2 = s_w + 7 * H;
    const long long r0 = ((long long)blockIdx.x * GKA_WARPS + warp) * 2;
    int id[2];
    float4 q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long r = r0 + h;
        id[h] = (r < a.m && lane < a.k) ? a.idx[r * a.k + lane] : -1;
        const long long rq = r < a.m ? r : 0;
        q[h] = a.q ? a.q[rq] : a.pts[rq];
    }
    float sc[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float u[3] = {(q[h].x - a.lo[0]) * a.inv_ext[0], (q[h].y - a.lo[1]) * a.inv_ext[1],
                            (q[h].z - a.lo[2]) * a.inv_ext[2]};
        float hj = 0.f;
        if (lane < H)
            hj = tanhf(fmaf(W1[lane], u[0], fmaf(W1[H + lane], u[1], fmaf(W1[2 * H + lane], u[2], b1[lane]))));
#pragma unroll
        for (int f = 0; f < 3; ++f)
            sc[h][f] = __expf(b2[f] + warp_sum(lane < H ? hj * W2[3 * lane + f] : 0.f));
    }
    float e[2], su[2], sv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        e[h] = INFINITY;
        su[h] = sv[h] = 0.f;
        if (id[h] >= 0) {
            const float4 p = a.pts[id[h]];
            const float2 s = a.wind[id[h]];
            const float dx = p.x - q[h].x, dy = p.y - q[h].y, dz = p.z - q[h].z, dt = p.w - q[h].w;
            e[h] = fmaf(sc[h][0], fmaf(dx, dx, dy * dy), fmaf(sc[h][1], dz * dz, sc[h][2] * (dt * dt)));
            su[h] = s.x;
            sv[h] = s.y;
        }
    }
    float emin[2] = {e[0], e[1]};
    for (int o = 16; o > 0; o >>= 1) {
        emin[0] = fminf(emin[0], __shfl_xor_sync(FULLMASK, emin[0], o));
        emin[1] = fminf(emin[1], __shfl_xor_sync(FULLMASK, emin[1], o));
    }
    float W[2], U[2], V[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float w = id[h] >= 0 ? expf(emin[h] - e[h]) : 0.f;
        W[h] = w;
        U[h] = fmaf(w, su[h], 0.f);
        V[h] = fmaf(w, sv[h], 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            W[h] += __shfl_xor_sync(FULLMASK, W[h], o);
            U[h] += __shfl_xor_sync(FULLMASK, U[h], o);
            V[h] += __shfl_xor_sync(FULLMASK, V[h], o);
        }
    }
    if (lane < 2 && r0 + lane < a.m) {
        const int h = lane;
        a.out[r0 + h] = make_float2(U[h] / W[h], V[h] / W[h]); // NaN for an empty context
    }
}

__global__ void __launch_bounds__(GKA_WARPS * 32) k_gkamlp(const __grid_constant__ GkaMlpArgs a)
{
    extern __shared__ float s_w[]; // [P] parameters, then [GKA_WARPS][P + 1] partials
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int H = a.H, P = a.P;
    const bool train = a.rows != nullptr;
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        s_w[i] = a.w[i];
    float *s_part = s_w + P;
    __syncthreads();
    const float *W1 = s_w, *b1 = s_w + 3 * H, *W2 = s_w + 4 * H, *b2 = s_w + 7 * H;
    const long long r = (long long)blockIdx.x * GKA_WARPS + warp;
    // this lane's gradient contributions: W1[0..2][lane], b1[lane], W2[lane][0..2], b2 (lane 0)
    float gW1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gW2[3] = {0.f, 0.f, 0.f}, gb2[3] = {0.f, 0.f, 0.f}, se = 0.f;
    if (r < a.m) {
        const long long row = train ? (long long)a.rows[r] : r;
        const float4 q = train ? a.pts[row] : (a.q ? a.q[r] : a.pts[r]);
        const float u[3] = {(q.x - a.lo[0]) * a.inv_ext[0], (q.y - a.lo[1]) * a.inv_ext[1],
                            (q.z - a.lo[2]) * a.inv_ext[2]};
        float hj = 0.f;
        if (lane < H)
            hj = tanhf(fmaf(W1[lane], u[0], fmaf(W1[H + lane], u[1], fmaf(W1[2 * H + lane], u[2], b1[lane]))));
        float th[3];
#pragma unroll
        for (int f = 0; f < 3; ++f)
            th[f] = b2[f] + warp_sum(lane < H ? hj * W2[3 * lane + f] : 0.f);
        const float sxy = __expf(th[0]), sz = __expf(th[1]), st = __expf(th[2]);
        float e[2], du[2][3], su[2], sv[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            const int id = j < a.k ? a.idx[row * a.k + j] : -1;
            ok[h] = id >= 0;
            e[h] = INFINITY;
            su[h] = sv[h] = 0.f;
            du[h][0] = du[h][1] = du[h][2] = 0.f;
            if (ok[h]) {
                const float4 p = a.pts[id];
                const float2 s = a.wind[id];
                const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z, dt = p.w - q.w;
                du[h][0] = fmaf(dx, dx, dy * dy);
                du[h][1] = dz * dz;
                du[h][2] = dt * dt;
                e[h] = fmaf(sxy, du[h][0], fmaf(sz, du[h][1], st * du[h][2]));
                su[h] = s.x;
                sv[h] = s.y;
            }
        }
        float emin = fminf(e[0], e[1]);
        for (int o = 16; o > 0; o >>= 1)
            emin = fminf(emin, __shfl_xor_sync(FULLMASK, emin, o));
        float w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            w[h] = ok[h] ? expf(emin - e[h]) : 0.f;
        const float W = warp_sum(w[0] + w[1]);
        const float U = warp_sum(fmaf(w[0], su[0], w[1] * su[1]));
        const float V = warp_sum(fmaf(w[0], sv[0], w[1] * sv[1]));
        const float pu = U / W, pv = V / W;
        if (!train) {
            if (lane == 0)
                a.out[r] = make_float2(pu, pv);
        } else if (W > 0.f) {
            const float2 t = a.wind[row];
            const float eu = pu - t.x, ev = pv - t.y;
            se = eu * eu + ev * ev;
            float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float proj = w[h] * fmaf(su[h] - pu, eu, (sv[h] - pv) * ev);
                c0 = fmaf(proj, du[h][0], c0);
                c1 = fmaf(proj, du[h][1], c1);
                c2 = fmaf(proj, du[h][2], c2);
            }
            const float f = -a.inv_B / W;
            const float dth[3] = {sxy * f * warp_sum(c0), sz * f * warp_sum(c1), st * f * warp_sum(c2)};
            if (lane < H) {
                float dh = 0.f;
#pragma unroll
                for (int g = 0; g < 3; ++g) {
                    gW2[g] = hj * dth[g];
                    dh = fmaf(W2[3 * lane + g], dth[g], dh);
                }
                const float da = dh * (1.0f - hj * hj);
                gW1[0] = u[0] * da;
                gW1[1] = u[1] * da;
                gW1[2] = u[2] * da;
                gb1 = da;
            }
            if (lane == 0) {
                gb2[0] = dth[0];
                gb2[1] = dth[1];
                gb2[2] = dth[2];
            }
        }
    }
    if (!train)
        return;
    // per-warp partials, then the block's sum in warp order
    float *wp = s_part + warp * (P + 1);
    if (lane < H) {
        wp[lane] = gW1[0];
        wp[H + lane] = gW1[1];
        wp[2 * H + lane] = gW1[2];
        wp[3 * H + lane] = gb1;
        wp[4 * H + 3 * lane] = gW2[0];
        wp[4 * H + 3 * lane + 1] = gW2[1];
        wp[4 * H + 3 * lane + 2] = gW2[2];
    }
    if (lane == 0) {
        wp[7 * H] = gb2[0];
        wp[7 * H + 1] = gb2[1];
        wp[7 * H + 2] = gb2[2];
        wp[P] = se;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= P; i += blockDim.x) {
        float acc = 0.f;
        for (int w2 = 0; w2 < GKA_WARPS; ++w2)
            acc += s_part[w2 * (P + 1) + i];
        a.part[(long long)blockIdx.x * (P + 1) + i] = acc;
    }
}

struct GkaMlpAdamArgs {
    const float *part;
    long long nblocks;
    int P;
    float *w, *m, *v;
    long long *step;
    float *grad_out;
    float *loss_out;
    float inv_2B;
    int update;
    float lr, b1, b2, eps, wd;
};

// One block: parameter i (thread i) sums its partials in block order.
__global__ void k_gkamlp_adam(const __grid_constant__ GkaMlpAdamArgs a)
{
    const int i = threadIdx.x;
    const long long t = a.update ? *a.step + 1 : 0;
    __syncthreads(); // every thread has read the count
    if (i <= a.P) {
        float g = 0.f;
        for (long long b = 0; b < a.nblocks; ++b)
            g += a.part[b * (a.P + 1) + i];
        if (i == a.P) {
            if (a.loss_out)
                *a.loss_out = g * a.inv_2B;
        } else {
            if (a.grad_out)
                a.grad_out[i] = g;
            if (a.update) {
                const float bc1 = -expm1f((float)t * log1pf(a.b1 - 1.0f));
                const float bc2 = -expm1f((float)t * log1pf(a.b2 - 1.0f));
                const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
                const float vv = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
                a.m[i] = m;
                a.v[i] = vv;
                const float wi = a.w[i];
                a.w[i] = wi - a.lr * ((m / bc1) / (sqrtf(vv / bc2) + a.eps) + a.wd * wi);
            }
        }
    }
    if (i == 0 && a.update)
        *a.step = t;
}

static uint64_t gka_splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" tnn_status tnn_gkamlp_create(const float *h_sigma, int32_t hidden, uint64_t seed,
                                        tnn_gkamlp **out)
{
    tnn_clear_error();
    TNN_ARG_CHECK(out != nullptr && h_sigma != nullptr, "NULL argument");
    *out = nullptr;
    TNN_ARG_CHECK(hidden >= 1 && hidden <= GKAMLP_HMAX, "hidden must be in [1, 32]");
    for (int i = 0; i < 3; ++i)
        TNN_ARG_CHECK(h_sigma[i] > 0.f && isfinite(h_sigma[i]), "sigma[%d] must be finite and > 0", i);
    tnn_gkamlp *g = new tnn_gkamlp();
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    g->H = hidden;
    g->P = 7 * hidden + 3;
    // W1, b1 ~ U(-1/sqrt(3), 1/sqrt(3)); W2 = 0 and b2 = log(sigma): the
    // model starts as plain GKA with the given scales
    std::vector<float> h(g->P, 0.f);
    uint64_t s = seed;
    const float bound = 1.0f / sqrtf(3.0f);
    for (int i = 0; i < 4 * hidden; ++i) {
        const double uu = (double)(gka_splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
        h[i] = (float)((2.0 * uu - 1.0) * bound);
    }
    for (int f = 0; f < 3; ++f)
        h[7 * hidden + f] = logf(h_sigma[f]);
    cudaError_t e = cudaMalloc(&g->w, g->P * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->m, g->P * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->v, g->P * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->step, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->w, h.data(), g->P * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(g->m, 0, g->P * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(g->v, 0, g->P * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemset(g->step, 0, sizeof(long long));
    if (e != cudaSuccess) {
        tnn_gkamlp_destroy(g);
        tnn_set_error("GKA-MLP allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TNN_ERR_OOM : TNN_ERR_CUDA;
    }
    *out = g;
    return TNN_OK;
}

extern "C" void tnn_gkamlp_destroy(tnn_gkamlp *g)
{
    if (!g)
        return;
    cudaFree(g->w);
    cudaFree(g->m);
    cudaFree(g->v);
    cudaFree(g->step);
    cudaFree(g->part);
    delete g;
}

extern "C" int64_t tnn_gkamlp_num_params(const tnn_gkamlp *g) { return g ? g->P : 0; }

extern "C" tnn_status tnn_gkamlp_get_params(const tnn_gkamlp *g, float *h_params, int64_t *h_step)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g != nullptr && h_params != nullptr, "NULL argument");
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    TNN_CUDA_TRY(cudaMemcpy(h_params, g->w, g->P * sizeof(float), cudaMemcpyDeviceToHost));
    if (h_step) {
        long long s = 0;
        TNN_CUDA_TRY(cudaMemcpy(&s, g->step, sizeof(s), cudaMemcpyDeviceToHost));
        *h_step = s;
    }
    return TNN_OK;
}

extern "C" tnn_status tnn_gkamlp_set_params(tnn_gkamlp *g, const float *h_params)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g != nullptr && h_params != nullptr, "NULL argument");
    TNN_CUDA_TRY(cudaDeviceSynchronize());
    TNN_CUDA_TRY(cudaMemcpy(g->w, h_params, g->P * sizeof(float), cudaMemcpyHostToDevice));
    TNN_CUDA_TRY(cudaMemset(g->m, 0, g->P * sizeof(float)));
    TNN_CUDA_TRY(cudaMemset(g->v, 0, g->P * sizeof(float)));
    TNN_CUDA_TRY(cudaMemset(g->step, 0, sizeof(long long)));
    return TNN_OK;
}

static void gkamlp_args(const tnn_gkamlp *g, const tnn_index *ix, const float *d_wind,
                        const int32_t *d_idx, int32_t k, GkaMlpArgs &a)
{
    memset(&a, 0, sizeof(a));
    a.pts = ix->pts;
    a.wind = (const float2 *)d_wind;
    a.idx = d_idx;
    a.k = k;
    a.H = g->H;
    a.P = g->P;
    a.w = g->w;
    for (int d = 0; d < 3; ++d) {
        const float ext = ix->bb_hi[d] - ix->bb_lo[d];
        a.lo[d] = ix->bb_lo[d];
        a.inv_ext[d] = ext > 0.f ? 1.0f / ext : 1.0f;
    }
}

extern "C" tnn_status tnn_gkamlp_forward(const tnn_gkamlp *g, const tnn_index *ix,
                                         const float *d_wind, const float *d_q, int64_t m,
                                         const int32_t *d_idx, int32_t k, float *d_uv,
                                         tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g && ix && d_wind && d_idx && d_uv, "NULL argument");
    TNN_ARG_CHECK(k >= 1 && k <= 64, "k must be in [1, 64]");
    TNN_ARG_CHECK(m >= 0 && m < (1ll << 31), "m out of range");
    TNN_ARG_CHECK(d_q != nullptr || m == ix->n, "self-query needs m == n_points");
    if (m == 0)
        return TNN_OK;
    GkaMlpArgs a;
    gkamlp_args(g, ix, d_wind, d_idx, k, a);
    a.q = (const float4 *)d_q;
    a.m = m;
    a.out = (float2 *)d_uv;
    if (k <= 32 && g->H <= 32)
        k_gkamlp_fwd_pair<<<(unsigned)((m + 2 * GKA_WARPS - 1) / (2 * GKA_WARPS)), GKA_WARPS * 32,
                            g->P * sizeof(float), (cudaStream_t)stream>>>(a);
    else
        k_gkamlp<<<(unsigned)((m + GKA_WARPS - 1) / GKA_WARPS), GKA_WARPS * 32, g->P * sizeof(float),
                   (cudaStream_t)stream>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}

extern "C" tnn_status tnn_gkamlp_train_step(tnn_gkamlp *g, const tnn_index *ix, const float *d_wind,
                                            const int32_t *d_rows, int64_t B, const int32_t *d_idx,
                                            int32_t k, const tnn_adamw_params *opt, float *d_loss,
                                            float *d_grad, tnn_stream_t stream)
{
    tnn_clear_error();
    TNN_ARG_CHECK(g && ix && d_wind && d_idx && d_rows, "NULL argument");
    TNN_ARG_CHECK(k >= 1 && k <= 64, "k must be in [1, 64]");
    TNN_ARG_CHECK(B >= 1 && B < (1ll << 31), "B out of range");
    if (opt)
        TNN_ARG_CHECK(opt->lr >= 0.f && opt->beta1 >= 0.f && opt->beta1 < 1.f && opt->beta2 >= 0.f &&
                          opt->beta2 < 1.f && opt->eps > 0.f && opt->weight_decay >= 0.f,
                      "invalid Adam parameters");
    TNN_ARG_CHECK(opt != nullptr || d_grad != nullptr, "nothing to do: no optimiser and no gradient output");
    const long long nb = (B + GKA_WARPS - 1) / GKA_WARPS;
    if (nb > g->cap) {
        cudaFree(g->part);
        g->part = nullptr;
        g->cap = 0;
        TNN_CUDA_TRY(cudaMalloc(&g->part, (size_t)nb * (g->P + 1) * sizeof(float)));
        g->cap = nb;
    }
    cudaStream_t st = (cudaStream_t)stream;
    GkaMlpArgs a;
    gkamlp_args(g, ix, d_wind, d_idx, k, a);
    a.rows = d_rows;
    a.m = B;
    a.part = g->part;
    a.inv_B = 1.0f / (float)B;
    const size_t smem = (g->P + GKA_WARPS * (g->P + 1)) * sizeof(float);
    k_gkamlp<<<(unsigned)nb, GKA_WARPS * 32, smem, st>>>(a);
    TNN_CUDA_TRY(cudaGetLastError());
    GkaMlpAdamArgs d;
    memset(&d, 0, sizeof(d));
    d.part = g->part;
    d.nblocks = nb;
    d.P = g->P;
    d.w = g->w;
    d.m = g->m;
    d.v = g->v;
    d.step = g->step;
    d.grad_out = d_grad;
    d.loss_out = d_loss;
    d.inv_2B = 1.0f / (2.0f * (float)B);
    d.update = opt != nullptr;
    if (opt) {
        d.lr = opt->lr;
        d.b1 = opt->beta1;
        d.b2 = opt->beta2;
        d.eps = opt->eps;
        d.wd = opt->weight_decay;
    }
    k_gkamlp_adam<<<1, 256, 0, st>>>(d);
    TNN_CUDA_TRY(cudaGetLastError());
    return TNN_OK;
}
