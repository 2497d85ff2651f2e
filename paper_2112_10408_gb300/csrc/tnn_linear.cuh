// Linear-search comparator (Sec. 3.6, Table 1 "Linear search"): every
// causally valid point is a candidate.  The index keeps a copy of the points
// ordered by time, so the valid set of a query is a prefix; the warp walks it
// from the most recent point backwards (nearest in time first, which fills
// the candidate lists with good keys early), one query per lane, 32 points
// per chunk staged in shared memory with the next chunk already in flight.
#pragma once
#include "tnn_device.cuh"

__global__ void __launch_bounds__(TNN_WARPS_PER_CTA * 32)
    k_linear_search(const __grid_constant__ KnnLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const size_t pw = smem_per_warp(L.L_max, L.kseg_max, SMEM_LINEAR);
    unsigned char *ws = smem + (threadIdx.x >> 5) * pw;
    unsigned long long *K = (unsigned long long *)ws + lane;
    unsigned char *rest = ws + (size_t)L.L_max * 256;
    float4 *pb = (float4 *)rest;   // [32]
    int *ib = (int *)(rest + 512); // [32]
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
        const float4 *__restrict__ pts_t = W->pts_t;
        const int32_t *__restrict__ idx_t = W->idx_t;
        const int Lw = W->L;

        float tmax = c.T32;
        for (int o = 16; o > 0; o >>= 1)
            tmax = fmaxf(tmax, __shfl_xor_sync(FULLMASK, tmax, o));
        const int hi = warp_count_less([&](int p) { return __ldg(&pts_t[p].w); }, W->n, tmax, lane);

        for (int i = 0; i < Lw; ++i)
            K[i * 32] = SENT;
        int nv = 0;
        unsigned long long tauk = SENT;
        float tau = INFINITY;

        float4 np_ = make_float4(0.f, 0.f, 0.f, 0.f);
        int ni = 0;
        if (hi > 0) {
            const int c0 = hi > 32 ? hi - 32 : 0;
            if (lane < hi - c0) {
                np_ = __ldg(pts_t + c0 + lane);
                ni = __ldg(idx_t + c0 + lane);
            }
        }
        for (int pos_hi = hi; pos_hi > 0;) {
            const int c0 = pos_hi > 32 ? pos_hi - 32 : 0;
            const int cnt = pos_hi - c0;
            __syncwarp();
            if (lane < cnt) {
                pb[lane] = np_;
                ib[lane] = ni;
            }
            __syncwarp();
            if (c0 > 0) {
                const int n0 = c0 > 32 ? c0 - 32 : 0;
                if (lane < c0 - n0) {
                    np_ = __ldg(pts_t + n0 + lane);
                    ni = __ldg(idx_t + n0 + lane);
                }
            }
#pragma unroll 4
            for (int i = cnt - 1; i >= 0; --i) {
                const float4 p = pb[i];
                const float d = dist32(c, s0, s1, s2, s3, p);
                if (p.w < c.T32 && d <= tau) {
                    const unsigned long long key = pack_key(d, ib[i]);
                    if (key < tauk) {
                        tauk = lane_push(K, Lw, nv, key);
                        tau = key_d(tauk);
                    }
                }
            }
            if (active)
                st.pairs += cnt;
            pos_hi = c0;
        }

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
    }
    flush_stats(L.scr, st);
}
