// Algorithm 1 (arXiv:1601.00072, Sec. 2.1) on the 256-bin grey-level
// histogram: the loop of the histogram-domain run (brFCM, cited in Sec. 3),
// shared by the single-image kernel and the batch kernels (one warp per run).
//
// Under Eq. 4 a pixel's memberships depend only on its grey level, so the
// center sums of Eq. 3 and J of Eq. 1 are sums over bins weighted by their
// pixel counts, and the stopping quantity is a maximum over the bins present.
#pragma once

#include "fcm_device.cuh"
#include "fcm_df.cuh"

namespace fcm {

constexpr int HNT = 256;  // threads of the pixel-pass CTAs

__device__ __forceinline__ bool grey_level(float v) {
    return v >= 0.0f && v <= 255.0f && v == rintf(v);  // false for NaN
}

// The loop runs in one warp: lane l holds grey levels l + 32 t, t < WB. A
// lane adds its eight bins' terms in FP32, then a double-float xor tree over
// the warp gives every lane the same totals, so every lane forms V^{k+1}
// (double-float quotients) itself: no block barrier, and a CTA of 32 threads
// per run lets the many runs of a batch share each SM. The loop body is kept
// small (bins two at a time, the tree's five levels rolled, U^{k-1} in shared
// memory): one warp per SM runs it from the instruction cache.
constexpr int WB = 256 / 32;

// Shared U of one warp's bins: s_up[(t * FCM_MAX_CLUSTERS + j) * 32 + lane]
// is cluster j of grey level lane + 32 t (conflict-free across the lanes).
__device__ __forceinline__ int up_at(int t, int j, int lane) { return (t * FCM_MAX_CLUSTERS + j) * 32 + lane; }

// N double-float sums over the warp, the five xor levels in a rolled loop
// (every level issues all N pairs of shuffles before the N merges).
template <int N>
__device__ __forceinline__ void warp_sum_df_rolled(DF (&d)[N]) {
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
        DF e[N];
#pragma unroll
        for (int q = 0; q < N; ++q) e[q] = DF{__shfl_xor_sync(0xffffffffu, d[q].hi, o), __shfl_xor_sync(0xffffffffu, d[q].lo, o)};
#pragma unroll
        for (int q = 0; q < N; ++q) d[q] = (lane & o) ? df_merge(e[q], d[q]) : df_merge(d[q], e[q]);
    }
}

// Iterations k = 1, 2, ... of Algorithm 1 on the bins of one run.
//   s_cnt the pixel counts of the bins (as floats), s_cnt[t * 32 + lane] for
//         grey level lane + 32 t.
//   v     in: V^1; out: V^k of the returned U^k. v64: the double-float
//         quotients behind v (in and out).
//   s_up  the warp's U (up_at): in, the bins' U^0 when the run started from
//         centers (from_u false); out, U^k. A run from memberships takes its
//         first stopping quantity d1 from the pixels instead.
//   J     out: J_k (Eq. 1) as a double-float.
template <int C, int MK>
__device__ __forceinline__ void solve_bins_warp(const float* s_cnt, bool from_u, float d1, float (&v)[C],
                                                DF (&v64)[C], float* s_up, float m, float inv_m1, float eps,
                                                int max_iter, int& flags, int& k_out, int& status_out,
                                                float& delta_out, DF& J) {
    constexpr int S = 2 * C + 1;
    const int lane = threadIdx.x & 31;
    int status = FCM_NOT_CONVERGED, k;
    float delta = 0.0f;
    for (k = 1;; ++k) {
        float acc[S];
#pragma unroll
        for (int q = 0; q < S; ++q) acc[q] = 0.0f;
        float mx = 0.0f;
        const bool first_from_u = from_u && k == 1;
#pragma unroll 1
        for (int t = 0; t < WB; t += 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float b = (float)(lane + 32 * (t + h));
                const float c = s_cnt[(t + h) * 32 + lane];
                float u[C], um[C];
                const float Ji = membership<C, MK>(b, v, m, inv_m1, u, um);
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    acc[j] = fmaf(c, um[j] * b, acc[j]);
                    acc[C + j] = fmaf(c, um[j], acc[C + j]);
                    float& upj = s_up[up_at(t + h, j, lane)];
                    if (c > 0.0f && !first_from_u) mx = fmaxf(mx, fabsf(u[j] - upj));
                    upj = u[j];
                }
                acc[2 * C] = fmaf(c, Ji, acc[2 * C]);
            }
        }
        DF tot[S];
#pragma unroll
        for (int q = 0; q < S; ++q) tot[q] = DF{acc[q], 0.0f};
        warp_sum_df_rolled<S>(tot);
        mx = warp_max(mx);
        delta = first_from_u ? d1 : mx;
        J = tot[2 * C];
        if (delta < eps) {
            status = FCM_OK;
            break;
        }
        if (k >= max_iter) break;
        // V^{k+1} (Eq. 3); an empty cluster keeps v_j
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (tot[C + j].hi > 0.0f) {
                v64[j] = df_div(tot[j], tot[C + j]);
                v[j] = v64[j].hi;
            } else {
                flags |= FCM_FLAG_EMPTY_CLUSTER;
            }
        }
    }
    k_out = k;
    status_out = status;
    delta_out = delta;
}

}  // namespace fcm
