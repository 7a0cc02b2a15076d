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
// per run lets the many runs of a batch share each SM.
constexpr int WB = 256 / 32;

// Iterations k = 1, 2, ... of Algorithm 1 on the bins of one run.
//   cnt   the pixel counts of the lane's bins (as floats).
//   v     in: V^1; out: V^k of the returned U^k. v64: the double-float
//         quotients behind v (in and out).
//   up    in: the bins' U^0 when the run started from centers (from_u
//         false); out: U^k. A run from memberships takes its first stopping
//         quantity d1 from the pixels instead.
//   J     out: J_k (Eq. 1) as a double-float.
template <int C, int MK>
__device__ __forceinline__ void solve_bins_warp(const float (&cnt)[WB], bool from_u, float d1, float (&v)[C],
                                                DF (&v64)[C], float (&up)[WB][C], float m, float inv_m1, float eps,
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
#pragma unroll
        for (int t = 0; t < WB; ++t) {
            const float b = (float)(lane + 32 * t);
            float u[C], um[C];
            const float Ji = membership<C, MK>(b, v, m, inv_m1, u, um);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                acc[j] = fmaf(cnt[t], um[j] * b, acc[j]);
                acc[C + j] = fmaf(cnt[t], um[j], acc[C + j]);
                if (cnt[t] > 0.0f && !first_from_u) mx = fmaxf(mx, fabsf(u[j] - up[t][j]));
                up[t][j] = u[j];
            }
            acc[2 * C] = fmaf(cnt[t], Ji, acc[2 * C]);
        }
        DF tot[S];
#pragma unroll
        for (int q = 0; q < S; ++q) tot[q] = DF{acc[q], 0.0f};
        warp_sum_df_n<S>(tot);
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
