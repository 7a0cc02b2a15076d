// Algorithm 1 (arXiv:1601.00072, Sec. 2.1) on the 256-bin grey-level
// histogram: the loop of the histogram-domain run (brFCM, cited in Sec. 3),
// shared by the single-image kernel and the batch kernel (one CTA per slice).
//
// Under Eq. 4 a pixel's memberships depend only on its grey level, so the
// center sums of Eq. 3 and J of Eq. 1 are sums over bins weighted by their
// pixel counts, and the stopping quantity is a maximum over the bins present.
#pragma once

#include "fcm_device.cuh"
#include "fcm_df.cuh"

namespace fcm {

constexpr int HNT = 256;  // threads of a bin-solver CTA: thread b holds grey level b

__device__ __forceinline__ bool grey_level(float v) {
    return v >= 0.0f && v <= 255.0f && v == rintf(v);  // false for NaN
}

// w * (hh + hl) as a double-float pair: the exact product w * hh (TwoProd by
// FMA) plus the small w * hl.
__device__ __forceinline__ DF weighted(float w, float hh, float hl) {
    const float p = w * hh;
    const float e = fmaf(w, hh, -p);
    DF d{p, 0.0f};
    df_add(d, fmaf(w, hl, e));
    return d;
}

// Shared scratch of the bin solver, sized for FCM_MAX_CLUSTERS.
struct BinScratch {
    DF wtot[HNT / 32][2 * FCM_MAX_CLUSTERS + 1];
    float wmax[HNT / 32];
    DF tot[2 * FCM_MAX_CLUSTERS + 1];  // after the solve: tot[2C] = J_k
    float s_v[FCM_MAX_CLUSTERS], s_delta;
    double s_v64[FCM_MAX_CLUSTERS];
    int s_empty;
};

// Iterations k = 1, 2, ... of Algorithm 1 on the bins, in one CTA of HNT
// threads; thread b holds grey level b and its pixel count cnt.
//   v     in: V^1 (the same in every thread); out: V^k of the returned U^k.
//   up    the bin's U^0 when the run started from centers (from_u false); a
//         run from memberships takes its first stopping quantity d1 from the
//         pass over the pixels instead.
//   u     out: the bin's U^k.
//   v64   threads j < C: in, the quotient behind V^1_j; out, behind V^k_j.
// Sums over the bins run in compensated FP32 (per-bin exact products,
// double-float warp trees, the eight warp totals merged in a fixed order by
// warp 0); an empty cluster keeps its center and sets the flag.
template <int C, int MK>
__device__ __forceinline__ void solve_bins(BinScratch& sc, unsigned long long cnt, bool from_u, float d1,
                                           float (&v)[C], float (&up)[C], float (&u)[C], double& v64, float m,
                                           float inv_m1, float eps, int max_iter, int& flags, int& k_out,
                                           int& status_out, float& delta_out) {
    constexpr int S = 2 * C + 1;
    const int b = threadIdx.x, lane = b & 31, warp = b >> 5;
    const bool present = cnt > 0ull;
    // the count as an unevaluated float pair (exact below 2^48)
    const float hh = (float)cnt, hl = (float)((double)cnt - (double)hh);
    float um[C];
    int status = FCM_NOT_CONVERGED, k = 1;
    float delta = 0.0f;
    for (k = 1;; ++k) {
        const float Ji = membership<C, MK>((float)b, v, m, inv_m1, u, um);
        DF s[S];
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            s[j] = weighted(um[j] * (float)b, hh, hl);
            s[C + j] = weighted(um[j], hh, hl);
            if (present && !(from_u && k == 1)) mx = fmaxf(mx, fabsf(u[j] - up[j]));
        }
        s[2 * C] = weighted(Ji, hh, hl);
#pragma unroll
        for (int q = 0; q < S; ++q) s[q] = warp_sum_df(s[q]);
        mx = warp_max(mx);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < S; ++q) sc.wtot[warp][q] = s[q];
            sc.wmax[warp] = mx;
        }
        __syncthreads();
        if (warp == 0) {
            // lane q merges sum q over the warps, in warp order
            if (lane < S) {
                DF t = sc.wtot[0][lane];
                for (int w = 1; w < HNT / 32; ++w) t = df_merge(t, sc.wtot[w][lane]);
                sc.tot[lane] = t;
            }
            float dm = lane < HNT / 32 ? sc.wmax[lane] : 0.0f;
            dm = warp_max(dm);
            __syncwarp();
            if (lane == 0) sc.s_delta = (from_u && k == 1) ? d1 : dm;
            // V^{k+1} (Eq. 3), computed by lane j; an empty cluster keeps v_j
            bool empty = false;
            if (lane < C) {
                const DF den = sc.tot[C + lane];
                if (den.hi > 0.0f) {
                    const DF q = df_div(sc.tot[lane], den);
                    sc.s_v[lane] = q.hi;
                    sc.s_v64[lane] = (double)q.hi + (double)q.lo;
                } else {
                    sc.s_v[lane] = v[lane];
                    sc.s_v64[lane] = v64;
                    empty = true;
                }
            }
            const unsigned em = __ballot_sync(0xffffffffu, empty);
            if (lane == 0) sc.s_empty = em != 0u;
        }
        __syncthreads();
        delta = sc.s_delta;
        if (delta < eps) {
            status = FCM_OK;
            break;
        }
        if (k >= max_iter) break;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            up[j] = u[j];
            v[j] = sc.s_v[j];
        }
        if (b < C) v64 = sc.s_v64[b];
        if (sc.s_empty) flags |= FCM_FLAG_EMPTY_CLUSTER;
        __syncthreads();  // s_v and the totals are reused by the next iteration
    }
    k_out = k;
    status_out = status;
    delta_out = delta;
}

}  // namespace fcm
