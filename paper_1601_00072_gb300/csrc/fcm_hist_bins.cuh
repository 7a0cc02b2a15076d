// Algorithm 1 (arXiv:1601.00072, Sec. 2.1) on the 256-bin grey-level
// histogram: the loop of the histogram-domain run (brFCM, cited in Sec. 3),
// shared by the single-image kernel and the batch kernels (one CTA per run).
//
// Under Eq. 4 a pixel's memberships depend only on its grey level, so the
// center sums of Eq. 3 and J of Eq. 1 are sums over bins weighted by their
// pixel counts, and the stopping quantity is a maximum over the bins present.
#pragma once

#include "fcm_device.cuh"
#include "fcm_df.cuh"

namespace fcm {

constexpr int HNT = 256;  // threads of the pixel-pass and bin-loop CTAs

__device__ __forceinline__ bool grey_level(float v) {
    return v >= 0.0f && v <= 255.0f && v == rintf(v);  // false for NaN
}

// The grey level of v when v is an integer in [0, 255], else -1 (the same
// test as grey_level, with the index). Adding 1.5 * 2^23 rounds any
// |v| < 2^22 to an integer held in the low mantissa bits; v is that integer
// exactly when subtracting the constant gives v back. NaN fails the
// comparison; infinities and values outside [0, 255] give an index outside
// [0, 255] (as unsigned).
__device__ __forceinline__ int grey_index(float v) {
    constexpr float kShift = 12582912.0f;  // 1.5 * 2^23
    const float t = __fadd_rn(v, kShift);
    const int g = __float_as_int(t) - __float_as_int(kShift);
    return ((unsigned)g <= 255u && __fsub_rn(t, kShift) == v) ? g : -1;
}

// The loop runs in one CTA of HNT threads, thread b holding grey level b.
// A sum over the bins is taken in two steps: a five-level FP32 xor tree in
// each warp (non-negative terms: at most five roundings, no cancellation),
// then the eight warp totals in double-float, by a three-level xor tree over
// groups of eight lanes that every warp evaluates alike. So every thread
// holds the same totals and forms the same V^{k+1} (double-float quotients),
// and one barrier per reduction suffices: the warp totals are double-buffered
// by the parity `par`, which every reduction flips.
constexpr int HNW = HNT / 32;
static_assert(HNW == 8, "the cross-warp tree takes eight warp totals");

struct BinScratch {
    float w[2][HNW][2 * FCM_MAX_CLUSTERS + 2];  // [parity][warp]: N sums, then one maximum
};

// N block sums and one block maximum: t[0..N-1] are this thread's terms and
// t[N] its maximum; on return every thread holds the totals tot[] and the
// maximum mx, the same in all threads. All HNT threads must call it.
template <int N>
__device__ __forceinline__ void block_sums(BinScratch& sc, int& par, float (&t)[N + 1], DF (&tot)[N], float& mx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float e[N + 1];
#pragma unroll
        for (int q = 0; q <= N; ++q) e[q] = __shfl_xor_sync(0xffffffffu, t[q], o);
#pragma unroll
        for (int q = 0; q < N; ++q) t[q] += e[q];  // a + b == b + a: every lane gets the same total
        t[N] = fmaxf(t[N], e[N]);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q <= N; ++q) sc.w[par][warp][q] = t[q];
    }
    __syncthreads();
    // lane l takes the total of warp l & 7 for sum 4 r + (l >> 3)
    const int g = lane >> 3, w = lane & 7;
#pragma unroll
    for (int r = 0; r < (N + 3) / 4; ++r) {
        const int q = 4 * r + g;
        DF d{q < N ? sc.w[par][w][q] : 0.0f, 0.0f};
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const DF e{__shfl_xor_sync(0xffffffffu, d.hi, o), __shfl_xor_sync(0xffffffffu, d.lo, o)};
            d = (lane & o) ? df_merge(e, d) : df_merge(d, e);  // lower warp first, in every lane
        }
#pragma unroll
        for (int gg = 0; gg < 4; ++gg)
            if (4 * r + gg < N)
                tot[4 * r + gg] = DF{__shfl_sync(0xffffffffu, d.hi, 8 * gg), __shfl_sync(0xffffffffu, d.lo, 8 * gg)};
    }
    mx = sc.w[par][0][N];
#pragma unroll
    for (int u = 1; u < HNW; ++u) mx = fmaxf(mx, sc.w[par][u][N]);
    par ^= 1;
}

// Iterations k = 1, 2, ... of Algorithm 1 on the bins of one run, in one CTA.
//   cnt   the pixel count of this thread's grey level (as a float).
//   from_u  the run started from U^0: its first stopping quantity is d1,
//         taken over the pixels (a run from centers has U^0 per grey level).
//   v, v64  in: V^1 (the same in every thread) and the double-float quotients
//         behind it; out: V^k of the returned U^k.
//   up    in: U^0 of this grey level (runs from centers); out: its U^k.
//   J     out: J_k (Eq. 1).
// An empty cluster keeps its center and sets the flag.
template <int C, int MK>
__device__ __forceinline__ void solve_bins(BinScratch& sc, int& par, float cnt, bool from_u, float d1,
                                           float (&v)[C], DF (&v64)[C], float (&up)[C], float m, float inv_m1,
                                           float eps, int max_iter, int& flags, int& k_out, int& status_out,
                                           float& delta_out, DF& J) {
    constexpr int S = 2 * C + 1;
    const float b = (float)threadIdx.x;
    int status = FCM_NOT_CONVERGED, k;
    float delta = 0.0f;
#pragma unroll 1
    for (k = 1;; ++k) {
        float u[C], um[C];
        const float Ji = membership<C, MK>(b, v, m, inv_m1, u, um);
        float t[S + 1], dm;
        DF tot[S];
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            t[j] = cnt * (um[j] * b);
            t[C + j] = cnt * um[j];
            if (cnt > 0.0f) mx = fmaxf(mx, fabsf(u[j] - up[j]));
            up[j] = u[j];
        }
        t[2 * C] = cnt * Ji;
        t[S] = mx;
        block_sums<S>(sc, par, t, tot, dm);
        delta = (from_u && k == 1) ? d1 : dm;
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
