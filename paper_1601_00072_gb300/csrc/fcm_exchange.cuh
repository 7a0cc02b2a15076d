// The cross-block exchange of the whole-run kernels (stored-U and U-free):
// after every pass each block has published its FP32 totals, slot-major
// (part[s * nb + b]), and met the others at a grid barrier; every block then
// forms the same grid totals in the same fixed order, so all blocks derive
// the same centers V^{k+1} (Eq. 3) and the same stop decision.
#pragma once

#include "fcm_device.cuh"
#include "fcm_df.cuh"

namespace fcm {

// Grid totals of S slots: slots 0..NS-1 are sums (double-float), the rest
// maxima. Warp w takes slots w, w + NW, ...; its lanes add the partials
// b = lane, lane + 32, ... in b order (the loop unrolled so that several L2
// loads are in flight at once), and a warp tree finishes each slot. Writes
// s_df[0..NS) and s_mx[0..S-NS).
template <int S, int NS, int NW>
__device__ __forceinline__ void grid_totals(const float* __restrict__ part, int nb, DF* s_df, float* s_mx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = warp; s < S; s += NW) {
        const float* ps = part + (int64_t)s * nb;
        if (s < NS) {
            DF d{0.0f, 0.0f};
#pragma unroll 6
            for (int b = lane; b < nb; b += 32) df_add(d, __ldcg(ps + b));
            d = warp_sum_df(d);
            if (lane == 0) s_df[s] = d;
        } else {
            float t = 0.0f;
#pragma unroll 6
            for (int b = lane; b < nb; b += 32) t = fmaxf(t, __ldcg(ps + b));
            t = warp_max(t);
            if (lane == 0) s_mx[s - NS] = t;
        }
    }
}

// V^{k+1}_j = num_j / den_j (Eq. 3) as a double-float quotient (about 44
// bits, FP32 instructions only), on threads j < C; an empty cluster (den = 0)
// is flagged and its quotient left 0.
template <int C>
__device__ __forceinline__ void grid_centers(const DF* s_df, DF* s_vq, int* s_empty) {
    if (threadIdx.x < C) {
        const int j = threadIdx.x;
        const DF den = s_df[C + j];
        const bool empty = !(den.hi > 0.0f);
        s_vq[j] = empty ? DF{0.0f, 0.0f} : df_div(s_df[j], den);
        s_empty[j] = empty;
    }
}

__device__ __forceinline__ double df_to_double(DF d) { return (double)d.hi + (double)d.lo; }

}  // namespace fcm
