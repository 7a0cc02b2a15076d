// Histogram-domain FCM on a batch of 8-bit slices: one CTA per slice.
//
// Each slice is one run of Algorithm 1 (arXiv:1601.00072, Sec. 2.1) on its
// own grey-level histogram (the brFCM reduction the paper cites, Sec. 3),
// with the iterates of the per-pixel run up to the order of rounding: a slice
// whose intensities are all integer grey levels 0..255 has memberships that
// depend only on the grey level, so after V^1 every iteration is a loop over
// 256 bins. Per slice, the CTA makes up to three passes over its pixels:
//   A. the histogram, input checks, and (from U^0) the sums of V^1 (Eq. 3);
//   B. (from U^0) the first stopping quantity max |f(x_i, V^1) - U^0_i|;
//   C. after the bin loop, U^k by table lookup.
// Sums run in FP32 over a few pixels, then in compensated FP32 (double-float)
// per thread, warp and CTA, with double-float quotients: no FP64 arithmetic
// before the results are written.
#include "fcm_batched.h"
#include "fcm_device.cuh"
#include "fcm_df.cuh"
#include "fcm_hist_bins.cuh"

namespace fcm {
namespace {

constexpr int BH_CHUNK = 4;  // pixels per thread whose loads are issued together

// Shared memory of one CTA, sized for FCM_MAX_CLUSTERS (one declaration in
// the kernel serves every C).
struct BhShared {
    unsigned hist[256];
    float T[256 * FCM_MAX_CLUSTERS];  // per grey level: U^1 (pass B), then U^k (pass C)
    DF wsum[HNT / 32][2 * FCM_MAX_CLUSTERS];
    DF tot[2 * FCM_MAX_CLUSTERS];
    float wmax[HNT / 32];
    float v1[FCM_MAX_CLUSTERS];
    double v164[FCM_MAX_CLUSTERS];
    int empty;
    BinScratch sc;
};

// Block totals of 2C double-floats, merged in warp order; every thread reads
// them from sh.tot afterwards.
template <int C>
__device__ __forceinline__ void block_df_sums(BhShared& sh, DF (&s)[2 * C]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * C; ++q) {
        const DF d = warp_sum_df(s[q]);
        if (lane == 0) sh.wsum[warp][q] = d;
    }
    __syncthreads();
    if (threadIdx.x < 2 * C) {
        const int q = threadIdx.x;
        DF t = sh.wsum[0][q];
        for (int w = 1; w < HNT / 32; ++w) t = df_merge(t, sh.wsum[w][q]);
        sh.tot[q] = t;
    }
    __syncthreads();
}

template <int C, int MK>
__device__ __noinline__ void bhist_slice(const SliceDesc& d, SliceResult& res, BhShared& sh) {
    const int64_t n = d.n;
    const float m = d.m, inv_m1 = d.inv_m1;
    const bool from_u = d.init == FCM_INIT_U;
    const float* __restrict__ x = d.x;
    const float* __restrict__ U0 = d.U0;
    const int b = threadIdx.x;
    sh.hist[b] = 0u;  // HNT == 256 threads, one bin each
    if (b == 0) sh.empty = 0;
    __syncthreads();

    // ---- pass A: histogram; from U^0 also the sums of V^1 ----
    DF acc[2 * C];
#pragma unroll
    for (int q = 0; q < 2 * C; ++q) acc[q] = DF{0.0f, 0.0f};
    bool bad = false;
    for (int64_t i0 = b; i0 < n; i0 += (int64_t)HNT * BH_CHUNK) {
        float xc[BH_CHUNK], uc[BH_CHUNK][C];
#pragma unroll
        for (int q = 0; q < BH_CHUNK; ++q) {
            const int64_t i = i0 + (int64_t)q * HNT;
            const bool in = i < n;
            xc[q] = in ? __ldg(x + i) : 0.0f;
#pragma unroll
            for (int j = 0; j < C; ++j) uc[q][j] = (in && from_u) ? __ldg(U0 + (int64_t)j * n + i) : 0.0f;
        }
        float num[C], den[C];
#pragma unroll
        for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
#pragma unroll
        for (int q = 0; q < BH_CHUNK; ++q) {
            if (i0 + (int64_t)q * HNT >= n) break;
            const float xi = xc[q];
            const bool good = grey_level(xi);
            bad |= !good;
            if (!good) continue;
            atomicAdd(&sh.hist[(int)xi], 1u);
            if (from_u) {
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float u0 = uc[q][j];
                    bad |= !(u0 >= 0.0f) || !finite_f(u0);
                    const float w = pow_m<MK>(u0, m);
                    num[j] = fmaf(w, xi, num[j]);
                    den[j] += w;
                }
            }
        }
        if (from_u) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                df_add(acc[j], num[j]);
                df_add(acc[C + j], den[j]);
            }
        }
    }
    if (!from_u) {
#pragma unroll
        for (int j = 0; j < C; ++j) bad |= !finite_f(d.V0[j]);
    }
    if (__syncthreads_or(bad)) {
        // not a grey-level slice (or a bad U^0 / V^0): nothing is written but
        // the status and V = V^0, as in the single-image histogram run
        if (b < C) {
            d.V[b] = d.V0[b];
            res.V64[b] = d.V0[b];
        }
        if (b == 0) {
            res.iters = 0;
            res.status = FCM_ERR_BAD_INPUT;
            res.flags = 0;
            res.delta = 0.0;
            res.J = 0.0;
        }
        return;
    }

    // ---- V^1 (Eq. 3): from the pixel sums, or from the bins with U^0 = f(b, V^0) ----
    const unsigned long long cnt = sh.hist[b];
    float up[C];
#pragma unroll
    for (int j = 0; j < C; ++j) up[j] = 0.0f;
    if (!from_u) {
        float v0[C], um0[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v0[j] = d.V0[j];
        membership<C, MK>((float)b, v0, m, inv_m1, up, um0);
        const float hh = (float)cnt, hl = (float)((double)cnt - (double)hh);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            acc[j] = weighted(um0[j] * (float)b, hh, hl);
            acc[C + j] = weighted(um0[j], hh, hl);
        }
    }
    block_df_sums<C>(sh, acc);
    if (b < C) {
        const DF den = sh.tot[C + b];
        if (den.hi > 0.0f) {
            const DF q = df_div(sh.tot[b], den);
            sh.v1[b] = q.hi;
            sh.v164[b] = (double)q.hi + (double)q.lo;
        } else {
            // an empty cluster keeps V^0, or 0 from a U^0
            sh.v1[b] = from_u ? 0.0f : d.V0[b];
            sh.v164[b] = sh.v1[b];
            atomicOr(&sh.empty, 1);
        }
    }
    __syncthreads();
    float v[C];
#pragma unroll
    for (int j = 0; j < C; ++j) v[j] = sh.v1[j];
    double v64 = b < C ? sh.v164[b] : 0.0;
    int flags = sh.empty ? FCM_FLAG_EMPTY_CLUSTER : 0;

    // ---- pass B (from U^0): first stopping quantity against every pixel ----
    float d1 = 0.0f;
    if (from_u) {
        {
            float u1[C], um1[C];
            membership<C, MK>((float)b, v, m, inv_m1, u1, um1);
#pragma unroll
            for (int j = 0; j < C; ++j) sh.T[b * C + j] = u1[j];
        }
        __syncthreads();
        float mx = 0.0f;
        for (int64_t i = b; i < n; i += HNT) {
            const int g = (int)__ldg(x + i);
#pragma unroll
            for (int j = 0; j < C; ++j) mx = fmaxf(mx, fabsf(sh.T[g * C + j] - __ldg(U0 + (int64_t)j * n + i)));
        }
        mx = warp_max(mx);
        if ((b & 31) == 0) sh.wmax[b >> 5] = mx;
        __syncthreads();
        d1 = sh.wmax[0];
        for (int w = 1; w < HNT / 32; ++w) d1 = fmaxf(d1, sh.wmax[w]);
        __syncthreads();  // sh.T is rewritten below
    }

    // ---- iterations on the bins ----
    float u[C];
    int k, status;
    float delta;
    solve_bins<C, MK>(sh.sc, cnt, from_u, d1, v, up, u, v64, m, inv_m1, d.eps, d.max_iter, flags, k, status, delta);
#pragma unroll
    for (int j = 0; j < C; ++j) sh.T[b * C + j] = u[j];
    __syncthreads();

    // ---- pass C: U^k by table lookup ----
    float* __restrict__ U = d.U;
    for (int64_t i = b; i < n; i += HNT) {
        const int g = (int)__ldg(x + i);
#pragma unroll
        for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + i, sh.T[g * C + j]);
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (b == j) {
            d.V[j] = v[j];
            res.V64[j] = v64;
        }
    }
    if (b == 0) {
        res.iters = k;
        res.status = status;
        res.flags = flags;
        res.delta = (double)delta;
        res.J = (double)sh.sc.tot[2 * C].hi + (double)sh.sc.tot[2 * C].lo;
    }
}

// One CTA per slice, in the order given (largest first).
__global__ void __launch_bounds__(HNT) k_bhist(const SliceDesc* __restrict__ descs, const int* __restrict__ order,
                                              int n_slices, SliceResult* __restrict__ results) {
    __shared__ BhShared sh;
    if ((int)blockIdx.x >= n_slices) return;
    const int s = order[blockIdx.x];
    const SliceDesc& d = descs[s];
    SliceResult& res = results[s];
#define FCM_BHIST_CASE(CC)                                                       \
    case CC:                                                                     \
        switch (d.mk) {                                                          \
            case M_TWO: bhist_slice<CC, M_TWO>(d, res, sh); break;               \
            case M_THREE: bhist_slice<CC, M_THREE>(d, res, sh); break;           \
            case M_ONE_HALF: bhist_slice<CC, M_ONE_HALF>(d, res, sh); break;     \
            default: bhist_slice<CC, M_GENERIC>(d, res, sh); break;              \
        }                                                                        \
        break;
    switch (d.C) {
        FCM_BHIST_CASE(1)
        FCM_BHIST_CASE(2)
        FCM_BHIST_CASE(3)
        FCM_BHIST_CASE(4)
        FCM_BHIST_CASE(5)
        FCM_BHIST_CASE(6)
        FCM_BHIST_CASE(7)
        FCM_BHIST_CASE(8)
        default: break;
    }
#undef FCM_BHIST_CASE
}

}  // namespace

cudaError_t launch_bhist(const SliceDesc* descs, const int* order, int n_slices, SliceResult* results,
                         cudaStream_t s) {
    k_bhist<<<n_slices, HNT, 0, s>>>(descs, order, n_slices, results);
    return cudaGetLastError();
}

}  // namespace fcm
