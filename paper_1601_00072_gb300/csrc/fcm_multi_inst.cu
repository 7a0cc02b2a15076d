// Multi-feature FCM: pixels with D channels (colour, or co-registered MR
// sequences), one cooperative launch per run.
//
// Compiled once per channel count with -DFCM_MULTI_D=1..4.
//
// Sec. 2.1 defines d_ij as a norm of x_i - v_j; with D channels it is the
// Euclidean norm over the channels, so Eq. 4 takes d_ij^2 = sum_d (x_id -
// v_jd)^2, Eq. 3 gives each center channel by channel, and Eq. 1 sums
// u_ij^m d_ij^2. The loop is Algorithm 1 with the readings of the scalar
// path (zero distance, L-infinity stopping test, empty clusters).
//
// Like the scalar recompute run, no U is stored between iterations: U^{k-1}
// comes from V^{k-1} through the same code, an iteration reads only x
// (4D bytes per pixel), and U^k is written once after the stop decision.
// Every block adds the per-block sums (compensated FP32 pairs) in the same
// order after a bounded grid barrier, so all blocks take the same decisions.
#include "fcm_device.cuh"
#include "fcm_multi.h"

#ifndef FCM_MULTI_D
#error "compile with -DFCM_MULTI_D=<channels>"
#endif

namespace fcm {
namespace {

constexpr int D = FCM_MULTI_D;
constexpr int MNT = 256;
constexpr int MNW = MNT / 32;
constexpr int MCHUNK = 4;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Memberships of one pixel from its squared distances d2[j] (Eq. 4 in the
// weight form w_j = (d2min / d2_j)^(1/(m-1)), u_j = w_j / sum_k w_k, with the
// zero-distance rule). A squared distance below the smallest normal float
// (2^-126) counts as zero, as the .ftz reciprocal and logarithm would read
// it. Returns the pixel's J term, d2min * S^(1-m).
template <int C, int MK>
__device__ __forceinline__ float membership_d2(const float (&d2)[C], float m, float inv_m1, float (&u)[C],
                                               float (&um)[C]) {
    float dmin = __int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < C; ++j) dmin = fminf(dmin, d2[j]);
    float Ji = 0.0f;
    if (dmin >= flt_min()) {
        float w[C];
        if (MK == M_TWO) {
#pragma unroll
            for (int j = 0; j < C; ++j) w[j] = dmin * rcp_approx(d2[j]);
        } else {
            const float l0 = lg2_approx(dmin);
#pragma unroll
            for (int j = 0; j < C; ++j) w[j] = ex2_approx(inv_m1 * (l0 - lg2_approx(d2[j])));
        }
        float S = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) S += w[j];
        const float r = rcp_approx(S);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = w[j] * r;
        Ji = (MK == M_TWO) ? dmin * r : dmin * ex2_approx((1.0f - m) * lg2_approx(S));
    } else {
        int nz = 0;
#pragma unroll
        for (int j = 0; j < C; ++j) nz += (d2[j] < flt_min());
        const float share = __fdiv_rn(1.0f, (float)nz);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = (d2[j] < flt_min()) ? share : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < C; ++j) um[j] = (MK == M_TWO) ? u[j] * u[j] : ex2_approx(m * lg2_approx(u[j]));
    return Ji;
}

template <int C>
__device__ __forceinline__ void dist2(const float (&xv)[D], const float* vs, float (&d2)[C]) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const float t = xv[d] - vs[j * D + d];
            s = fmaf(t, t, s);
        }
        d2[j] = s;
    }
}

// Pass 0 is INIT (V^1 from U^0, or from U^0 = f(x, V^0)); pass p >= 1 is
// iteration p; the pass after the stop decision writes U^k.
template <int C, int MK, bool FROM_U>
__global__ void __launch_bounds__(MNT) k_fcm_run_multi(MultiState* __restrict__ st, float* __restrict__ partials) {
    constexpr int NS = C * D + C + 1;  // num[C][D], den[C], J (compensated)
    constexpr int S = NS + 3;          // then max|dU|, bad input, timeout
    __shared__ float s_v[C * D], s_vp[C * D];
    __shared__ float s_w[MNW][2 * NS + 3];
    __shared__ DF s_df[NS];
    __shared__ float s_mx[3];
    __shared__ int s_err;

    const float* __restrict__ x = st->x;
    const float* __restrict__ U0 = st->U0;
    float* __restrict__ U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1, eps = st->eps;
    const int max_iter = st->max_iter;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < C * D; t += MNT) s_v[t] = s_vp[t] = st->V0[t];
    if (threadIdx.x == 0) s_err = 0;
    double v64 = threadIdx.x < C * D ? (double)st->V0[threadIdx.x] : 0.0;  // thread t keeps the FP64 quotient
    int flags = 0;
    __syncthreads();

    const int64_t stride = (int64_t)gridDim.x * MNT;
    bool emit = false, stop = false;
    int status = FCM_NOT_CONVERGED, iters = 0;
    for (int p = 0;; ++p) {
        // ---- the pass over this thread's pixels ----
        DF acc[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) acc[q] = DF{0.0f, 0.0f};
        float dmax = 0.0f;
        bool bad = false;
        if (p == 0 && !FROM_U && threadIdx.x < C * D) bad |= !finite_f(s_v[threadIdx.x]);
        for (int64_t i0 = (int64_t)blockIdx.x * MNT + threadIdx.x; i0 < n; i0 += stride * MCHUNK) {
            float num[C * D], den[C], J = 0.0f;
#pragma unroll
            for (int q = 0; q < C * D; ++q) num[q] = 0.0f;
#pragma unroll
            for (int j = 0; j < C; ++j) den[j] = 0.0f;
            for (int c = 0; c < MCHUNK; ++c) {
                const int64_t i = i0 + (int64_t)c * stride;
                if (i >= n) break;
                float xv[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xv[d] = __ldg(x + (int64_t)d * n + i);
                float u[C], um[C];
                if (emit) {
                    float d2[C];
                    dist2<C>(xv, s_v, d2);
                    membership_d2<C, MK>(d2, m, inv_m1, u, um);
#pragma unroll
                    for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + i, u[j]);
                    continue;
                }
                if (p == 0) {
#pragma unroll
                    for (int d = 0; d < D; ++d) bad |= !finite_f(xv[d]);
                }
                if (p == 0 && FROM_U) {
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const float u0 = __ldg(U0 + (int64_t)j * n + i);
                        bad |= !(u0 >= 0.0f) || !finite_f(u0);
                        um[j] = (MK == M_TWO) ? u0 * u0 : ex2_approx(m * lg2_approx(u0));
                    }
                } else {
                    float d2[C];
                    dist2<C>(xv, s_v, d2);
                    J += membership_d2<C, MK>(d2, m, inv_m1, u, um);
                    if (p >= 1) {
                        float uo[C];
                        if (p == 1 && FROM_U) {
#pragma unroll
                            for (int j = 0; j < C; ++j) uo[j] = __ldg(U0 + (int64_t)j * n + i);
                        } else {
                            float d2p[C], ump[C];
                            dist2<C>(xv, s_vp, d2p);
                            membership_d2<C, MK>(d2p, m, inv_m1, uo, ump);
                        }
#pragma unroll
                        for (int j = 0; j < C; ++j) dmax = fmaxf(dmax, fabsf(u[j] - uo[j]));
                    }
                }
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    den[j] += um[j];
#pragma unroll
                    for (int d = 0; d < D; ++d) num[j * D + d] = fmaf(um[j], xv[d], num[j * D + d]);
                }
            }
#pragma unroll
            for (int q = 0; q < C * D; ++q) df_add(acc[q], num[q]);
#pragma unroll
            for (int j = 0; j < C; ++j) df_add(acc[C * D + j], den[j]);
            df_add(acc[NS - 1], J);
        }
        if (emit) break;

        // ---- block totals -> partials[p & 1], slot-major (hi, lo) pairs ----
#pragma unroll
        for (int q = 0; q < NS; ++q) acc[q] = warp_sum_df(acc[q]);
        const float wm = warp_max(dmax), wb = warp_max(bad ? 1.0f : 0.0f);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                s_w[warp][2 * q] = acc[q].hi;
                s_w[warp][2 * q + 1] = acc[q].lo;
            }
            s_w[warp][2 * NS] = wm;
            s_w[warp][2 * NS + 1] = wb;
            s_w[warp][2 * NS + 2] = 0.0f;
        }
        __syncthreads();
        float* part = partials + (int64_t)(p & 1) * (2 * S) * gridDim.x;
        if (threadIdx.x < S) {
            const int q = threadIdx.x;
            if (q < NS) {
                DF t = DF{s_w[0][2 * q], s_w[0][2 * q + 1]};
                for (int w = 1; w < MNW; ++w) t = df_merge(t, DF{s_w[w][2 * q], s_w[w][2 * q + 1]});
                __stcg(part + (int64_t)(2 * q) * gridDim.x + blockIdx.x, t.hi);
                __stcg(part + (int64_t)(2 * q + 1) * gridDim.x + blockIdx.x, t.lo);
            } else {
                float t = 0.0f;
                for (int w = 0; w < MNW; ++w) t = fmaxf(t, s_w[w][2 * NS + (q - NS)]);
                __stcg(part + (int64_t)(2 * q) * gridDim.x + blockIdx.x, t);
            }
        }
        __syncthreads();
        // ---- bounded grid barrier ----
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&st->ticket, 1u);
            // bounded by st->lim: grid_spins polls 128 ns apart, for the
            // grid's arrivals plus st->lim.phantoms (0 unless a test injects
            // a barrier that never fills)
            const unsigned target = (unsigned)(p + 1) * gridDim.x + st->lim.phantoms;
            const uint32_t limit = st->lim.grid_spins;
            uint32_t spins = 0;
            while (ld_acquire_u32(&st->ticket) < target) {
                if (++spins > limit) {
                    s_err = 1;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_err) {
            status = FCM_ERR_TIMEOUT;
            iters = p;
            break;
        }
        // ---- cross-block sums, the same fixed order in every block ----
        for (int q = warp; q < S; q += MNW) {
            const float* ph = part + (int64_t)(2 * q) * gridDim.x;
            if (q < NS) {
                const float* pl = ph + gridDim.x;
                DF d{0.0f, 0.0f};
                for (int b = lane; b < (int)gridDim.x; b += 32) d = df_merge(d, DF{__ldcg(ph + b), __ldcg(pl + b)});
                d = warp_sum_df(d);
                if (lane == 0) s_df[q] = d;
            } else {
                float t = 0.0f;
                for (int b = lane; b < (int)gridDim.x; b += 32) t = fmaxf(t, __ldcg(ph + b));
                t = warp_max(t);
                if (lane == 0) s_mx[q - NS] = t;
            }
        }
        __syncthreads();
        const float delta = s_mx[0];
        const bool badin = s_mx[1] != 0.0f;
        bool update = false;
        if (p == 0) {
            if (badin) {
                status = FCM_ERR_BAD_INPUT;
                stop = true;
            } else {
                update = true;
            }
        } else {
            if (delta < eps) {
                status = FCM_OK;
                iters = p;
                stop = emit = true;
            } else if (p >= max_iter) {
                status = FCM_NOT_CONVERGED;
                iters = p;
                stop = emit = true;
            } else {
                update = true;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->delta = delta;
                st->J = (double)s_df[NS - 1].hi + (double)s_df[NS - 1].lo;
            }
        }
        if (update) {
            // V^{p+1}_jd = num_jd / den_j in FP64 (Eq. 3); an empty cluster
            // keeps its center (first pass: V^0, or 0 from a U^0)
            float nv = 0.0f;
            bool empty = false;
            if (threadIdx.x < C * D) {
                const int t = threadIdx.x, j = t / D;
                const double num = (double)s_df[t].hi + (double)s_df[t].lo;
                const double den = (double)s_df[C * D + j].hi + (double)s_df[C * D + j].lo;
                empty = !(den > 0.0);
                if (!empty) {
                    v64 = num / den;
                    nv = (float)v64;
                } else {
                    nv = (p == 0 && FROM_U) ? 0.0f : s_v[t];
                    v64 = nv;
                }
            }
            if (__syncthreads_or(empty)) flags |= FCM_FLAG_EMPTY_CLUSTER;
            if (threadIdx.x < C * D) {
                s_vp[threadIdx.x] = s_v[threadIdx.x];
                s_v[threadIdx.x] = nv;
            }
        }
        __syncthreads();
        if (stop && !emit) break;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < C * D) {
            st->V[threadIdx.x] = s_v[threadIdx.x];
            st->V64[threadIdx.x] = v64;
        }
        if (threadIdx.x == 0) {
            st->status = status;
            st->iters = iters;
            st->flags = flags;
        }
    }
}

template <int C, int MK>
void fill(MultiTable& t) {
    t.run[D][C][MK == M_TWO ? 0 : 1][0] = k_fcm_run_multi<C, MK, true>;
    t.run[D][C][MK == M_TWO ? 0 : 1][1] = k_fcm_run_multi<C, MK, false>;
}

template <int C>
void fill_c(MultiTable& t) {
    fill<C, M_TWO>(t);
    fill<C, M_GENERIC>(t);
}

}  // namespace

#define FCM_CAT2(a, b) a##b
#define FCM_CAT(a, b) FCM_CAT2(a, b)
void FCM_CAT(register_multi_d, FCM_MULTI_D)(MultiTable& t) {
    fill_c<1>(t);
    fill_c<2>(t);
    fill_c<3>(t);
    fill_c<4>(t);
    fill_c<5>(t);
    fill_c<6>(t);
    fill_c<7>(t);
    fill_c<8>(t);
}

}  // namespace fcm
