// The whole single-image run without storing U between iterations.
//
// Compiled once per cluster count with -DFCM_INST_C=<C>.
//
// Algorithm 1 (Sec. 2.1) needs U^{k-1} only for the stopping quantity
// max |U^k - U^{k-1}|. Here U^{k-1} is recomputed from V^{k-1} with the same
// code that would have produced it (Eq. 4; bit-identical, same inputs), so an
// iteration reads only x: 4 bytes per pixel instead of 4 + 8C. For the 256^3
// volume x is 67 MB and stays in the 129 MB L2 across iterations, so the
// iterations trade HBM traffic for arithmetic. U^0 (when given) is read in
// pass 0 and iteration 1; U^k is written once, in an extra pass after the
// stop decision.
//
// Structure as the stored-U run kernel: one cooperative launch, each warp
// streams its own 128-pixel tiles through a private ring of TMA bulk copies
// across all passes, every block adds the per-block sums in the same order
// after a bounded grid barrier, so all blocks take the same decisions.
#include "fcm_bounds.cuh"
#include "fcm_device.cuh"
#include "fcm_exchange.cuh"
#include "fcm_internal.h"
#include "fcm_recompute.h"
#include "fcm_tma.cuh"

#ifndef FCM_INST_C
#error "compile with -DFCM_INST_C=<clusters>"
#endif

namespace fcm {
namespace {

constexpr int WTILE = WARP_TILE;
// Wait bounds come from st->lim: mbarrier waits of tma_polls suspensions of
// about 1 ms; the grid barrier polls grid_spins times, 128 ns apart, for the
// grid's arrivals plus st->lim.phantoms (0 unless a test injects a barrier
// that never fills).

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int C, int INIT>
struct RcShape {
    static constexpr int ROWS = INIT == P_ACCUM0 ? 1 + C : 1;  // x, then the rows of U^0
    static constexpr int STAGE_FLOATS = ROWS * WTILE;
    static constexpr int BLOCKS_PER_SM = C <= 4 ? 3 : 2;
    static constexpr int RAW = ((BLOCKS_PER_SM == 3 ? 72 : 108) * 1024) / (NWARP * STAGE_FLOATS * 4);
    static constexpr int STAGES = RAW < 2 ? 2 : (RAW > 8 ? 8 : RAW);
    static constexpr int SMEM_BYTES = NWARP * STAGES * STAGE_FLOATS * 4;
};

template <int C>
struct RcAcc {
    f2 num2[C], den2[C], J2;
    float num[C], den[C], J, dmax;
    bool bad;
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            num2[j] = den2[j] = pack2(0.0f, 0.0f);
            num[j] = den[j] = 0.0f;
        }
        J2 = pack2(0.0f, 0.0f);
        J = dmax = 0.0f;
        bad = false;
    }
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            num[j] += lo2(num2[j]) + hi2(num2[j]);
            den[j] += lo2(den2[j]) + hi2(den2[j]);
        }
        J += lo2(J2) + hi2(J2);
    }
};

enum RcKind : int { RC_ACCUM0 = 0, RC_INITV = 1, RC_ITER_U0 = 2, RC_ITER = 3, RC_EMIT = 4 };

// One warp tile at sb (x, then the U^0 rows when they were copied): lane l
// takes pixels 2l, 2l+1 and 64+2l, 65+2l (cnt is a multiple of 4).
template <int C, int MK, int KIND>
__device__ __forceinline__ void rc_tile(const float* sb, int cnt, int64_t i0, int lane, float* U, int64_t n,
                                        const float (&v)[C], const f2 (&v2)[C], const float (&vp)[C],
                                        const f2 (&vp2)[C], float m, float inv_m1, uint64_t pol_u, RcAcc<C>& a) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int pp = q * (WTILE / 2) + 2 * lane;
        if (pp >= cnt) continue;
        const float2 xv = lds2(sb + pp);
        if (KIND == RC_ACCUM0) {
            a.bad |= !finite_f(xv.x) || !finite_f(xv.y);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float2 u0 = lds2(sb + (1 + j) * WTILE + pp);
                a.bad |= !(u0.x >= 0.0f) || !finite_f(u0.x) || !(u0.y >= 0.0f) || !finite_f(u0.y);
                const float w0 = pow_m<MK>(u0.x, m), w1 = pow_m<MK>(u0.y, m);
                a.num[j] = fmaf(w0, xv.x, fmaf(w1, xv.y, a.num[j]));
                a.den[j] += w0 + w1;
            }
            continue;
        }
        const f2 xq = pack2(xv.x, xv.y);
        f2 u2[C], um2[C];
        if (KIND == RC_EMIT) {
            membership_pair<C, MK>(xq, v2, m, inv_m1, v, u2, um2);
#pragma unroll
            for (int j = 0; j < C; ++j) st_hint2(U + (int64_t)j * n + i0 + pp, u2[j], pol_u);
            continue;
        }
        if (KIND == RC_INITV) a.bad |= !finite_f(xv.x) || !finite_f(xv.y);
        a.J2 = add2(a.J2, membership_pair<C, MK>(xq, v2, m, inv_m1, v, u2, um2));
        f2 uo2[C];
        if (KIND == RC_ITER_U0) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float2 u0 = lds2(sb + (1 + j) * WTILE + pp);
                uo2[j] = pack2(u0.x, u0.y);
            }
        } else if (KIND == RC_ITER) {
            f2 tmp[C];
            membership_pair<C, MK>(xq, vp2, m, inv_m1, vp, uo2, tmp);
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            a.num2[j] = fma2(um2[j], xq, a.num2[j]);
            a.den2[j] = add2(a.den2[j], um2[j]);
            if (KIND == RC_ITER || KIND == RC_ITER_U0) {
                float da, db;
                unpack2(sub2(u2[j], uo2[j]), da, db);
                a.dmax = fmaxf(a.dmax, fmaxf(fabsf(da), fabsf(db)));
            }
        }
    }
}

// Pass 0 is INIT (V^1 from U^0, or from U^0 = f(x, V^0)); pass p >= 1 is
// iteration p; the pass after the stop decision writes U^k.
template <int C, int MK, int INIT>
__global__ void __launch_bounds__(NT, (C <= 4 ? 3 : 2)) k_fcm_run_rc(RunState* __restrict__ st,
                                                                     double* __restrict__ partials_raw) {
    using Sh = RcShape<C, INIT>;
    constexpr int S = 2 * C + 4;
    extern __shared__ __align__(128) float ring_all[];
    __shared__ __align__(8) uint64_t full_all[NWARP][Sh::STAGES];
    __shared__ float s_red[NWARP][S];
    __shared__ DF s_df[2 * C + 1];
    __shared__ float s_mx[3];
    __shared__ DF s_vq[C];
    __shared__ int s_empty[C];
    __shared__ int s_err;

    const float* __restrict__ x = st->x;
    const float* U0 = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1, eps = st->eps;
    const int max_iter = st->max_iter;
    unsigned* gbar = &st->ticket;
    float* partials = reinterpret_cast<float*>(partials_raw);

    float v[C], vp[C];
    f2 v2[C], vp2[C];
    DF v64[C];  // the double-float quotients behind v, converted to FP64 only when written
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = vp[j] = st->V0[j];
        v2[j] = vp2[j] = pack2(v[j], v[j]);
        v64[j] = DF{v[j], 0.0f};
    }
    int flags = 0;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* ring = ring_all + warp * (Sh::STAGES * Sh::STAGE_FLOATS);
    uint64_t* full = full_all[warp];
    const int64_t nwarps = (int64_t)gridDim.x * NWARP;
    const int64_t gw = (int64_t)blockIdx.x * NWARP + warp;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    const int nk = (int)(ntiles > gw ? (ntiles - 1 - gw) / nwarps + 1 : 0);
    const int look = nk < Sh::STAGES ? nk : Sh::STAGES;
    const int64_t tile_stride = nwarps * (int64_t)WTILE;
    const int npass = 2 + max_iter;  // INIT, max_iter iterations, the U write
    const uint32_t wait_limit = st->lim.tma_polls, grid_spins = st->lim.grid_spins;
    const unsigned phantoms = st->lim.phantoms;
    const uint64_t pol_x = policy_evict_last();
    const uint64_t pol_u = policy_evict_first();

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < Sh::STAGES; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();

    // Issue side (lane 0): pass ip, tile ik of the next load, ring slot is.
    int ip = 0, ik = 0, is = 0;
    int64_t issued = 0;
    auto issue_next = [&]() {
        if (ip >= npass || nk == 0) return;
        const int64_t i0 = gw * (int64_t)WTILE + ik * tile_stride;
        const uint32_t bytes = (uint32_t)min((int64_t)WTILE, n - i0) * 4u;  // multiple of 16
        const bool with_u = INIT == P_ACCUM0 && ip <= 1;
        float* dst = ring + is * Sh::STAGE_FLOATS;
        if (!in_bounds(i0 >= 0 && i0 < n && i0 % 4 == 0, &st->bounds)) {
            mbar_expect_tx(&full[is], 0u);  // arrive without copies: the consumer's tile is empty
            ++issued;
            if (++ik == nk) {
                ik = 0;
                ++ip;
            }
            if (++is == Sh::STAGES) is = 0;
            return;
        }
        mbar_expect_tx(&full[is], bytes * (with_u ? 1 + C : 1));
        bulk_g2s(dst, x + i0, bytes, &full[is], pol_x);
        if (with_u) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                bulk_g2s(dst + (1 + j) * WTILE, U0 + (int64_t)j * n + i0, bytes, &full[is], pol_u);
        }
        ++issued;
        if (++ik == nk) {
            ik = 0;
            ++ip;
        }
        if (++is == Sh::STAGES) is = 0;
    };
    if (lane == 0)
        for (int t = 0; t < look; ++t) issue_next();

    int cs = 0;
    uint32_t parity = 0;
    int64_t consumed = 0;
    bool stop = false, err = false, emit = false;
    int status = FCM_NOT_CONVERGED, iters = 0;
    RcAcc<C> a;

    for (int p = 0;; ++p) {
        a.reset();
        if (p == 0 && INIT == P_INITV) {
#pragma unroll
            for (int j = 0; j < C; ++j) a.bad |= !finite_f(v[j]);
        }
        // ---- the pass over this warp's tiles ----
        int64_t i0 = gw * (int64_t)WTILE;
        for (int k = 0; k < nk; ++k, i0 += tile_stride) {
            const bool ok = mbar_wait_bounded(&full[cs], parity, wait_limit);
            if (__any_sync(0xffffffffu, !ok)) {
                err = true;
                break;
            }
            const int cnt = (int)min((int64_t)WTILE, n - i0);
            const float* sb = ring + cs * Sh::STAGE_FLOATS;
            if (emit)
                rc_tile<C, MK, RC_EMIT>(sb, cnt, i0, lane, U, n, v, v2, vp, vp2, m, inv_m1, pol_u, a);
            else if (p == 0 && INIT == P_ACCUM0)
                rc_tile<C, MK, RC_ACCUM0>(sb, cnt, i0, lane, U, n, v, v2, vp, vp2, m, inv_m1, pol_u, a);
            else if (p == 0)
                rc_tile<C, MK, RC_INITV>(sb, cnt, i0, lane, U, n, v, v2, vp, vp2, m, inv_m1, pol_u, a);
            else if (p == 1 && INIT == P_ACCUM0)
                rc_tile<C, MK, RC_ITER_U0>(sb, cnt, i0, lane, U, n, v, v2, vp, vp2, m, inv_m1, pol_u, a);
            else
                rc_tile<C, MK, RC_ITER>(sb, cnt, i0, lane, U, n, v, v2, vp, vp2, m, inv_m1, pol_u, a);
            __syncwarp();
            ++consumed;
            if (lane == 0) issue_next();
            if (++cs == Sh::STAGES) {
                cs = 0;
                parity ^= 1u;
            }
        }
        if (emit) break;
        if (!(p == 0 && INIT == P_ACCUM0)) a.fold();

        // ---- block totals (FP32 over the 8 warps) -> partials[p & 1] ----
        {
            float vals[S];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                vals[j] = a.num[j];
                vals[C + j] = a.den[j];
            }
            vals[2 * C] = a.J;
            vals[2 * C + 1] = a.dmax;
            vals[2 * C + 2] = a.bad ? 1.0f : 0.0f;
            vals[2 * C + 3] = err ? 1.0f : 0.0f;
#pragma unroll
            for (int s = 0; s < S; ++s) vals[s] = (s <= 2 * C) ? warp_sum(vals[s]) : warp_max(vals[s]);
            if (lane == 0) {
#pragma unroll
                for (int s = 0; s < S; ++s) s_red[warp][s] = vals[s];
            }
        }
        __syncthreads();
        float* part = partials + (int64_t)(p & 1) * S * gridDim.x;
        if (threadIdx.x < S) {
            const int s = threadIdx.x;
            float t = s_red[0][s];
#pragma unroll
            for (int w = 1; w < NWARP; ++w) t = (s <= 2 * C) ? t + s_red[w][s] : fmaxf(t, s_red[w][s]);
            __stcg(part + (int64_t)s * gridDim.x + blockIdx.x, t);
        }
        __syncthreads();
        // ---- bounded grid barrier ----
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(gbar, 1u);
            const unsigned target = (unsigned)(p + 1) * gridDim.x + phantoms;
            uint32_t spins = 0;
            while (ld_acquire_u32(gbar) < target) {
                if (++spins > grid_spins) {
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
        // ---- cross-block sums and V^{p+1}, the same fixed order in every block ----
        grid_totals<S, 2 * C + 1, NWARP>(part, (int)gridDim.x, s_df, s_mx);
        __syncthreads();
        grid_centers<C>(s_df, s_vq, s_empty);
        __syncthreads();
        const float delta = s_mx[0];
        const bool bad = s_mx[1] != 0.0f, tmo = s_mx[2] != 0.0f;
        bool update = false;
        if (tmo) {
            status = FCM_ERR_TIMEOUT;
            iters = p;
            stop = true;
        } else if (p == 0) {
            if (bad) {
                status = FCM_ERR_BAD_INPUT;
                iters = 0;
                stop = true;
            } else {
                update = true;
            }
        } else {
            if (blockIdx.x == 0 && threadIdx.x == 0 && st->trace) {
                double* t = st->trace + (int64_t)(p - 1) * (2 + C);
                t[0] = delta;
                t[1] = df_to_double(s_df[2 * C]);
#pragma unroll
                for (int j = 0; j < C; ++j) t[2 + j] = df_to_double(v64[j]);
            }
            if (delta < eps) {
                status = FCM_OK;
                iters = p;
                stop = true;
                emit = true;
            } else if (p >= max_iter) {
                status = FCM_NOT_CONVERGED;
                iters = p;
                stop = true;
                emit = true;
            } else {
                update = true;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->delta = delta;
                st->J = df_to_double(s_df[2 * C]);
            }
        }
        if (update) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                vp[j] = v[j];
                vp2[j] = v2[j];
                if (s_empty[j]) {
                    // an empty cluster keeps its center (first pass: V^0, or 0 from a U^0)
                    flags |= FCM_FLAG_EMPTY_CLUSTER;
                    if (p == 0 && INIT == P_ACCUM0) {
                        v[j] = 0.0f;
                        v64[j] = DF{0.0f, 0.0f};
                    }
                } else {
                    v[j] = s_vq[j].hi;
                    v64[j] = s_vq[j];
                }
                v2[j] = pack2(v[j], v[j]);
            }
        }
        __syncthreads();  // s_df / s_vq are rewritten by the next pass
        if (stop && !emit) break;
    }

    // copies issued for passes that will not run: let them land
    if (lane == 0) {
        int ds = cs;
        uint32_t dp = parity;
        for (int64_t q = consumed; q < issued; ++q) {
            mbar_wait_bounded(&full[ds], dp, wait_limit);
            if (++ds == Sh::STAGES) {
                ds = 0;
                dp ^= 1u;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            st->V[j] = v[j];
            st->V64[j] = df_to_double(v64[j]);
        }
        st->status = status;
        st->iters = iters;
        st->k = iters;
        st->flags = flags;
        st->done = 1;
        st->Uprev = st->U;
    }
}

template <int C, int MK>
void fill_rc(RcTable& t) {
    t.run[C][MK][0] = k_fcm_run_rc<C, MK, P_ACCUM0>;
    t.run[C][MK][1] = k_fcm_run_rc<C, MK, P_INITV>;
    t.smem[C][0] = RcShape<C, P_ACCUM0>::SMEM_BYTES;
    t.smem[C][1] = RcShape<C, P_INITV>::SMEM_BYTES;
}

}  // namespace

#define FCM_CAT2(a, b) a##b
#define FCM_CAT(a, b) FCM_CAT2(a, b)
void FCM_CAT(register_rc_c, FCM_INST_C)(RcTable& t) {
    fill_rc<FCM_INST_C, M_TWO>(t);
    fill_rc<FCM_INST_C, M_THREE>(t);
    fill_rc<FCM_INST_C, M_ONE_HALF>(t);
    fill_rc<FCM_INST_C, M_GENERIC>(t);
}

}  // namespace fcm
