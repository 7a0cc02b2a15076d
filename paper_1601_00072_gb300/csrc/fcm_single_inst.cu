// The fused single-image FCM pass, instantiated for one cluster count.
//
// Compiled once per C in 1..8 with -DFCM_INST_C=<C>, so the eight kernel
// families build in parallel.
//
// One launch of a P_ITER pass is one iteration of Algorithm 1
// (arXiv:1601.00072, Sec. 2.1): every pixel's memberships U^k are computed
// from the centers V^k held in registers (Eq. 4) and written in place over
// U^{k-1} (cluster-major rows, the paper's 1-D layout of Sec. 5.1), while
// FP32 accumulators collect the center numerators sum u^m x and denominators
// sum u^m (Eq. 3), the objective sum u^m d^2 (Eq. 1) and the largest change
// |u^k - u^{k-1}| (the stopping quantity of Algorithm 1 step 3). The paper's
// four center kernels per cluster (Sec. 4.2) and one membership kernel per
// cluster (Sec. 4.3) become this single pass.
//
// Two kernels move the pixels:
//  * k_fcm_pass_tma (n % 4 == 0, 16-byte aligned rows): a persistent block
//    walks 1024-pixel tiles; thread 0 streams each tile's x and U rows into a
//    multi-stage shared-memory ring with 1-D TMA bulk copies completing on
//    mbarriers, so the bytes in flight do not depend on register occupancy;
//    the threads read 4 pixels each from shared memory and store U^k with
//    128-bit stores. x carries an L2 evict-last hint (it is re-read every
//    iteration and fits in L2), U an evict-first hint.
//  * k_fcm_pass_ldg (any n): grid-stride loop with scalar loads.
//
// Reduction: warp shuffle -> shared memory -> one FP64 partial per block ->
// the last block to finish (ticket counter) sums the partials in FP64 in
// block order, forms V^{k+1}, decides convergence on the device (the paper
// does this on the host, Sec. 4.3) and sets the CUDA-graph WHILE condition.
// No block waits for another: the ticket only elects the finisher.
#include "fcm_device.cuh"
#include "fcm_internal.h"
#include "fcm_tma.cuh"

#ifndef FCM_INST_C
#error "compile with -DFCM_INST_C=<cluster count>"
#endif

namespace fcm {
namespace {

// Bound of every mbarrier wait (polls); TMA tiles land in microseconds.
constexpr uint32_t WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int C, int MK, int PASS>
__device__ __forceinline__ void pixel_step(float xp, const float (&v)[C], float m, float inv_m1,
                                           const float* uo, float* un, float (&num)[C],
                                           float (&den)[C], float& Jacc, float& dmax, bool& bad) {
    if (PASS == P_ACCUM0) {
        bad |= !finite_f(xp);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float u0 = uo[j];
            bad |= !(u0 >= 0.0f) || !finite_f(u0);
            const float w = pow_m<MK>(u0, m);
            num[j] = fmaf(w, xp, num[j]);
            den[j] += w;
        }
    } else {
        if (PASS == P_INITV) bad |= !finite_f(xp);
        float u[C], um[C];
        Jacc += membership<C, MK>(xp, v, m, inv_m1, u, um);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            num[j] = fmaf(um[j], xp, num[j]);
            den[j] += um[j];
            un[j] = u[j];
            if (PASS == P_ITER) dmax = fmaxf(dmax, fabsf(u[j] - uo[j]));
        }
    }
}

// Start of every pass: loop guard and the host-loop "finished" check.
// Returns false when the block has nothing to do.
__device__ __forceinline__ bool pass_prologue(RunState* st, int pass, cudaGraphConditionalHandle cond,
                                              int use_cond) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) {
        // Loop guard, independent of the last-block election: a run never
        // needs more than 1 + max_iter passes, so a graph that keeps going
        // past that is stopped with a timeout status instead of spinning.
        const int L = atomicAdd(&st->launches, 1);
        if (L > st->max_iter + 1) {
            st->status = FCM_ERR_TIMEOUT;
            st->done = 1;
            cudaGraphSetConditional(cond, 0);
        }
    }
    // Host-driven mode launches iterations ahead; a finished run makes them
    // no-ops (uniform across the grid: every block reads the same flag,
    // written by an earlier launch).
    if (pass == P_ITER && *reinterpret_cast<volatile int*>(&st->done)) return false;
    return true;
}

// Block reduction, FP64 partial, last-block combine and loop control.
// Slots: num[C], den[C], J, max|dU|, bad-input flag, timeout flag.
template <int C, int PASS>
__device__ __forceinline__ void finish_pass(RunState* st, double* partials,
                                            cudaGraphConditionalHandle cond, int use_cond,
                                            const float (&num)[C], const float (&den)[C], float Jacc,
                                            float dmax, bool bad, bool tmo) {
    constexpr int S = 2 * C + 4;
    static_assert(S <= SLOTS_MAX, "partial slots");
    __shared__ float s_red[NWARP][S];
    __shared__ double s_red64[NWARP][S];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        float vals[S];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            vals[j] = num[j];
            vals[C + j] = den[j];
        }
        vals[2 * C] = Jacc;
        vals[2 * C + 1] = dmax;
        vals[2 * C + 2] = bad ? 1.0f : 0.0f;
        vals[2 * C + 3] = tmo ? 1.0f : 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s) vals[s] = (s <= 2 * C) ? warp_sum(vals[s]) : warp_max(vals[s]);
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) s_red[warp][s] = vals[s];
        }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            double a = lane < NWARP ? (double)s_red[lane][s] : 0.0;
            a = (s <= 2 * C) ? warp_sum(a) : warp_max_d(a);
            if (lane == 0) __stcg(partials + (int64_t)blockIdx.x * S + s, a);
        }
        if (lane == 0) {
            __threadfence();
            const unsigned t = atomicAdd(&st->ticket, 1u);
            s_last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!s_last) return;

    // ---- last block: FP64 combine of all partials in block order ----
    __threadfence();
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const double p = __ldcg(partials + (int64_t)b * S + s);
            acc[s] = (s <= 2 * C) ? acc[s] + p : fmax(acc[s], p);
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = (s <= 2 * C) ? warp_sum(acc[s]) : warp_max_d(acc[s]);
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) s_red64[warp][s] = acc[s];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double a = s_red64[0][s];
        for (int w = 1; w < NWARP; ++w) a = (s <= 2 * C) ? a + s_red64[w][s] : fmax(a, s_red64[w][s]);
        tot[s] = a;
    }

    int cont = 1;
    if (tot[2 * C + 3] != 0.0) {
        st->status = FCM_ERR_TIMEOUT;
        st->done = 1;
        st->iters = st->k;
        cont = 0;
    } else if (PASS == P_ACCUM0 || PASS == P_INITV) {
        if (tot[2 * C + 2] != 0.0) {
            st->status = FCM_ERR_BAD_INPUT;
            st->done = 1;
            st->iters = 0;
            cont = 0;
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                double vj;
                if (tot[C + j] > 0.0) {
                    vj = tot[j] / tot[C + j];
                } else {
                    vj = (PASS == P_INITV) ? (double)st->V0[j] : 0.0;
                    st->flags |= FCM_FLAG_EMPTY_CLUSTER;
                }
                st->V64[j] = vj;
                st->V[j] = (float)vj;
            }
            st->k = 1;
            if (PASS == P_INITV) st->Uprev = st->U;  // U^0 now lives in U
        }
    } else {
        st->Uprev = st->U;  // from now on U^{k-1} is read where U^k was written
        const int k = st->k;
        const float delta = (float)tot[2 * C + 1];
        const double J = tot[2 * C];
        st->delta = delta;
        st->J = J;
        if (st->trace) {
            double* t = st->trace + (int64_t)(k - 1) * (2 + C);
            t[0] = delta;
            t[1] = J;
#pragma unroll
            for (int j = 0; j < C; ++j) t[2 + j] = st->V64[j];
        }
        if (delta < st->eps) {
            st->status = FCM_OK;
            st->iters = k;
            st->done = 1;
            cont = 0;
        } else if (k >= st->max_iter) {
            st->status = FCM_NOT_CONVERGED;
            st->iters = k;
            st->done = 1;
            cont = 0;
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (tot[C + j] > 0.0) {
                    const double vj = tot[j] / tot[C + j];
                    st->V64[j] = vj;
                    st->V[j] = (float)vj;
                } else {
                    st->flags |= FCM_FLAG_EMPTY_CLUSTER;  // keep v_j
                }
            }
            st->k = k + 1;
        }
    }
    st->ticket = 0;
    if (use_cond) cudaGraphSetConditional(cond, cont);
}

template <int C>
struct PassVars {
    float v[C];
    float num[C], den[C];
    float Jacc = 0.0f, dmax = 0.0f;
    bool bad = false;
};

template <int C, int PASS>
__device__ __forceinline__ void load_centers(const RunState* st, PassVars<C>& pv) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
        pv.v[j] = (PASS == P_INITV) ? st->V0[j] : st->V[j];
        pv.num[j] = pv.den[j] = 0.0f;
        if (PASS == P_INITV) pv.bad |= !finite_f(pv.v[j]);
    }
}

// ---------------------------------------------------------------------------
// Any n: grid-stride loop, scalar loads.
// ---------------------------------------------------------------------------
template <int C, int MK, int PASS>
__global__ void __launch_bounds__(NT) k_fcm_pass_ldg(RunState* __restrict__ st, double* __restrict__ partials,
                                                      cudaGraphConditionalHandle cond, int use_cond) {
    if (!pass_prologue(st, PASS, cond, use_cond)) return;
    const float* __restrict__ x = st->x;
    // U^{k-1} and U^k may be the same buffer (the in-place update): no
    // __restrict__ on them. Each element is read and then written by the
    // same thread only.
    const float* Uold = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1;
    PassVars<C> pv;
    load_centers<C, PASS>(st, pv);
    const int64_t gstride = (int64_t)gridDim.x * NT;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += gstride) {
        float uop[C], unp[C];
        const float xp = __ldg(x + i);
#pragma unroll
        for (int j = 0; j < C; ++j) uop[j] = (PASS != P_INITV) ? __ldcs(Uold + (int64_t)j * n + i) : 0.0f;
        pixel_step<C, MK, PASS>(xp, pv.v, m, inv_m1, uop, unp, pv.num, pv.den, pv.Jacc, pv.dmax, pv.bad);
        if (PASS != P_ACCUM0) {
#pragma unroll
            for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + i, unp[j]);
        }
    }
    finish_pass<C, PASS>(st, partials, cond, use_cond, pv.num, pv.den, pv.Jacc, pv.dmax, pv.bad, false);
}

// ---------------------------------------------------------------------------
// n % 4 == 0, 16-byte aligned rows: TMA bulk-copy ring.
// ---------------------------------------------------------------------------
constexpr int TPX = 4;                 // pixels per thread per tile
constexpr int TILE = NT * TPX;         // 1024 pixels

template <int PASS, int C>
struct TmaShape {
    static constexpr int ROWS = (PASS == P_INITV) ? 1 : 1 + C;   // x, then U^{k-1} rows
    static constexpr int STAGE_FLOATS = ROWS * TILE;
    static constexpr int RAW = (100 * 1024) / (STAGE_FLOATS * 4);
    static constexpr int STAGES = RAW < 2 ? 2 : (RAW > 6 ? 6 : RAW);
    static constexpr int SMEM_BYTES = STAGES * STAGE_FLOATS * 4;
};

template <int C, int MK, int PASS>
__global__ void __launch_bounds__(NT, 2) k_fcm_pass_tma(RunState* __restrict__ st, double* __restrict__ partials,
                                                         cudaGraphConditionalHandle cond, int use_cond) {
    using Sh = TmaShape<PASS, C>;
    extern __shared__ __align__(128) float ring[];
    __shared__ __align__(8) uint64_t full[Sh::STAGES];
    if (!pass_prologue(st, PASS, cond, use_cond)) return;

    const float* __restrict__ x = st->x;
    const float* Uold = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1;
    PassVars<C> pv;
    load_centers<C, PASS>(st, pv);

    const int64_t ntiles = (n + TILE - 1) / TILE;
    const int64_t nk = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t pol_x = policy_evict_last();
    const uint64_t pol_u = policy_evict_first();

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < Sh::STAGES; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // Thread 0 only: start the copies of this block's k-th tile into stage s.
    auto issue = [&](int64_t k, int s) {
        const int64_t i0 = (blockIdx.x + k * gridDim.x) * (int64_t)TILE;
        const uint32_t bytes = (uint32_t)min((int64_t)TILE, n - i0) * 4u;  // multiple of 16
        float* dst = ring + s * Sh::STAGE_FLOATS;
        mbar_expect_tx(&full[s], bytes * Sh::ROWS);
        bulk_g2s(dst, x + i0, bytes, &full[s], pol_x);
        if (PASS != P_INITV) {
#pragma unroll
            for (int j = 0; j < C; ++j) bulk_g2s(dst + (1 + j) * TILE, Uold + (int64_t)j * n + i0, bytes, &full[s], pol_u);
        }
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < Sh::STAGES && s < nk; ++s) issue(s, s);

    bool tmo = false;
    const int p0 = threadIdx.x * TPX;
    for (int64_t k = 0; k < nk; ++k) {
        const int s = (int)(k % Sh::STAGES);
        const uint32_t parity = (uint32_t)((k / Sh::STAGES) & 1);
        const bool ok = mbar_wait_bounded(&full[s], parity, WAIT_LIMIT);
        const int64_t i0 = (blockIdx.x + k * gridDim.x) * (int64_t)TILE;
        const int64_t cnt = min((int64_t)TILE, n - i0);
        if (ok && p0 < cnt) {
            const float* sb = ring + s * Sh::STAGE_FLOATS;
            const float4 xv = lds4(sb + p0);
            float4 uo[C], un[C];
            if (PASS != P_INITV) {
#pragma unroll
                for (int j = 0; j < C; ++j) uo[j] = lds4(sb + (1 + j) * TILE + p0);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float uop[C], unp[C];
#pragma unroll
                for (int j = 0; j < C; ++j) uop[j] = (PASS != P_INITV) ? comp(uo[j], p) : 0.0f;
                pixel_step<C, MK, PASS>(comp(xv, p), pv.v, m, inv_m1, uop, unp, pv.num, pv.den, pv.Jacc,
                                        pv.dmax, pv.bad);
#pragma unroll
                for (int j = 0; j < C; ++j) set_comp(un[j], p, unp[j]);
            }
            if (PASS != P_ACCUM0) {
#pragma unroll
                for (int j = 0; j < C; ++j) st_hint4(U + (int64_t)j * n + i0 + p0, un[j], pol_u);
            }
        }
        // every thread is done with stage s (and agrees on any timeout)
        if (__syncthreads_or(!ok)) {
            tmo = true;
            if (threadIdx.x == 0) {
                // let the copies still in flight land before the block exits
                const int64_t last = min(nk, k + (int64_t)Sh::STAGES);
                for (int64_t kk = k; kk < last; ++kk)
                    mbar_wait_bounded(&full[kk % Sh::STAGES], (uint32_t)((kk / Sh::STAGES) & 1), WAIT_LIMIT);
            }
            break;
        }
        if (threadIdx.x == 0 && k + Sh::STAGES < nk) issue(k + Sh::STAGES, s);
    }
    finish_pass<C, PASS>(st, partials, cond, use_cond, pv.num, pv.den, pv.Jacc, pv.dmax, pv.bad, tmo);
}

template <int C, int MK, int PASS>
void fill_pass(SingleTable& t) {
    t.k[C][MK][PASS][0] = k_fcm_pass_ldg<C, MK, PASS>;
    t.k[C][MK][PASS][1] = k_fcm_pass_tma<C, MK, PASS>;
    t.smem[C][MK][PASS][0] = 0;
    t.smem[C][MK][PASS][1] = TmaShape<PASS, C>::SMEM_BYTES;
}

template <int C, int MK>
void fill_mk(SingleTable& t) {
    fill_pass<C, MK, P_ACCUM0>(t);
    fill_pass<C, MK, P_INITV>(t);
    fill_pass<C, MK, P_ITER>(t);
}

}  // namespace

#define FCM_CAT2(a, b) a##b
#define FCM_CAT(a, b) FCM_CAT2(a, b)
void FCM_CAT(register_single_c, FCM_INST_C)(SingleTable& t) {
    fill_mk<FCM_INST_C, M_TWO>(t);
    fill_mk<FCM_INST_C, M_THREE>(t);
    fill_mk<FCM_INST_C, M_ONE_HALF>(t);
    fill_mk<FCM_INST_C, M_GENERIC>(t);
}

}  // namespace fcm
