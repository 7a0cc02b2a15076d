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
//  * k_fcm_pass_tma (n % 4 == 0, 16-byte aligned rows): persistent warps
//    each stream 128-pixel tiles of x and of the C rows of U through a private
//    multi-stage shared-memory ring filled by 1-D TMA bulk copies that
//    complete on mbarriers, so the bytes in flight do not depend on register
//    occupancy and no warp waits for another; each lane reads 4 pixels from
//    shared memory and stores U^k with 128-bit stores. x carries an L2
//    evict-last hint (it is re-read every iteration and fits in L2), U an
//    evict-first hint.
//  * k_fcm_pass_ldg (any n): grid-stride loop with scalar loads.
//
// Reduction: warp shuffle -> shared memory -> one FP64 partial per block ->
// the last block to finish (ticket counter) sums the partials in FP64 in
// block order, forms V^{k+1}, decides convergence on the device (the paper
// does this on the host, Sec. 4.3) and sets the CUDA-graph WHILE condition.
// No block waits for another: the ticket only elects the finisher.
#include <climits>

#include "fcm_bounds.cuh"
#include "fcm_device.cuh"
#include "fcm_exchange.cuh"
#include "fcm_internal.h"
#include "fcm_tma.cuh"

#ifndef FCM_INST_C
#error "compile with -DFCM_INST_C=<cluster count>"
#endif

namespace fcm {
namespace {

// Every mbarrier wait is bounded by st->lim.tma_polls suspensions of about
// 1 ms (2048 by default, about 2 s); TMA tiles land in microseconds.

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

// Block reduction, per-block partials, last-block combine and loop control.
// Slots: num[C], den[C], J, max|dU|, bad-input flag, timeout flag.
//
// The finisher runs when the pass's memory traffic is over, so it is kept
// short: within a block the 8 warp totals are added in FP32 (8 terms); the
// block totals go to slot-major FP32 partials[slot * gridDim.x + block]; the
// last block to finish gives one slot to each warp, whose lanes add the block
// totals in FP64 in a fixed order (lane-strided, then a shuffle tree), so the
// cross-block sums of up to 10^7-pixel terms are FP64 and deterministic.
template <int C, int PASS>
__device__ __forceinline__ void finish_pass(RunState* st, double* partials_raw,
                                            cudaGraphConditionalHandle cond, int use_cond,
                                            const float (&num)[C], const float (&den)[C], float Jacc,
                                            float dmax, bool bad, bool tmo) {
    constexpr int S = 2 * C + 4;
    static_assert(S <= SLOTS_MAX, "partial slots");
    float* partials = reinterpret_cast<float*>(partials_raw);
    __shared__ float s_red[NWARP][S];
    __shared__ double s_tot[S];
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
    if (threadIdx.x < S) {
        const int s = threadIdx.x;
        float a = s_red[0][s];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) a = (s <= 2 * C) ? a + s_red[w][s] : fmaxf(a, s_red[w][s]);
        __stcg(partials + (int64_t)s * gridDim.x + blockIdx.x, a);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&st->ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;

    // ---- last block: one slot per warp, FP64 over the block totals ----
    __threadfence();
    for (int s = warp; s < S; s += NWARP) {
        const float* ps = partials + (int64_t)s * gridDim.x;
        double a = 0.0;
        if (s <= 2 * C) {
            for (int b = lane; b < (int)gridDim.x; b += 32) a += (double)__ldcg(ps + b);
            a = warp_sum(a);
        } else {
            for (int b = lane; b < (int)gridDim.x; b += 32) a = fmax(a, (double)__ldcg(ps + b));
            a = warp_max_d(a);
        }
        if (lane == 0) s_tot[s] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[S];
#pragma unroll
    for (int s = 0; s < S; ++s) tot[s] = s_tot[s];

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
// n % 4 == 0, 16-byte aligned rows: one TMA bulk-copy ring per warp.
// ---------------------------------------------------------------------------
constexpr int WTILE = WARP_TILE;       // 128 pixels per warp tile: 2 steps of 2 per lane

template <int PASS, int C>
struct TmaShape {
    static constexpr int ROWS = (PASS == P_INITV) ? 1 : 1 + C;    // x, then U^{k-1} rows
    static constexpr int STAGE_FLOATS = ROWS * WTILE;              // one warp's stage
    // two blocks per SM with about 108 KB of ring each: deeper per-warp rings
    // stream HBM better here than a third block with shallower ones
    static constexpr int BLOCKS_PER_SM = 2;
    static constexpr int RAW = (108 * 1024) / (NWARP * STAGE_FLOATS * 4);
    static constexpr int STAGES = RAW < 2 ? 2 : (RAW > 8 ? 8 : RAW);
    static constexpr int SMEM_BYTES = NWARP * STAGES * STAGE_FLOATS * 4;
};

// Per-thread accumulators of one pass: packed pairs for the membership passes,
// scalars for the first pass from a given U^0.
template <int C>
struct Acc {
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
    // fold the packed halves into the scalar sums
    __device__ __forceinline__ void fold() {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            num[j] += lo2(num2[j]) + hi2(num2[j]);
            den[j] += lo2(den2[j]) + hi2(den2[j]);
        }
        J += lo2(J2) + hi2(J2);
    }
};

// One warp tile held in shared memory at sb (x, then the C rows of U^{k-1}
// unless PASS == P_INITV): lane l handles pixels 2l, 2l+1 and 64+2l, 65+2l.
// Writes U^k (not for P_ACCUM0) and accumulates the pass's sums.
template <int C, int MK, int PASS>
__device__ __forceinline__ void tile_work(const float* sb, int cnt, int64_t i0, int lane, float* U, int64_t n,
                                          const float (&v)[C], const f2 (&v2)[C], float m, float inv_m1,
                                          uint64_t pol_u, Acc<C>& a) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int pp = q * (WTILE / 2) + 2 * lane;
        if (pp >= cnt) continue;  // cnt is a multiple of 4: pp + 1 < cnt too
        const float2 xv = lds2(sb + pp);
        float2 uo[C];
        if (PASS != P_INITV) {
#pragma unroll
            for (int j = 0; j < C; ++j) uo[j] = lds2(sb + (1 + j) * WTILE + pp);
        }
        if (PASS == P_ACCUM0) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float uop[C], unp[C];
#pragma unroll
                for (int j = 0; j < C; ++j) uop[j] = p == 0 ? uo[j].x : uo[j].y;
                pixel_step<C, MK, PASS>(p == 0 ? xv.x : xv.y, v, m, inv_m1, uop, unp, a.num, a.den, a.J,
                                        a.dmax, a.bad);
            }
        } else {
            if (PASS == P_INITV) a.bad |= !finite_f(xv.x) || !finite_f(xv.y);
            const f2 xq = pack2(xv.x, xv.y);
            f2 u2[C], um2[C];
            a.J2 = add2(a.J2, membership_pair<C, MK>(xq, v2, m, inv_m1, v, u2, um2));
#pragma unroll
            for (int j = 0; j < C; ++j) {
                a.num2[j] = fma2(um2[j], xq, a.num2[j]);
                a.den2[j] = add2(a.den2[j], um2[j]);
                if (PASS == P_ITER) {
                    float da, db;
                    unpack2(sub2(u2[j], pack2(uo[j].x, uo[j].y)), da, db);
                    a.dmax = fmaxf(a.dmax, fmaxf(fabsf(da), fabsf(db)));
                }
                st_hint2(U + (int64_t)j * n + i0 + pp, u2[j], pol_u);
            }
        }
    }
}

// Every warp streams its own 128-pixel tiles (warp tile t = global warp id
// + k * number of warps) through a private ring of STAGES shared-memory
// stages: lane 0 issues the bulk copies of x and the C rows of U^{k-1} and
// arms the stage's mbarrier with the byte count; all lanes wait on it, each
// lane processes 4 pixels, and after __syncwarp lane 0 refills the stage with
// the warp's tile k + STAGES. Warps never wait for one another.
template <int C, int MK, int PASS>
__global__ void __launch_bounds__(NT, 2) k_fcm_pass_tma(RunState* __restrict__ st, double* __restrict__ partials,
                                                         cudaGraphConditionalHandle cond, int use_cond) {
    using Sh = TmaShape<PASS, C>;
    extern __shared__ __align__(128) float ring_all[];
    __shared__ __align__(8) uint64_t full_all[NWARP][Sh::STAGES];
    if (!pass_prologue(st, PASS, cond, use_cond)) return;

    const float* __restrict__ x = st->x;
    const float* Uold = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1;
    float v[C];
    f2 v2[C];
    Acc<C> a;
    a.reset();
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = (PASS == P_INITV) ? st->V0[j] : st->V[j];
        v2[j] = pack2(v[j], v[j]);
        if (PASS == P_INITV) a.bad |= !finite_f(v[j]);
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* ring = ring_all + warp * (Sh::STAGES * Sh::STAGE_FLOATS);
    uint64_t* full = full_all[warp];
    const int64_t nwarps = (int64_t)gridDim.x * NWARP;
    const int64_t gw = (int64_t)blockIdx.x * NWARP + warp;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    const int64_t nk = ntiles > gw ? (ntiles - 1 - gw) / nwarps + 1 : 0;
    const uint64_t pol_x = policy_evict_last();
    const uint64_t pol_u = policy_evict_first();

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < Sh::STAGES; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncwarp();

    // Lane 0 only: start the copies of this warp's k-th tile into stage s.
    auto issue = [&](int64_t k, int s) {
        const int64_t i0 = (gw + k * nwarps) * (int64_t)WTILE;
        const uint32_t bytes = (uint32_t)min((int64_t)WTILE, n - i0) * 4u;  // multiple of 16
        float* dst = ring + s * Sh::STAGE_FLOATS;
        if (!in_bounds(i0 >= 0 && i0 < n && i0 % 4 == 0 && s < Sh::STAGES, &st->bounds)) {
            mbar_expect_tx(&full[s], 0u);  // arrive without copies: the consumer skips the tile
            return;
        }
        mbar_expect_tx(&full[s], bytes * Sh::ROWS);
        bulk_g2s(dst, x + i0, bytes, &full[s], pol_x);
        if (PASS != P_INITV) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                bulk_g2s(dst + (1 + j) * WTILE, Uold + (int64_t)j * n + i0, bytes, &full[s], pol_u);
        }
    };
    if (lane == 0)
        for (int s = 0; s < Sh::STAGES && s < nk; ++s) issue(s, s);

    bool tmo = false;
    int s = 0;
    uint32_t parity = 0;
    const uint32_t wait_limit = st->lim.tma_polls;
    int64_t i0 = gw * (int64_t)WTILE;
    const int64_t tile_stride = nwarps * (int64_t)WTILE;
    for (int64_t k = 0; k < nk; ++k, i0 += tile_stride) {
        const bool ok = mbar_wait_bounded(&full[s], parity, wait_limit);
        if (__any_sync(0xffffffffu, !ok)) {
            tmo = true;
            if (lane == 0) {
                // let the copies still in flight land before the warp leaves
                const int64_t last = min(nk, k + (int64_t)Sh::STAGES);
                for (int64_t kk = k; kk < last; ++kk)
                    mbar_wait_bounded(&full[kk % Sh::STAGES], (uint32_t)((kk / Sh::STAGES) & 1), wait_limit);
            }
            break;
        }
        const int cnt = (int)min((int64_t)WTILE, n - i0);
        tile_work<C, MK, PASS>(ring + s * Sh::STAGE_FLOATS, cnt, i0, lane, U, n, v, v2, m, inv_m1, pol_u, a);
        __syncwarp();  // every lane is done reading stage s
        if (lane == 0 && k + Sh::STAGES < nk) issue(k + Sh::STAGES, s);
        if (++s == Sh::STAGES) {
            s = 0;
            parity ^= 1u;
        }
    }
    if (PASS != P_ACCUM0) a.fold();
    finish_pass<C, PASS>(st, partials, cond, use_cond, a.num, a.den, a.J, a.dmax, a.bad, tmo);
}

// ---------------------------------------------------------------------------
// The whole run in one cooperative launch (n % 4 == 0, aligned rows).
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The grid barrier polls at most st->lim.grid_spins times, 128 ns apart
// (2^23, about 1 s, by default), and waits for st->lim.phantoms arrivals
// beyond the grid's own (0 unless a test injects a barrier that never fills).

// Tiles are dealt in two parts. Every warp keeps the same fixed share of tiles
// in every pass (tile gw + k * nwarps, k < ks), so the U tile it reads from
// that share in pass p + 1 is one it wrote itself in pass p. Its ring
// therefore streams one sequence of loads across passes (a proxy fence orders
// the warp's stores before its own TMA re-read) and keeps DRAM busy while the
// grid exchanges the 2C + 4 sums of a pass. The rest of each pass is taken in
// chunks of DCHUNK consecutive tiles from a per-pass counter, so warps on SMs
// that stream faster take more of it and the warps finish a pass together
// (with fixed shares alone, the slowest SMs took about 1.5x as long as the
// fastest). A warp reaches the shared part of pass p only after its fixed
// share of pass p, which it starts after the grid barrier of pass p - 1, so
// every tile it takes was written before that barrier. The counter grab is
// issued one chunk ahead, so its latency hides behind the chunk's copies. After each pass every block
// publishes its FP32 totals, waits at a bounded grid barrier (co-residency is
// guaranteed by the cooperative launch), and computes the cross-block sums in
// the same fixed order as every other block, so all blocks derive the same
// V^{k+1} and the same stop decision. Pass 0 is INIT (V^1 from U^0, or U^0
// from V^0); pass p >= 1 is iteration p of Algorithm 1.
template <int C, int MK, int INIT>
__global__ void __launch_bounds__(NT, 2) k_fcm_run_tma(RunState* __restrict__ st,
                                                                      double* __restrict__ partials_raw) {
    using Sh = TmaShape<P_ITER, C>;
    constexpr int S = 2 * C + 4;
    extern __shared__ __align__(128) float ring_all[];
    __shared__ __align__(8) uint64_t full_all[NWARP][Sh::STAGES];
    __shared__ float s_red[NWARP][S];
    __shared__ DF s_df[2 * C + 1];
    __shared__ float s_mx[3];
    __shared__ DF s_vq[C];
    __shared__ int s_empty[C];
    __shared__ int s_err;
    // what each ring stage holds: tile and pass (pass INT_MAX: nothing)
    __shared__ int64_t s_tile[NWARP][Sh::STAGES];
    __shared__ int s_pass[NWARP][Sh::STAGES];
    __shared__ IssueState s_iss[NWARP];

    const float* __restrict__ x = st->x;
    const float* U0 = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1, eps = st->eps;
    const int max_iter = st->max_iter;
    unsigned* gbar = &st->ticket;
    float* partials = reinterpret_cast<float*>(partials_raw);

    float v[C];
    f2 v2[C];
    DF v64[C];  // the double-float quotients behind v, converted to FP64 only when written
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = st->V0[j];
        v2[j] = pack2(v[j], v[j]);
        v64[j] = DF{v[j], 0.0f};
    }
    int flags = 0;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* ring = ring_all + warp * (Sh::STAGES * Sh::STAGE_FLOATS);
    uint64_t* full = full_all[warp];
    const int64_t nwarps = (int64_t)gridDim.x * NWARP;
    const int64_t gw = (int64_t)blockIdx.x * NWARP + warp;
    const int64_t ntiles = (n + WTILE - 1) / WTILE;
    // fixed share: ks tiles per warp, when every warp has more than a ring of
    // them; otherwise every tile is dealt in fixed shares (nk per warp)
    const int64_t ks = ntiles * (int64_t)st->static_pct / 100 / nwarps;
    const bool shared_part = st->static_pct < 100 && ks > Sh::STAGES;
    const int nk = shared_part ? (int)ks : (int)(ntiles > gw ? (ntiles - 1 - gw) / nwarps + 1 : 0);
    const int64_t n_fixed = shared_part ? ks * nwarps : ntiles;
    const int64_t n_chunks = (ntiles - n_fixed + DCHUNK - 1) / DCHUNK;
    const int look = nk < Sh::STAGES ? nk : Sh::STAGES;
    const int npass = 1 + max_iter;  // passes the run can take
    const uint32_t wait_limit = st->lim.tma_polls, grid_spins = st->lim.grid_spins;
    const unsigned phantoms = st->lim.phantoms;
    const uint64_t pol_x = policy_evict_last();
    const uint64_t pol_u = policy_evict_first();

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < Sh::STAGES; ++s) {
            mbar_init(&full[s], 1);
            s_pass[warp][s] = INT_MAX;
        }
        mbar_fence_init();
    }
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();

    // Issue side (lane 0), kept in shared memory so that it takes no
    // registers during the tile work: pass ip, index ik in the fixed share,
    // the chunk being issued (next tile cb, cl tiles left), the grab for the
    // next chunk, ring slot is, and the copies issued so far.
    IssueState& q = s_iss[warp];
    if (lane == 0) q = IssueState{0, 0, 0, 0, 0, 0, 0u};
    auto issue_tile = [&](int64_t tile, int ip) {
        const int64_t i0 = tile * WTILE;
        const uint32_t bytes = (uint32_t)min((int64_t)WTILE, n - i0) * 4u;  // multiple of 16
        const bool with_u = !(ip == 0 && INIT == P_INITV);
        const float* Usrc = (ip == 0 || (ip == 1 && INIT == P_ACCUM0)) ? U0 : U;
        const int is = q.is;
        float* dst = ring + is * Sh::STAGE_FLOATS;
        s_pass[warp][is] = ip;
        if (!in_bounds(tile >= 0 && tile < ntiles && is < Sh::STAGES, &st->bounds)) {
            s_tile[warp][is] = -1;  // the consumer skips it
            mbar_expect_tx(&full[is], 0u);  // arrive without copies
            ++q.issued;
            q.is = is + 1 == Sh::STAGES ? 0 : is + 1;
            return;
        }
        s_tile[warp][is] = tile;
        mbar_expect_tx(&full[is], bytes * (with_u ? 1 + C : 1));
        bulk_g2s(dst, x + i0, bytes, &full[is], pol_x);
        if (with_u) {
#pragma unroll
            for (int j = 0; j < C; ++j)
                bulk_g2s(dst + (1 + j) * WTILE, Usrc + (int64_t)j * n + i0, bytes, &full[is], pol_u);
        }
        ++q.issued;
        q.is = is + 1 == Sh::STAGES ? 0 : is + 1;
    };
    auto issue_next = [&]() {
        while (q.ip < npass && nk > 0) {
            const int ip = q.ip;
            if (q.ik < nk) {
                const int64_t tile = gw + (int64_t)q.ik * nwarps;
                if (++q.ik == nk && shared_part) q.grab = atomicAdd(&st->dyn[ip & 1], 1u);  // first chunk, ahead
                issue_tile(tile, ip);
                return;
            }
            if (q.cl == 0) {
                if (shared_part && (int64_t)q.grab < n_chunks) {
                    q.cb = n_fixed + (int64_t)q.grab * DCHUNK;
                    q.cl = (int)min((int64_t)DCHUNK, ntiles - q.cb);
                    q.grab = atomicAdd(&st->dyn[ip & 1], 1u);  // the chunk after this one, ahead
                } else {
                    ++q.ip;  // pass ip is dealt out: on to the next pass's fixed share
                    q.ik = 0;
                    continue;
                }
            }
            --q.cl;
            issue_tile(q.cb++, ip);
            return;
        }
        s_pass[warp][q.is] = INT_MAX;  // nothing more to load
    };
    if (lane == 0)
        for (int t = 0; t < look; ++t) issue_next();
    __syncwarp();

    int cs = 0;  // consume side: ring slot and phase parity
    uint32_t parity = 0;
    int64_t consumed = 0;
    bool stop = false, err = false;
    int status = FCM_NOT_CONVERGED, iters = 0;
    Acc<C> a;

    for (int p = 0; !stop; ++p) {
        a.reset();
        if (p == 0 && INIT == P_INITV) {
#pragma unroll
            for (int j = 0; j < C; ++j) a.bad |= !finite_f(v[j]);
        }
        // ---- the pass over this warp's tiles: the ring's items of pass p ----
        while (s_pass[warp][cs] == p) {
            const bool ok = mbar_wait_bounded(&full[cs], parity, wait_limit);
            if (__any_sync(0xffffffffu, !ok)) {
                err = true;
                break;
            }
            const int64_t tile = s_tile[warp][cs];
            const int64_t i0 = tile * WTILE;
            const int cnt = (int)min((int64_t)WTILE, n - i0);
            const float* sb = ring + cs * Sh::STAGE_FLOATS;
            if (kBoundsChecks && tile < 0) {
                // a copy the guards skipped: nothing to compute or store
            } else if (p == 0) {
                tile_work<C, MK, INIT>(sb, cnt, i0, lane, U, n, v, v2, m, inv_m1, pol_u, a);
            } else {
                tile_work<C, MK, P_ITER>(sb, cnt, i0, lane, U, n, v, v2, m, inv_m1, pol_u, a);
            }
            // this lane's stores of U must precede any TMA re-read of the tile:
            // the warp's own (fixed share, next pass) or another warp's after
            // the grid barrier (shared part)
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncwarp();
            ++consumed;
            if (lane == 0) issue_next();
            __syncwarp();  // the stage records written by lane 0
            if (++cs == Sh::STAGES) {
                cs = 0;
                parity ^= 1u;
            }
        }
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
        // the loads this warp issues from here on may read U tiles that other
        // warps wrote before the barrier
        if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        // every chunk of pass p was taken before this barrier; its counter
        // serves pass p + 2, whose first grab follows the next barrier
        if (blockIdx.x == 0 && threadIdx.x == 0) st->dyn[p & 1] = 0u;
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
            } else if (p >= max_iter) {
                status = FCM_NOT_CONVERGED;
                iters = p;
                stop = true;
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
    }

    // copies issued for passes that will not run: let them land
    if (lane == 0) {
        int ds = cs;
        uint32_t dp = parity;
        for (int64_t t = consumed; t < q.issued; ++t) {
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
    t.run[C][MK][0] = k_fcm_run_tma<C, MK, P_ACCUM0>;
    t.run[C][MK][1] = k_fcm_run_tma<C, MK, P_INITV>;
    t.run_smem[C] = TmaShape<P_ITER, C>::SMEM_BYTES;
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
