// The fused single-image FCM pass, instantiated for one cluster count.
//
// Compiled once per C in 1..8 with -DFCM_INST_C=<C>, so the eight kernel
// families build in parallel.
//
// One launch of k_fcm_pass<P_ITER> is one iteration of Algorithm 1
// (arXiv:1601.00072, Sec. 2.1): every thread walks the pixels grid-stride,
// four at a time with 128-bit loads (x, then U^{k-1} row by row, cluster-major
// as in the paper's Sec. 5.1 layout), computes U^k from the centers V^k held
// in registers (Eq. 4), writes U^k in place, and accumulates in FP32 the
// center numerators sum u^m x and denominators sum u^m (Eq. 3), the objective
// term sum u^m d^2 (Eq. 1) and the largest change |u^k - u^{k-1}| (the
// stopping quantity of Algorithm 1 step 3). The paper's four center kernels
// per cluster (Sec. 4.2) and membership kernel per cluster (Sec. 4.3) become
// this one pass.
//
// Reduction: warp shuffle -> shared memory -> one FP64 partial per block ->
// the last block to finish (ticket counter) sums the partials in FP64 in
// block order, forms V^{k+1}, decides convergence on the device (the paper
// does this on the host, Sec. 4.3) and sets the CUDA-graph WHILE condition.
// No block waits for another: the ticket only elects the finisher.
#include "fcm_device.cuh"
#include "fcm_internal.h"

#ifndef FCM_INST_C
#error "compile with -DFCM_INST_C=<cluster count>"
#endif

namespace fcm {
namespace {

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

template <int C, int MK, int PASS, int VEC>
__global__ void __launch_bounds__(NT) k_fcm_pass(RunState* __restrict__ st,
                                                  double* __restrict__ partials,
                                                  cudaGraphConditionalHandle cond, int use_cond) {
    constexpr int S = 2 * C + 2;
    if (PASS == P_ITER) {
        // Host-driven mode launches iterations ahead; a finished run makes
        // them no-ops (uniform across the grid: every block reads the same
        // flag, written by an earlier launch).
        if (*reinterpret_cast<volatile int*>(&st->done)) return;
    }
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
    const float* __restrict__ x = st->x;
    // U^{k-1} and U^k may be the same buffer (the in-place update): no
    // __restrict__ on them. Each element is read and then written by the
    // same thread only.
    const float* Uold = st->Uprev;
    float* U = st->U;
    const int64_t n = st->n;
    const float m = st->m, inv_m1 = st->inv_m1;
    float v[C];
#pragma unroll
    for (int j = 0; j < C; ++j) v[j] = (PASS == P_INITV) ? st->V0[j] : st->V[j];

    float num[C], den[C];
#pragma unroll
    for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
    float Jacc = 0.0f, dmax = 0.0f;
    bool bad = false;
    if (PASS == P_INITV) {
#pragma unroll
        for (int j = 0; j < C; ++j) bad |= !finite_f(v[j]);
    }

    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * NT;
    if (VEC == 4) {
        const int64_t nq = n >> 2;  // n % 4 == 0 and 16-byte aligned rows
        for (int64_t q = gtid; q < nq; q += gstride) {
            const int64_t i0 = q << 2;
            const float4 xv = ld_x4(x + i0);
            float4 uo[C], un[C];
            if (PASS != P_INITV) {
#pragma unroll
                for (int j = 0; j < C; ++j) uo[j] = ld_u4(Uold + (int64_t)j * n + i0);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                float uop[C], unp[C];
#pragma unroll
                for (int j = 0; j < C; ++j) uop[j] = (PASS != P_INITV) ? comp(uo[j], p) : 0.0f;
                pixel_step<C, MK, PASS>(comp(xv, p), v, m, inv_m1, uop, unp, num, den, Jacc, dmax, bad);
#pragma unroll
                for (int j = 0; j < C; ++j) set_comp(un[j], p, unp[j]);
            }
            if (PASS != P_ACCUM0) {
#pragma unroll
                for (int j = 0; j < C; ++j) st_u4(U + (int64_t)j * n + i0, un[j]);
            }
        }
    } else {
        for (int64_t i = gtid; i < n; i += gstride) {
            float uop[C], unp[C];
            const float xp = __ldg(x + i);
#pragma unroll
            for (int j = 0; j < C; ++j) uop[j] = (PASS != P_INITV) ? __ldcs(Uold + (int64_t)j * n + i) : 0.0f;
            pixel_step<C, MK, PASS>(xp, v, m, inv_m1, uop, unp, num, den, Jacc, dmax, bad);
            if (PASS != P_ACCUM0) {
#pragma unroll
                for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + i, unp[j]);
            }
        }
    }

    // ---- block reduction: warp shuffle (FP32) -> shared -> FP64 partial ----
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
        vals[2 * C + 1] = (PASS == P_ITER) ? dmax : (bad ? 1.0f : 0.0f);
#pragma unroll
        for (int s = 0; s < S - 1; ++s) vals[s] = warp_sum(vals[s]);
        vals[S - 1] = warp_max(vals[S - 1]);
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
            a = (s == S - 1) ? warp_max_d(a) : warp_sum(a);
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
            acc[s] = (s == S - 1) ? fmax(acc[s], p) : acc[s] + p;
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = (s == S - 1) ? warp_max_d(acc[s]) : warp_sum(acc[s]);
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
        for (int w = 1; w < NWARP; ++w) a = (s == S - 1) ? fmax(a, s_red64[w][s]) : a + s_red64[w][s];
        tot[s] = a;
    }

    int cont = 1;
    if (PASS == P_ACCUM0 || PASS == P_INITV) {
        if (tot[S - 1] != 0.0) {
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
        const float delta = (float)tot[S - 1];
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

template <int C, int MK>
void fill_mk(SingleTable& t) {
    t.k[C][MK][P_ACCUM0][0] = k_fcm_pass<C, MK, P_ACCUM0, 1>;
    t.k[C][MK][P_ACCUM0][1] = k_fcm_pass<C, MK, P_ACCUM0, 4>;
    t.k[C][MK][P_INITV][0] = k_fcm_pass<C, MK, P_INITV, 1>;
    t.k[C][MK][P_INITV][1] = k_fcm_pass<C, MK, P_INITV, 4>;
    t.k[C][MK][P_ITER][0] = k_fcm_pass<C, MK, P_ITER, 1>;
    t.k[C][MK][P_ITER][1] = k_fcm_pass<C, MK, P_ITER, 4>;
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
