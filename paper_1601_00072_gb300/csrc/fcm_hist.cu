// Histogram-domain FCM for images of integer grey levels 0..255.
//
// When every intensity is one of 256 grey levels, the membership of a pixel
// under Eq. 4 depends only on its grey level, so after the first center
// update the whole of Algorithm 1 (Sec. 2.1) can run on the 256-bin
// histogram: the center sums of Eq. 3 and J of Eq. 1 become sums over bins
// weighted by their pixel counts, and the stopping quantity max |U^k - U^{k-1}|
// is a maximum over the bins that occur. This is the grey-level reduction the
// paper cites among related GPU work (brFCM, Sec. 3); the results equal the
// per-pixel run's up to the order of rounding.
//
// Per run: one pass over the pixels builds the histogram (and, from U^0, the
// sums of V^1); with U^0 given, a second pass takes the first stopping
// quantity against the pixels' U^0; one CTA then iterates on the bins; a last
// pass writes U^k by table lookup. HBM traffic is 4 + 4C bytes per pixel for
// each of the (up to) three passes instead of 4 + 8C per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "fcm.h"
#include "fcm_bounds.cuh"
#include "fcm_device.cuh"
#include "fcm_df.cuh"
#include "fcm_hist_bins.cuh"
#include "fcm_runtime.h"

namespace fcm {

struct alignas(16) HistState {
    unsigned long long hist[256];
    double V64[FCM_MAX_CLUSTERS];
    float V[FCM_MAX_CLUSTERS];
    float V0[FCM_MAX_CLUSTERS];
    double delta, J;
    unsigned d1bits;  // max |U^1 - U^0| over the pixels, as float bits (from U^0)
    int bad;
    int iters, status, flags;
    unsigned bounds;  // FCM_FLAG_BOUNDS from a FCM_DEBUG_BOUNDS build's guards
};

struct HistWorkspace {
    HistState* d_st = nullptr;
    HistState* h_st = nullptr;  // pinned
    double* part = nullptr;
    int part_blocks = 0;
    float* table = nullptr;  // [256][C] final memberships of each grey level
};

}  // namespace fcm

using namespace fcm;

namespace {

constexpr int HCHUNK = 4;  // pixels per thread whose loads are issued together in the first pass

// Pass over the pixels: histogram, input checks, and (from U^0) the
// numerators and denominators of V^1 (Eq. 3) as per-block FP64 slots. A
// negative U^0 entry is caught here; a NaN or infinite one makes the sums of
// V^1 non-finite, which the next kernel rejects (so does an entry whose u^m
// overflows FP32).
// Up to C = 4, four blocks per SM fit in 64 registers (a few bytes spill at
// C = 4): twice the warps of an unbounded build to cover the loads' latency.
template <int C, int MK, bool FROM_U>
__global__ void __launch_bounds__(HNT, C <= 4 ? 4 : 2) k_hist_pass0(const float* __restrict__ x, const float* __restrict__ U0,
                                                   int64_t n, float m, HistState* st, double* __restrict__ part) {
    __shared__ unsigned hs[HNT / 32][256];  // one sub-histogram per warp
    __shared__ float w[HNT / 32][4 * C];
    for (int t = threadIdx.x; t < (HNT / 32) * 256; t += HNT) (&hs[0][0])[t] = 0u;
    __syncthreads();
    DF acc[2 * C];
#pragma unroll
    for (int q = 0; q < 2 * C; ++q) acc[q] = DF{0.0f, 0.0f};
    bool bad = false;
    float umin = 0.0f;  // smallest U^0 entry seen (negative entries are bad input)
    const int64_t stride = (int64_t)gridDim.x * HNT;
    const int lane_id = threadIdx.x & 31;
    unsigned* hw = hs[threadIdx.x >> 5];
    // the loop bounds are the same for all lanes of a warp (its first lane's
    // index); lanes past n load nothing and count nothing
    for (int64_t i0 = (int64_t)blockIdx.x * HNT + threadIdx.x; i0 - lane_id < n; i0 += stride * HCHUNK) {
        // the chunk's loads are all issued before any is used
        float xc[HCHUNK], uc[HCHUNK][FROM_U ? C : 1];
#pragma unroll
        for (int q = 0; q < HCHUNK; ++q) {
            const int64_t i = i0 + (int64_t)q * stride;
            const bool in = i < n;
            xc[q] = in ? __ldg(x + i) : 0.0f;
            if (FROM_U) {
#pragma unroll
                for (int j = 0; j < C; ++j) uc[q][j] = in ? __ldg(U0 + (int64_t)j * n + i) : 0.0f;
            }
        }
        float num[C], den[C];
#pragma unroll
        for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
#pragma unroll
        for (int q = 0; q < HCHUNK; ++q) {
            const int64_t i = i0 + (int64_t)q * stride;
            if (i - lane_id >= n) break;  // warp-uniform
            const bool in = i < n;
            const float xi = xc[q];
            const int g = grey_index(xi);
            const bool good = in && g >= 0;
            bad |= in && !good;
            // shared-memory atomics: lanes of a warp on the same grey level are
            // serialised by the hardware; counts are exact in any order
            if (good) atomicAdd(&hw[g], 1u);
            if (FROM_U && good) {
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float u0 = uc[q][j];
                    umin = fminf(umin, u0);  // NaN and infinities show in the sums instead
                    const float wt = pow_m<MK>(u0, m);
                    num[j] = fmaf(wt, xi, num[j]);
                    den[j] += wt;
                }
            }
        }
        if (FROM_U) {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                df_add(acc[j], num[j]);
                df_add(acc[C + j], den[j]);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += HNT) {
        unsigned t = 0u;
        for (int v = 0; v < HNT / 32; ++v) t += hs[v][b];
        if (t) atomicAdd(&st->hist[b], (unsigned long long)t);
    }
    if (__syncthreads_or(bad || umin < 0.0f) && threadIdx.x == 0) atomicOr(&st->bad, 1);
    if (!FROM_U) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 2 * C; ++q) {
        const DF d = warp_sum_df(acc[q]);
        if (lane == 0) {
            w[warp][2 * q] = d.hi;
            w[warp][2 * q + 1] = d.lo;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * C) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int v = 0; v < HNT / 32; ++v) t += (double)w[v][2 * q] + (double)w[v][2 * q + 1];
        part[(int64_t)blockIdx.x * 2 * C + q] = t;
    }
}

// Block-wide FP64 sums of S values per thread and one float maximum, the same
// fixed order in every call; every thread receives the totals.
template <int S>
__device__ __forceinline__ void block_sums(double (&v)[S], float& mx, double (*red)[S + 1], double* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < S; ++q) v[q] = warp_sum(v[q]);
    mx = warp_max(mx);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < S; ++q) red[warp][q] = v[q];
        red[warp][S] = (double)mx;
    }
    __syncthreads();
    if (threadIdx.x <= S) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int u = 0; u < HNT / 32; ++u) t = q < S ? t + red[u][q] : fmax(t, red[u][q]);
        tot[q] = t;
    }
    __syncthreads();
}

// V^1: from the pass-0 slots (U^0 given), or from the bins with
// U^0 = f(grey level, V^0) (Eq. 4 then Eq. 3). One CTA.
template <int C, int MK, bool FROM_U>
__global__ void __launch_bounds__(HNT) k_hist_init(HistState* st, const double* __restrict__ part, int nblocks,
                                                  float m, float inv_m1) {
    __shared__ double red[HNT / 32][2 * C + 1];
    __shared__ double tot[2 * C + 1];
    bool bad = st->bad != 0;
    if (!FROM_U) {
#pragma unroll
        for (int j = 0; j < C; ++j) bad |= !finite_f(st->V0[j]);
    }
    if (bad) {
        if (threadIdx.x == 0) {
            st->bad = 1;
            st->status = FCM_ERR_BAD_INPUT;
            st->iters = 0;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                st->V[j] = st->V0[j];
                st->V64[j] = st->V0[j];
            }
        }
        return;
    }
    if (FROM_U) {
        // thread t adds slots t, t + HNT, ... of every sum; then one block sum
        double s[2 * C];
        float mx = 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * C; ++q) s[q] = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += HNT) {
#pragma unroll
            for (int q = 0; q < 2 * C; ++q) s[q] += part[(int64_t)b * 2 * C + q];
        }
        block_sums<2 * C>(s, mx, red, tot);
        bool finite = true;
#pragma unroll
        for (int q = 0; q < 2 * C; ++q) finite &= isfinite(tot[q]);
        if (!finite) {
            // a NaN or infinite U^0 entry (pass 0 checks only for negative ones)
            if (threadIdx.x == 0) {
                st->bad = 1;
                st->status = FCM_ERR_BAD_INPUT;
                st->iters = 0;
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    st->V[j] = st->V0[j];
                    st->V64[j] = st->V0[j];
                }
            }
            return;
        }
    } else {
        const int b = threadIdx.x;
        const double hb = (double)st->hist[b];
        float v0[C], u[C], um[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v0[j] = st->V0[j];
        membership<C, MK>((float)b, v0, m, inv_m1, u, um);
        double s[2 * C];
        float mx = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            s[j] = hb * (double)um[j] * (double)b;
            s[C + j] = hb * (double)um[j];
        }
        block_sums<2 * C>(s, mx, red, tot);
    }
    if (threadIdx.x == 0) {
        int flags = 0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const double den = tot[C + j];
            if (den > 0.0) {
                st->V64[j] = tot[j] / den;
                st->V[j] = (float)st->V64[j];
            } else {
                flags |= FCM_FLAG_EMPTY_CLUSTER;  // V^0 kept, or 0 from a U^0
                st->V[j] = FROM_U ? 0.0f : st->V0[j];
                st->V64[j] = st->V[j];
            }
        }
        st->flags = flags;
    }
}

// The first stopping quantity from U^0: max over pixels and clusters of
// |f(x_i, V^1)_j - U^0_ij|, with f tabulated per grey level.
template <int C, int MK>
__global__ void __launch_bounds__(HNT) k_hist_delta1(const float* __restrict__ x, const float* __restrict__ U0,
                                                    int64_t n, float m, float inv_m1, HistState* st) {
    __shared__ float T[256][C];
    __shared__ float wm[HNT / 32];
    if (st->bad) return;
    {
        float v[C], u[C], um[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = st->V[j];
        membership<C, MK>((float)threadIdx.x, v, m, inv_m1, u, um);
#pragma unroll
        for (int j = 0; j < C; ++j) T[threadIdx.x][j] = u[j];
    }
    __syncthreads();
    float d = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * HNT;
    for (int64_t i = (int64_t)blockIdx.x * HNT + threadIdx.x; i < n; i += stride) {
        const int b = (int)__ldg(x + i);
        if (!in_bounds(b >= 0 && b < 256, &st->bounds)) continue;
#pragma unroll
        for (int j = 0; j < C; ++j) d = fmaxf(d, fabsf(T[b][j] - __ldg(U0 + (int64_t)j * n + i)));
    }
    d = warp_max(d);
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int u = 0; u < HNT / 32; ++u) t = fmaxf(t, wm[u]);
        atomicMax(&st->d1bits, __float_as_uint(t));  // non-negative floats order as their bits
    }
}

// Algorithm 1 on the bins, one CTA (solve_bins: thread b holds grey level b).
template <int C, int MK, bool FROM_U>
__global__ void __launch_bounds__(HNT) k_hist_solve(HistState* st, float* __restrict__ table, float m, float inv_m1,
                                                   float eps, int max_iter) {
    __shared__ BinScratch sc;
    if (st->bad) return;
    const int b = threadIdx.x;
    float v[C], up[C];
    DF v64[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = st->V[j];
        const double q = st->V64[j];
        v64[j] = DF{(float)q, (float)(q - (double)(float)q)};
        up[j] = 0.0f;
    }
    if (!FROM_U) {
        float v0[C], um0[C];
#pragma unroll
        for (int j = 0; j < C; ++j) v0[j] = st->V0[j];
        membership<C, MK>((float)b, v0, m, inv_m1, up, um0);
    }
    const float cnt = (float)st->hist[b];
    int flags = st->flags, par = 0;
    int k, status;
    float delta;
    DF J;
    solve_bins<C, MK>(sc, par, cnt, FROM_U, FROM_U ? __uint_as_float(st->d1bits) : 0.0f, v, v64, up, m, inv_m1,
                      eps, max_iter, flags, k, status, delta, J);
#pragma unroll
    for (int j = 0; j < C; ++j) table[b * C + j] = up[j];
    if (b == 0) {
        st->iters = k;
        st->status = status;
        st->flags = flags;
        st->delta = (double)delta;
        st->J = (double)J.hi + (double)J.lo;
    }
#pragma unroll
    for (int j = 0; j < C; ++j)
        if (b == j) {
            st->V[j] = v[j];
            st->V64[j] = (double)v64[j].hi + (double)v64[j].lo;
        }
}

// U^k by table lookup: U_ij = table[x_i][j].
template <int C>
__global__ void __launch_bounds__(HNT) k_hist_emit(const float* __restrict__ x, int64_t n,
                                                  const float* __restrict__ table, const HistState* st,
                                                  float* __restrict__ U) {
    __shared__ float T[256 * C];
    if (st->bad) return;
    for (int t = threadIdx.x; t < 256 * C; t += HNT) T[t] = table[t];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * HNT;
    for (int64_t i = (int64_t)blockIdx.x * HNT + threadIdx.x; i < n; i += stride) {
        const int b = (int)__ldg(x + i);
        if (!in_bounds(b >= 0 && b < 256, const_cast<unsigned*>(&st->bounds))) continue;
#pragma unroll
        for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + i, T[b * C + j]);
    }
}

typedef void (*Pass0Fn)(const float*, const float*, int64_t, float, HistState*, double*);
typedef void (*InitFn)(HistState*, const double*, int, float, float);
typedef void (*Delta1Fn)(const float*, const float*, int64_t, float, float, HistState*);
typedef void (*SolveFn)(HistState*, float*, float, float, float, int);
typedef void (*EmitFn)(const float*, int64_t, const float*, const HistState*, float*);

struct HistKernels {
    Pass0Fn pass0[2];
    InitFn init[2];
    Delta1Fn delta1;
    SolveFn solve[2];
    EmitFn emit;
};

template <int C, int MK>
HistKernels kernels_cm() {
    return HistKernels{{k_hist_pass0<C, MK, false>, k_hist_pass0<C, MK, true>},
                       {k_hist_init<C, MK, false>, k_hist_init<C, MK, true>},
                       k_hist_delta1<C, MK>,
                       {k_hist_solve<C, MK, false>, k_hist_solve<C, MK, true>},
                       k_hist_emit<C>};
}

template <int C>
HistKernels kernels_c(int mk) {
    switch (mk) {
        case M_TWO: return kernels_cm<C, M_TWO>();
        case M_THREE: return kernels_cm<C, M_THREE>();
        case M_ONE_HALF: return kernels_cm<C, M_ONE_HALF>();
        default: return kernels_cm<C, M_GENERIC>();
    }
}

HistKernels kernels_for(int C, int mk) {
    switch (C) {
        case 1: return kernels_c<1>(mk);
        case 2: return kernels_c<2>(mk);
        case 3: return kernels_c<3>(mk);
        case 4: return kernels_c<4>(mk);
        case 5: return kernels_c<5>(mk);
        case 6: return kernels_c<6>(mk);
        case 7: return kernels_c<7>(mk);
        default: return kernels_c<8>(mk);
    }
}

bool device_buffer(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call); \
    } while (0)

void fcm_release_hist(fcm_ctx* h) {
    if (!h || !h->hist) return;
    HistWorkspace* w = h->hist;
    cudaFree(w->d_st);
    cudaFree(w->part);
    cudaFree(w->table);
    cudaFreeHost(w->h_st);
    delete w;
    h->hist = nullptr;
}

extern "C" int fcm_run_hist(fcm_handle h, const float* x, int64_t n, int C, float m, float eps, int max_iter,
                            int init_mode, const float* U0, float* U, float* V, fcm_report* rep) {
    NvtxRange nvtx_range("fcm_run_hist");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!x || !U || !V) return ctx_invalid(h, "null x, U or V");
    if (n < 1 || n > ((int64_t)1 << 40)) return ctx_invalid(h, "n must be in [1, 2^40]");
    if (C < 1 || C > FCM_MAX_CLUSTERS) return ctx_invalid(h, "C must be in [1, 8]");
    if (!(m > 1.0f) || !std::isfinite(m)) return ctx_invalid(h, "m must be a finite number > 1");
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return ctx_invalid(h, "eps must be finite and >= 0");
    if (max_iter < 1) return ctx_invalid(h, "max_iter must be >= 1");
    if (init_mode != FCM_INIT_U && init_mode != FCM_INIT_V) return ctx_invalid(h, "bad init_mode");
    const bool from_u = init_mode == FCM_INIT_U;
    if (from_u && !U0) U0 = U;
    if (!device_buffer(x) || !device_buffer(U) || (from_u && !device_buffer(U0)))
        return ctx_invalid(h, "x, U and U0 must be device memory");
    const bool V_dev = device_buffer(V);
    DeviceGuard g(h->device);
    if (!h->hist) h->hist = new HistWorkspace();
    HistWorkspace* w = h->hist;
    if (!w->d_st) CK(dev_malloc(h, &w->d_st, sizeof(HistState)));
    if (!w->h_st) CK(host_malloc(h, &w->h_st, sizeof(HistState)));
    if (!w->table) CK(dev_malloc(h, &w->table, sizeof(float) * 256 * FCM_MAX_CLUSTERS));
    const int64_t want = (n + (int64_t)HNT * HCHUNK - 1) / ((int64_t)HNT * HCHUNK);
    const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)h->num_sms * 8));
    if (w->part_blocks < nblocks) {
        cudaFree(w->part);
        w->part = nullptr;
        w->part_blocks = 0;
        CK(dev_malloc(h, &w->part, sizeof(double) * 2 * FCM_MAX_CLUSTERS * nblocks));
        w->part_blocks = nblocks;
    }
    HistState* hs = w->h_st;
    std::memset(hs, 0, sizeof(HistState));
    hs->status = FCM_ERR_TIMEOUT;  // overwritten by the solver
    if (!from_u && !V_dev) std::memcpy(hs->V0, V, sizeof(float) * C);
    CK(cudaMemcpyAsync(w->d_st, hs, sizeof(HistState), cudaMemcpyHostToDevice, h->stream));
    if (!from_u && V_dev)
        CK(cudaMemcpyAsync(&w->d_st->V0, V, sizeof(float) * C, cudaMemcpyDeviceToDevice, h->stream));

    const HistKernels k = kernels_for(C, mkind_of(m));
    const float inv_m1 = (float)(1.0 / ((double)m - 1.0));
    const int fu = from_u ? 1 : 0;
    k.pass0[fu]<<<nblocks, HNT, 0, h->stream>>>(x, from_u ? U0 : nullptr, n, m, w->d_st, w->part);
    k.init[fu]<<<1, HNT, 0, h->stream>>>(w->d_st, w->part, nblocks, m, inv_m1);
    if (from_u) k.delta1<<<nblocks, HNT, 0, h->stream>>>(x, U0, n, m, inv_m1, w->d_st);
    k.solve[fu]<<<1, HNT, 0, h->stream>>>(w->d_st, w->table, m, inv_m1, eps, max_iter);
    k.emit<<<nblocks, HNT, 0, h->stream>>>(x, n, w->table, w->d_st, U);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(hs, w->d_st, sizeof(HistState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(V, &w->d_st->V, sizeof(float) * C, V_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->iters = hs->iters;
        rep->status = hs->status;
        rep->flags = hs->flags | (int)hs->bounds;
        rep->C = C;
        rep->delta = hs->delta;
        rep->J = hs->J;
        for (int j = 0; j < C; ++j) rep->V64[j] = hs->V64[j];
        rep->launches = from_u ? 5 : 4;
    }
    if (hs->status == FCM_ERR_BAD_INPUT) h->last_error = "x must hold integer grey levels 0..255 (and U0 be valid)";
    return hs->status;
}
