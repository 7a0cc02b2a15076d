// Batched FCM: many independent slices in one persistent launch.
//
// Compiled once per block size with -DFCM_BATCH_NT=256 or 512.
//
// Each slice is one run of Algorithm 1 (arXiv:1601.00072, Sec. 2.1) with its
// own n, C, m, eps and max_iter. The grid is persistent: CTAs (or thread-block
// clusters) take slices from a work queue ordered by decreasing size (LPT),
// so the largest slices start first and the small ones fill the tail.
//
//  * Big slices (n >= plan.big) are shared by all K CTAs of a cluster: each
//    CTA takes a contiguous 1/K of the pixels; after every pass the CTAs
//    exchange their block totals through distributed shared memory at a
//    hardware cluster barrier and add them in rank order, so every rank
//    derives the same centers and the same stop decision.
//  * Once the queue reaches small slices, every CTA works alone.
//
// No U is stored between iterations: U^{k-1} is recomputed from V^{k-1} with
// the same code that produced it (bit-identical), so an iteration reads only
// x, which sits in shared memory when the CTA's share fits. U^0 (when given)
// is read in the first two passes; U^k is written once, after the last
// iteration. All per-pixel arithmetic is the single-image pass's (Eq. 4 in
// packed FP32x2 pairs); sums run in FP32 over chunks of a few pixels, then in
// compensated FP32 per thread, warp, CTA and cluster (no FP64 instruction in
// the iteration loop).
#include "fcm_batched.h"
#include "fcm_device.cuh"
#include "fcm_df.cuh"

#ifndef FCM_BATCH_NT
#error "compile with -DFCM_BATCH_NT=<threads per CTA>"
#endif

namespace fcm {
namespace {

constexpr int NTB = FCM_BATCH_NT;
constexpr int NWB = NTB / 32;
// Up to 128 registers per thread (the recompute loop keeps two center sets
// and packed accumulators live): one 512-thread CTA or two 256-thread CTAs
// per SM, with 192 KB or 96 KB of x staging each.
constexpr int XCAP = NTB == 512 ? 49152 : 24576;
constexpr int MIN_BLOCKS = NTB == 512 ? 1 : 2;
constexpr int SBMAX = 2 * FCM_MAX_CLUSTERS + 3;  // num[C], den[C], J, max|dU|, bad

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned k;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(k));
    return k;
}
// Hardware barrier of all threads of all CTAs of the cluster, with release /
// acquire ordering of their shared-memory writes.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(const void* local, unsigned rank) {
    uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(local)), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_dsmem_f2(const float2* local, unsigned rank) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(dsmem_addr(local, rank))
                 : "memory");
    return v;
}
__device__ __forceinline__ int ld_dsmem_s32(const int* local, unsigned rank) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(dsmem_addr(local, rank)) : "memory");
    return v;
}

struct BatchShared {
    float w[NWB][2 * SBMAX];  // warp totals: (hi, lo) of each sum, then the maxima
    // block totals (sums as hi/lo double-floats, maxima in x), double-buffered
    // for the cluster or team exchange, and every rank's, gathered for the
    // rank-order sum
    float2 red[2][SBMAX];
    float2 xch[TEAM_MAX][SBMAX];
    DF tot[SBMAX];            // slice totals (the same on every rank); maxima in .hi
    DF vq[FCM_MAX_CLUSTERS];  // next centers, double-float quotients
    float vcur[FCM_MAX_CLUSTERS], vprev[FCM_MAX_CLUSTERS];  // centers, for the scalar path
    int idx;
    int team_err;             // a team barrier gave up
    int item[3];              // team schedule: slice, seat, team size
};

// A slice shared by a team of CTAs of the team schedule (any CTAs of the
// grid, not one cluster): after every pass each rank writes its block totals
// to global slots, arrives at the slice's barrier counter and waits, bounded,
// for the whole team; then every rank adds the team's totals in rank order.
// slots == nullptr: no team (a lone CTA, or a cluster exchanging through
// distributed shared memory).
struct TeamCtx {
    float2* slots;        // [T][2][SBMAX], this slice's
    unsigned* ctr;        // this slice's barrier counter (zero before the batch)
    uint32_t spins;       // polls, 128 ns apart, before the barrier gives up
    uint32_t phantoms;    // arrivals beyond the team's (0 unless a test injects a barrier that never fills)
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Per-thread pass sums: compensated (double-float) num, den and J, plus the
// maxima. Threads add pixels in FP32 over chunks of CHUNK pairs and fold each
// chunk into these, so the rounding of a thread's sum does not grow with the
// size of its share of the slice.
constexpr int CHUNK = 8;

template <int C>
struct SliceAcc {
    DF s[2 * C + 1];
    float dmax;
    bool bad;
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int t = 0; t < 2 * C + 1; ++t) s[t] = DF{0.0f, 0.0f};
        dmax = 0.0f;
        bad = false;
    }
};

// Totals of one pass over the slice: double-float warp sums, the CTA's warps
// merged in warp order, then (K > 1) the K CTAs in rank order through
// distributed shared memory, all in compensated FP32 (no FP64 instruction:
// a few threads would run a long FP64 chain while the rest wait at the
// barrier). Leaves sh.tot and the double-float quotients sh.vq = num / den.
template <int C>
__device__ __forceinline__ void slice_reduce(BatchShared& sh, SliceAcc<C>& a, unsigned r, unsigned K, int& parity,
                                             int& npass, const TeamCtx& tc) {
    constexpr int S = 2 * C + 3;
    constexpr int NS = 2 * C + 1;  // compensated sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const DF d = warp_sum_df(a.s[t]);
        if (lane == 0) {
            sh.w[warp][2 * t] = d.hi;
            sh.w[warp][2 * t + 1] = d.lo;
        }
    }
    const float dm = warp_max(a.dmax), bd = warp_max(a.bad ? 1.0f : 0.0f);
    if (lane == 0) {
        sh.w[warp][2 * NS] = dm;
        sh.w[warp][2 * NS + 1] = bd;
    }
    __syncthreads();
    if (threadIdx.x < S) {
        const int s = threadIdx.x;
        float2 t;
        if (s < NS) {
            DF d{sh.w[0][2 * s], sh.w[0][2 * s + 1]};
            for (int w = 1; w < NWB; ++w) d = df_merge(d, DF{sh.w[w][2 * s], sh.w[w][2 * s + 1]});
            t = make_float2(d.hi, d.lo);
        } else {
            float mx = sh.w[0][2 * NS + (s - NS)];
            for (int w = 1; w < NWB; ++w) mx = fmaxf(mx, sh.w[w][2 * NS + (s - NS)]);
            t = make_float2(mx, 0.0f);
        }
        sh.red[parity][s] = t;
        if (tc.slots) __stcg(&tc.slots[((int64_t)r * 2 + parity) * SBMAX + s], t);
    }
    ++npass;
    if (K > 1 && tc.slots) {
        // team: arrive, wait (bounded) for every rank's totals of this pass
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(tc.ctr, 1u);
            const unsigned target = (unsigned)npass * K + tc.phantoms;
            uint32_t spins = 0;
            while (ld_acquire_gpu(tc.ctr) < target) {
                if (++spins > tc.spins) {
                    sh.team_err = 1;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        __syncthreads();
        for (int t = threadIdx.x; t < (int)K * S; t += NTB)
            sh.xch[t / S][t % S] = __ldcg(&tc.slots[((int64_t)(t / S) * 2 + parity) * SBMAX + (t % S)]);
    } else if (K > 1) {
        cluster_sync();
        // all remote reads at once (one thread per rank and value)
        for (int t = threadIdx.x; t < (int)K * S; t += NTB) sh.xch[t / S][t % S] = ld_dsmem_f2(&sh.red[parity][t % S], t / S);
    }
    __syncthreads();
    // thread s combines value s in rank order; thread j < C also combines
    // den_j the same way (equal to total C + j) and forms v_j = num_j / den_j
    const int par = parity;
    auto at = [&](unsigned q, int s) {
        const float2 v = K > 1 ? sh.xch[q][s] : sh.red[par][s];
        return DF{v.x, v.y};
    };
    if (threadIdx.x < S) {
        const int s = threadIdx.x;
        DF t = at(0, s);
        for (unsigned q = 1; q < K; ++q) t = (s < NS) ? df_merge(t, at(q, s)) : DF{fmaxf(t.hi, at(q, s).hi), 0.0f};
        sh.tot[s] = t;
        if (s < C) {
            DF den = at(0, C + s);
            for (unsigned q = 1; q < K; ++q) den = df_merge(den, at(q, C + s));
            sh.vq[s] = den.hi > 0.0f ? df_div(t, den) : DF{0.0f, 0.0f};
        }
    }
    parity ^= 1;
    __syncthreads();
}

// Where a CTA reads its share of x during the iterations: FP32 values (in
// shared memory, or in global memory when the share does not fit), or bytes
// in shared memory when every value of the share is an integer grey level
// 0..255 (exact, and four times the pixels per byte of shared memory). The
// choice is the same for the whole CTA.
struct XSrc {
    const float* f;
    const uint8_t* b;
    bool bytes;
    __device__ __forceinline__ float at(int i) const { return bytes ? (float)b[i] : f[i]; }
    __device__ __forceinline__ float2 pair(int q) const {
        if (bytes) {
            const uchar2 v = *reinterpret_cast<const uchar2*>(b + 2 * q);
            return make_float2((float)v.x, (float)v.y);
        }
        return *reinterpret_cast<const float2*>(f + 2 * q);
    }
};

template <int C, int MK>
__device__ __noinline__ void process_slice(const SliceDesc& d, SliceResult& res, unsigned r, unsigned K, float* xs,
                                           BatchShared& sh, bool resume, int cap, const TeamCtx& tc) {
    const int64_t n = d.n;
    int64_t share = (n + K - 1) / K;
    share += share & 1;  // even, so only the last pixel of the slice can be unpaired
    const int64_t lo = min(n, (int64_t)r * share), hi = min(n, lo + share);
    const int cnt = (int)(hi - lo);
    if (threadIdx.x < C) {
        sh.vcur[threadIdx.x] = resume ? res.vcur[threadIdx.x] : d.V0[threadIdx.x];
        sh.vprev[threadIdx.x] = resume ? res.vprev[threadIdx.x] : d.V0[threadIdx.x];
    }
    XSrc xl{d.x + lo, reinterpret_cast<const uint8_t*>(xs), false};
    if (cnt <= XCAP) {
        for (int i = threadIdx.x; i < cnt; i += NTB) xs[i] = __ldg(d.x + lo + i);
        xl.f = xs;
    } else if (cnt <= 4 * XCAP) {
        uint8_t* xb = reinterpret_cast<uint8_t*>(xs);
        bool ok = true;
        for (int i = threadIdx.x; i < cnt; i += NTB) {
            const float v = __ldg(d.x + lo + i);
            const bool g = v >= 0.0f && v <= 255.0f && v == rintf(v);
            ok &= g;
            xb[i] = g ? (uint8_t)v : (uint8_t)0;
        }
        xl.bytes = __syncthreads_and(ok);
    }
    __syncthreads();
    const int npair = cnt >> 1;
    const bool odd_tail = (cnt & 1) && threadIdx.x == 0;  // the slice's last pixel, alone
    const float m = d.m, inv_m1 = d.inv_m1;
    const bool from_u = d.init == FCM_INIT_U;
    const float* U0 = d.U0;
    float (&v)[C] = *reinterpret_cast<float(*)[C]>(sh.vcur);
    float (&vp)[C] = *reinterpret_cast<float(*)[C]>(sh.vprev);

    f2 v2[C], vp2[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v2[j] = pack2(v[j], v[j]);
        vp2[j] = pack2(vp[j], vp[j]);
    }
    int parity = 0, npass = 0, flags = resume ? res.flags : 0;
    if (threadIdx.x == 0) sh.team_err = 0;
    SliceAcc<C> a;
    int status = FCM_NOT_CONVERGED, iters = 0;
    // delta, J and the centers behind V (double-floats) in FP32 arithmetic;
    // FP64 only when the result is written
    float delta = 0.0f;
    DF Jk{0.0f, 0.0f};
    DF v64[C];
    bool ok0 = true;
    if (resume) {
        // a parked slice: V^k and V^{k-1} as saved, iteration k = iters + 1 next
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const float hi = (float)res.V64[j];
            v64[j] = DF{hi, (float)(res.V64[j] - (double)hi)};
        }
        iters = res.iters;
    } else {
    // ---- pass 0: V^1 from U^0 (Eq. 3), or U^0 = membership(V^0) (Eq. 4) ----
    a.reset();
    if (!from_u) {
#pragma unroll
        for (int j = 0; j < C; ++j) a.bad |= !finite_f(d.V0[j]);
    }
    for (int p0 = threadIdx.x; p0 < npair; p0 += NTB * CHUNK) {
        float num[C], den[C];
#pragma unroll
        for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
        for (int q = 0, p = p0; q < CHUNK && p < npair; ++q, p += NTB) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = 2 * p + h;
                const float xi = xl.at(i);
                a.bad |= !finite_f(xi);
                if (from_u) {
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const float u0 = __ldg(U0 + (int64_t)j * n + lo + i);
                        a.bad |= !(u0 >= 0.0f) || !finite_f(u0);
                        const float w = pow_m<MK>(u0, m);
                        num[j] = fmaf(w, xi, num[j]);
                        den[j] += w;
                    }
                } else {
                    float u[C], um[C];
                    membership<C, MK>(xi, v, m, inv_m1, u, um);
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        num[j] = fmaf(um[j], xi, num[j]);
                        den[j] += um[j];
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            df_add(a.s[j], num[j]);
            df_add(a.s[C + j], den[j]);
        }
    }
    if (odd_tail) {
        const float xi = xl.at(cnt - 1);
        a.bad |= !finite_f(xi);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            float w;
            if (from_u) {
                const float u0 = __ldg(U0 + (int64_t)j * n + lo + cnt - 1);
                a.bad |= !(u0 >= 0.0f) || !finite_f(u0);
                w = pow_m<MK>(u0, m);
            } else {
                float u[C], um[C];
                membership<C, MK>(xi, v, m, inv_m1, u, um);
                w = um[j];
            }
            df_add(a.s[j], w * xi);
            df_add(a.s[C + j], w);
        }
    }
    slice_reduce<C>(sh, a, r, K, parity, npass, tc);
#pragma unroll
    for (int j = 0; j < C; ++j) v64[j] = DF{d.V0[j], 0.0f};
    ok0 = sh.tot[2 * C + 2].hi == 0.0f;
    }
    bool parked = false, gave_up = sh.team_err != 0;
    if (gave_up) {
        status = FCM_ERR_TIMEOUT;
    } else if (!ok0) {
        status = FCM_ERR_BAD_INPUT;
    } else {
        float vn[C];
        if (!resume) {
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (sh.tot[C + j].hi > 0.0f) {
                v64[j] = sh.vq[j];
                vn[j] = sh.vq[j].hi;
            } else {
                flags |= FCM_FLAG_EMPTY_CLUSTER;  // V^0 kept, or 0 from a U^0
                vn[j] = from_u ? 0.0f : d.V0[j];
                v64[j] = DF{vn[j], 0.0f};
            }
            v2[j] = pack2(vn[j], vn[j]);
        }
        __syncthreads();
        if (threadIdx.x < C) sh.vcur[threadIdx.x] = vn[threadIdx.x];
        __syncthreads();
        }
        // ---- iterations: U^k from V^k, U^{k-1} recomputed from V^{k-1} ----
        for (int k = iters + 1;; ++k) {
            if (k > cap) {
                // first phase of a two-phase batch: park before iteration k
                parked = true;
                break;
            }
            a.reset();
            const bool prev_given = from_u && k == 1;
            for (int p0 = threadIdx.x; p0 < npair; p0 += NTB * CHUNK) {
                f2 num2[C], den2[C], J2 = pack2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < C; ++j) num2[j] = den2[j] = pack2(0.0f, 0.0f);
                for (int q = 0, p = p0; q < CHUNK && p < npair; ++q, p += NTB) {
                    const float2 xv = xl.pair(p);
                    const f2 xq = pack2(xv.x, xv.y);
                    f2 u2[C], um2[C];
                    J2 = add2(J2, membership_pair<C, MK>(xq, v2, m, inv_m1, v, u2, um2));
                    f2 uo2[C];
                    if (prev_given) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const float* r0 = U0 + (int64_t)j * n + lo + 2 * p;
                            uo2[j] = pack2(__ldg(r0), __ldg(r0 + 1));
                        }
                    } else {
                        f2 tmp[C];
                        membership_pair<C, MK>(xq, vp2, m, inv_m1, vp, uo2, tmp);
                    }
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        num2[j] = fma2(um2[j], xq, num2[j]);
                        den2[j] = add2(den2[j], um2[j]);
                        float da, db;
                        unpack2(sub2(u2[j], uo2[j]), da, db);
                        a.dmax = fmaxf(a.dmax, fmaxf(fabsf(da), fabsf(db)));
                    }
                }
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    df_add(a.s[j], lo2(num2[j]) + hi2(num2[j]));
                    df_add(a.s[C + j], lo2(den2[j]) + hi2(den2[j]));
                }
                df_add(a.s[2 * C], lo2(J2) + hi2(J2));
            }
            if (odd_tail) {
                const float xi = xl.at(cnt - 1);
                float u[C], um[C], uo[C], umo[C];
                df_add(a.s[2 * C], membership<C, MK>(xi, v, m, inv_m1, u, um));
                if (prev_given) {
#pragma unroll
                    for (int j = 0; j < C; ++j) uo[j] = __ldg(U0 + (int64_t)j * n + lo + cnt - 1);
                } else {
                    membership<C, MK>(xi, vp, m, inv_m1, uo, umo);
                }
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    df_add(a.s[j], um[j] * xi);
                    df_add(a.s[C + j], um[j]);
                    a.dmax = fmaxf(a.dmax, fabsf(u[j] - uo[j]));
                }
            }
            slice_reduce<C>(sh, a, r, K, parity, npass, tc);
            delta = sh.tot[2 * C + 1].hi;
            Jk = sh.tot[2 * C];
            iters = k;
            if (sh.team_err) {
                status = FCM_ERR_TIMEOUT;
                gave_up = true;
                break;
            }
            if (delta < d.eps) {
                status = FCM_OK;
                break;
            }
            if (k >= d.max_iter) {
                status = FCM_NOT_CONVERGED;
                break;
            }
#pragma unroll
            for (int j = 0; j < C; ++j) {
                vp2[j] = v2[j];
                vn[j] = v[j];
                if (sh.tot[C + j].hi > 0.0f) {
                    v64[j] = sh.vq[j];
                    vn[j] = sh.vq[j].hi;
                    v2[j] = pack2(vn[j], vn[j]);
                } else {
                    flags |= FCM_FLAG_EMPTY_CLUSTER;  // keep v_j
                }
            }
            __syncthreads();  // every thread has read sh.vcur
            if (threadIdx.x < C) {
                sh.vprev[threadIdx.x] = sh.vcur[threadIdx.x];
                sh.vcur[threadIdx.x] = vn[threadIdx.x];
            }
            __syncthreads();
        }
        // ---- U^k, written once (a parked slice writes it in the second phase) ----
        float* U = d.U;
        for (int p = threadIdx.x; p < (parked || gave_up ? 0 : npair); p += NTB) {
            const float2 xv = xl.pair(p);
            f2 u2[C], um2[C];
            membership_pair<C, MK>(pack2(xv.x, xv.y), v2, m, inv_m1, v, u2, um2);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                float a0, b0;
                unpack2(u2[j], a0, b0);
                float* row = U + (int64_t)j * n + lo + 2 * p;
                __stcs(row, a0);
                __stcs(row + 1, b0);
            }
        }
        if (odd_tail && !parked && !gave_up) {
            float u[C], um[C];
            membership<C, MK>(xl.at(cnt - 1), v, m, inv_m1, u, um);
#pragma unroll
            for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + lo + cnt - 1, u[j]);
        }
    }
    if (r == 0 && threadIdx.x == 0) {
        res.iters = iters;
        res.status = parked ? SLICE_PARKED : status;
        res.flags = flags;
        res.delta = (double)delta;
        res.J = (double)Jk.hi + (double)Jk.lo;
#pragma unroll
        for (int j = 0; j < C; ++j) {
            res.V64[j] = (double)v64[j].hi + (double)v64[j].lo;
            if (parked) {
                res.vcur[j] = v[j];
                res.vprev[j] = vp[j];
            } else {
                d.V[j] = v[j];
            }
        }
    }
    // no rank of a cluster leaves the slice (and reuses its shared memory)
    // while another may still read it; a team exchanges through global slots
    // of its own slice and needs no such wait
    if (K > 1 && !tc.slots) cluster_sync();
    __syncthreads();
}

__device__ __forceinline__ void run_slice(const SliceDesc& d, SliceResult& res, unsigned r, unsigned K, float* xs,
                                          BatchShared& sh, bool resume, int cap, const TeamCtx& tc) {
#define FCM_BATCH_CASE(CC)                                                                  \
    case CC:                                                                                \
        switch (d.mk) {                                                                     \
            case M_TWO: process_slice<CC, M_TWO>(d, res, r, K, xs, sh, resume, cap, tc); break;              \
            case M_THREE: process_slice<CC, M_THREE>(d, res, r, K, xs, sh, resume, cap, tc); break;          \
            case M_ONE_HALF: process_slice<CC, M_ONE_HALF>(d, res, r, K, xs, sh, resume, cap, tc); break;    \
            default: process_slice<CC, M_GENERIC>(d, res, r, K, xs, sh, resume, cap, tc); break;             \
        }                                                                                   \
        break;
    switch (d.C) {
        FCM_BATCH_CASE(1)
        FCM_BATCH_CASE(2)
        FCM_BATCH_CASE(3)
        FCM_BATCH_CASE(4)
        FCM_BATCH_CASE(5)
        FCM_BATCH_CASE(6)
        FCM_BATCH_CASE(7)
        FCM_BATCH_CASE(8)
        default: break;
    }
#undef FCM_BATCH_CASE
}

__global__ void __launch_bounds__(NTB, MIN_BLOCKS)
    k_fcm_batched(const SliceDesc* __restrict__ descs, const int* __restrict__ order, int n_slices,
                  SliceResult* __restrict__ results, BatchCtl* __restrict__ ctl, int64_t big, int phase,
                  int cap) {
    extern __shared__ __align__(16) float xs[];
    __shared__ BatchShared sh;
    const unsigned K = cluster_size(), r = cluster_rank();
    const bool resume = phase == 1;
    // the second phase takes only the slices the first one parked (their
    // status was written by the earlier launch; no one else writes it now)
    auto wanted = [&](int s) { return !resume || __ldcg(&results[s].status) == SLICE_PARKED; };
    bool solo = K == 1;
    int first_solo = -1;
    // ---- the cluster shares the big slices ----
    while (!solo) {
        if (r == 0 && threadIdx.x == 0) sh.idx = (int)atomicAdd(&ctl->next, 1u);
        cluster_sync();
        const int idx = ld_dsmem_s32(&sh.idx, 0);
        cluster_sync();  // every rank has read the index before rank 0 takes another
        if (idx >= n_slices) return;
        const int s = order[idx];
        if (!wanted(s)) continue;
        if (descs[s].n >= big) {
            run_slice(descs[s], results[s], r, K, xs, sh, resume, cap, TeamCtx{});
            continue;
        }
        // the queue has reached the small slices: every CTA works alone now
        solo = true;
        if (r == 0) first_solo = s;
    }
    if (first_solo >= 0) run_slice(descs[first_solo], results[first_solo], 0, 1, xs, sh, resume, cap, TeamCtx{});
    for (;;) {
        if (threadIdx.x == 0) sh.idx = (int)atomicAdd(&ctl->next, 1u);
        __syncthreads();
        const int idx = sh.idx;
        __syncthreads();
        if (idx >= n_slices) return;
        const int s = order[idx];
        if (!wanted(s)) continue;
        run_slice(descs[s], results[s], 0, 1, xs, sh, resume, cap, TeamCtx{});
    }
}

// The team schedule: one cooperative launch (every CTA resident), no
// clusters. The queue holds one item per seat: a slice with a team of T CTAs
// appears T times in a row, seats 0..T-1, so the CTAs that take them form its
// team; the host orders the items by team time, longest first. Only the team
// at the head of the queue can be incomplete, and every other team finishes
// and frees its CTAs, so every team fills; each barrier wait is bounded
// nonetheless.
__global__ void __launch_bounds__(NTB, MIN_BLOCKS)
    k_fcm_teams(TeamArgs a) {
    extern __shared__ __align__(16) float xs[];
    __shared__ BatchShared sh;
    for (;;) {
        if (threadIdx.x == 0) {
            const int idx = (int)atomicAdd(&a.ctl->next, 1u);
            if (idx < a.hdr->max_rounds) {
                const int4 it = a.items[idx];
                sh.item[0] = it.x;
                sh.item[1] = it.y;
                sh.item[2] = it.z;
            } else {
                sh.item[0] = -1;
            }
        }
        __syncthreads();
        const int s = sh.item[0], seat = sh.item[1], T = sh.item[2];
        __syncthreads();
        if (s < 0) return;
        TeamCtx tc{};
        if (T > 1) {
            tc.slots = a.slots + (int64_t)a.slot_base[s] * 2 * SBMAX;
            tc.ctr = a.counters + s;
            tc.spins = a.hdr->wait_spins;
            tc.phantoms = a.hdr->phantoms;
        }
        run_slice(a.descs[s], a.results[s], (unsigned)seat, (unsigned)T, xs, sh, false, 0x7fffffff, tc);
    }
}

}  // namespace

#define FCM_CAT2(a, b) a##b
#define FCM_CAT(a, b) FCM_CAT2(a, b)
BatchKernel FCM_CAT(batched_kernel_, FCM_BATCH_NT)() {
    return BatchKernel{k_fcm_batched, XCAP * (int)sizeof(float), XCAP, k_fcm_teams};
}

}  // namespace fcm
