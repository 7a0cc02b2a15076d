// Batched FCM, round-synchronous schedule.
//
// Compiled once per block size with -DFCM_ROUNDS_NT=256 or 512.
//
// Each slice is one run of Algorithm 1 (arXiv:1601.00072, Sec. 2.1), as in
// the slice-queue kernel, with the same per-pixel arithmetic. Here every slice
// takes the same step in the same round: round 0 is pass 0 (V^1 from U^0, or
// from U^0 = f(x, V^0)), round k >= 1 is iteration k, and the round after a
// slice's stop decision writes its U^k.
//
// In each round the slices still running are laid end to end in work units
// (pixels, padded to an even count, times a per-pixel cost weight 2C + 1) and
// cut into gridDim.x equal, contiguous chunks, one per CTA (never smaller than
// min_chunk pixels of the heaviest weight, so a nearly finished batch uses
// fewer CTAs). A slice that needs many iterations is thus spread over the
// whole GPU in its late rounds instead of holding a few SMs while the rest
// idle, and every round's work is balanced.
//
// A CTA's chunk is one segment (a whole number of pixel pairs, possibly none)
// of each slice it crosses. A slice inside one chunk is decided by that CTA at
// once. Otherwise each segment writes FP64 block sums to its own slot; the
// last segment of the slice to finish the round (a ticket per slice) adds the
// slots in order, takes the step's decision and writes the next centers. Rounds are separated by a
// bounded grid barrier (the launch is cooperative, so all CTAs are resident).
// Whether a slice runs in round r is read from its end_round, which a
// finaliser only moves from "open" to r + 1 (or to -1 in round 0) during
// round r; every CTA sees the same set for round r whichever value it reads,
// so all derive the same chunks. No U is stored between iterations: U^{k-1}
// is recomputed from V^{k-1}, so an iteration reads only x.
#include "fcm_batched.h"
#include "fcm_device.cuh"

#ifndef FCM_ROUNDS_NT
#error "compile with -DFCM_ROUNDS_NT=<threads per CTA>"
#endif

namespace fcm {
namespace {

constexpr int NTR = FCM_ROUNDS_NT;
constexpr int NWR = NTR / 32;
constexpr int MIN_BLOCKS_R = NTR == 512 ? 1 : 2;
constexpr int SR = ROUND_SUMS;
constexpr int OPEN = 0x7fffffff;

// Pixels are added in FP32 over chunks of CHUNK pairs, then in compensated
// FP32 per thread and warp, then in FP64 across warps and segments.
constexpr int CHUNK = 8;

// The round barrier polls at most hdr->wait_spins times, 128 ns apart (about
// 1 s by default), for the grid's arrivals plus hdr->phantoms (0 unless a
// test injects a barrier that never fills).

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

struct RoundShared {
    float w[NWR][2 * SR];  // warp totals: (hi, lo) of each sum, then the maxima
    double tot[SR];
    int64_t chunk, beg, end;
    int last, stop;
};

template <int C>
struct SegAcc {
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

// Block sums of one segment: into sh.tot when the segment is the whole of the
// slice's round (K == 0), else into its slot, value q at part[q * K].
template <int C>
__device__ __forceinline__ void store_segment(SegAcc<C>& a, RoundShared& sh, double* part, int K) {
    constexpr int NS = 2 * C + 1, S = 2 * C + 3;
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
        const int q = threadIdx.x;
        double t = 0.0;
        if (q < NS) {
            for (int w = 0; w < NWR; ++w) t += (double)sh.w[w][2 * q] + (double)sh.w[w][2 * q + 1];
        } else {
            for (int w = 0; w < NWR; ++w) t = fmax(t, (double)sh.w[w][2 * NS + (q - NS)]);
        }
        if (K == 0) {
            sh.tot[q] = t;
        } else {
            __stcg(part + (int64_t)q * K, t);
            __threadfence();  // before the segment's ticket
        }
    }
}

// Pass 0 over pixels [lo, lo + cnt) of a slice: the numerators and
// denominators of V^1 (Eq. 3) from U^0, or from U^0 = f(x, V^0) (Eq. 4), and
// the input checks.
template <int C, int MK>
__device__ __noinline__ void seg_pass0(const SliceDesc* __restrict__ d, int64_t lo, int64_t cnt, RoundShared& sh,
                                       double* part, int K) {
    const float* x = d->x + lo;
    const float* U0 = d->U0;
    const int64_t n = d->n;
    const float m = d->m, inv_m1 = d->inv_m1;
    const bool from_u = d->init == FCM_INIT_U;
    float v[C];
#pragma unroll
    for (int j = 0; j < C; ++j) v[j] = d->V0[j];
    SegAcc<C> a;
    a.reset();
    if (!from_u && lo == 0) {
#pragma unroll
        for (int j = 0; j < C; ++j) a.bad |= !finite_f(v[j]);
    }
    for (int64_t i0 = threadIdx.x; i0 < cnt; i0 += (int64_t)NTR * CHUNK) {
        float num[C], den[C];
#pragma unroll
        for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
        float xc[CHUNK];
#pragma unroll
        for (int q = 0; q < CHUNK; ++q) {
            const int64_t i = i0 + (int64_t)q * NTR;
            xc[q] = i < cnt ? __ldg(x + i) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < CHUNK; ++q) {
            const int64_t i = i0 + (int64_t)q * NTR;
            if (i >= cnt) break;
            const float xi = xc[q];
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
#pragma unroll
        for (int j = 0; j < C; ++j) {
            df_add(a.s[j], num[j]);
            df_add(a.s[C + j], den[j]);
        }
    }
    store_segment<C>(a, sh, part, K);
}

// Iteration k over pixels [lo, lo + cnt): U^k from V^k (Eq. 4) with its J
// term (Eq. 1), the sums of V^{k+1} (Eq. 3), and max |U^k - U^{k-1}| with
// U^{k-1} recomputed from V^{k-1} (or read from U^0 when k = 1 and the run
// started from U^0). lo is even; only the slice's last pixel can be unpaired.
template <int C, int MK>
__device__ __noinline__ void seg_iter(const SliceDesc* __restrict__ d, const RoundSlice* st, int64_t lo,
                                      int64_t cnt, bool prev_given, RoundShared& sh, double* part, int K) {
    const float* x = d->x + lo;
    const float* U0 = d->U0;
    const int64_t n = d->n;
    const float m = d->m, inv_m1 = d->inv_m1;
    float v[C], vp[C];
    f2 v2[C], vp2[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = __ldcg(&st->vcur[j]);
        vp[j] = __ldcg(&st->vprev[j]);
        v2[j] = pack2(v[j], v[j]);
        vp2[j] = pack2(vp[j], vp[j]);
    }
    SegAcc<C> a;
    a.reset();
    const int64_t npair = cnt >> 1;
    const float2* x2 = reinterpret_cast<const float2*>(x);
    for (int64_t p0 = threadIdx.x; p0 < npair; p0 += (int64_t)NTR * CHUNK) {
        f2 num2[C], den2[C], J2 = pack2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < C; ++j) num2[j] = den2[j] = pack2(0.0f, 0.0f);
        for (int64_t q = 0, p = p0; q < CHUNK && p < npair; ++q, p += NTR) {
            const float2 xv = __ldg(x2 + p);
            const f2 xq = pack2(xv.x, xv.y);
            f2 u2[C], um2[C], uo2[C];
            J2 = add2(J2, membership_pair<C, MK>(xq, v2, m, inv_m1, v, u2, um2));
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
    if ((cnt & 1) && threadIdx.x == 0) {  // the slice's last pixel, alone
        const float xi = x[cnt - 1];
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
    store_segment<C>(a, sh, part, K);
}

// The final memberships U^k from the final V^k, written once.
template <int C, int MK>
__device__ __noinline__ void seg_emit(const SliceDesc* __restrict__ d, const RoundSlice* st, int64_t lo,
                                      int64_t cnt) {
    const float* x = d->x + lo;
    float* U = d->U;
    const int64_t n = d->n;
    const float m = d->m, inv_m1 = d->inv_m1;
    float v[C];
    f2 v2[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        v[j] = __ldcg(&st->vcur[j]);
        v2[j] = pack2(v[j], v[j]);
    }
    const int64_t npair = cnt >> 1;
    const float2* x2 = reinterpret_cast<const float2*>(x);
    for (int64_t p0 = threadIdx.x; p0 < npair; p0 += (int64_t)NTR * CHUNK) {
        float2 xc[CHUNK];
#pragma unroll
        for (int q = 0; q < CHUNK; ++q) {
            const int64_t p = p0 + (int64_t)q * NTR;
            xc[q] = p < npair ? __ldg(x2 + p) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < CHUNK; ++q) {
            const int64_t p = p0 + (int64_t)q * NTR;
            if (p >= npair) break;
            f2 u2[C], um2[C];
            membership_pair<C, MK>(pack2(xc[q].x, xc[q].y), v2, m, inv_m1, v, u2, um2);
#pragma unroll
            for (int j = 0; j < C; ++j) {
                float a0, b0;
                unpack2(u2[j], a0, b0);
                float* row = U + (int64_t)j * n + lo + 2 * p;
                __stcs(row, a0);
                __stcs(row + 1, b0);
            }
        }
    }
    if ((cnt & 1) && threadIdx.x == 0) {
        float u[C], um[C];
        membership<C, MK>(x[cnt - 1], v, m, inv_m1, u, um);
#pragma unroll
        for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * n + lo + cnt - 1, u[j]);
    }
}

enum SegKind : int { K_PASS0 = 0, K_ITER = 1, K_EMIT = 2 };

template <int C>
__device__ __forceinline__ void seg_c(int kind, int mk, const SliceDesc* d, const RoundSlice* st, int64_t lo,
                                      int64_t cnt, bool prev_given, RoundShared& sh, double* part, int K) {
#define FCM_ROUND_MK(MKV)                                                                   \
    case MKV:                                                                               \
        if (kind == K_PASS0) seg_pass0<C, MKV>(d, lo, cnt, sh, part, K);                   \
        else if (kind == K_ITER) seg_iter<C, MKV>(d, st, lo, cnt, prev_given, sh, part, K); \
        else seg_emit<C, MKV>(d, st, lo, cnt);                                              \
        break;
    switch (mk) {
        FCM_ROUND_MK(M_TWO)
        FCM_ROUND_MK(M_THREE)
        FCM_ROUND_MK(M_ONE_HALF)
        default:
            FCM_ROUND_MK(M_GENERIC)
    }
#undef FCM_ROUND_MK
}

__device__ __forceinline__ void run_segment(int kind, const SliceDesc* d, const RoundSlice* st, int64_t lo,
                                            int64_t cnt, bool prev_given, RoundShared& sh, double* part, int K) {
    const int mk = d->mk;
    switch (d->C) {
        case 1: seg_c<1>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 2: seg_c<2>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 3: seg_c<3>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 4: seg_c<4>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 5: seg_c<5>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 6: seg_c<6>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        case 7: seg_c<7>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
        default: seg_c<8>(kind, mk, d, st, lo, cnt, prev_given, sh, part, K); break;
    }
}

// The totals of a slice split over nseg segments: its slots in order (one
// warp per sum, lanes over slots, FP64, fixed xor tree), into sh.tot.
__device__ void gather(int C, const double* part, int K, int nseg, RoundShared& sh) {
    const int S = 2 * C + 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < S; q += NWR) {
        const double* pq = part + (int64_t)q * K;
        double acc = 0.0;
        if (q <= 2 * C) {
            for (int i = lane; i < nseg; i += 32) acc += __ldcg(pq + i);
            acc = warp_sum(acc);
        } else {
            for (int i = lane; i < nseg; i += 32) acc = fmax(acc, __ldcg(pq + i));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        }
        if (lane == 0) sh.tot[q] = acc;
    }
}

// The step of Algorithm 1 that ends round r for slice s, from its totals in
// sh.tot, by thread 0: V^1 after pass 0, else the stop test and V^{k+1}.
// The grid barrier that ends the round orders these writes before any reader.
__device__ void decide(const RoundsArgs& a, int s, int r, const RoundShared& sh) {
    const SliceDesc* d = a.descs + s;
    RoundSlice* st = a.state + s;
    const int C = d->C;
    const double* tot = sh.tot;
    st->ticket = 0u;  // every segment of this round has arrived
    SliceResult* res = a.results + s;
    int flags = st->flags;
    if (r == 0) {
        if (tot[2 * C + 2] != 0.0) {
            res->iters = 0;
            res->status = FCM_ERR_BAD_INPUT;
            res->flags = 0;
            res->delta = 0.0;
            res->J = 0.0;
            for (int j = 0; j < C; ++j) {
                res->V64[j] = d->V0[j];
                d->V[j] = d->V0[j];
            }
            st->end_round = -1;
            atomicSub(&a.ctl->undecided, 1u);
            return;
        }
        const bool from_u = d->init == FCM_INIT_U;
        for (int j = 0; j < C; ++j) {
            const double den = tot[C + j];
            float vn;
            double v64;
            if (den > 0.0) {
                v64 = tot[j] / den;
                vn = (float)v64;
            } else {
                flags |= FCM_FLAG_EMPTY_CLUSTER;  // V^0 kept, or 0 from a U^0
                vn = from_u ? 0.0f : d->V0[j];
                v64 = vn;
            }
            st->vprev[j] = d->V0[j];
            st->vcur[j] = vn;
            st->v64[j] = v64;
        }
        st->flags = flags;
        return;
    }
    const double delta = tot[2 * C + 1], J = tot[2 * C];
    const bool converged = delta < (double)d->eps;
    if (converged || r >= d->max_iter) {
        res->iters = r;
        res->status = converged ? FCM_OK : FCM_NOT_CONVERGED;
        res->flags = flags;
        res->delta = delta;
        res->J = J;
        for (int j = 0; j < C; ++j) {
            res->V64[j] = st->v64[j];
            d->V[j] = st->vcur[j];
        }
        st->end_round = r + 1;
        atomicMax(&a.ctl->last_round, r + 1);
        atomicSub(&a.ctl->undecided, 1u);
        return;
    }
    for (int j = 0; j < C; ++j) {
        const double den = tot[C + j];
        st->vprev[j] = st->vcur[j];
        if (den > 0.0) {
            const double q = tot[j] / den;
            st->v64[j] = q;
            st->vcur[j] = (float)q;
        } else {
            flags |= FCM_FLAG_EMPTY_CLUSTER;  // keep v_j
        }
    }
    st->flags = flags;
}

// Cost weight of one pixel of a slice with C clusters (its work grows
// about linearly in C).
__device__ __forceinline__ int64_t pixel_weight(int C) { return 2 * C + 1; }

// Work units slice s contributes to round r: its size padded to even times
// its pixel weight, or 0 when it does not run.
__device__ __forceinline__ int64_t round_units(const RoundsArgs& a, int s, int r) {
    if (r > 0) {
        const int er = __ldcg(&a.state[s].end_round);
        if (r > er) return 0;  // also er = -1
    }
    const SliceDesc& d = a.descs[s];
    return (d.n + (d.n & 1)) * pixel_weight(d.C);
}

__global__ void __launch_bounds__(NTR, MIN_BLOCKS_R) k_fcm_rounds(RoundsArgs a) {
    extern __shared__ int64_t pre[];  // [n_slices + 1]: prefix of this round's pixels
    __shared__ RoundShared sh;
    __shared__ int64_t wsum[NWR];
    const int ns = a.hdr->n_slices, max_rounds = a.hdr->max_rounds;
    const int per = (ns + NTR - 1) / NTR;  // slices per thread in the scan
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r <= max_rounds; ++r) {
        // ---- exclusive prefix of the pixels of the slices in this round ----
        const int e0 = min(ns, (int)threadIdx.x * per), e1 = min(ns, e0 + per);
        int64_t mine = 0;
        for (int e = e0; e < e1; ++e) mine += round_units(a, e, r);
        int64_t inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int64_t base = 0;
        for (int w = 0; w < warp; ++w) base += wsum[w];
        int64_t run = base + inc - mine;
        for (int e = e0; e < e1; ++e) {
            pre[e] = run;
            run += round_units(a, e, r);
        }
        if (threadIdx.x == NTR - 1) {
            int64_t total = 0;
            for (int w = 0; w < NWR; ++w) total += wsum[w];
            pre[ns] = total;
            int64_t c = (total + gridDim.x - 1) / gridDim.x;
            // at least min_chunk pixels of the heaviest weight, so no slice
            // has more segments than its ceil(n / min_chunk) + 2 slots
            c = max(c, (int64_t)a.min_chunk * pixel_weight(FCM_MAX_CLUSTERS));
            sh.chunk = c;
            sh.beg = min(total, (int64_t)blockIdx.x * c);
            sh.end = min(total, sh.beg + c);
        }
        __syncthreads();
        const int64_t chunk = sh.chunk, beg = sh.beg, end = sh.end;
        if (beg < end) {
            // first slice whose pixels reach past beg
            int lo_s = 0, hi_s = ns - 1;
            while (lo_s < hi_s) {
                const int mid = (lo_s + hi_s) >> 1;
                if (pre[mid + 1] > beg) hi_s = mid;
                else lo_s = mid + 1;
            }
            for (int s = lo_s; s < ns && pre[s] < end; ++s) {
                const int64_t p0 = pre[s], p1 = pre[s + 1];
                if (p1 == p0) continue;
                const SliceDesc* d = a.descs + s;
                RoundSlice* st = a.state + s;
                int kind = K_PASS0;
                if (r > 0) kind = r < __ldcg(&st->end_round) ? K_ITER : K_EMIT;
                // pixel range: unit offsets in the slice, down to a whole pair
                const int64_t pair_units = 2 * pixel_weight(d->C);
                const int64_t npad = d->n + (d->n & 1);
                const int64_t lo = beg <= p0 ? 0 : (beg - p0) / pair_units * 2;
                const int64_t hi = end >= p1 ? npad : (end - p0) / pair_units * 2;
                const int64_t cnt = max((int64_t)0, min(hi, d->n) - lo);
                const int sb = __ldg(a.slot_base + s), K = __ldg(a.slot_base + s + 1) - sb;
                const int b0 = (int)(p0 / chunk), nseg = (int)((p1 - 1) / chunk) - b0 + 1;
                double* part = a.partials + (int64_t)sb * SR;
                const bool prev_given = r == 1 && d->init == FCM_INIT_U;
                // a slice inside this chunk is decided here at once, with no slot
                run_segment(kind, d, st, lo, cnt, prev_given, sh, part + (blockIdx.x - b0), nseg == 1 ? 0 : K);
                if (kind == K_EMIT) continue;
                __syncthreads();  // the segment's totals or slot stores are issued
                if (nseg > 1) {
                    if (threadIdx.x == 0) {
                        __threadfence();
                        const unsigned old = atomicAdd(&st->ticket, 1u);
                        const int last = (int)(old + 1 == (unsigned)nseg);
                        if (last) __threadfence();
                        sh.last = last;
                    }
                    __syncthreads();
                    if (!sh.last) continue;
                    gather(d->C, part, K, nseg, sh);
                    __syncthreads();
                }
                if (threadIdx.x == 0) decide(a, s, r, sh);
                __syncthreads();
            }
        }
        // ---- bounded grid barrier, then the common stop test ----
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctl->bar, 1u);
            const unsigned target = (unsigned)(r + 1) * gridDim.x + a.hdr->phantoms;
            const uint32_t limit = a.hdr->wait_spins;
            uint32_t spins = 0;
            int stop = 0;
            while (ld_acquire_u32(&a.ctl->bar) < target) {
                if (++spins > limit) {
                    atomicExch(&a.ctl->timeout, 1u);
                    stop = 1;
                    break;
                }
                __nanosleep(128);
            }
            if (!stop) {
                __threadfence();
                const unsigned und = ld_acquire_u32(&a.ctl->undecided);
                const int lr = (int)ld_acquire_u32(reinterpret_cast<const unsigned*>(&a.ctl->last_round));
                stop = und == 0u && r >= lr;
            }
            sh.stop = stop;
        }
        __syncthreads();
        if (sh.stop) break;
    }
}

// State of every slice before a batch: open, no ticket, results marked as
// timed out until the slice's decision overwrites them.
__global__ void k_rounds_init(RoundSlice* state, SliceResult* results, RoundCtl* ctl, int n_slices) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        ctl->bar = 0u;
        ctl->undecided = (unsigned)n_slices;
        ctl->last_round = 0;
        ctl->timeout = 0u;
    }
    if (s >= n_slices) return;
    RoundSlice& st = state[s];
    st.end_round = OPEN;
    st.flags = 0;
    st.ticket = 0u;
    SliceResult& r = results[s];
    r.iters = 0;
    r.status = FCM_ERR_TIMEOUT;
    r.flags = 0;
    r.delta = 0.0;
    r.J = 0.0;
}

}  // namespace

#define FCM_CAT2(a, b) a##b
#define FCM_CAT(a, b) FCM_CAT2(a, b)
RoundsKernel FCM_CAT(rounds_kernel_, FCM_ROUNDS_NT)() {
    return RoundsKernel{k_fcm_rounds, k_rounds_init};
}

}  // namespace fcm
