// Histogram-domain FCM on batches of 8-bit slices, with the pixel passes
// spread over the whole GPU.
//
// Each run is one start of Algorithm 1 (arXiv:1601.00072, Sec. 2.1) on one
// slice, carried out on the slice's 256-bin grey-level histogram (the brFCM
// reduction the paper cites, Sec. 3): under Eq. 4 a pixel's memberships depend
// only on its grey level, so after V^1 every iteration is a loop over the
// bins, with the iterates of the per-pixel run up to the order of rounding.
//
// Kernels, in stream order (each pixel pass takes one CTA per BIN_CHUNK
// pixels of any slice, so a large slice is shared by many SMs):
//   A  histogram, input checks, one pixel index per grey level, and the
//      per-chunk sums of V^1 (Eq. 3) for slices started from U^0;
//   S0 per run (one CTA, a thread per grey level): V^1, then the first stopping quantity
//      delta_1 = max_i |f(x_i, V^1) - U^0_i| is bounded from below by the
//      recorded pixel of every grey level; when that bound already reaches
//      eps, the first iteration cannot stop and the run proceeds on the bins;
//   B  only for runs whose bound could not decide: delta_1 exactly, over all
//      pixels (it is needed when U^0 is close to a fixed point, or when
//      max_iter is 1);
//   S1 the runs of B, with the exact delta_1;
//   C  U^k by table lookup for the runs that write their slice.
// The results are those of the exact algorithm: the bound only skips pass B
// when it proves the stop decision it would feed. The pixel sums of V^1 run in
// FP32 over a few pixels, then in compensated FP32 (double-float) per thread,
// warp, CTA and chunk, merged in chunk order: the iterates do not depend on
// the schedule. The bin loop sums 256 non-negative terms in FP32 within each
// warp (a fixed tree, at most five roundings), then across the eight warps in
// double-float.
#include <cstring>
#include <vector>

#include "fcm_batched.h"
#include "fcm_bounds.cuh"
#include "fcm_device.cuh"
#include "fcm_df.cuh"
#include "fcm_hist_bins.cuh"
#include "fcm_runtime.h"

namespace fcm {
namespace {

constexpr int BNT = HNT;                 // threads of every kernel here (one per grey level)
constexpr unsigned BAD_BOUNDS = 4u;      // bit 2 of BinArgs::bad
constexpr int BNW = BNT / 32;
constexpr int PX_PER_THREAD = BIN_CHUNK / BNT;
// pixels per thread whose loads pass A issues together: more for fewer
// clusters (each pixel loads x and C memberships), as many as fit in the
// registers of three CTAs per SM without spilling
template <int C>
constexpr int loads_a() { return C <= 3 ? 8 : (C == 4 ? 6 : 4); }
constexpr int LOADS_C = 8;               // pixels per thread whose x loads pass C issues together

__device__ __forceinline__ float uint_to_floatbits(unsigned u) { return __uint_as_float(u); }

// ---------------------------------------------------------------------------
// Pass A
// ---------------------------------------------------------------------------

struct PassAShared {
    unsigned sub[BNW][256];  // per-warp histograms (less contention on busy bins)
    int rep[256];
    DF wsum[BNW][2 * FCM_MAX_CLUSTERS];
};

template <int C, int MK>
__device__ __noinline__ void pass_a_chunk(const BinArgs& a, const SliceDesc& d, int s, int k, int lo, int hi,
                                          bool from_u, PassAShared& sh) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float* __restrict__ x = d.x;
    const float* __restrict__ U0 = d.U0;
    const int64_t n = d.n;
    const float m = d.m;
    DF acc[2 * C];
#pragma unroll
    for (int q = 0; q < 2 * C; ++q) acc[q] = DF{0.0f, 0.0f};
    bool bad_x = false, bad_u = false;
    unsigned* hw = sh.sub[warp];
    constexpr int LOADS = loads_a<C>();
    for (int i0 = lo + t; i0 < hi; i0 += BNT * LOADS) {
        float xc[LOADS], uc[LOADS][C];
#pragma unroll
        for (int q = 0; q < LOADS; ++q) {
            const int i = i0 + q * BNT;
            const bool in = i < hi;
            xc[q] = in ? __ldg(x + i) : 0.0f;
#pragma unroll
            for (int j = 0; j < C; ++j) uc[q][j] = (in && from_u) ? __ldg(U0 + (int64_t)j * n + i) : 0.0f;
        }
        float num[C], den[C];
#pragma unroll
        for (int j = 0; j < C; ++j) num[j] = den[j] = 0.0f;
#pragma unroll
        for (int q = 0; q < LOADS; ++q) {
            const int i = i0 + q * BNT;
            if (i >= hi) break;
            const float xi = xc[q];
            const int g = grey_index(xi);
            bad_x |= g < 0;
            if (g < 0) continue;
            atomicAdd(&hw[g], 1u);
            sh.rep[g] = i;  // any pixel of the grey level will do
            if (from_u) {
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float u0 = uc[q][j];
                    bad_u |= !(u0 >= 0.0f) || !finite_f(u0);
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
    if (from_u) {
#pragma unroll
        for (int q = 0; q < 2 * C; ++q) {
            const DF dd = warp_sum_df(acc[q]);
            if (lane == 0) sh.wsum[warp][q] = dd;
        }
    }
    // bit 0: some x is not a grey level; bit 1: U^0 has a negative or non-finite value
    const int bx = __syncthreads_or(bad_x), bu = __syncthreads_or(bad_u);
    if ((bx || bu) && t == 0) atomicOr(&a.bad[s], (bx ? 1u : 0u) | (bu ? 2u : 0u));
    {
        unsigned c = 0;
#pragma unroll
        for (int w = 0; w < BNW; ++w) c += sh.sub[w][t];
        if (c) atomicAdd(&a.hist[(int64_t)s * 256 + t], c);
        if (sh.rep[t] >= 0) a.rep[(int64_t)s * 256 + t] = sh.rep[t];
    }
    if (from_u && t < 2 * C) {
        DF tot = sh.wsum[0][t];
        for (int w = 1; w < BNW; ++w) tot = df_merge(tot, sh.wsum[w][t]);
        a.part[(int64_t)k * 2 * FCM_MAX_CLUSTERS + t] = make_float2(tot.hi, tot.lo);
    }
}

__global__ void __launch_bounds__(BNT, 3) k_bins_pass_a(BinArgs a) {
    __shared__ PassAShared sh;
    const int k = blockIdx.x;
    if (k >= a.n_chunks) return;
    const BinChunk ch = a.chunks[k];
    const int s = ch.slice;
    const SliceDesc& d = a.descs[s];
    const int lo = ch.lo, hi = (int)min((int64_t)lo + BIN_CHUNK, d.n);
    const bool from_u = a.slice_urun[s] >= 0;
    for (int i = threadIdx.x; i < BNW * 256; i += BNT) (&sh.sub[0][0])[i] = 0u;
    sh.rep[threadIdx.x] = -1;
    __syncthreads();
#define FCM_BINS_A(CC)                                                                        \
    case CC:                                                                                  \
        switch (d.mk) {                                                                       \
            case M_TWO: pass_a_chunk<CC, M_TWO>(a, d, s, k, lo, hi, from_u, sh); break;       \
            case M_THREE: pass_a_chunk<CC, M_THREE>(a, d, s, k, lo, hi, from_u, sh); break;   \
            case M_ONE_HALF: pass_a_chunk<CC, M_ONE_HALF>(a, d, s, k, lo, hi, from_u, sh); break; \
            default: pass_a_chunk<CC, M_GENERIC>(a, d, s, k, lo, hi, from_u, sh); break;      \
        }                                                                                     \
        break;
    switch (d.C) {
        FCM_BINS_A(1)
        FCM_BINS_A(2)
        FCM_BINS_A(3)
        FCM_BINS_A(4)
        FCM_BINS_A(5)
        FCM_BINS_A(6)
        FCM_BINS_A(7)
        FCM_BINS_A(8)
        default: break;
    }
#undef FCM_BINS_A
}

// ---------------------------------------------------------------------------
// Solve: one CTA per run, thread b holding grey level b
// ---------------------------------------------------------------------------

constexpr int SNT = HNT;

template <int C, int MK>
__device__ __noinline__ void solve_run(const BinArgs& a, int r, const BinRun& run, const SliceDesc& d,
                                       BinScratch& sc, DF* s_tot) {
    const int s = run.slice, b = threadIdx.x;
    const bool from_u = run.init == BIN_FROM_U;
    const float m = d.m, inv_m1 = d.inv_m1;
    SliceResult& res = a.results[r];
    float v0[C];
#pragma unroll
    for (int j = 0; j < C; ++j)
        v0[j] = run.init == BIN_FROM_V_DEV ? a.v0_dev[(int64_t)s * a.v0_stride + j]
                                           : (run.init == BIN_FROM_V ? d.V0[j] : 0.0f);
    // a run from U^0 needs good x and U^0; a run from centers only good x
    bool bad = (a.bad[s] & (from_u ? 3u : 1u)) != 0u;
    if (!from_u) {
#pragma unroll
        for (int j = 0; j < C; ++j) bad |= !finite_f(v0[j]);
    }
    if (bad) {
        // not a grey-level slice (or a bad U^0 / V^0): the status, and V = V^0
        if (b < C) {
            if (run.write_u) d.V[b] = v0[b];
            res.V64[b] = v0[b];
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
    const float cnt = (float)a.hist[(int64_t)s * 256 + b];
    int par = 0, flags = 0;
    float v[C], up[C];
    DF v64[C];

    // ---- V^1 (Eq. 3): from the chunk sums of pass A, or from the bins with U^0 = f(b, V^0) ----
    if (from_u) {
        // thread q < 2C merges sum q over the slice's chunks, in chunk order
        if (b < 2 * C) {
            DF mine{0.0f, 0.0f};
            for (int c = a.chunk_base[s]; c < a.chunk_base[s + 1]; ++c) {
                const float2 p = a.part[(int64_t)c * 2 * FCM_MAX_CLUSTERS + b];
                mine = df_merge(mine, DF{p.x, p.y});
            }
            s_tot[b] = mine;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < C; ++j) {
            up[j] = 0.0f;
            if (s_tot[C + j].hi > 0.0f) {
                v64[j] = df_div(s_tot[j], s_tot[C + j]);
                v[j] = v64[j].hi;
            } else {
                v[j] = v0[j];  // an empty cluster keeps 0 from a U^0
                v64[j] = DF{v0[j], 0.0f};
                flags = FCM_FLAG_EMPTY_CLUSTER;
            }
        }
    } else {
        float um[C], t[2 * C + 1], dummy;
        DF tot[2 * C];
        membership<C, MK>((float)b, v0, m, inv_m1, up, um);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            t[j] = cnt * (um[j] * (float)b);
            t[C + j] = cnt * um[j];
        }
        t[2 * C] = 0.0f;
        block_sums<2 * C>(sc, par, t, tot, dummy);
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (tot[C + j].hi > 0.0f) {
                v64[j] = df_div(tot[j], tot[C + j]);
                v[j] = v64[j].hi;
            } else {
                v[j] = v0[j];  // an empty cluster keeps V^0
                v64[j] = DF{v0[j], 0.0f};
                flags = FCM_FLAG_EMPTY_CLUSTER;
            }
        }
    }
    float* T = a.table + (int64_t)r * 256 * FCM_MAX_CLUSTERS;

    // ---- the first stopping quantity, from U^0 ----
    float d1 = 0.0f;
    if (from_u) {
        if (a.phase == 0) {
            // U^1 per grey level, kept for pass B; the recorded pixel of each
            // grey level gives a lower bound of delta_1
            float u1[C], um1[C], t[2], lb;
            DF tot[1];
            membership<C, MK>((float)b, v, m, inv_m1, u1, um1);
#pragma unroll
            for (int j = 0; j < C; ++j) T[b * FCM_MAX_CLUSTERS + j] = u1[j];
            t[0] = 0.0f;
            t[1] = 0.0f;
            const int rp = a.rep[(int64_t)s * 256 + b];
            if (rp >= 0) {
#pragma unroll
                for (int j = 0; j < C; ++j) t[1] = fmaxf(t[1], fabsf(u1[j] - __ldg(d.U0 + (int64_t)j * d.n + rp)));
            }
            block_sums<1>(sc, par, t, tot, lb);
            if (!(lb >= d.eps) || d.max_iter == 1) {
                if (b == 0) a.need_b[r] = 1;  // pass B takes delta_1 over every pixel; S1 resumes
                return;
            }
            d1 = lb;  // proves delta_1 >= eps: the run goes on to iteration 2
        } else {
            d1 = uint_to_floatbits(a.d1[r]);
        }
    }

    // ---- iterations on the bins ----
    int k, status;
    float delta;
    DF J;
    solve_bins<C, MK>(sc, par, cnt, from_u, d1, v, v64, up, m, inv_m1, d.eps, d.max_iter, flags, k, status, delta, J);
#pragma unroll
    for (int j = 0; j < C; ++j) T[b * FCM_MAX_CLUSTERS + j] = up[j];
#pragma unroll
    for (int j = 0; j < C; ++j)
        if (b == j) {
            if (run.write_u) d.V[j] = v[j];
            res.V64[j] = (double)v64[j].hi + (double)v64[j].lo;
        }
    if (b == 0) {
        res.iters = k;
        res.status = status;
        res.flags = flags;
        res.delta = (double)delta;
        res.J = (double)J.hi + (double)J.lo;
    }
}

__global__ void __launch_bounds__(SNT, 2) k_bins_solve(BinArgs a) {
    __shared__ BinScratch sc;
    __shared__ DF s_tot[2 * FCM_MAX_CLUSTERS];
    const int r = blockIdx.x;
    if (r >= a.n_runs) return;
    if (a.phase == 1 && !a.need_b[r]) return;
    const BinRun run = a.runs[r];
    const SliceDesc& d = a.descs[run.slice];
#define FCM_BINS_S(CC)                                                                   \
    case CC:                                                                             \
        switch (d.mk) {                                                                  \
            case M_TWO: solve_run<CC, M_TWO>(a, r, run, d, sc, s_tot); break;          \
            case M_THREE: solve_run<CC, M_THREE>(a, r, run, d, sc, s_tot); break;      \
            case M_ONE_HALF: solve_run<CC, M_ONE_HALF>(a, r, run, d, sc, s_tot); break; \
            default: solve_run<CC, M_GENERIC>(a, r, run, d, sc, s_tot); break;         \
        }                                                                                \
        break;
    switch (d.C) {
        FCM_BINS_S(1)
        FCM_BINS_S(2)
        FCM_BINS_S(3)
        FCM_BINS_S(4)
        FCM_BINS_S(5)
        FCM_BINS_S(6)
        FCM_BINS_S(7)
        FCM_BINS_S(8)
        default: break;
    }
#undef FCM_BINS_S
}

// ---------------------------------------------------------------------------
// Pass B: delta_1 over every pixel, for the runs that need it
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BNT) k_bins_pass_b(BinArgs a) {
    __shared__ float T[256 * FCM_MAX_CLUSTERS];
    __shared__ float wmax[BNW];
    const int k = blockIdx.x;
    if (k >= a.n_chunks) return;
    const BinChunk ch = a.chunks[k];
    const int r = a.slice_urun[ch.slice];
    if (r < 0 || !a.need_b[r]) return;
    const SliceDesc& d = a.descs[ch.slice];
    const int C = d.C;
    const float* Tg = a.table + (int64_t)r * 256 * FCM_MAX_CLUSTERS;
    for (int i = threadIdx.x; i < 256 * FCM_MAX_CLUSTERS; i += BNT) T[i] = Tg[i];
    __syncthreads();
    const int lo = ch.lo, hi = (int)min((int64_t)lo + BIN_CHUNK, d.n);
    float mx = 0.0f;
    for (int i = lo + threadIdx.x; i < hi; i += BNT) {
        const int g = (int)__ldg(d.x + i);  // grey levels only: pass A checked them
        if (!in_bounds(g >= 0 && g < 256, &a.bad[ch.slice], BAD_BOUNDS)) continue;
        for (int j = 0; j < C; ++j) mx = fmaxf(mx, fabsf(T[g * FCM_MAX_CLUSTERS + j] - __ldg(d.U0 + (int64_t)j * d.n + i)));
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = wmax[0];
        for (int w = 1; w < BNW; ++w) t = fmaxf(t, wmax[w]);
        atomicMax(&a.d1[r], __float_as_uint(t));  // non-negative floats order as their bits
    }
}

// ---------------------------------------------------------------------------
// Pass C: U^k by table lookup
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BNT) k_bins_pass_c(BinArgs a) {
    __shared__ float T[256 * FCM_MAX_CLUSTERS];
    const int k = blockIdx.x;
    if (k >= a.n_chunks) return;
    const BinChunk ch = a.chunks[k];
    const int r = a.slice_wrun[ch.slice];
    if (r < 0 || a.results[r].status < 0) return;  // nothing to write, or a rejected slice
    const SliceDesc& d = a.descs[ch.slice];
    const int C = d.C;
    const float* Tg = a.table + (int64_t)r * 256 * FCM_MAX_CLUSTERS;
    for (int i = threadIdx.x; i < 256 * FCM_MAX_CLUSTERS; i += BNT) T[i] = Tg[i];
    __syncthreads();
    const int lo = ch.lo, hi = (int)min((int64_t)lo + BIN_CHUNK, d.n);
    float* __restrict__ U = d.U;
    for (int i0 = lo + threadIdx.x; i0 < hi; i0 += BNT * LOADS_C) {
        int g[LOADS_C];
#pragma unroll
        for (int q = 0; q < LOADS_C; ++q) {
            const int i = i0 + q * BNT;
            g[q] = i < hi ? (int)__ldg(d.x + i) : 0;
        }
#pragma unroll
        for (int q = 0; q < LOADS_C; ++q) {
            const int i = i0 + q * BNT;
            if (i >= hi) break;
            if (!in_bounds(g[q] >= 0 && g[q] < 256, &a.bad[ch.slice], BAD_BOUNDS)) continue;
            for (int j = 0; j < C; ++j) __stcs(U + (int64_t)j * d.n + i, T[g[q] * FCM_MAX_CLUSTERS + j]);
        }
    }
}

// FCM_DEBUG_BOUNDS builds only, last in stream order: the runs of a slice
// whose guards skipped an access report FCM_FLAG_BOUNDS.
__global__ void k_bins_bounds_flags(BinArgs a) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n_runs; r += gridDim.x * blockDim.x)
        if (a.bad[a.runs[r].slice] & BAD_BOUNDS) a.results[r].flags |= FCM_FLAG_BOUNDS;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct BinWorkspace {
    int slice_cap = 0, chunk_cap = 0, run_cap = 0;
    // device, per slice
    unsigned* hist = nullptr;
    int* rep = nullptr;
    unsigned* bad = nullptr;
    int* slice_ints = nullptr;  // chunk_base [n + 1], then the U^0 run and the writing run of each slice
    // device, per chunk
    BinChunk* chunks = nullptr;
    float2* part = nullptr;
    // device, per run
    BinRun* runs = nullptr;
    float* table = nullptr;
    unsigned* d1 = nullptr;
    int* need_b = nullptr;
    SliceResult* results = nullptr;
    // pinned host staging of the tables uploaded before each batch
    BinChunk* h_chunks = nullptr;
    int* h_slice_ints = nullptr;  // the same, staged
    BinRun* h_runs = nullptr;
};

}  // namespace fcm

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call); \
    } while (0)

namespace fcm {

void release_bins(fcm_ctx* h) {
    if (!h || !h->bins) return;
    BinWorkspace* w = h->bins;
    void* dev[] = {w->hist, w->rep, w->bad, w->slice_ints, w->chunks,
                   w->part, w->runs, w->table, w->d1, w->need_b, w->results};
    for (void* p : dev) cudaFree(p);
    void* host[] = {w->h_chunks, w->h_slice_ints, w->h_runs};
    for (void* p : host) cudaFreeHost(p);
    delete w;
    h->bins = nullptr;
}

namespace {

// Frees a buffer and allocates it again with `count` elements.
template <typename T>
int regrow_dev(fcm_ctx* h, T** p, size_t count) {
    cudaFree(*p);
    *p = nullptr;
    CK(dev_malloc(h, p, sizeof(T) * count));
    return 0;
}
template <typename T>
int regrow_host(fcm_ctx* h, T** p, size_t count) {
    cudaFreeHost(*p);
    *p = nullptr;
    CK(host_malloc(h, p, sizeof(T) * count));
    return 0;
}

int ensure_bins(fcm_ctx* h, int ns, int nc, int nr) {
    if (!h->bins) h->bins = new BinWorkspace();
    BinWorkspace* w = h->bins;
    int rc = 0;
    if (w->slice_cap < ns) {
        const int cap = ns < 64 ? 64 : ns;
        w->slice_cap = 0;  // stays 0 until every buffer below is in place
        if ((rc = regrow_dev(h, &w->hist, (size_t)cap * 256)) || (rc = regrow_dev(h, &w->rep, (size_t)cap * 256)) ||
            (rc = regrow_dev(h, &w->bad, cap)) || (rc = regrow_dev(h, &w->slice_ints, 3 * (size_t)cap + 1)) ||
            (rc = regrow_host(h, &w->h_slice_ints, 3 * (size_t)cap + 1)))
            return rc;
        w->slice_cap = cap;
    }
    if (w->chunk_cap < nc) {
        const int cap = nc + nc / 4 + 64;
        w->chunk_cap = 0;
        if ((rc = regrow_dev(h, &w->chunks, cap)) || (rc = regrow_dev(h, &w->part, (size_t)cap * 2 * FCM_MAX_CLUSTERS)) ||
            (rc = regrow_host(h, &w->h_chunks, cap)))
            return rc;
        w->chunk_cap = cap;
    }
    if (w->run_cap < nr) {
        const int cap = nr < 64 ? 64 : nr;
        w->run_cap = 0;
        if ((rc = regrow_dev(h, &w->runs, cap)) ||
            (rc = regrow_dev(h, &w->table, (size_t)cap * 256 * FCM_MAX_CLUSTERS)) ||
            (rc = regrow_dev(h, &w->d1, cap)) || (rc = regrow_dev(h, &w->need_b, cap)) ||
            (rc = regrow_dev(h, &w->results, cap)) || (rc = regrow_host(h, &w->h_runs, cap)))
            return rc;
        w->run_cap = cap;
    }
    return 0;
}

}  // namespace

int bins_run(fcm_ctx* h, const SliceDesc* h_desc, const SliceDesc* d_desc, int ns, const BinRun* runs, int nr,
             const float* v0_dev, int v0_stride, SliceResult* h_results) {
    int64_t nc64 = 0;
    for (int s = 0; s < ns; ++s) nc64 += (h_desc[s].n + BIN_CHUNK - 1) / BIN_CHUNK;
    if (nc64 > (1 << 30)) return ctx_invalid(h, "batch too large for the histogram-domain run");
    const int nc = (int)nc64;
    int rc = ensure_bins(h, ns, nc, nr);
    if (rc) return rc;
    BinWorkspace* w = h->bins;
    int* base = w->h_slice_ints;
    int* urun = base + (ns + 1);
    int* wrun = urun + ns;
    int k = 0;
    for (int s = 0; s < ns; ++s) {
        base[s] = k;
        for (int64_t lo = 0; lo < h_desc[s].n; lo += BIN_CHUNK) w->h_chunks[k++] = BinChunk{s, (int)lo};
        urun[s] = wrun[s] = -1;
    }
    base[ns] = k;
    bool write_any = false;
    for (int r = 0; r < nr; ++r) {
        const BinRun& q = runs[r];
        if (q.slice < 0 || q.slice >= ns) return ctx_invalid(h, "bin run: bad slice index");
        if (q.init == BIN_FROM_U) {
            if (urun[q.slice] >= 0) return ctx_invalid(h, "bin runs: two starts from U^0 of one slice");
            urun[q.slice] = r;
        }
        if (q.write_u) {
            if (wrun[q.slice] >= 0) return ctx_invalid(h, "bin runs: two runs write one slice");
            wrun[q.slice] = r;
            write_any = true;
        }
        w->h_runs[r] = q;
    }
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(w->chunks, w->h_chunks, sizeof(BinChunk) * nc, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->slice_ints, base, sizeof(int) * (3 * (size_t)ns + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(w->runs, w->h_runs, sizeof(BinRun) * nr, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w->hist, 0, sizeof(unsigned) * 256 * (size_t)ns, st));
    CK(cudaMemsetAsync(w->rep, 0xff, sizeof(int) * 256 * (size_t)ns, st));  // -1: no pixel yet
    CK(cudaMemsetAsync(w->bad, 0, sizeof(unsigned) * ns, st));
    CK(cudaMemsetAsync(w->d1, 0, sizeof(unsigned) * nr, st));
    CK(cudaMemsetAsync(w->need_b, 0, sizeof(int) * nr, st));
    BinArgs a;
    std::memset(&a, 0, sizeof(a));
    a.descs = d_desc;
    a.chunks = w->chunks;
    a.chunk_base = w->slice_ints;
    a.runs = w->runs;
    a.slice_urun = w->slice_ints + (ns + 1);
    a.slice_wrun = w->slice_ints + (2 * ns + 1);
    a.v0_dev = v0_dev;
    a.v0_stride = v0_stride;
    a.n_slices = ns;
    a.n_chunks = nc;
    a.n_runs = nr;
    a.hist = w->hist;
    a.rep = w->rep;
    a.bad = w->bad;
    a.part = w->part;
    a.table = w->table;
    a.d1 = w->d1;
    a.need_b = w->need_b;
    a.results = w->results;
    CK(launch_bins(a, write_any, st));
    if (h_results) CK(cudaMemcpyAsync(h_results, w->results, sizeof(SliceResult) * nr, cudaMemcpyDeviceToHost, st));
    return 0;
}

cudaError_t launch_bins(const BinArgs& a0, bool write_any, cudaStream_t s) {
    BinArgs a = a0;
    a.phase = 0;
    if (a.n_chunks > 0) k_bins_pass_a<<<a.n_chunks, BNT, 0, s>>>(a);
    k_bins_solve<<<a.n_runs, SNT, 0, s>>>(a);
    if (a.n_chunks > 0) k_bins_pass_b<<<a.n_chunks, BNT, 0, s>>>(a);
    a.phase = 1;
    k_bins_solve<<<a.n_runs, SNT, 0, s>>>(a);
    if (write_any && a.n_chunks > 0) k_bins_pass_c<<<a.n_chunks, BNT, 0, s>>>(a);
    if (kBoundsChecks && a.n_runs > 0) k_bins_bounds_flags<<<(a.n_runs + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fcm
