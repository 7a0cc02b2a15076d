// Learned warm start: a small network from a slice's grey-level histogram to
// initial centers V^0, trained and run on the GPU by the kernels below. The
// paper starts from random memberships (Algorithm 1 step 2); this is an
// addition of this library, judged by how many FCM iterations it saves.
//
//   f  = [histogram / n (256 bins of round(clip(x, 0, 255))), onehot(C) (8)]
//   a1 = GELU(W1 f + b1)   (128)      a2 = GELU(W2 a1 + b2)   (128)
//   y  = W3 a2 + b3        (8)        V^0 = sort(255 * y[:C])
//   loss = sum_{b, j < C_b} (y_bj - t_bj)^2 / sum_b C_b
//
// Weights W[out, in] are kept as FP32 master copies (updated by Adam) and
// used as BF16 in every product; activations, accumulation, gradients and
// optimiser state are FP32. The products are small (batch <= a few hundred,
// widths <= 264): a shared-memory tiled SIMT GEMM with fused bias/GELU
// epilogues covers them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "fcm.h"
#include "fcm_batched.h"
#include "fcm_runtime.h"

using namespace fcm;

namespace fcm {

constexpr int D_HIST = 256, D_ONE = 8, D_IN = D_HIST + D_ONE, D_H = 128, D_OUT = 8;
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + D_H * D_IN, OFF_W2 = OFF_B1 + D_H, OFF_B2 = OFF_W2 + D_H * D_H,
                  OFF_W3 = OFF_B2 + D_H, OFF_B3 = OFF_W3 + D_OUT * D_H, N_PARAMS = OFF_B3 + D_OUT;
static_assert(N_PARAMS == FCM_MODEL_PARAMS, "parameter count");

struct MlpWorkspace {
    bool ready = false;
    float* master = nullptr;   // FP32 parameters
    __nv_bfloat16* wbf = nullptr;  // BF16 copies used in the products
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    int64_t step = 0;
    int bcap = 0;
    float *xb = nullptr, *tb = nullptr, *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr,
          *dy = nullptr, *dz2 = nullptr, *dz1 = nullptr, *loss = nullptr;
    int* cb = nullptr;
    int* idx = nullptr;
    int idx_cap = 0;
    // features of the slices of one predict call
    float* feats = nullptr;
    int feat_cap = 0;
    void* hdesc_dev = nullptr;
    int hdesc_cap = 0;
    float* v0 = nullptr;  // [feat_cap][9]: sorted initial centers and a usability flag
    // warm-started batches: the predictions and the judge's results, pinned
    float* h_v0 = nullptr;            // [judge_cap][9]
    SliceResult* h_judge = nullptr;   // [2 * judge_cap]: cold runs, then warm runs
    int judge_cap = 0;
    unsigned* counts = nullptr;  // [counts_cap][256] grey-level counters, kept zero between calls
    int counts_cap = 0;
    std::unordered_set<const void*> known_device;  // slice x pointers already checked
};

}  // namespace fcm

namespace {

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

template <typename T>
__device__ __forceinline__ float ld(const T* p, int64_t i);
template <>
__device__ __forceinline__ float ld<float>(const float* p, int64_t i) {
    return p[i];
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
    return __bfloat162float(p[i]);
}

enum Epi : int { E_NONE = 0, E_BIAS = 1, E_BIAS_GELU = 2, E_GELU_GRAD = 3 };

// C[m, n] = sum_k A(m, k) B(k, n), A(m, k) = A[m * as_m + k * as_k], likewise
// B. Epilogues: + bias[n]; + bias[n] then GELU (Z and A both stored); times
// GELU'(Z[m, n]) (backward through a GELU). 32 x 32 output tile per block,
// 256 threads with 2 x 2 outputs each, K in steps of 32 through shared memory.
constexpr int TT = 32;
template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(const TA* __restrict__ A, int64_t as_m, int64_t as_k,
                                              const TB* __restrict__ B, int64_t bs_k, int64_t bs_n, int M, int N,
                                              int K, const float* __restrict__ bias, const float* __restrict__ Zin,
                                              float* __restrict__ Cout, float* __restrict__ Aout, int ldc) {
    __shared__ float sa[TT][TT + 1], sb[TT][TT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * TT, n0 = blockIdx.x * TT;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += TT) {
        for (int t = threadIdx.x; t < TT * TT; t += 256) {
            const int r = t / TT, c = t % TT;
            const int m = m0 + r, k = k0 + c;
            sa[r][c] = (m < M && k < K) ? ld<TA>(A, (int64_t)m * as_m + (int64_t)k * as_k) : 0.0f;
            const int kk = k0 + r, n = n0 + c;
            sb[r][c] = (kk < K && n < N) ? ld<TB>(B, (int64_t)kk * bs_k + (int64_t)n * bs_n) : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TT; ++k) {
            const float a0 = sa[ty * 2][k], a1 = sa[ty * 2 + 1][k];
            const float b0 = sb[k][tx * 2], b1 = sb[k][tx * 2 + 1];
            acc[0][0] = fmaf(a0, b0, acc[0][0]);
            acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]);
            acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
            if (m >= M || n >= N) continue;
            float v = acc[i][j];
            const int64_t o = (int64_t)m * ldc + n;
            if (EPI == E_BIAS || EPI == E_BIAS_GELU) v += bias[n];
            if (EPI == E_GELU_GRAD) v *= gelu_grad(Zin[o]);
            Cout[o] = v;
            if (EPI == E_BIAS_GELU) Aout[o] = gelu(v);
        }
}

// db[n] = sum_m dZ[m, n], in a fixed order.
__global__ void k_colsum(const float* __restrict__ dZ, int M, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += dZ[(int64_t)m * N + n];
    db[n] = s;
}

// Masked MSE and its gradient dY (one block, fixed-order reduction).
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, const int* __restrict__ Cs, int B,
                       float* __restrict__ dY, float* __restrict__ loss) {
    __shared__ float s_l[256], s_c[256];
    float l = 0.0f, c = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) c += (float)Cs[b];
    s_c[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_c[threadIdx.x] += s_c[threadIdx.x + o];
        __syncthreads();
    }
    const float cnt = s_c[0];
    for (int t = threadIdx.x; t < B * D_OUT; t += blockDim.x) {
        const int b = t / D_OUT, j = t % D_OUT;
        const float r = j < Cs[b] ? Y[t] - T[t] : 0.0f;
        dY[t] = 2.0f * r / cnt;
        l = fmaf(r, r, l);
    }
    s_l[threadIdx.x] = l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_l[threadIdx.x] += s_l[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s_l[0] / cnt;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wbf, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wbf[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wbf[i] = __float2bfloat16_rn(w[i]);
}

// Rows idx[r] of the feature, target and C arrays into contiguous batches.
__global__ void k_gather(const float* __restrict__ F, const float* __restrict__ T, const int* __restrict__ Cs,
                         const int* __restrict__ idx, int B, float* __restrict__ Fb, float* __restrict__ Tb,
                         int* __restrict__ Cb) {
    const int r = blockIdx.x;
    if (r >= B) return;
    const int64_t s = idx[r];
    for (int t = threadIdx.x; t < D_IN; t += blockDim.x) Fb[(int64_t)r * D_IN + t] = F[s * D_IN + t];
    if (threadIdx.x < D_OUT) Tb[(int64_t)r * D_OUT + threadIdx.x] = T[s * D_OUT + threadIdx.x];
    if (threadIdx.x == 0) Cb[r] = Cs[s];
}

struct HistDesc {
    const float* x;
    int64_t n;
    int C;
    int pad;
};

// Histogram features in two steps. k_hist_counts: block (s, c) counts the
// grey levels round(clip(x)) of chunk c (FEAT_CHUNK pixels) of slice s in
// shared memory and adds them to the slice's 256 counters; non-finite pixels
// count in no bin. k_features: one block per slice turns its counters into
// the normalised histogram and onehot(C), and clears them for the next call.
constexpr int FEAT_CHUNK = 32768;

__global__ void k_hist_counts(const HistDesc* __restrict__ d, int ns, unsigned* __restrict__ counts) {
    __shared__ unsigned int h[D_HIST];
    const int s = blockIdx.x;
    const int64_t lo = (int64_t)blockIdx.y * FEAT_CHUNK;
    if (s >= ns || lo >= d[s].n) return;
    for (int b = threadIdx.x; b < D_HIST; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const float* x = d[s].x;
    const int64_t hi = min(d[s].n, lo + FEAT_CHUNK);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float v = __ldg(x + i);
        if (!(v == v) || fabsf(v) == __int_as_float(0x7f800000)) continue;
        const int b = (int)fminf(fmaxf(rintf(v), 0.0f), 255.0f);
        atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < D_HIST; b += blockDim.x)
        if (h[b]) atomicAdd(&counts[(int64_t)s * D_HIST + b], h[b]);
}

__global__ void k_features(const HistDesc* __restrict__ d, int ns, unsigned* __restrict__ counts,
                           float* __restrict__ F) {
    const int s = blockIdx.x;
    if (s >= ns) return;
    const float inv = 1.0f / (float)d[s].n;
    float* f = F + (int64_t)s * D_IN;
    unsigned* c = counts + (int64_t)s * D_HIST;
    for (int b = threadIdx.x; b < D_HIST; b += blockDim.x) {
        f[b] = (float)c[b] * inv;
        c[b] = 0u;
    }
    if (threadIdx.x < D_ONE) f[D_HIST + threadIdx.x] = (threadIdx.x == d[s].C - 1) ? 1.0f : 0.0f;
}

// Initial centers from the network output, one thread per slice: the first C
// outputs times 255, sorted ascending (insertion sort of at most 8), and a flag
// telling whether they can start a run (all finite, neighbours more than 1e-3
// apart). Row s of P holds V0[0..7] then the flag (1 or 0).
__global__ void k_v0(const HistDesc* __restrict__ d, const float* __restrict__ y, int ns, float* __restrict__ P) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int C = d[s].C;
    float v[D_OUT];
#pragma unroll
    for (int j = 0; j < D_OUT; ++j) v[j] = j < C ? 255.0f * y[(int64_t)s * D_OUT + j] : 0.0f;
    bool ok = true;
    for (int j = 0; j < C; ++j) ok &= (v[j] == v[j]) && fabsf(v[j]) != __int_as_float(0x7f800000);
    for (int j = 1; j < C; ++j) {
        const float t = v[j];
        int k = j - 1;
        while (k >= 0 && v[k] > t) {
            v[k + 1] = v[k];
            --k;
        }
        v[k + 1] = t;
    }
    for (int j = 1; j < C; ++j) ok &= v[j] - v[j - 1] > 1e-3f;
    float* o = P + (int64_t)s * (D_OUT + 1);
#pragma unroll
    for (int j = 0; j < D_OUT; ++j) o[j] = v[j];
    o[D_OUT] = ok ? 1.0f : 0.0f;
}

}  // namespace

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ctx_fail(h, e_, #call); \
    } while (0)

namespace {

dim3 tiles(int M, int N) { return dim3((N + TT - 1) / TT, (M + TT - 1) / TT); }

int ensure_mlp(fcm_ctx* h, int bcap) {
    if (!h->mlp) h->mlp = new MlpWorkspace();
    MlpWorkspace* w = h->mlp;
    // each buffer is allocated when missing, so a call after a failed
    // allocation completes the workspace
    if (!w->master) CK(dev_malloc(h, &w->master, sizeof(float) * N_PARAMS));
    if (!w->wbf) CK(dev_malloc(h, &w->wbf, sizeof(__nv_bfloat16) * N_PARAMS));
    if (!w->adam_m) CK(dev_malloc(h, &w->adam_m, sizeof(float) * N_PARAMS));
    if (!w->adam_v) CK(dev_malloc(h, &w->adam_v, sizeof(float) * N_PARAMS));
    if (!w->grad) CK(dev_malloc(h, &w->grad, sizeof(float) * N_PARAMS));
    if (!w->loss) CK(dev_malloc(h, &w->loss, sizeof(float)));
    if (w->bcap < bcap) {
        float** bufs[] = {&w->xb, &w->tb, &w->z1, &w->a1, &w->z2, &w->a2, &w->y, &w->dy, &w->dz2, &w->dz1};
        const int64_t sizes[] = {D_IN, D_OUT, D_H, D_H, D_H, D_H, D_OUT, D_OUT, D_H, D_H};
        w->bcap = 0;  // stays 0 until every buffer below is in place
        for (int i = 0; i < 10; ++i) {
            cudaFree(*bufs[i]);
            *bufs[i] = nullptr;
            CK(dev_malloc(h, bufs[i], sizeof(float) * sizes[i] * bcap));
        }
        cudaFree(w->cb);
        w->cb = nullptr;
        CK(dev_malloc(h, &w->cb, sizeof(int) * bcap));
        w->bcap = bcap;
    }
    return 0;
}

// Forward pass of B rows of X (device, row stride D_IN) into w->y.
int forward(fcm_ctx* h, const float* X, int B) {
    MlpWorkspace* w = h->mlp;
    cudaStream_t s = h->stream;
    k_gemm<float, __nv_bfloat16, E_BIAS_GELU><<<tiles(B, D_H), 256, 0, s>>>(
        X, D_IN, 1, w->wbf + OFF_W1, 1, D_IN, B, D_H, D_IN, w->master + OFF_B1, nullptr, w->z1, w->a1, D_H);
    k_gemm<float, __nv_bfloat16, E_BIAS_GELU><<<tiles(B, D_H), 256, 0, s>>>(
        w->a1, D_H, 1, w->wbf + OFF_W2, 1, D_H, B, D_H, D_H, w->master + OFF_B2, nullptr, w->z2, w->a2, D_H);
    k_gemm<float, __nv_bfloat16, E_BIAS><<<tiles(B, D_OUT), 256, 0, s>>>(
        w->a2, D_H, 1, w->wbf + OFF_W3, 1, D_H, B, D_OUT, D_H, w->master + OFF_B3, nullptr, w->y, nullptr, D_OUT);
    CK(cudaGetLastError());
    return 0;
}

// Loss and gradients (into w->grad) of B rows: X [B, D_IN], T [B, D_OUT], Cs [B].
int backward(fcm_ctx* h, const float* X, const float* T, const int* Cs, int B) {
    MlpWorkspace* w = h->mlp;
    cudaStream_t s = h->stream;
    int rc = forward(h, X, B);
    if (rc) return rc;
    k_loss<<<1, 256, 0, s>>>(w->y, T, Cs, B, w->dy, w->loss);
    // layer 3: dW3 = dY^T a2, db3; dZ2 = (dY W3) * GELU'(z2)
    k_gemm<float, float, E_NONE><<<tiles(D_OUT, D_H), 256, 0, s>>>(
        w->dy, 1, D_OUT, w->a2, D_H, 1, D_OUT, D_H, B, nullptr, nullptr, w->grad + OFF_W3, nullptr, D_H);
    k_colsum<<<1, 128, 0, s>>>(w->dy, B, D_OUT, w->grad + OFF_B3);
    k_gemm<float, __nv_bfloat16, E_GELU_GRAD><<<tiles(B, D_H), 256, 0, s>>>(
        w->dy, D_OUT, 1, w->wbf + OFF_W3, D_H, 1, B, D_H, D_OUT, nullptr, w->z2, w->dz2, nullptr, D_H);
    // layer 2
    k_gemm<float, float, E_NONE><<<tiles(D_H, D_H), 256, 0, s>>>(
        w->dz2, 1, D_H, w->a1, D_H, 1, D_H, D_H, B, nullptr, nullptr, w->grad + OFF_W2, nullptr, D_H);
    k_colsum<<<1, 128, 0, s>>>(w->dz2, B, D_H, w->grad + OFF_B2);
    k_gemm<float, __nv_bfloat16, E_GELU_GRAD><<<tiles(B, D_H), 256, 0, s>>>(
        w->dz2, D_H, 1, w->wbf + OFF_W2, D_H, 1, B, D_H, D_H, nullptr, w->z1, w->dz1, nullptr, D_H);
    // layer 1
    k_gemm<float, float, E_NONE><<<tiles(D_H, D_IN), 256, 0, s>>>(
        w->dz1, 1, D_H, X, D_IN, 1, D_H, D_IN, B, nullptr, nullptr, w->grad + OFF_W1, nullptr, D_IN);
    k_colsum<<<1, 128, 0, s>>>(w->dz1, B, D_H, w->grad + OFF_B1);
    CK(cudaGetLastError());
    return 0;
}

// splitmix64 (Steele, Lea & Flood 2014) and Box-Muller for the initial weights.
uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

bool device_mem(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int upload_params(fcm_ctx* h, const float* host) {
    MlpWorkspace* w = h->mlp;
    CK(cudaMemcpyAsync(w->master, host, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(w->adam_m, 0, sizeof(float) * N_PARAMS, h->stream));
    CK(cudaMemsetAsync(w->adam_v, 0, sizeof(float) * N_PARAMS, h->stream));
    k_to_bf16<<<(unsigned)((N_PARAMS + 255) / 256), 256, 0, h->stream>>>(w->master, w->wbf, N_PARAMS);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    w->step = 0;
    w->ready = true;
    return 0;
}

// The acceptance rule of a warm-started slice against the cold start: its
// sorted centers within 1e-4 of the cold start's (relative to max(|v|, 1)),
// or a fixed point whose J is no larger (relative slack 1e-5, above the FP32
// kernels' resolution of J). Random starts of the same slice often end at
// different local minima of J (Eq. 1), so a warm start that finds a lower
// minimum than the cold one is as valid a result.
bool warm_accepted(const double* Vw, double Jw, int status_w, const double* Vc, double Jc, int C) {
    double a[FCM_MAX_CLUSTERS], b[FCM_MAX_CLUSTERS];
    for (int j = 0; j < C; ++j) {
        a[j] = Vw[j];
        b[j] = Vc[j];
    }
    std::sort(a, a + C);
    std::sort(b, b + C);
    double err = 0.0;
    for (int j = 0; j < C; ++j) err = std::max(err, std::fabs(a[j] - b[j]) / std::max(std::fabs(b[j]), 1.0));
    if (err <= 1e-4) return true;
    return status_w >= 0 && Jw <= Jc * (1.0 + 1e-5);
}

int need_model(fcm_ctx* h) {
    if (!h->mlp || !h->mlp->ready) return ctx_invalid(h, "no model: call fcm_model_init, _load or _set_params");
    return 0;
}

}  // namespace

void fcm_release_mlp(fcm_ctx* h) {
    if (!h || !h->mlp) return;
    MlpWorkspace* w = h->mlp;
    void* ps[] = {w->master, w->wbf, w->adam_m, w->adam_v, w->grad, w->xb, w->tb, w->z1, w->a1, w->z2,
                  w->a2, w->y, w->dy, w->dz2, w->dz1, w->loss, w->cb, w->idx, w->feats, w->hdesc_dev, w->v0, w->counts};
    for (void* p : ps) cudaFree(p);
    cudaFreeHost(w->h_v0);
    cudaFreeHost(w->h_judge);
    delete w;
    h->mlp = nullptr;
}

int fcm_features_impl(fcm_ctx* h, const fcm_slice* slices, int n, float* feats) {
    if (!h || !slices || n < 1 || !feats) return FCM_ERR_INVALID_ARG;
    if (!device_mem(feats)) return ctx_invalid(h, "features must be device memory");
    DeviceGuard g(h->device);
    int rc = ensure_mlp(h, 1);
    if (rc) return rc;
    MlpWorkspace* w = h->mlp;
    std::vector<HistDesc> d(n);
    for (int i = 0; i < n; ++i) {
        if (!slices[i].x || slices[i].n < 1 || slices[i].C < 1 || slices[i].C > FCM_MAX_CLUSTERS)
            return ctx_invalid(h, "slice: bad x, n or C");
        if (!w->known_device.count(slices[i].x)) {
            if (!device_mem(slices[i].x)) return ctx_invalid(h, "slice: x must be device memory");
            if (w->known_device.size() > (1u << 16)) w->known_device.clear();
            w->known_device.insert(slices[i].x);
        }
        d[i] = HistDesc{slices[i].x, slices[i].n, slices[i].C, 0};
    }
    if (w->hdesc_cap < n) {
        cudaFree(w->hdesc_dev);
        w->hdesc_dev = nullptr;
        w->hdesc_cap = 0;
        CK(dev_malloc(h, &w->hdesc_dev, sizeof(HistDesc) * n));
        w->hdesc_cap = n;
    }
    CK(cudaMemcpyAsync(w->hdesc_dev, d.data(), sizeof(HistDesc) * n, cudaMemcpyHostToDevice, h->stream));
    if (w->counts_cap < n) {
        cudaFree(w->counts);
        w->counts = nullptr;
        w->counts_cap = 0;
        CK(dev_malloc(h, &w->counts, sizeof(unsigned) * D_HIST * n));
        CK(cudaMemsetAsync(w->counts, 0, sizeof(unsigned) * D_HIST * n, h->stream));
        w->counts_cap = n;
    }
    int64_t chunks = 1;
    for (int i = 0; i < n; ++i) chunks = std::max<int64_t>(chunks, (d[i].n + FEAT_CHUNK - 1) / FEAT_CHUNK);
    if (chunks > 65535) return ctx_invalid(h, "slice too large for the feature kernel");
    k_hist_counts<<<dim3((unsigned)n, (unsigned)chunks), 512, 0, h->stream>>>((const HistDesc*)w->hdesc_dev, n,
                                                                              w->counts);
    CK(cudaGetLastError());
    k_features<<<n, 256, 0, h->stream>>>((const HistDesc*)w->hdesc_dev, n, w->counts, feats);
    CK(cudaGetLastError());
    return FCM_OK;
}

// Features, forward pass and k_v0 for a batch, queued on the handle's stream:
// row i of w->v0 receives slice i's sorted V^0 and its usability flag.
int predict_v0_launch(fcm_ctx* h, const fcm_slice* slices, int n) {
    MlpWorkspace* w = h->mlp;
    if (w->feat_cap < n) {
        cudaFree(w->feats);
        cudaFree(w->v0);
        w->feats = nullptr;
        w->v0 = nullptr;
        w->feat_cap = 0;
        CK(dev_malloc(h, &w->feats, sizeof(float) * D_IN * n));
        CK(dev_malloc(h, &w->v0, sizeof(float) * (D_OUT + 1) * n));
        w->feat_cap = n;
    }
    int rc;
    if ((rc = fcm_features_impl(h, slices, n, w->feats))) return rc;
    if ((rc = ensure_mlp(h, n))) return rc;
    if ((rc = forward(h, w->feats, n))) return rc;
    k_v0<<<(n + 127) / 128, 128, 0, h->stream>>>((const HistDesc*)w->hdesc_dev, w->y, n, w->v0);
    CK(cudaGetLastError());
    return FCM_OK;
}

// Features, forward pass and k_v0 for a batch; fills each slice's V0 and sets
// FCM_INIT_V. ok (when given) receives the usability flag of each prediction.
int predict_v0(fcm_ctx* h, fcm_slice* slices, int n, std::vector<unsigned char>* ok) {
    if (!h || !slices || n < 1) return FCM_ERR_INVALID_ARG;
    int rc = need_model(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    if ((rc = predict_v0_launch(h, slices, n))) return rc;
    MlpWorkspace* w = h->mlp;
    std::vector<float> P((size_t)n * (D_OUT + 1));
    CK(cudaMemcpyAsync(P.data(), w->v0, sizeof(float) * P.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (ok) ok->assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const float* r = &P[(size_t)i * (D_OUT + 1)];
        for (int j = 0; j < FCM_MAX_CLUSTERS; ++j) slices[i].V0[j] = j < slices[i].C ? r[j] : 0.0f;
        slices[i].init_mode = FCM_INIT_V;
        if (ok) (*ok)[i] = r[D_OUT] != 0.0f;
    }
    return FCM_OK;
}

extern "C" {

int fcm_model_init(fcm_handle h, uint64_t seed) {
    if (!h) return FCM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    int rc = ensure_mlp(h, 1);
    if (rc) return rc;
    // He-normal weights (std sqrt(2 / fan_in)), zero hidden biases, output
    // biases spread over (0, 1) so an untrained net predicts ordered centers.
    std::vector<float> p(N_PARAMS, 0.0f);
    uint64_t s = seed;
    auto fill = [&](int64_t off, int fan_out, int fan_in) {
        const double sd = std::sqrt(2.0 / fan_in);
        for (int64_t i = 0; i < (int64_t)fan_out * fan_in; ++i) {
            const double u1 = uniform01(s), u2 = uniform01(s);
            p[off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    };
    fill(OFF_W1, D_H, D_IN);
    fill(OFF_W2, D_H, D_H);
    fill(OFF_W3, D_OUT, D_H);
    for (int j = 0; j < D_OUT; ++j) p[OFF_B3 + j] = (float)(j + 1) / (D_OUT + 1);
    return upload_params(h, p.data());
}

int fcm_model_set_params(fcm_handle h, const float* params, int64_t count) {
    if (!h || !params || count != N_PARAMS) return FCM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    int rc = ensure_mlp(h, 1);
    if (rc) return rc;
    return upload_params(h, params);
}

int fcm_model_get_params(fcm_handle h, float* params, int64_t count) {
    if (!h || !params || count != N_PARAMS) return FCM_ERR_INVALID_ARG;
    int rc = need_model(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    CK(cudaMemcpyAsync(params, h->mlp->master, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FCM_OK;
}

int fcm_model_save(fcm_handle h, const char* path) {
    if (!h || !path) return FCM_ERR_INVALID_ARG;
    std::vector<float> p(N_PARAMS);
    int rc = fcm_model_get_params(h, p.data(), N_PARAMS);
    if (rc) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return ctx_invalid(h, "cannot open the model file for writing");
    const int32_t head[5] = {0x57434D46 /* "FMCW" */, 1, D_IN, D_H, D_OUT};
    const bool ok = std::fwrite(head, sizeof(head), 1, f) == 1 &&
                    std::fwrite(p.data(), sizeof(float), N_PARAMS, f) == (size_t)N_PARAMS;
    std::fclose(f);
    return ok ? FCM_OK : ctx_invalid(h, "short write of the model file");
}

int fcm_model_load(fcm_handle h, const char* path) {
    if (!h || !path) return FCM_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return ctx_invalid(h, "cannot open the model file");
    int32_t head[5];
    std::vector<float> p(N_PARAMS);
    const bool ok = std::fread(head, sizeof(head), 1, f) == 1 && head[0] == 0x57434D46 && head[1] == 1 &&
                    head[2] == D_IN && head[3] == D_H && head[4] == D_OUT &&
                    std::fread(p.data(), sizeof(float), N_PARAMS, f) == (size_t)N_PARAMS;
    std::fclose(f);
    if (!ok) return ctx_invalid(h, "not a model file of this network");
    return fcm_model_set_params(h, p.data(), N_PARAMS);
}

int fcm_model_forward(fcm_handle h, const float* feats, int B, float* out) {
    if (!h || !feats || !out || B < 1) return FCM_ERR_INVALID_ARG;
    int rc = need_model(h);
    if (rc) return rc;
    if (!device_mem(feats) || !device_mem(out)) return ctx_invalid(h, "features and output must be device memory");
    DeviceGuard g(h->device);
    if ((rc = ensure_mlp(h, B))) return rc;
    if ((rc = forward(h, feats, B))) return rc;
    CK(cudaMemcpyAsync(out, h->mlp->y, sizeof(float) * B * D_OUT, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FCM_OK;
}

int fcm_model_loss_grad(fcm_handle h, const float* feats, const float* targets, const int* Cs, int B, float* grad,
                        float* loss) {
    if (!h || !feats || !targets || !Cs || B < 1 || !grad || !loss) return FCM_ERR_INVALID_ARG;
    int rc = need_model(h);
    if (rc) return rc;
    if (!device_mem(feats) || !device_mem(targets) || !device_mem(Cs))
        return ctx_invalid(h, "features, targets and C must be device memory");
    DeviceGuard g(h->device);
    if ((rc = ensure_mlp(h, B))) return rc;
    if ((rc = backward(h, feats, targets, Cs, B))) return rc;
    CK(cudaMemcpyAsync(grad, h->mlp->grad, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(loss, h->mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FCM_OK;
}

int fcm_model_train(fcm_handle h, const float* feats, const float* targets, const int* Cs, int n, int epochs,
                    int batch, float lr, uint64_t seed, float* last_loss) {
    NvtxRange nvtx_range("fcm_model_train");
    if (!h || !feats || !targets || !Cs || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
        return FCM_ERR_INVALID_ARG;
    int rc = need_model(h);
    if (rc) return rc;
    if (!device_mem(feats) || !device_mem(targets) || !device_mem(Cs))
        return ctx_invalid(h, "features, targets and C must be device memory");
    DeviceGuard g(h->device);
    batch = std::min(batch, n);
    if ((rc = ensure_mlp(h, batch))) return rc;
    MlpWorkspace* w = h->mlp;
    if (w->idx_cap < n) {
        cudaFree(w->idx);
        w->idx = nullptr;
        w->idx_cap = 0;
        CK(dev_malloc(h, &w->idx, sizeof(int) * n));
        w->idx_cap = n;
    }
    std::vector<int> perm(n);
    uint64_t s = seed;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double epoch_loss = 0.0;
    float lh = 0.0f;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int)(splitmix64(s) % (uint64_t)(i + 1))]);
        CK(cudaMemcpyAsync(w->idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
        epoch_loss = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 + batch <= n; b0 += batch, ++nb) {  // full batches only
            k_gather<<<batch, 128, 0, h->stream>>>(feats, targets, Cs, w->idx + b0, batch, w->xb, w->tb, w->cb);
            if ((rc = backward(h, w->xb, w->tb, w->cb, batch))) return rc;
            ++w->step;
            const float c1 = 1.0f - std::pow(b1, (float)w->step), c2 = 1.0f - std::pow(b2, (float)w->step);
            k_adam<<<(unsigned)((N_PARAMS + 255) / 256), 256, 0, h->stream>>>(w->master, w->grad, w->adam_m,
                                                                               w->adam_v, w->wbf, N_PARAMS, lr, b1,
                                                                               b2, eps, c1, c2);
            if (e == epochs - 1) {
                CK(cudaMemcpyAsync(&lh, w->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
                CK(cudaStreamSynchronize(h->stream));
                epoch_loss += lh;
            }
        }
        CK(cudaGetLastError());
        if (e == epochs - 1 && nb > 0) epoch_loss /= nb;
    }
    CK(cudaStreamSynchronize(h->stream));
    if (last_loss) *last_loss = (float)epoch_loss;
    return FCM_OK;
}

int fcm_features(fcm_handle h, const fcm_slice* slices, int n, float* feats) {
    NvtxRange nvtx_range("fcm_features");
    const int rc = fcm_features_impl(h, slices, n, feats);
    if (rc) return rc;
    DeviceGuard g(h->device);
    CK(cudaStreamSynchronize(h->stream));
    return FCM_OK;
}

int fcm_predict_centers(fcm_handle h, fcm_slice* slices, int n) {
    NvtxRange nvtx_range("fcm_predict_centers");
    return predict_v0(h, slices, n, nullptr);
}

int fcm_run_batched_warm(fcm_handle h, fcm_slice* slices, int n, int options, int* n_cold) {
    NvtxRange nvtx_range("fcm_run_batched_warm");
    if (!h || !slices || n < 1) return FCM_ERR_INVALID_ARG;
    if (n_cold) *n_cold = 0;
    for (int i = 0; i < n; ++i)
        if (!slices[i].U0 || slices[i].U0 == slices[i].U)
            return ctx_invalid(h, "warm-started batch: every slice needs its own U0 (the cold start judges and "
                                  "replaces the warm start)");
    int rc = need_model(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    MlpWorkspace* w = h->mlp;

    // 1. the network's V^0 of every slice, on the device
    if ((rc = predict_v0_launch(h, slices, n))) return rc;

    // 2. the judge: every slice on its grey-level histogram, from its U^0
    //    (plain cold-start FCM) and from the predicted V^0, read from the device
    if (w->judge_cap < n) {
        cudaFreeHost(w->h_v0);
        cudaFreeHost(w->h_judge);
        w->h_v0 = nullptr;
        w->h_judge = nullptr;
        w->judge_cap = 0;
        CK(host_malloc(h, &w->h_v0, sizeof(float) * (D_OUT + 1) * n));
        CK(host_malloc(h, &w->h_judge, sizeof(SliceResult) * 2 * n));
        w->judge_cap = n;
    }
    std::vector<fcm_slice> from_u(slices, slices + n);
    for (fcm_slice& q : from_u) {
        q.init_mode = FCM_INIT_U;
        q.iters_hint = 0;
    }
    SliceDesc *hd = nullptr, *dd = nullptr;
    if ((rc = batch_descs(h, from_u.data(), n, (int64_t)1 << 31, &hd, &dd))) return rc;
    std::vector<BinRun> runs(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        runs[i] = BinRun{i, BIN_FROM_U, 0, 0};
        runs[n + i] = BinRun{i, BIN_FROM_V_DEV, 0, 0};
    }
    if ((rc = bins_run(h, hd, dd, n, runs.data(), 2 * n, w->v0, D_OUT + 1, w->h_judge))) return rc;
    CK(cudaMemcpyAsync(w->h_v0, w->v0, sizeof(float) * (D_OUT + 1) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));

    // 3. a slice starts warm when the prediction is usable and the judge
    //    accepts the fixed point it leads to; the others start cold. Each
    //    slice carries the iterations its start took on the histogram.
    std::vector<const SliceResult*> cold_ref(n, nullptr);
    int64_t hint_sum = 0, hint_cnt = 0;
    for (int i = 0; i < n; ++i) {
        const SliceResult& c = w->h_judge[i];
        const SliceResult& wr = w->h_judge[n + i];
        const float* P = w->h_v0 + (size_t)i * (D_OUT + 1);
        fcm_slice& s = slices[i];
        const bool judged = c.status >= 0;  // a grey-level slice with a valid U^0
        if (judged) cold_ref[i] = &c;
        const bool warm = judged && P[D_OUT] != 0.0f && wr.status == FCM_OK && !(wr.flags & FCM_FLAG_EMPTY_CLUSTER) &&
                          warm_accepted(wr.V64, wr.J, wr.status, c.V64, c.J, s.C);
        for (int j = 0; j < FCM_MAX_CLUSTERS; ++j) s.V0[j] = (warm && j < s.C) ? P[j] : 0.0f;
        s.init_mode = warm ? FCM_INIT_V : FCM_INIT_U;
        s.iters_hint = judged ? (warm ? wr.iters : c.iters) : 0;
        if (s.iters_hint > 0) {
            hint_sum += s.iters_hint;
            ++hint_cnt;
        }
    }
    // a slice the histogram cannot judge (not all grey levels) gets the mean
    for (int i = 0; i < n; ++i)
        if (slices[i].iters_hint <= 0) slices[i].iters_hint = hint_cnt ? (int)(hint_sum / hint_cnt) : 1;

    // 4. the batch, costliest slices first
    const int st = fcm_run_batched(h, slices, n, options);
    if (st == FCM_ERR_INVALID_ARG || st == FCM_ERR_CUDA || st == FCM_ERR_OOM) return st;

    // 5. every warm result against the cold start's fixed point: a warm run
    //    that did not converge, emptied a cluster, or ended elsewhere with a
    //    larger J is run again from its U^0
    std::vector<int> redo;
    for (int i = 0; i < n; ++i) {
        const fcm_slice& s = slices[i];
        if (s.init_mode != FCM_INIT_V) continue;
        const bool ok = s.status == FCM_OK && !(s.flags & FCM_FLAG_EMPTY_CLUSTER) && cold_ref[i] &&
                        warm_accepted(s.V64, s.J, s.status, cold_ref[i]->V64, cold_ref[i]->J, s.C);
        if (!ok) redo.push_back(i);
    }
    int worst = st;
    if (!redo.empty()) {
        std::vector<fcm_slice> sub(redo.size());
        for (size_t t = 0; t < redo.size(); ++t) {
            sub[t] = slices[redo[t]];
            sub[t].init_mode = FCM_INIT_U;
            sub[t].iters_hint = cold_ref[redo[t]] ? cold_ref[redo[t]]->iters : 0;
        }
        const int st2 = fcm_run_batched(h, sub.data(), (int)sub.size(), options | FCM_BATCH_NO_TUNE);
        if (st2 == FCM_ERR_INVALID_ARG || st2 == FCM_ERR_CUDA || st2 == FCM_ERR_OOM) return st2;
        for (size_t t = 0; t < redo.size(); ++t) slices[redo[t]] = sub[t];
        worst = FCM_OK;
        for (int i = 0; i < n; ++i) {
            if (slices[i].status < 0 && worst >= 0) worst = slices[i].status;
            if (slices[i].status == FCM_NOT_CONVERGED && worst == FCM_OK) worst = FCM_NOT_CONVERGED;
        }
    }
    if (n_cold) {
        int c = 0;
        for (int i = 0; i < n; ++i) c += slices[i].init_mode == FCM_INIT_U;
        *n_cold = c;
    }
    return worst;
}

}  // extern "C"
