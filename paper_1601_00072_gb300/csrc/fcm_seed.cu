// The random initial membership of Algorithm 1 step 2 (arXiv:1601.00072,
// Sec. 2.1: "initialize U randomly"), drawn on the device.
//
// Each pixel's column of U^0 is a uniform Dirichlet(1, ..., 1) draw: C
// independent standard exponentials E_j = -ln r_j, normalised to sum 1. The
// uniforms come from the counter-based generator Philox4x32-10 (Salmon,
// Moraes, Dror and Shaw, SC'11), so every pixel's draw depends only on its
// index and the seed, in any launch shape: pixel i uses counter
// (i mod 2^32, i div 2^32, b, 0) under key (seed mod 2^32, seed div 2^32),
// block b = j div 4 and word j mod 4 for cluster j; a word w gives
// r = (2 floor(w / 512) + 1) / 2^24 in (0, 1), exact in FP32 (an odd integer
// below 2^24 times a power of two).
#include <cuda_runtime.h>

#include <algorithm>

#include "fcm.h"
#include "fcm_runtime.h"

using namespace fcm;

namespace {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;  // round multipliers
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;  // key increments

// Ten rounds of Philox4x32 on c under (k0, k1): a round takes the 64-bit
// products of words 0 and 2 with the multipliers and gives
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const uint32_t hi0 = __umulhi(PHILOX_M0, c[0]), lo0 = PHILOX_M0 * c[0];
        const uint32_t hi1 = __umulhi(PHILOX_M1, c[2]), lo1 = PHILOX_M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

template <int C>
__global__ void __launch_bounds__(256) k_dirichlet(float* __restrict__ U, int64_t n, uint32_t k0, uint32_t k1) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float e[C];
#pragma unroll
        for (int b = 0; b < (C + 3) / 4; ++b) {
            uint32_t c[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), (uint32_t)b, 0u};
            philox4x32_10(c, k0, k1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * b + q;
                if (j < C) e[j] = -logf((float)(2u * (c[q] >> 9) + 1u) * 5.9604644775390625e-8f);  // * 2^-24
            }
        }
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) s += e[j];
#pragma unroll
        for (int j = 0; j < C; ++j) U[(int64_t)j * n + i] = e[j] / s;
    }
}

typedef void (*DirFn)(float*, int64_t, uint32_t, uint32_t);
const DirFn k_dir[FCM_MAX_CLUSTERS + 1] = {nullptr,           k_dirichlet<1>, k_dirichlet<2>, k_dirichlet<3>,
                                           k_dirichlet<4>,    k_dirichlet<5>, k_dirichlet<6>, k_dirichlet<7>,
                                           k_dirichlet<8>};

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int fcm_init_dirichlet(fcm_handle h, int64_t n, int C, uint64_t seed, float* U) {
    NvtxRange nvtx_range("fcm_init_dirichlet");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (n < 1 || n > ((int64_t)1 << 40) || C < 1 || C > FCM_MAX_CLUSTERS || !U)
        return ctx_invalid(h, "n >= 1, C in [1, 8] and a device U are required");
    if (!on_device(U)) return ctx_invalid(h, "U must be device memory");
    DeviceGuard g(h->device);
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)h->num_sms * 16);
    k_dir[C]<<<blocks, 256, 0, h->stream>>>(U, n, (uint32_t)seed, (uint32_t)(seed >> 32));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_fail(h, e, "k_dirichlet");
    return FCM_OK;
}

int fcm_run_seeded(fcm_handle h, const float* x, int64_t n, int C, float m, float eps, int max_iter,
                   uint64_t seed, float* U, float* V, int options, fcm_report* rep) {
    NvtxRange nvtx_range("fcm_run_seeded");
    const int rc = fcm_init_dirichlet(h, n, C, seed, U);
    if (rc) return rc;
    return fcm_run(h, x, n, C, m, eps, max_iter, FCM_INIT_U, nullptr, U, V, options, rep);
}

}  // extern "C"
