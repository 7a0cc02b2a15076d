// Defuzzification and the Dice similarity of the result against ground truth.
//
// After the run each pixel takes the cluster of its largest membership
// (Sec. 2.1; ties go to the lowest cluster index), which a map sends to a
// tissue class. The paper scores a segmentation per class by the Dice
// similarity coefficient DSC = 2 |PR n GT| / (|PR| + |GT|) (Sec. 5.2, Eq. 5).
// One pass over U and the truth labels counts |PR_c|, |GT_c| and
// |PR_c n GT_c| in shared memory, then in 64-bit global counters; the counts
// are exact integers, so the result does not depend on the order of the adds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "fcm.h"
#include "fcm_runtime.h"

using namespace fcm;

namespace {

constexpr int DNT = 256;
constexpr int MAX_CLASSES = 16;

struct DscArgs {
    int class_of_cluster[FCM_MAX_CLUSTERS];
};

// counts: [3 * n_classes] of |PR_c|, |GT_c|, |PR_c n GT_c|; bad: a truth label
// outside [0, n_classes) was seen.
template <int C>
__global__ void __launch_bounds__(DNT) k_dsc(const float* __restrict__ U, const uint8_t* __restrict__ truth,
                                             int64_t n, DscArgs map, int n_classes,
                                             unsigned long long* __restrict__ counts, int* bad) {
    __shared__ unsigned sc[3 * MAX_CLASSES];
    for (int t = threadIdx.x; t < 3 * MAX_CLASSES; t += DNT) sc[t] = 0u;
    __syncthreads();
    bool b = false;
    const int64_t stride = (int64_t)gridDim.x * DNT;
    for (int64_t i = (int64_t)blockIdx.x * DNT + threadIdx.x; i < n; i += stride) {
        int best = 0;
        float bu = __ldg(U + i);
#pragma unroll
        for (int j = 1; j < C; ++j) {
            const float u = __ldg(U + (int64_t)j * n + i);
            if (u > bu) {
                bu = u;
                best = j;
            }
        }
        const int p = map.class_of_cluster[best], g = __ldg(truth + i);
        if (g >= n_classes) {
            b = true;
            continue;
        }
        atomicAdd(&sc[3 * p], 1u);
        atomicAdd(&sc[3 * g + 1], 1u);
        if (p == g) atomicAdd(&sc[3 * p + 2], 1u);
    }
    if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1);
    for (int t = threadIdx.x; t < 3 * n_classes; t += DNT)
        if (sc[t]) atomicAdd(&counts[t], (unsigned long long)sc[t]);
}

typedef void (*DscFn)(const float*, const uint8_t*, int64_t, DscArgs, int, unsigned long long*, int*);

DscFn dsc_kernel(int C) {
    switch (C) {
        case 1: return k_dsc<1>;
        case 2: return k_dsc<2>;
        case 3: return k_dsc<3>;
        case 4: return k_dsc<4>;
        case 5: return k_dsc<5>;
        case 6: return k_dsc<6>;
        case 7: return k_dsc<7>;
        default: return k_dsc<8>;
    }
}

bool on_device(const void* p) {
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

extern "C" int fcm_dsc(fcm_handle h, const float* U, int64_t n, int C, const uint8_t* truth,
                       const int* class_of_cluster, int n_classes, int64_t* counts, double* dsc) {
    NvtxRange nvtx_range("fcm_dsc");
    if (!h) return FCM_ERR_INVALID_ARG;
    if (!U || !truth || !class_of_cluster || !dsc) return ctx_invalid(h, "null U, truth, map or dsc");
    if (n < 1 || C < 1 || C > FCM_MAX_CLUSTERS) return ctx_invalid(h, "n >= 1 and C in [1, 8]");
    if (n_classes < 1 || n_classes > MAX_CLASSES) return ctx_invalid(h, "n_classes must be in [1, 16]");
    DscArgs map;
    std::memset(&map, 0, sizeof(map));
    for (int j = 0; j < C; ++j) {
        if (class_of_cluster[j] < 0 || class_of_cluster[j] >= n_classes)
            return ctx_invalid(h, "class_of_cluster entries must be in [0, n_classes)");
        map.class_of_cluster[j] = class_of_cluster[j];
    }
    if (!on_device(U) || !on_device(truth)) return ctx_invalid(h, "U and truth must be device memory");
    DeviceGuard g(h->device);
    unsigned long long* d_counts = nullptr;
    int* d_bad = nullptr;
    // a small scratch, allocated per call: the score is an evaluation step
    CK(cudaMallocAsync((void**)&d_counts, sizeof(unsigned long long) * 3 * MAX_CLASSES + sizeof(int), h->stream));
    d_bad = reinterpret_cast<int*>(d_counts + 3 * MAX_CLASSES);
    CK(cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * 3 * MAX_CLASSES + sizeof(int), h->stream));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + DNT - 1) / DNT, (int64_t)h->num_sms * 8));
    dsc_kernel(C)<<<blocks, DNT, 0, h->stream>>>(U, truth, n, map, n_classes, d_counts, d_bad);
    cudaError_t le = cudaGetLastError();
    unsigned long long hc[3 * MAX_CLASSES + 1];
    if (le == cudaSuccess)
        le = cudaMemcpyAsync(hc, d_counts, sizeof(unsigned long long) * 3 * MAX_CLASSES + sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream);
    if (le == cudaSuccess) le = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(d_counts, h->stream);
    if (le != cudaSuccess) return ctx_fail(h, le, "dsc pass");
    int bad_flag;
    std::memcpy(&bad_flag, &hc[3 * MAX_CLASSES], sizeof(int));
    if (bad_flag) return ctx_invalid(h, "truth labels must be in [0, n_classes)");
    for (int c = 0; c < n_classes; ++c) {
        const unsigned long long pr = hc[3 * c], gt = hc[3 * c + 1], both = hc[3 * c + 2];
        dsc[c] = (pr + gt) == 0 ? 1.0 : 2.0 * (double)both / (double)(pr + gt);
        if (counts) {
            counts[3 * c] = (int64_t)pr;
            counts[3 * c + 1] = (int64_t)gt;
            counts[3 * c + 2] = (int64_t)both;
        }
    }
    return FCM_OK;
}
