// Shared definitions of the batched FCM path (host runtime and kernels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fcm.h"

namespace fcm {

// Device-side copy of one slice's arguments.
struct alignas(16) SliceDesc {
    const float* x;
    const float* U0;  // initial memberships (FCM_INIT_U); may equal U
    float* U;         // final memberships, written once at the end
    float* V;         // final centers (device)
    int64_t n;
    int C;
    int mk;           // fuzzifier kind (MKind)
    float m, inv_m1, eps;
    int max_iter;
    int init;         // FCM_INIT_U or FCM_INIT_V
    int pad;
    float V0[FCM_MAX_CLUSTERS];  // initial centers (FCM_INIT_V), copied before the run
};

struct alignas(16) SliceResult {
    int iters;
    int status;
    int flags;
    int pad;
    double delta;
    double J;
    double V64[FCM_MAX_CLUSTERS];
};

struct alignas(128) BatchCtl {
    unsigned int next;  // work-queue head (index into the LPT order)
    unsigned int pad[31];
};

// Launch shape of the batched kernel.
struct BatchPlan {
    int block;      // threads per CTA: 256 or 512
    int cluster;    // CTAs per cluster: 1, 2, 4 or 8
    int64_t big;    // slices with n >= big are shared by a whole cluster
};

typedef void (*BatchFn)(const SliceDesc*, const int*, int, SliceResult*, BatchCtl*, int64_t);

// Kernel of each block size, and its dynamic shared memory (x staging).
struct BatchKernel {
    BatchFn fn;
    int smem;
    int xcap;  // pixels of x one CTA keeps in shared memory
};

BatchKernel batched_kernel_256();
BatchKernel batched_kernel_512();

}  // namespace fcm
