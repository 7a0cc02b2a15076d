// Multi-feature FCM (D channels per pixel): device state and kernel table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fcm.h"
#include "fcm_internal.h"

namespace fcm {

constexpr int MULTI_MAX_D = 4;

struct alignas(128) MultiState {
    const float* x;   // [D][n], channel-major
    const float* U0;  // [C][n] (from U^0), else null
    float* U;         // [C][n] out
    int64_t n;
    float m, inv_m1, eps;
    int max_iter;
    float V0[FCM_MAX_CLUSTERS * MULTI_MAX_D];    // [C][D]
    float V[FCM_MAX_CLUSTERS * MULTI_MAX_D];     // out
    double V64[FCM_MAX_CLUSTERS * MULTI_MAX_D];  // out: FP64 quotients behind V
    double delta, J;
    int iters, status, flags;
    unsigned ticket;  // grid barrier arrivals
    WaitLimits lim;
};

typedef void (*MultiFn)(MultiState*, float*);

struct MultiTable {
    // [D][C][0 = m == 2, 1 = any m][0 = from U^0, 1 = from V^0]
    MultiFn run[MULTI_MAX_D + 1][FCM_MAX_CLUSTERS + 1][2][2];
};

void register_multi_d1(MultiTable&);
void register_multi_d2(MultiTable&);
void register_multi_d3(MultiTable&);
void register_multi_d4(MultiTable&);

}  // namespace fcm
