// Double-float (compensated FP32) arithmetic beyond the sums of
// fcm_device.cuh, for kernels whose per-iteration reductions must avoid FP64
// instructions: on this GPU a dependent FP64 add takes about 64 cycles and an
// FP64 division about 630, against 4.6 and 51 in FP32.
#pragma once

#include "fcm_device.cuh"

namespace fcm {

// Quotient of two double-float values, as a double-float (one FP32 division
// and a residual correction): accurate to about 2^-44 relative.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q0 = a.hi / b.hi;
    const float p = q0 * b.hi;
    const float e = fmaf(q0, b.hi, -p);  // q0 * b.hi = p + e exactly
    const float r = ((a.hi - p) - e + a.lo) - q0 * b.lo;
    const float q1 = r / b.hi;
    const float s = q0 + q1;
    return DF{s, q1 - (s - q0)};
}

}  // namespace fcm
