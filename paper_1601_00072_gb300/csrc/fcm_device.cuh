// Device-side building blocks of the FCM pixel pass (sm_103a).
//
// Membership (Eq. 4 of arXiv:1601.00072) is evaluated in its weight form:
//   u_j = w_j / sum_k w_k,   w_j = (q_j)^(1/(m-1)),   q_j = d2min / d2_j,
// which equals 1 / sum_k (d_j / d_k)^(2/(m-1)) after dividing numerator and
// denominator by sum_k w_k; the common factor d2min^(1/(m-1)) keeps every
// weight in (0, 1], so no weight or sum can overflow even for tiny distances.
// A pixel at distance exactly 0 from one or more centers gives those clusters
// equal shares and the others 0 (Bezdek's rule; the paper leaves d = 0 open).
// "Exactly 0" means (x - v)^2 == 0 in FP32 with flush-to-zero.
//
// Specialisations of the fuzzifier avoid general powers on the hot path:
//   m = 2    w = q                u^m = u*u
//   m = 3    w = sqrt(q)          u^m = u*u*u
//   m = 1.5  w = q*q              u^m = u*sqrt(u)
//   other m  w = 2^((log2 q)/(m-1))   u^m = 2^(m log2 u)
// using the PTX approximate instructions (rcp, rsqrt, sqrt, lg2, ex2), whose
// documented error is at most a few ulp in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fcm {

enum MKind : int { M_TWO = 0, M_THREE = 1, M_ONE_HALF = 2, M_GENERIC = 3, M_KINDS = 4 };

__host__ __device__ inline int mkind_of(float m) {
    return m == 2.0f ? M_TWO : m == 3.0f ? M_THREE : m == 1.5f ? M_ONE_HALF : M_GENERIC;
}

__device__ __forceinline__ float rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float a) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float lg2_approx(float a) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float ex2_approx(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// u^m for the specialised fuzzifiers (u in [0, 1]).
template <int MK>
__device__ __forceinline__ float pow_m(float u, float m) {
    if (MK == M_TWO) return u * u;
    if (MK == M_THREE) return u * u * u;
    if (MK == M_ONE_HALF) return u * sqrt_approx(u);
    return ex2_approx(m * lg2_approx(u));  // lg2(0) = -inf -> ex2(-inf) = 0
}

// Memberships of one pixel x against C centers v (Eq. 4). Writes u[j] and
// um[j] = u[j]^m; returns this pixel's term of J_m, sum_j u_j^m d_j^2 (Eq. 1).
template <int C, int MK>
__device__ __forceinline__ float membership(float x, const float (&v)[C], float m,
                                            float inv_m1, float (&u)[C], float (&um)[C]) {
    float d2[C];
    float dmin = __int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const float d = x - v[j];
        d2[j] = __fmul_rn(d, d);
        dmin = fminf(dmin, d2[j]);
    }
    if (dmin > 0.0f) {
        float w[C];
        if (MK == M_GENERIC) {
            const float l0 = lg2_approx(dmin);
#pragma unroll
            for (int j = 0; j < C; ++j) w[j] = ex2_approx(inv_m1 * (l0 - lg2_approx(d2[j])));
        } else if (MK == M_THREE) {
            const float s0 = sqrt_approx(dmin);
#pragma unroll
            for (int j = 0; j < C; ++j) w[j] = s0 * rsqrt_approx(d2[j]);
        } else {
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const float q = dmin * rcp_approx(d2[j]);
                w[j] = (MK == M_ONE_HALF) ? q * q : q;
            }
        }
        float S = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) S += w[j];
        const float r = rcp_approx(S);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = w[j] * r;
    } else {
        int nz = 0;
#pragma unroll
        for (int j = 0; j < C; ++j) nz += (d2[j] == 0.0f);
        const float share = __fdiv_rn(1.0f, (float)nz);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = (d2[j] == 0.0f) ? share : 0.0f;
    }
    float Ji = 0.0f;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        um[j] = pow_m<MK>(u[j], m);
        Ji = fmaf(um[j], d2[j], Ji);
    }
    return Ji;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float comp(const float4& a, int p) {
    return p == 0 ? a.x : p == 1 ? a.y : p == 2 ? a.z : a.w;
}
__device__ __forceinline__ void set_comp(float4& a, int p, float v) {
    if (p == 0) a.x = v; else if (p == 1) a.y = v; else if (p == 2) a.z = v; else a.w = v;
}

// Read-only streaming load of the intensities (non-coherent path).
__device__ __forceinline__ float4 ld_x4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
// Memberships are read once and overwritten by the same thread: evict-first.
__device__ __forceinline__ float4 ld_u4(const float* p) {
    return __ldcs(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st_u4(float* p, float4 v) {
    __stcs(reinterpret_cast<float4*>(p), v);
}

__device__ __forceinline__ bool finite_f(float a) {
    return (__float_as_uint(a) & 0x7f800000u) != 0x7f800000u;
}

}  // namespace fcm
