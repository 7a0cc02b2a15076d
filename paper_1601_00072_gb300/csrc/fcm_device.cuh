// Device-side building blocks of the FCM pixel pass (sm_103a).
//
// Membership (Eq. 4 of arXiv:1601.00072) is evaluated in its weight form:
//   u_j = w_j / sum_k w_k,   w_j = (q_j)^(1/(m-1)),   q_j = d2min / d2_j,
// which equals 1 / sum_k (d_j / d_k)^(2/(m-1)) after dividing numerator and
// denominator by sum_k w_k; the common factor keeps every weight in (0, 1], so
// no weight or sum can overflow. When some squared distance d2 = (x - v)^2
// falls below the smallest normal float (2^-126) although the distances
// themselves are normal, q_j is formed as (|d|min / |d_j|)^2 instead, from the
// distances, which do not underflow.
// A pixel at distance 0 from one or more centers gives those clusters equal
// shares and the others 0 (Bezdek's rule; the paper leaves d = 0 open).
// "Distance 0" means |x - v| below 2^-126, i.e. zero once the FP32
// approximate instructions flush subnormal operands to zero.
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

// Smallest normal FP32 value: distances (and sums of products of distances)
// below it count as zero, as the .ftz instructions would read them.
__device__ __forceinline__ float flt_min() { return __int_as_float(0x00800000); }

// Memberships of one pixel x against C centers v (Eq. 4). Writes u[j] and
// um[j] = u[j]^m; returns this pixel's term of J_m, sum_j u_j^m d_j^2 (Eq. 1),
// through its closed form under Eq. 4: with u_j = w_j / S and
// w_j = (d2min / d2_j)^(1/(m-1)), u_j^m d2_j = d2min w_j / S^m, so the term is
// d2min * S^(1-m) (and 0 when the pixel sits on a center).
template <int C, int MK>
__device__ __forceinline__ float membership(float x, const float (&v)[C], float m, float inv_m1,
                                            float (&u)[C], float (&um)[C]) {
    float d2[C], ad[C];
    float dmin = __int_as_float(0x7f800000), amin = dmin;
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const float d = x - v[j];
        ad[j] = fabsf(d);
        d2[j] = __fmul_rn(d, d);
        dmin = fminf(dmin, d2[j]);
        amin = fminf(amin, ad[j]);
    }
    float Ji = 0.0f;
    if (amin >= flt_min()) {
        float w[C];
        if (dmin >= flt_min()) {
            // every squared distance is a normal float: ratios of the squares
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
        } else {
            // tiny distances: ratios of the distances themselves
            if (MK == M_GENERIC) {
                const float l0 = lg2_approx(amin), e = 2.0f * inv_m1;
#pragma unroll
                for (int j = 0; j < C; ++j) w[j] = ex2_approx(e * (l0 - lg2_approx(ad[j])));
            } else {
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const float r = amin * rcp_approx(ad[j]);
                    const float q = r * r;
                    w[j] = (MK == M_THREE) ? r : (MK == M_ONE_HALF) ? q * q : q;
                }
            }
        }
        float S = 0.0f;
#pragma unroll
        for (int j = 0; j < C; ++j) S += w[j];
        const float r = rcp_approx(S);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = w[j] * r;
        // dmin may be subnormal or 0 for tiny distances: the J term is then tiny or 0
        if (MK == M_TWO) Ji = dmin * r;
        else if (MK == M_THREE) Ji = dmin * r * r;
        else if (MK == M_ONE_HALF) Ji = dmin * sqrt_approx(r);
        else Ji = dmin * ex2_approx((1.0f - m) * lg2_approx(S));
    } else {
        int nz = 0;
#pragma unroll
        for (int j = 0; j < C; ++j) nz += (ad[j] < flt_min());
        const float share = __fdiv_rn(1.0f, (float)nz);
#pragma unroll
        for (int j = 0; j < C; ++j) u[j] = (ad[j] < flt_min()) ? share : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < C; ++j) um[j] = pow_m<MK>(u[j], m);
    return Ji;
}

// ---------------------------------------------------------------------------
// Two pixels at once with the packed FP32x2 instructions of sm_100+ (PTX
// add/sub/mul/fma.rn.f32x2). A pair lives in one 64-bit register pair:
// the low half is the first pixel.
// ---------------------------------------------------------------------------
typedef uint64_t f2;

__device__ __forceinline__ f2 pack2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(f2 r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ float lo2(f2 r) { float a, b; unpack2(r, a, b); return a; }
__device__ __forceinline__ float hi2(f2 r) { float a, b; unpack2(r, a, b); return b; }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 abs2(f2 a) { return a & 0x7fffffff7fffffffull; }

// Memberships of two pixels (packed x2) against C centers (each packed as
// (v_j, v_j)), Eq. 4. Writes u2[j], um2[j] = u^m and returns the pair of J
// terms sum_j u_j^m d_j^2.
//
// m = 2 and m = 3 use the product form: with b_j = d_j^2 (m = 2) or |d_j|
// (m = 3) the weights 1/b_j share the denominator prod_k b_k, so
//   u_j = P_j / sum_k P_k,   P_j = prod_{k != j} b_k,
// one reciprocal per pixel; a pixel equal to exactly one center gets u = 1
// there and 0 elsewhere without a special case. The J term is u_j b_j for any
// j when m = 2 (both equal 1 / sum_k 1/d_k^2), and (u_j b_j)^2 when m = 3.
// A pixel whose sum_k P_k is 0 (two or more centers hit exactly), below the
// smallest normal float (products of tiny distances), or not finite (products
// out of FP32 range) takes the scalar weight form above, as do the other
// fuzzifiers.
template <int C, int MK>
__device__ __forceinline__ f2 membership_pair(f2 x2, const f2 (&v2)[C], float m, float inv_m1,
                                              const float (&v)[C], f2 (&u2)[C], f2 (&um2)[C]) {
    if (MK == M_TWO || MK == M_THREE) {
        f2 b[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            const f2 d = sub2(x2, v2[j]);
            b[j] = (MK == M_TWO) ? mul2(d, d) : abs2(d);
        }
        f2 P[C];
        if (C == 1) {
            P[0] = pack2(1.0f, 1.0f);
        } else {
            f2 pre[C], suf[C];
#pragma unroll
            for (int j = 1; j < C; ++j) pre[j] = (j == 1) ? b[0] : mul2(pre[j - 1], b[j - 1]);
#pragma unroll
            for (int j = C - 2; j >= 0; --j) suf[j] = (j == C - 2) ? b[C - 1] : mul2(suf[j + 1], b[j + 1]);
#pragma unroll
            for (int j = 0; j < C; ++j) P[j] = (j == 0) ? suf[0] : (j == C - 1) ? pre[C - 1] : mul2(pre[j], suf[j]);
        }
        f2 S = P[0];
#pragma unroll
        for (int j = 1; j < C; ++j) S = add2(S, P[j]);
        float s0, s1;
        unpack2(S, s0, s1);
        // a sum below the smallest normal float would be flushed to zero by
        // the reciprocal: those pixels take the scalar form
        const float inf = __int_as_float(0x7f800000);
        if (s0 >= flt_min() && s0 < inf && s1 >= flt_min() && s1 < inf) {
            const f2 r = pack2(rcp_approx(s0), rcp_approx(s1));
#pragma unroll
            for (int j = 0; j < C; ++j) {
                u2[j] = mul2(P[j], r);
                const f2 uu = mul2(u2[j], u2[j]);
                um2[j] = (MK == M_TWO) ? uu : mul2(uu, u2[j]);
            }
            const f2 t = mul2(u2[0], b[0]);
            return (MK == M_TWO) ? t : mul2(t, t);
        }
    }
    // scalar weight form, one pixel at a time
    float xa, xb;
    unpack2(x2, xa, xb);
    float ua[C], uma[C], ub[C], umb[C];
    const float ja = membership<C, MK>(xa, v, m, inv_m1, ua, uma);
    const float jb = membership<C, MK>(xb, v, m, inv_m1, ub, umb);
#pragma unroll
    for (int j = 0; j < C; ++j) {
        u2[j] = pack2(ua[j], ub[j]);
        um2[j] = pack2(uma[j], umb[j]);
    }
    return pack2(ja, jb);
}

// Compensated FP32 ("double-float") sum, hi + lo, with Knuth's TwoSum: long
// sums of the center numerators/denominators and of J carry about 44 bits
// while using only FP32 instructions.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add(DF& a, float b) {
    const float s = __fadd_rn(a.hi, b);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ DF df_merge(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    const float hi = __fadd_rn(s, lo);  // Fast2Sum renormalisation (|s| >= |lo|)
    return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// Warp-wide double-float sum (xor tree, fixed order).
__device__ __forceinline__ DF warp_sum_df(DF d) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF e{__shfl_xor_sync(0xffffffffu, d.hi, o), __shfl_xor_sync(0xffffffffu, d.lo, o)};
        d = (lane & o) ? df_merge(e, d) : df_merge(d, e);
    }
    return d;
}

// N warp-wide double-float sums at once: every level of the xor tree issues
// the shuffles of all N sums before their merges, so the N chains of five
// dependent levels overlap instead of running one after another. Each sum is
// the same as warp_sum_df's (same operands, same order).
template <int N>
__device__ __forceinline__ void warp_sum_df_n(DF (&d)[N]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF e[N];
#pragma unroll
        for (int q = 0; q < N; ++q) e[q] = DF{__shfl_xor_sync(0xffffffffu, d[q].hi, o), __shfl_xor_sync(0xffffffffu, d[q].lo, o)};
#pragma unroll
        for (int q = 0; q < N; ++q) d[q] = (lane & o) ? df_merge(e[q], d[q]) : df_merge(d[q], e[q]);
    }
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
