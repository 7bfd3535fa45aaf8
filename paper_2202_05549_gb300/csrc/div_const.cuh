// Correctly rounded division by a small integer constant.
#pragma once

#include <cuda_runtime.h>

namespace lt {

// a / C rounded to nearest, by Markstein's correction step (P. Markstein,
// "Computation of elementary functions on the IBM RISC System/6000
// processor", IBM J. Res. Dev. 34(1), 1990): with y = RN(1/C) and
// q0 = RN(a*y) within one ulp of a/C, the remainder r = a - C*q0 is exact in
// one FMA and RN(q0 + r*y) is the correctly rounded quotient.  Zero, tiny
// and huge magnitudes, infinities and NaN take the IEEE division.  Three
// instructions instead of a full division; lt_selftest_div_const checks it
// against __fdiv_rn on all 2^32 inputs for C = 5 and C = 7.
template <int C>
__device__ __forceinline__ float div_const_rn(float a) {
    constexpr float y = 1.0f / (float)C;  // RN(1/C)
    const float m = fabsf(a);
    if (!(m >= 1e-30f && m <= 1e30f)) return __fdiv_rn(a, (float)C);
    const float q0 = __fmul_rn(a, y);
    const float r = __fmaf_rn(-q0, (float)C, a);
    return __fmaf_rn(r, y, q0);
}

// The same for four values at once, with one range test for the four: the
// smallest and the largest magnitude must lie in [1e-30, 1e30] (the largest
// is taken NaN-propagating, so that a NaN fails the test); otherwise each
// value goes through div_const_rn.  Results equal div_const_rn's element by
// element; the saving is the per-value test and branch.
__device__ __forceinline__ float max_nan(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

template <int C>
__device__ __forceinline__ float4 div4_const_rn(float4 a) {
    constexpr float y = 1.0f / (float)C;
    const float ax = fabsf(a.x), ay = fabsf(a.y), az = fabsf(a.z), aw = fabsf(a.w);
    const float lo = fminf(fminf(ax, ay), fminf(az, aw));
    const float hi = max_nan(max_nan(ax, ay), max_nan(az, aw));
    if (lo >= 1e-30f && hi <= 1e30f) {
        const float qx = __fmul_rn(a.x, y), qy = __fmul_rn(a.y, y), qz = __fmul_rn(a.z, y), qw = __fmul_rn(a.w, y);
        return make_float4(__fmaf_rn(__fmaf_rn(-qx, (float)C, a.x), y, qx),
                           __fmaf_rn(__fmaf_rn(-qy, (float)C, a.y), y, qy),
                           __fmaf_rn(__fmaf_rn(-qz, (float)C, a.z), y, qz),
                           __fmaf_rn(__fmaf_rn(-qw, (float)C, a.w), y, qw));
    }
    return make_float4(div_const_rn<C>(a.x), div_const_rn<C>(a.y), div_const_rn<C>(a.z), div_const_rn<C>(a.w));
}

}  // namespace lt
