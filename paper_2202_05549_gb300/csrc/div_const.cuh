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

}  // namespace lt
