// Exhaustive device self-test of the constant divisions the stencils use.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lightning.h"
#include "div_const.cuh"

namespace lt {
namespace {

// Every 32-bit pattern a: div_const_rn<C>(a) must equal __fdiv_rn(a, C) bit
// for bit (any two NaNs count as equal).  Grid-stride over all 2^32 inputs.
template <int C>
__global__ void div_const_check(unsigned long long *mismatches) {
    unsigned long long bad = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const float a = __uint_as_float((uint32_t)i);
        const float got = div_const_rn<C>(a), want = __fdiv_rn(a, (float)C);
        const bool same = __float_as_uint(got) == __float_as_uint(want) || (got != got && want != want);
        bad += same ? 0 : 1;
    }
    if (bad) atomicAdd(mismatches, bad);
}

// div4_const_rn against __fdiv_rn: every pattern a in each of the four
// positions, next to three in-range values, so that the one range test for
// the four must send every out-of-range a (zero, tiny, huge, inf, NaN) to
// the exact path.
template <int C>
__global__ void div4_const_check(unsigned long long *mismatches) {
    unsigned long long bad = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
        const float a = __uint_as_float((uint32_t)i);
        float v[4] = {1.0f, 0.3f, 7.5f, 123.0f};
        v[i & 3] = a;
        const float4 got = div4_const_rn<C>(make_float4(v[0], v[1], v[2], v[3]));
        const float g[4] = {got.x, got.y, got.z, got.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float want = __fdiv_rn(v[k], (float)C);
            const bool same = __float_as_uint(g[k]) == __float_as_uint(want) || (g[k] != g[k] && want != want);
            bad += same ? 0 : 1;
        }
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace
}  // namespace lt

extern "C" lt_status lt_selftest_div_const(int32_t device, int32_t divisor, uint64_t *mismatches) {
    if (!mismatches || (divisor != 5 && divisor != 7)) return LT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return LT_ERR_CUDA;
    unsigned long long *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(*d)) != cudaSuccess) return LT_ERR_CUDA;
    cudaError_t e = cudaMemset(d, 0, sizeof(*d));
    if (e == cudaSuccess) {
        if (divisor == 5) {
            lt::div_const_check<5><<<152 * 8, 256>>>(d);
            lt::div4_const_check<5><<<152 * 8, 256>>>(d);
        } else {
            lt::div_const_check<7><<<152 * 8, 256>>>(d);
            lt::div4_const_check<7><<<152 * 8, 256>>>(d);
        }
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return LT_ERR_CUDA;
    *mismatches = h;
    return LT_OK;
}
