// Device-side lookup of the task that owns a CTA of an Execute launch.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace lt {

// One division when every task has the same CTA count (uniform tilings, set
// by the runtime in ExecParams.uniform_ctas); otherwise a binary search on
// cta_begin.  The division needs no memory access, so a CTA reaches its first
// data load after a single dependent read (its task record).
__device__ __forceinline__ int task_of(const ExecTask *t, const ExecParams &p, uint32_t cta) {
    if (p.uniform_ctas > 0) return (int)(cta / (uint32_t)p.uniform_ctas);
    int lo = 0, hi = p.ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (t[mid].cta_begin <= cta)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace lt
