// Global -> shared copies that bypass registers (cp.async, 16 bytes).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lt {

// Copy 16 bytes from global `src` to shared `dst` (both 16-byte aligned),
// cached in L2 only; with valid == false nothing is read and dst is zeroed
// (src must still be a valid global address).
__device__ __forceinline__ void cp_async16(float *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

// Wait for every cp.async this thread issued (the caller then synchronises
// the CTA before reading what other threads copied).
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

}  // namespace lt
