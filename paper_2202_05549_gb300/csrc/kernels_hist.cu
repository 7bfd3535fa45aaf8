// 256-bin histogram built-in: "global i => read X[i], reduce(+) H[:]"
// (the reduce(f) access mode of Sec. 2.3).  Every superblock counts its
// elements into its own partial H (a temporary the runtime zeroes); the
// runtime then sums the partials in superblock order (Sec. 2.4).  Inside a
// superblock each CTA counts into shared memory (one copy per warp, to cut
// contention on skewed data) and adds its counts to the partial with
// integer atomics, which are exact and order-independent.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"
#include "task_lookup.cuh"

namespace lt {
namespace {

constexpr int HT = 256;                  // threads per CTA
constexpr int64_t HCHUNK = 64 * 1024;    // bytes of X per CTA

__device__ __forceinline__ void count4(uint32_t w, uint32_t *h) {
    atomicAdd(&h[w & 255u], 1u);
    atomicAdd(&h[(w >> 8) & 255u], 1u);
    atomicAdd(&h[(w >> 16) & 255u], 1u);
    atomicAdd(&h[w >> 24], 1u);
}

__global__ void __launch_bounds__(HT) hist256_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ uint32_t sh[HT / 32][256];
    for (int i = threadIdx.x; i < (HT / 32) * 256; i += HT) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t n = p.shape[0][0];
    const int64_t lo = t.t_lo[0] + (int64_t)(blockIdx.x - t.cta_begin) * HCHUNK;
    const int64_t hi = min(min(lo + HCHUNK, t.t_hi[0] + 1), n);  // exclusive
    const uint8_t *x = (const uint8_t *)t.v[0].base;
    const int64_t sx = t.v[0].s[0];
    uint32_t *h = sh[threadIdx.x >> 5];
    if (lo < hi) {
        // 16-byte vector body when X is contiguous; scalar head and tail
        int64_t a = lo, b = hi;
        if (sx == 1) {
            uint64_t addr = t.v[0].base + (uint64_t)lo;
            a = lo + (int64_t)((16 - (addr & 15)) & 15);
            if (a > hi) a = hi;
            b = a + (hi - a) / 16 * 16;
            for (int64_t i = lo + threadIdx.x; i < a; i += HT) atomicAdd(&h[x[i]], 1u);
            const uint4 *v = (const uint4 *)(x + a);
            const int64_t nv = (b - a) / 16;
            for (int64_t i = threadIdx.x; i < nv; i += HT) {
                uint4 w = __ldg(v + i);
                count4(w.x, h);
                count4(w.y, h);
                count4(w.z, h);
                count4(w.w, h);
            }
            for (int64_t i = b + threadIdx.x; i < hi; i += HT) atomicAdd(&h[x[i]], 1u);
        } else {
            for (int64_t i = lo + threadIdx.x; i < hi; i += HT) atomicAdd(&h[x[i * sx]], 1u);
        }
    }
    __syncthreads();
    uint32_t *out = (uint32_t *)t.v[1].base;
    const int64_t so = t.v[1].s[0];
    for (int bin = threadIdx.x; bin < 256; bin += HT) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < HT / 32; ++w) s += sh[w][bin];
        if (s) atomicAdd(&out[bin * so], s);
    }
}

// Row reduction "global [i, j] => read A[i, j], reduce(f) S[i]": one warp per
// row of the superblock; each lane folds columns lane, lane+32, ... from the
// identity, then the warp combines lanes in a fixed shuffle tree, so the
// partial of every row is deterministic.
constexpr int RW = 8;  // warps (rows) per CTA

__device__ __forceinline__ float rop(int op, float a, float b) {
    switch (op) {
        case 0: return __fadd_rn(a, b);
        case 1: return __fmul_rn(a, b);
        case 2: return fminf(a, b);
        default: return fmaxf(a, b);
    }
}

__global__ void __launch_bounds__(RW * 32) rowreduce_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], x1 = min(t.t_hi[0], NX - 1);
    const int64_t y1 = min(t.t_hi[1], NY - 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = t.t_lo[1] + (int64_t)(blockIdx.x - t.cta_begin) * RW + warp;
    if (i > y1 || x1 < x0) return;  // warp-uniform
    const int op = p.red_op;
    const float ident = op == 0 ? 0.0f : op == 1 ? 1.0f : op == 2 ? __int_as_float(0x7f800000) : __int_as_float(0xff800000);
    const DView A = t.v[0], S = t.v[1];
    const float *row = (const float *)A.base + i * A.s[0];
    float acc = ident;
    for (int64_t j = x0 + lane; j <= x1; j += 32) acc = rop(op, acc, row[j * A.s[1]]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = rop(op, acc, __shfl_down_sync(0xffffffffu, acc, off));
    if (lane == 0) ((float *)S.base)[i * S.s[0]] = acc;
}

}  // namespace

namespace k {

uint32_t prepare_rowreduce(ExecTask *t, int n, ExecParams &p) {
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t h = std::min(t[i].t_hi[1], p.shape[0][0] - 1) - t[i].t_lo[1] + 1;
        int64_t w = std::min(t[i].t_hi[0], p.shape[0][1] - 1) - t[i].t_lo[0] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = (h > 0 && w > 0) ? (uint32_t)((h + RW - 1) / RW) : 0;
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_rowreduce(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    rowreduce_kernel<<<ctas, RW * 32, 0, st>>>(dev, p);
    return cudaGetLastError();
}


uint32_t prepare_hist256(ExecTask *t, int n, ExecParams &p) {
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t hi = std::min(t[i].t_hi[0], p.shape[0][0] - 1);
        int64_t len = hi - t[i].t_lo[0] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = len > 0 ? (uint32_t)((len + HCHUNK - 1) / HCHUNK) : 0;
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_hist256(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    hist256_kernel<<<ctas, HT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
