// Element-wise built-ins over 2-D f32 arrays: the per-operation pieces of a
// diffusion step and of its adjoint when each is a launch of its own (the
// unfused "plain" form that the fused and checkpointed adjoint is compared
// against).  Explicit _rn intrinsics, no contraction.
//   EWISE2D   C = A + B  (value parameter op = 0)   or   C = A * B  (op = 1)
//             "global [i, j] => read A[i, j], read B[i, j], write C[i, j]"
//   MULADD2D  C = C + A * B
//             "global [i, j] => read A[i, j], read B[i, j], readwrite C[i, j]"
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"
#include "task_lookup.cuh"

namespace lt {
namespace {

constexpr int ET = 256;     // threads per CTA
constexpr int EROWS = 8;    // rows per CTA
constexpr int ECOLS = 512;  // columns per CTA: 128 threads x 4 columns ... two row halves per pass

// MODE 0: C = A + B, 1: C = A * B, 2: C = C + A * B.  VEC: rows 16-byte
// aligned in every view and tasks starting on a 4-aligned column (float4).
template <int MODE, bool VEC>
__global__ void __launch_bounds__(ET) ewise_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    const uint32_t gx = (uint32_t)((x1 - x0 + ECOLS) / ECOLS);
    const uint32_t local = blockIdx.x - t.cta_begin;
    const int64_t r0 = y0 + (int64_t)(local / gx) * EROWS, c0 = x0 + (int64_t)(local % gx) * ECOLS;
    const DView A = t.v[0], B = t.v[1], C = t.v[2];
    const float *a = (const float *)A.base, *b = (const float *)B.base;
    float *c = (float *)C.base;
    auto op = [](float x, float y, float z) {
        if (MODE == 0) return __fadd_rn(x, y);
        if (MODE == 1) return __fmul_rn(x, y);
        return __fadd_rn(z, __fmul_rn(x, y));
    };
    // each thread: columns c0 + 4 * (threadIdx.x % 128) .. +3 of rows r0 + threadIdx.x / 128 + 2k
    const int64_t j = c0 + 4 * (int64_t)(threadIdx.x % 128);
    if (j > x1) return;
    const bool full = VEC && j + 3 <= x1;
    float4 av[EROWS / 2], bv[EROWS / 2], cv[EROWS / 2];
#pragma unroll
    for (int k = 0; k < EROWS / 2; ++k) {
        const int64_t i = r0 + threadIdx.x / 128 + 2 * k;
        if (i > y1 || !full) continue;
        av[k] = *(const float4 *)(a + i * A.s[0] + j);
        bv[k] = *(const float4 *)(b + i * B.s[0] + j);
        if (MODE == 2) cv[k] = *(const float4 *)(c + i * C.s[0] + j);
    }
#pragma unroll
    for (int k = 0; k < EROWS / 2; ++k) {
        const int64_t i = r0 + threadIdx.x / 128 + 2 * k;
        if (i > y1) continue;
        if (full) {
            float4 o;
            o.x = op(av[k].x, bv[k].x, MODE == 2 ? cv[k].x : 0.f);
            o.y = op(av[k].y, bv[k].y, MODE == 2 ? cv[k].y : 0.f);
            o.z = op(av[k].z, bv[k].z, MODE == 2 ? cv[k].z : 0.f);
            o.w = op(av[k].w, bv[k].w, MODE == 2 ? cv[k].w : 0.f);
            *(float4 *)(c + i * C.s[0] + j) = o;
        } else {
            for (int m = 0; m < 4 && j + m <= x1; ++m) {
                float *cp = c + i * C.s[0] + (j + m) * C.s[1];
                *cp = op(a[i * A.s[0] + (j + m) * A.s[1]], b[i * B.s[0] + (j + m) * B.s[1]], MODE == 2 ? *cp : 0.f);
            }
        }
    }
}

bool ewise_vec_ok(const ExecTask *t, int n) {
    for (int i = 0; i < n; ++i) {
        if (t[i].t_lo[0] % 4 != 0) return false;
        for (int a = 0; a < 3; ++a) {
            const DView &v = t[i].v[a];
            if (v.s[1] != 1 || (v.s[0] % 4) != 0 || (v.base % 16) != 0) return false;
        }
    }
    return true;
}

uint32_t ewise_prepare(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    p.variant = ewise_vec_ok(t, n) ? 1 : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        const int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = (w > 0 && h > 0) ? (uint32_t)(((w + ECOLS - 1) / ECOLS) * ((h + EROWS - 1) / EROWS)) : 0;
        total += t[i].cta_count;
    }
    return total;
}

template <int MODE>
cudaError_t ewise_launch(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 1)
        ewise_kernel<MODE, true><<<ctas, ET, 0, st>>>(dev, p);
    else
        ewise_kernel<MODE, false><<<ctas, ET, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace

namespace k {

uint32_t prepare_ewise(ExecTask *t, int n, ExecParams &p) {
    if (p.i[0] != 0 && p.i[0] != 1) return 0xFFFFFFFFu;  // op: 0 add, 1 multiply
    return ewise_prepare(t, n, p);
}

cudaError_t launch_ewise(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    return p.i[0] == 0 ? ewise_launch<0>(dev, ctas, p, st) : ewise_launch<1>(dev, ctas, p, st);
}

uint32_t prepare_muladd(ExecTask *t, int n, ExecParams &p) { return ewise_prepare(t, n, p); }

cudaError_t launch_muladd(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    return ewise_launch<2>(dev, ctas, p, st);
}

}  // namespace k
}  // namespace lt
