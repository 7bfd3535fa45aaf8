// Variable-coefficient diffusion and its adjoint (an extension beyond the
// paper: differentiation of a chunked stencil launch).
//
// Forward, "global [i, j] => read U[i-1:i+1, j-1:j+1], read K[i, j], write V[i, j]":
//     (L u)_ij = (((u_{i-1,j} + u_{i+1,j}) + u_{i,j-1}) + u_{i,j+1}) - 4 u_ij
//     V = U + K * (L U)            (zero outside the domain)
// Adjoint of one step, with the annotation transposed so that the forward
// halo READ becomes a halo REDUCE(+):
//     "global [i, j] => read L1[i, j], read K[i, j], read U[i-1:i+1, j-1:j+1],
//                       readwrite G[i, j], reduce(+) L0[i-1:i+1, j-1:j+1]"
// Thread (i,j) owns s = K_ij L1_ij and contributes L1_ij - 4 s to L0_ij and s
// to its four neighbours; it also accumulates G_ij += L1_ij (L U)_ij.  Summed
// over all threads this is L0 = L1 + L(K L1) (L is symmetric) and the
// kappa-gradient term.  Each superblock gathers, for every cell of its
// reduce region, the contributions of its OWN threads (own term first, then
// north, south, west, east) into its partial; the runtime adds the partials
// in superblock order, so the result is deterministic.
// All arithmetic is f32 with explicit _rn intrinsics (no contraction).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace lt {
namespace {

__device__ __forceinline__ int find_task_d(const ExecTask *t, int n, uint32_t cta) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (t[mid].cta_begin <= cta)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float at2(const DView &v, int64_t i, int64_t j) {
    return ((const float *)v.base)[i * v.s[0] + j * v.s[1]];
}

__device__ __forceinline__ float lap5(float c, float n, float s, float w, float e) {
    return __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(n, s), w), e), __fmul_rn(4.0f, c));
}

constexpr int DT = 256;  // threads per CTA, one cell each

__global__ void __launch_bounds__(DT) diffusion_fwd_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = find_task_d(tasks, p.ntasks, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    const int64_t w = x1 - x0 + 1;
    const int64_t cell = (int64_t)(blockIdx.x - t.cta_begin) * DT + threadIdx.x;
    if (w <= 0 || cell >= w * (y1 - y0 + 1)) return;
    const int64_t i = y0 + cell / w, j = x0 + cell % w;
    const DView U = t.v[0], K = t.v[1], V = t.v[2];
    float c = at2(U, i, j);
    float n = i > 0 ? at2(U, i - 1, j) : 0.f;
    float s = i + 1 < NY ? at2(U, i + 1, j) : 0.f;
    float we = j > 0 ? at2(U, i, j - 1) : 0.f;
    float e = j + 1 < NX ? at2(U, i, j + 1) : 0.f;
    float k = at2(K, i, j);
    ((float *)V.base)[i * V.s[0] + j * V.s[1]] = __fadd_rn(c, __fmul_rn(k, lap5(c, n, s, we, e)));
}

__global__ void __launch_bounds__(DT) diffusion_adj_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = find_task_d(tasks, p.ntasks, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    // the superblock's cells (thread box clipped to the domain)
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    // its reduce region: one cell wider, clipped
    const int64_t rx0 = max(x0 - 1, (int64_t)0), ry0 = max(y0 - 1, (int64_t)0);
    const int64_t rx1 = min(x1 + 1, NX - 1), ry1 = min(y1 + 1, NY - 1);
    const int64_t w = rx1 - rx0 + 1;
    const int64_t cell = (int64_t)(blockIdx.x - t.cta_begin) * DT + threadIdx.x;
    if (cell >= w * (ry1 - ry0 + 1)) return;
    const int64_t i = ry0 + cell / w, j = rx0 + cell % w;
    const DView L1 = t.v[0], K = t.v[1], U = t.v[2], G = t.v[3], L0 = t.v[4];
    auto in_sb = [&](int64_t a, int64_t b) { return a >= y0 && a <= y1 && b >= x0 && b <= x1; };
    auto src = [&](int64_t a, int64_t b) { return __fmul_rn(at2(K, a, b), at2(L1, a, b)); };
    float acc = 0.f;
    if (in_sb(i, j)) {
        const float l1 = at2(L1, i, j);
        acc = __fsub_rn(l1, __fmul_rn(4.0f, __fmul_rn(at2(K, i, j), l1)));
        float c = at2(U, i, j);
        float n = i > 0 ? at2(U, i - 1, j) : 0.f;
        float s = i + 1 < NY ? at2(U, i + 1, j) : 0.f;
        float we = j > 0 ? at2(U, i, j - 1) : 0.f;
        float e = j + 1 < NX ? at2(U, i, j + 1) : 0.f;
        float *g = (float *)G.base + i * G.s[0] + j * G.s[1];
        *g = __fadd_rn(*g, __fmul_rn(l1, lap5(c, n, s, we, e)));
    }
    if (i - 1 >= 0 && in_sb(i - 1, j)) acc = __fadd_rn(acc, src(i - 1, j));
    if (i + 1 < NY && in_sb(i + 1, j)) acc = __fadd_rn(acc, src(i + 1, j));
    if (j - 1 >= 0 && in_sb(i, j - 1)) acc = __fadd_rn(acc, src(i, j - 1));
    if (j + 1 < NX && in_sb(i, j + 1)) acc = __fadd_rn(acc, src(i, j + 1));
    ((float *)L0.base)[i * L0.s[0] + j * L0.s[1]] = acc;
}

}  // namespace

namespace k {

uint32_t prepare_diffusion(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        uint64_t cells = (w > 0 && h > 0) ? (uint64_t)(w * h) : 0;
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)((cells + DT - 1) / DT);
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_diffusion(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    diffusion_fwd_kernel<<<ctas, DT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

uint32_t prepare_diffusion_adj(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t x0 = t[i].t_lo[0], y0 = t[i].t_lo[1];
        int64_t x1 = std::min(t[i].t_hi[0], NX - 1), y1 = std::min(t[i].t_hi[1], NY - 1);
        uint64_t cells = 0;
        if (x1 >= x0 && y1 >= y0) {
            int64_t w = std::min(x1 + 1, NX - 1) - std::max<int64_t>(x0 - 1, 0) + 1;
            int64_t h = std::min(y1 + 1, NY - 1) - std::max<int64_t>(y0 - 1, 0) + 1;
            cells = (uint64_t)(w * h);
        }
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)((cells + DT - 1) / DT);
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_diffusion_adj(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    diffusion_adj_kernel<<<ctas, DT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
