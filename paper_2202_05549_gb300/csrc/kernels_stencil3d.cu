// 3-D 7-point Jacobi built-in:
//   "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]"
//   V = ((((((U + U[k-1]) + U[k+1]) + U[i-1]) + U[i+1]) + U[j-1]) + U[j+1]) / 7
// zero outside the domain, __fadd_rn in that fixed order, then a correctly
// rounded division by 7 (div_const_rn).
// Each CTA owns a 16 x 128 (i, j) tile and sweeps a run of planes along k:
// the current plane is staged in shared memory (with a one-cell ring) for
// the i and j neighbours, the planes above and below stay in registers.
#include <cuda_runtime.h>

#include <algorithm>

#include "div_const.cuh"
#include "kernels.cuh"
#include "task_lookup.cuh"

namespace lt {
namespace {

constexpr int ST = 256;           // threads per CTA
constexpr int SY = 16, SX = 128;  // (i, j) tile
constexpr int SKR = 32;           // planes per CTA (k run)
constexpr int SQ = SX / 4;        // float4 groups per tile row
constexpr int SPITCH = SX + 8;    // shared pitch, 4 cells of room each side
constexpr int GPT = SY * SQ / ST; // float4 groups per thread (2)

__device__ __forceinline__ float j7(float c, float zm, float zp, float ym, float yp, float xm, float xp) {
    float a = __fadd_rn(c, zm);
    a = __fadd_rn(a, zp);
    a = __fadd_rn(a, ym);
    a = __fadd_rn(a, yp);
    a = __fadd_rn(a, xm);
    a = __fadd_rn(a, xp);
    return div_const_rn<7>(a);
}

struct Geo3 {
    int64_t NZ, NY, NX;
    int64_t x0, x1, y0, y1, z0, z1;  // output box (clipped)
};

__device__ __forceinline__ bool geo3(const ExecTask &t, const ExecParams &p, Geo3 *g) {
    g->NZ = p.shape[0][0];
    g->NY = p.shape[0][1];
    g->NX = p.shape[0][2];
    g->x0 = t.t_lo[0];
    g->y0 = t.t_lo[1];
    g->z0 = t.t_lo[2];
    g->x1 = min(t.t_hi[0], g->NX - 1);
    g->y1 = min(t.t_hi[1], g->NY - 1);
    g->z1 = min(t.t_hi[2], g->NZ - 1);
    return g->x1 >= g->x0 && g->y1 >= g->y0 && g->z1 >= g->z0;
}

__device__ __forceinline__ const float *row3(const DView &v, int64_t k, int64_t i) {
    return (const float *)v.base + k * v.s[0] + i * v.s[1];
}

__global__ void __launch_bounds__(ST) jacobi3d_vec_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ __align__(16) float pl[SY + 2][SPITCH];
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    Geo3 g;
    if (!geo3(t, p, &g)) return;
    const uint32_t gx = (uint32_t)((g.x1 - g.x0 + SX) / SX), gy = (uint32_t)((g.y1 - g.y0 + SY) / SY);
    uint32_t local = blockIdx.x - t.cta_begin;  // 32-bit split: no 64-bit division in the prologue
    const int64_t tx0 = g.x0 + (int64_t)(local % gx) * SX;
    local /= gx;
    const int64_t ty0 = g.y0 + (int64_t)(local % gy) * SY;
    local /= gy;
    const int64_t kz0 = g.z0 + (int64_t)local * SKR, kz1 = min(kz0 + SKR - 1, g.z1);
    const DView U = t.v[0], V = t.v[1];
    // readable box (the annotation's region, clipped)
    const int64_t cmin = max(g.x0 - 1, (int64_t)0), cmax = min(g.x1 + 1, g.NX - 1);
    const int64_t rmin = max(g.y0 - 1, (int64_t)0), rmax = min(g.y1 + 1, g.NY - 1);
    const int64_t zmax = min(g.z1 + 1, g.NZ - 1);
    auto load4 = [&](int64_t k, int64_t i, int64_t j) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k >= 0 && k <= zmax && k >= g.z0 - 1 && i >= rmin && i <= rmax && j <= cmax) {
            v = *(const float4 *)(row3(U, k, i) + j);
            if (j + 1 > cmax) v.y = 0.f;
            if (j + 2 > cmax) v.z = 0.f;
            if (j + 3 > cmax) v.w = 0.f;
        }
        return v;
    };
    float4 prev[GPT], cur[GPT];
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const int e = threadIdx.x + q * ST, li = e / SQ, c = e % SQ;
        prev[q] = load4(kz0 - 1, ty0 + li, tx0 + 4 * c);
        cur[q] = load4(kz0, ty0 + li, tx0 + 4 * c);
    }
    for (int64_t k = kz0; k <= kz1; ++k) {
        // stage plane k with its ring
        for (int e = threadIdx.x; e < (SY + 2) * SQ; e += ST) {
            const int li = e / SQ, c = e % SQ;
            *(float4 *)&pl[li][4 + 4 * c] = load4(k, ty0 - 1 + li, tx0 + 4 * c);
        }
        for (int e = threadIdx.x; e < 2 * (SY + 2); e += ST) {
            const int li = e >> 1;
            const int64_t i = ty0 - 1 + li, j = (e & 1) ? tx0 + SX : tx0 - 1;
            float v = 0.f;
            if (i >= rmin && i <= rmax && j >= cmin && j <= cmax) v = row3(U, k, i)[j];
            pl[li][(e & 1) ? 4 + SX : 3] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GPT; ++q) {
            const int e = threadIdx.x + q * ST, li = e / SQ + 1, c = e % SQ;
            const int64_t i = ty0 + li - 1, j = tx0 + 4 * c;
            const float4 nx = load4(k + 1, i, j);
            if (i <= g.y1 && j <= g.x1) {
                const int cc = 4 + 4 * c;
                const float zm[4] = {prev[q].x, prev[q].y, prev[q].z, prev[q].w};
                const float zp[4] = {nx.x, nx.y, nx.z, nx.w};
                float o[4];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    o[m] = j7(pl[li][cc + m], zm[m], zp[m], pl[li - 1][cc + m], pl[li + 1][cc + m], pl[li][cc + m - 1],
                              pl[li][cc + m + 1]);
                float *dst = (float *)V.base + k * V.s[0] + i * V.s[1] + j;
                if (j + 3 <= g.x1) {
                    *(float4 *)dst = make_float4(o[0], o[1], o[2], o[3]);
                } else {
                    for (int m = 0; m < 4 && j + m <= g.x1; ++m) dst[m] = o[m];
                }
            }
            prev[q] = cur[q];
            cur[q] = nx;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(ST) jacobi3d_scalar_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    Geo3 g;
    if (!geo3(t, p, &g)) return;
    const int64_t w = g.x1 - g.x0 + 1, h = g.y1 - g.y0 + 1;
    const int64_t cell = (int64_t)(blockIdx.x - t.cta_begin) * ST + threadIdx.x;
    if (cell >= w * h * (g.z1 - g.z0 + 1)) return;
    const int64_t j = g.x0 + cell % w, i = g.y0 + (cell / w) % h, k = g.z0 + cell / (w * h);
    const DView U = t.v[0], V = t.v[1];
    auto at = [&](int64_t a, int64_t b, int64_t c) {
        return ((const float *)U.base)[a * U.s[0] + b * U.s[1] + c * U.s[2]];
    };
    const float v = j7(at(k, i, j), k > 0 ? at(k - 1, i, j) : 0.f, k + 1 < g.NZ ? at(k + 1, i, j) : 0.f,
                       i > 0 ? at(k, i - 1, j) : 0.f, i + 1 < g.NY ? at(k, i + 1, j) : 0.f,
                       j > 0 ? at(k, i, j - 1) : 0.f, j + 1 < g.NX ? at(k, i, j + 1) : 0.f);
    ((float *)V.base)[k * V.s[0] + i * V.s[1] + j * V.s[2]] = v;
}

}  // namespace

namespace k {

uint32_t prepare_jacobi3d(ExecTask *t, int n, ExecParams &p) {
    const int64_t NZ = p.shape[0][0], NY = p.shape[0][1], NX = p.shape[0][2];
    bool vec = true;
    for (int i = 0; i < n && vec; ++i) {
        if (t[i].t_lo[0] % 4 != 0) vec = false;
        for (int a = 0; a < 2; ++a) {
            const DView &v = t[i].v[a];
            if (v.s[2] != 1 || v.s[1] % 4 != 0 || v.s[0] % 4 != 0 || v.base % 16 != 0) vec = false;
        }
    }
    p.variant = vec ? 1 : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        int64_t d = std::min(t[i].t_hi[2], NZ - 1) - t[i].t_lo[2] + 1;
        uint64_t c = 0;
        if (w > 0 && h > 0 && d > 0)
            c = vec ? (uint64_t)((w + SX - 1) / SX) * (uint64_t)((h + SY - 1) / SY) * (uint64_t)((d + SKR - 1) / SKR)
                    : (uint64_t)((w * h * d + ST - 1) / ST);
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)c;
        total += (uint32_t)c;
    }
    return total;
}

cudaError_t launch_jacobi3d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 1)
        jacobi3d_vec_kernel<<<ctas, ST, 0, st>>>(dev, p);
    else
        jacobi3d_scalar_kernel<<<ctas, ST, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
