// 3-D 7-point Jacobi built-in:
//   "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]"
//   V = ((((((U + U[k-1]) + U[k+1]) + U[i-1]) + U[i+1]) + U[j-1]) + U[j+1]) / 7
// zero outside the domain, __fadd_rn in that fixed order, then a correctly
// rounded division by 7 (div_const_rn).
// The vector kernel computes register strips of one plane (below); the
// scalar kernel takes tasks whose rows are not 16-byte aligned.
#include <cuda_runtime.h>

#include <algorithm>

#include "div_const.cuh"
#include "kernels.cuh"
#include "task_lookup.cuh"

namespace lt {
namespace {

constexpr int ST = 256;  // threads per CTA of the scalar kernel

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

// Vector kernel: each warp computes J3R rows x 128 columns (4 per lane) of
// one plane k.  It loads everything first (planes k-1 and k+1 over its rows,
// plane k over its rows and the one above and below, and the column outside
// the strip for lanes 0 and 31), then computes: no shared memory, no
// barriers, and 3*J3R+2 independent 16-byte loads per lane in flight, as in
// the 2-D kernel.  The neighbouring planes a warp reads are re-read by the
// warps of planes k-1 and k+1; CTAs are ordered plane by plane (j fastest,
// then i, then k), so those reads come from L2.
constexpr int J3R = 8;   // output rows per warp
constexpr int J3W = 4;   // warps per CTA, side by side along j

__global__ void __launch_bounds__(J3W * 32) jacobi3d_vec_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    Geo3 g;
    if (!geo3(t, p, &g)) return;
    const uint32_t gx = (uint32_t)((g.x1 - g.x0 + J3W * 128) / (J3W * 128));
    const uint32_t gy = (uint32_t)((g.y1 - g.y0 + J3R) / J3R);
    uint32_t local = blockIdx.x - t.cta_begin;  // 32-bit split: no 64-bit division in the prologue
    const uint32_t tx = local % gx;
    local /= gx;
    const int64_t r0 = g.y0 + (int64_t)(local % gy) * J3R;
    const int64_t k = g.z0 + (int64_t)(local / gy);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t js = g.x0 + (int64_t)(tx * J3W + warp) * 128;
    if (js > g.x1 || r0 > g.y1) return;  // warp-uniform
    const int64_t j0 = js + 4 * lane;
    const DView U = t.v[0], V = t.v[1];
    // readable box (the annotation's region, clipped)
    const int64_t cmin = max(g.x0 - 1, (int64_t)0), cmax = min(g.x1 + 1, g.NX - 1);
    const int64_t rmin = max(g.y0 - 1, (int64_t)0), rmax = min(g.y1 + 1, g.NY - 1);
    const int64_t zmin = max(g.z0 - 1, (int64_t)0), zmax = min(g.z1 + 1, g.NZ - 1);
    const bool ldc = j0 <= cmax;
    // guarded loads only; the columns past cmax are cleared after every load
    // is in flight (clearing right after each load would wait for it)
    auto ld4 = [&](int64_t kk, int64_t i) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ldc && kk >= zmin && kk <= zmax && i >= rmin && i <= rmax) v = *(const float4 *)(row3(U, kk, i) + j0);
        return v;
    };
    auto clip = [&](float4 &v) {
        if (j0 + 1 > cmax) v.y = 0.f;
        if (j0 + 2 > cmax) v.z = 0.f;
        if (j0 + 3 > cmax) v.w = 0.f;
    };
    // the column left of the strip (lane 0) or right of it (lane 31)
    const int64_t jx = lane == 0 ? j0 - 1 : j0 + 4;
    const bool ldx = (lane == 0 || lane == 31) && jx >= cmin && jx <= cmax && k >= zmin && k <= zmax;
    float4 zm[J3R], zp[J3R], pc[J3R + 2];
    float xo[J3R];
#pragma unroll
    for (int m = 0; m < J3R + 2; ++m) pc[m] = ld4(k, r0 - 1 + m);
#pragma unroll
    for (int m = 0; m < J3R; ++m) {
        zm[m] = ld4(k - 1, r0 + m);
        zp[m] = ld4(k + 1, r0 + m);
        const int64_t i = r0 + m;
        xo[m] = (ldx && i >= rmin && i <= rmax) ? row3(U, k, i)[jx] : 0.f;
    }
#pragma unroll
    for (int m = 0; m < J3R + 2; ++m) clip(pc[m]);
#pragma unroll
    for (int m = 0; m < J3R; ++m) {
        clip(zm[m]);
        clip(zp[m]);
    }
    float *vb = (float *)V.base;
#pragma unroll
    for (int m = 0; m < J3R; ++m) {
        const float4 mid = pc[m + 1], up = pc[m], dn = pc[m + 2], lo = zm[m], hi = zp[m];
        const float w_in = __shfl_up_sync(0xffffffffu, mid.w, 1);
        const float e_in = __shfl_down_sync(0xffffffffu, mid.x, 1);
        const float w = lane == 0 ? xo[m] : w_in;
        const float e = lane == 31 ? xo[m] : e_in;
        const int64_t i = r0 + m;
        if (i > g.y1 || j0 > g.x1) continue;
        float4 o;
        o.x = j7(mid.x, lo.x, hi.x, up.x, dn.x, w, mid.y);
        o.y = j7(mid.y, lo.y, hi.y, up.y, dn.y, mid.x, mid.z);
        o.z = j7(mid.z, lo.z, hi.z, up.z, dn.z, mid.y, mid.w);
        o.w = j7(mid.w, lo.w, hi.w, up.w, dn.w, mid.z, e);
        float *dst = vb + k * V.s[0] + i * V.s[1] + j0;
        if (j0 + 3 <= g.x1) {
            *(float4 *)dst = o;
        } else {
            dst[0] = o.x;
            if (j0 + 1 <= g.x1) dst[1] = o.y;
            if (j0 + 2 <= g.x1) dst[2] = o.z;
        }
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
            c = vec ? (uint64_t)((w + J3W * 128 - 1) / (J3W * 128)) * (uint64_t)((h + J3R - 1) / J3R) * (uint64_t)d
                    : (uint64_t)((w * h * d + ST - 1) / ST);
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)c;
        total += (uint32_t)c;
    }
    return total;
}

cudaError_t launch_jacobi3d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 1)
        jacobi3d_vec_kernel<<<ctas, J3W * 32, 0, st>>>(dev, p);
    else
        jacobi3d_scalar_kernel<<<ctas, ST, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
