// Device bodies shared by the stencil kernels (single launches and the
// batched persistent kernel).
//   V[i,j] = ((((U[i,j] + U[i-1,j]) + U[i+1,j]) + U[i,j-1]) + U[i,j+1]) / 5,
// zero outside the NY x NX domain, __fadd_rn in that order and a correctly
// rounded division (no contraction).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "div_const.cuh"
#include "kernels.cuh"

namespace lt {

constexpr int JR = 16;      // output rows per warp strip
constexpr int JCOLS = 128;  // columns per warp strip (4 per lane)

__device__ __forceinline__ float sum5(float c, float n, float s, float w, float e) {
    float acc = __fadd_rn(c, n);
    acc = __fadd_rn(acc, s);
    acc = __fadd_rn(acc, w);
    return __fadd_rn(acc, e);
}

__device__ __forceinline__ float j5(float c, float n, float s, float w, float e) {
    return div_const_rn<5>(sum5(c, n, s, w, e));
}

template <bool L2ONLY>
__device__ __forceinline__ float4 ld4(const float *p) {
    if (L2ONLY) return __ldcg((const float4 *)p);
    return *(const float4 *)p;
}

template <bool L2ONLY>
__device__ __forceinline__ float ld1(const float *p) {
    if (L2ONLY) return __ldcg(p);
    return *p;
}

// One warp computes output rows r0 .. min(r0+R-1, ye) of the 128-column
// strip starting at column js (js <= xe, js % 4 == 0), reading U (row
// stride su) and writing V (row stride sv); both are views indexed with
// global indices whose rows are 16-byte aligned.  All R+2 input rows are
// loaded before any arithmetic; horizontal neighbours come from the
// adjacent lanes.  L2ONLY loads bypass L1 (data written by other SMs in the
// same kernel).  Columns read: up to min(xe+1, NX-1), in 4-aligned groups.
template <bool L2ONLY, int R = JR>
__device__ __forceinline__ void jacobi_strip(const float *ub, int64_t su, float *vb, int64_t sv, int64_t NY,
                                             int64_t NX, int64_t js, int64_t r0, int64_t xe, int64_t ye, int lane) {
    const int64_t j0 = js + lane * 4;
    const int64_t rlast = min(r0 + R - 1, ye);
    const int64_t cmax = min(xe + 1, NX - 1);  // last column that may be read
    const bool ld = j0 <= cmax;
    const int kr = (int)(rlast - r0);  // output rows r0 .. r0+kr (0 <= kr < R): a 32-bit test per row
    float4 row[R + 2];
    float side[R];  // lane 0: the west halo column, lane 31: the east one
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        row[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t r = r0 - 1 + k;
        if (ld && r >= 0 && r < NY && r <= rlast + 1) row[k] = ld4<L2ONLY>(ub + r * su + j0);
    }
    const bool side_ok = lane == 0 ? (j0 - 1 >= 0 && ld) : (lane == 31 && j0 + 4 <= cmax);
    if (L2ONLY) {
        // (the batch kernel) the halo column's address computed for each row
        const int64_t sc = lane == 0 ? j0 - 1 : j0 + 4;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            side[k] = 0.f;
            if (side_ok && k <= kr) side[k] = ld1<L2ONLY>(ub + (r0 + k) * su + sc);
        }
    } else {
        // (the single-launch kernels) a pointer that walks down the halo
        // column: fewer instructions there, more registers in the batch
        // kernel (measured both ways on each)
        const float *sp = ub + r0 * su + (lane == 0 ? j0 - 1 : j0 + 4);
#pragma unroll
        for (int k = 0; k < R; ++k, sp += su) {
            side[k] = 0.f;
            if (side_ok && k <= kr) side[k] = ld1<L2ONLY>(sp);
        }
    }
    // columns of this lane that lie outside the domain read as 0 (the last
    // strip of a row of the grid only)
    if (j0 + 3 > NX - 1) {
#pragma unroll
        for (int k = 0; k < R + 2; ++k) {
            if (j0 + 1 > NX - 1) row[k].y = 0.f;
            if (j0 + 2 > NX - 1) row[k].z = 0.f;
            row[k].w = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t r = r0 + k;
        const float4 up = row[k], mid = row[k + 1], dn = row[k + 2];
        float w_in = __shfl_up_sync(0xffffffffu, mid.w, 1);
        float e_in = __shfl_down_sync(0xffffffffu, mid.x, 1);
        float w = lane == 0 ? side[k] : w_in;
        float e = lane == 31 ? side[k] : e_in;
        if (k > kr || j0 > xe) continue;
        const float4 o = div4_const_rn<5>(make_float4(sum5(mid.x, up.x, dn.x, w, mid.y),
                                                      sum5(mid.y, up.y, dn.y, mid.x, mid.z),
                                                      sum5(mid.z, up.z, dn.z, mid.y, mid.w),
                                                      sum5(mid.w, up.w, dn.w, mid.z, e)));
        float *dst = vb + r * sv + j0;
        if (j0 + 3 <= xe) {
            *(float4 *)dst = o;
        } else {
            dst[0] = o.x;
            if (j0 + 1 <= xe) dst[1] = o.y;
            if (j0 + 2 <= xe) dst[2] = o.z;
        }
    }
}

// Write-through replicas (ExecParams.reps): thread `cell` of the CTAs that
// follow the tasks' CTAs computes one replica cell from the input view of the
// task that owns it, with the same operations as that task, and stores it to
// the replica's view.
__device__ __forceinline__ void jacobi_replica_cell(const ExecTask *tasks, const ExecParams &p, uint64_t cell) {
    if (cell >= p.rep_cells) return;
    int lo = 0, hi = (int)p.nreps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.reps[mid].cell_begin <= cell)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ReplicaTarget &r = p.reps[lo];
    const uint64_t l = cell - r.cell_begin, w = (uint64_t)(r.hi[1] - r.lo[1] + 1);
    const int64_t i = r.lo[0] + (int64_t)(l / w), j = r.lo[1] + (int64_t)(l % w);
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const DView U = tasks[r.task].v[0];
    const float *u = (const float *)U.base;
    auto at = [&](int64_t a, int64_t b) { return u[a * U.s[0] + b * U.s[1]]; };
    const float c = at(i, j);
    const float n = i > 0 ? at(i - 1, j) : 0.f;
    const float s = i + 1 < NY ? at(i + 1, j) : 0.f;
    const float wv = j > 0 ? at(i, j - 1) : 0.f;
    const float e = j + 1 < NX ? at(i, j + 1) : 0.f;
    ((float *)r.dst.base)[i * r.dst.s[0] + j * r.dst.s[1]] = j5(c, n, s, wv, e);
}

// Write-through replicas by warp units (ExecParams.runits): a row unit is
// the strip body with one row, reading the owning task's input view and
// storing into the replica's view; any other unit computes 32 cells, one per
// lane, as jacobi_replica_cell does.  Same operations as the owning task.
__device__ __forceinline__ void jacobi_replica_unit(const ExecTask *tasks, const ExecParams &p, uint32_t unit,
                                                    int lane) {
    if (unit >= p.nunits) return;
    const ReplicaUnit u = p.runits[unit];
    const ReplicaTarget &r = p.reps[u.rep];
    const DView U = tasks[r.task].v[0];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    if (u.row) {
        jacobi_strip<false, 1>((const float *)U.base, U.s[0], (float *)r.dst.base, r.dst.s[0], NY, NX,
                               r.lo[1] + (int64_t)u.off, r.lo[0], r.hi[1], r.lo[0], lane);
        return;
    }
    const uint64_t w = (uint64_t)(r.hi[1] - r.lo[1] + 1), cells = w * (uint64_t)(r.hi[0] - r.lo[0] + 1);
    const uint64_t l = (uint64_t)u.off + (uint64_t)lane;
    if (l >= cells) return;
    const int64_t i = r.lo[0] + (int64_t)(l / w), j = r.lo[1] + (int64_t)(l % w);
    const float *uu = (const float *)U.base;
    auto at = [&](int64_t a, int64_t b) { return uu[a * U.s[0] + b * U.s[1]]; };
    const float c = at(i, j);
    const float n = i > 0 ? at(i - 1, j) : 0.f;
    const float s = i + 1 < NY ? at(i + 1, j) : 0.f;
    const float wv = j > 0 ? at(i, j - 1) : 0.f;
    const float e = j + 1 < NX ? at(i, j + 1) : 0.f;
    ((float *)r.dst.base)[i * r.dst.s[0] + j * r.dst.s[1]] = j5(c, n, s, wv, e);
}

}  // namespace lt
