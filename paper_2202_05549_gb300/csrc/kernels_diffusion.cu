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

#include "async_copy.cuh"
#include "kernels.cuh"
#include "task_lookup.cuh"

namespace lt {
namespace {

__device__ __forceinline__ float at2(const DView &v, int64_t i, int64_t j) {
    return ((const float *)v.base)[i * v.s[0] + j * v.s[1]];
}

__device__ __forceinline__ float lap5(float c, float n, float s, float w, float e) {
    return __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(n, s), w), e), __fmul_rn(4.0f, c));
}

constexpr int DT = 256;            // threads per CTA
constexpr int TY = 32, TX = 128;   // cells per CTA tile
constexpr int SP = TX + 2 + 1;     // shared row pitch (halo + bank padding)

// Tiles of TY x TX cells over the box [by0, by1] x [bx0, bx1].
// (32-bit split: a 64-bit division costs registers and latency in every CTA)
__device__ __forceinline__ void tile_of(uint32_t local, int64_t bx0, int64_t bx1, int64_t by0, int64_t *ty0,
                                        int64_t *tx0) {
    const uint32_t gx = (uint32_t)((bx1 - bx0 + TX) / TX);
    *ty0 = by0 + (int64_t)(local / gx) * TY;
    *tx0 = bx0 + (int64_t)(local % gx) * TX;
}

// LAP: the Laplacian alone, G = L U (views U, G); else V = U + K (L U) (views U, K, V).
template <bool LAP>
__global__ void __launch_bounds__(DT) diffusion_fwd_scalar_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ float su[TY + 2][SP];
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    int64_t ty0, tx0;
    tile_of(blockIdx.x - t.cta_begin, x0, x1, y0, &ty0, &tx0);
    const DView U = t.v[0], K = t.v[1], V = t.v[LAP ? 1 : 2];
    // U over the tile plus a one-cell ring (zero outside the domain)
    for (int e = threadIdx.x; e < (TY + 2) * (TX + 2); e += DT) {
        const int li = e / (TX + 2), lj = e % (TX + 2);
        const int64_t i = ty0 - 1 + li, j = tx0 - 1 + lj;
        su[li][lj] = (i >= 0 && i < NY && j >= 0 && j < NX && i <= y1 + 1 && j <= x1 + 1) ? at2(U, i, j) : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TY * TX; e += DT) {
        const int li = e / TX + 1, lj = e % TX + 1;
        const int64_t i = ty0 + li - 1, j = tx0 + lj - 1;
        if (i > y1 || j > x1) continue;
        const float c = su[li][lj];
        const float l = lap5(c, su[li - 1][lj], su[li + 1][lj], su[li][lj - 1], su[li][lj + 1]);
        ((float *)V.base)[i * V.s[0] + j * V.s[1]] = LAP ? l : __fadd_rn(c, __fmul_rn(at2(K, i, j), l));
    }
}

__global__ void __launch_bounds__(DT) diffusion_adj_scalar_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ float ss[TY + 2][SP];  // s = K * L1 of the superblock's own cells, 0 elsewhere
    __shared__ float su[TY + 2][SP];  // u_t
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    // the superblock's cells (thread box clipped to the domain)
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    // its reduce region: one cell wider, clipped
    const int64_t rx0 = max(x0 - 1, (int64_t)0), ry0 = max(y0 - 1, (int64_t)0);
    const int64_t rx1 = min(x1 + 1, NX - 1), ry1 = min(y1 + 1, NY - 1);
    int64_t ty0, tx0;
    tile_of(blockIdx.x - t.cta_begin, rx0, rx1, ry0, &ty0, &tx0);
    const DView L1 = t.v[0], K = t.v[1], U = t.v[2], G = t.v[3], L0 = t.v[4];
    for (int e = threadIdx.x; e < (TY + 2) * (TX + 2); e += DT) {
        const int li = e / (TX + 2), lj = e % (TX + 2);
        const int64_t i = ty0 - 1 + li, j = tx0 - 1 + lj;
        const bool sb = i >= y0 && i <= y1 && j >= x0 && j <= x1;
        ss[li][lj] = sb ? __fmul_rn(at2(K, i, j), at2(L1, i, j)) : 0.f;
        su[li][lj] = (sb || (i >= 0 && i < NY && j >= 0 && j < NX && i >= y0 - 1 && i <= y1 + 1 && j >= x0 - 1 &&
                             j <= x1 + 1))
                         ? at2(U, i, j)
                         : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TY * TX; e += DT) {
        const int li = e / TX + 1, lj = e % TX + 1;
        const int64_t i = ty0 + li - 1, j = tx0 + lj - 1;
        if (i > ry1 || j > rx1) continue;
        float acc = 0.f;
        if (i >= y0 && i <= y1 && j >= x0 && j <= x1) {
            const float l1 = at2(L1, i, j);
            acc = __fsub_rn(l1, __fmul_rn(4.0f, ss[li][lj]));
            const float c = su[li][lj];
            float *g = (float *)G.base + i * G.s[0] + j * G.s[1];
            *g = __fadd_rn(*g, __fmul_rn(l1, lap5(c, su[li - 1][lj], su[li + 1][lj], su[li][lj - 1], su[li][lj + 1])));
        }
        // contributions of the superblock's neighbours of (i, j): north, south, west, east
        acc = __fadd_rn(acc, ss[li - 1][lj]);
        acc = __fadd_rn(acc, ss[li + 1][lj]);
        acc = __fadd_rn(acc, ss[li][lj - 1]);
        acc = __fadd_rn(acc, ss[li][lj + 1]);
        ((float *)L0.base)[i * L0.s[0] + j * L0.s[1]] = acc;
    }
}

// ---------------------------------------------------------------- vector variants
// Tiles start on 4-aligned global columns; every view is row-major with
// 16-byte aligned rows, so float4 groups are aligned in every chunk and
// partial (storage is padded to 128-byte column boundaries).  Elements of a
// group that lie outside what the annotation lets the kernel read are
// zeroed after the load (the group itself stays inside the padded storage).
constexpr int VQ = TX / 4;          // float4 groups per tile row
constexpr int VP = TX + 8;          // shared pitch: 4 columns of halo room each side

__device__ __forceinline__ float4 ld4v(const DView &v, int64_t i, int64_t j) {
    return *(const float4 *)((const float *)v.base + i * v.s[0] + j);
}
__device__ __forceinline__ float sel(bool b, float x) { return b ? x : 0.f; }

// Both vector kernels issue every load of a thread (its staging groups, its
// ring cells and the groups its compute phase needs) before using any, then
// mask, stage and compute: no load waits behind another.
constexpr int NS = ((TY + 2) * VQ + DT - 1) / DT;  // staging groups per thread (last one partial)
constexpr int NC = TY * VQ / DT;                   // compute groups per thread
static_assert(TY * VQ % DT == 0, "compute groups divide evenly");

template <bool LAP>
__global__ void __launch_bounds__(DT) diffusion_fwd_vec_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ __align__(16) float su[TY + 2][VP];
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    int64_t ty0, tx0;
    tile_of(blockIdx.x - t.cta_begin, x0, x1, y0, &ty0, &tx0);
    const DView U = t.v[0], K = t.v[1], V = t.v[LAP ? 1 : 2];
    const int64_t cmax = min(x1 + 1, NX - 1), rmin = max(y0 - 1, (int64_t)0), rmax = min(y1 + 1, NY - 1);
    float4 uv[NS], kv[NC];
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) {
        const int e = threadIdx.x + s2 * DT;
        const int li = e / VQ, q = e % VQ;
        const int64_t i = ty0 - 1 + li, j = tx0 + 4 * q;
        uv[s2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < (TY + 2) * VQ && i >= rmin && i <= rmax && j <= cmax) uv[s2] = ld4v(U, i, j);
    }
#pragma unroll
    for (int c2 = 0; c2 < NC; ++c2) {
        const int e = threadIdx.x + c2 * DT;
        const int64_t i = ty0 + e / VQ, j = tx0 + 4 * (e % VQ);
        kv[c2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!LAP && i <= y1 && j <= x1) kv[c2] = ld4v(K, i, j);
    }
    float ring = 0.f;
    const int re = threadIdx.x;
    const int64_t ri = ty0 - 1 + (re >> 1), rj = (re & 1) ? tx0 + TX : tx0 - 1;
    if (re < 2 * (TY + 2) && ri >= rmin && ri <= rmax && rj >= 0 && rj <= cmax) ring = at2(U, ri, rj);
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) {
        const int e = threadIdx.x + s2 * DT;
        if (e >= (TY + 2) * VQ) break;
        const int li = e / VQ, q = e % VQ;
        const int64_t j = tx0 + 4 * q;
        float4 v = uv[s2];
        v.y = sel(j + 1 <= cmax, v.y);
        v.z = sel(j + 2 <= cmax, v.z);
        v.w = sel(j + 3 <= cmax, v.w);
        *(float4 *)&su[li][4 + 4 * q] = v;
    }
    if (re < 2 * (TY + 2)) su[re >> 1][(re & 1) ? 4 + TX : 3] = ring;
    __syncthreads();
#pragma unroll
    for (int c2 = 0; c2 < NC; ++c2) {
        const int e = threadIdx.x + c2 * DT;
        const int li = e / VQ + 1, q = e % VQ;
        const int64_t i = ty0 + li - 1, j = tx0 + 4 * q;
        if (i > y1 || j > x1) continue;
        const int c = 4 + 4 * q;
        const float kk[4] = {kv[c2].x, kv[c2].y, kv[c2].z, kv[c2].w};
        float o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float cc = su[li][c + m];
            const float l = lap5(cc, su[li - 1][c + m], su[li + 1][c + m], su[li][c + m - 1], su[li][c + m + 1]);
            o[m] = LAP ? l : __fadd_rn(cc, __fmul_rn(kk[m], l));
        }
        float *dst = (float *)V.base + i * V.s[0] + j;
        if (j + 3 <= x1) {
            *(float4 *)dst = make_float4(o[0], o[1], o[2], o[3]);
        } else {
            for (int m = 0; m < 4 && j + m <= x1; ++m) dst[m] = o[m];
        }
    }
}

__global__ void __launch_bounds__(DT, 2) diffusion_adj_vec_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    __shared__ __align__(16) float ss[TY + 2][VP];
    __shared__ __align__(16) float su[TY + 2][VP];
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    const int64_t rx0 = max(x0 - 1, (int64_t)0), ry0 = max(y0 - 1, (int64_t)0);
    const int64_t rx1 = min(x1 + 1, NX - 1), ry1 = min(y1 + 1, NY - 1);
    const int64_t ax0 = rx0 & ~(int64_t)3;  // tiles start on 4-aligned columns
    int64_t ty0, tx0;
    tile_of(blockIdx.x - t.cta_begin, ax0, rx1, ry0, &ty0, &tx0);
    const DView L1 = t.v[0], K = t.v[1], U = t.v[2], G = t.v[3], L0 = t.v[4];
    // staging: s = K * L1 over the superblock's own cells (0 elsewhere), u over the U read region
    float4 kv[NS], lv[NS], uv[NS], l1c[NC], gc[NC];  // gc: loaded after the barrier, before the compute
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) {
        const int e = threadIdx.x + s2 * DT;
        const int li = e / VQ, q = e % VQ;
        const int64_t i = ty0 - 1 + li, j = tx0 + 4 * q;
        kv[s2] = lv[s2] = uv[s2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < (TY + 2) * VQ) {
            if (i >= y0 && i <= y1 && j + 3 >= x0 && j <= x1) {  // group meets the superblock
                kv[s2] = ld4v(K, i, j);
                lv[s2] = ld4v(L1, i, j);
            }
            if (i >= ry0 && i <= ry1 && j + 3 >= rx0 && j <= rx1) uv[s2] = ld4v(U, i, j);  // meets U's region
        }
    }
#pragma unroll
    for (int c2 = 0; c2 < NC; ++c2) {
        const int e = threadIdx.x + c2 * DT;
        const int64_t i = ty0 + e / VQ, j = tx0 + 4 * (e % VQ);
        l1c[c2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i >= y0 && i <= y1 && j + 3 >= x0 && j <= x1) l1c[c2] = ld4v(L1, i, j);
    }
    float rs = 0.f, ru = 0.f;
    const int re = threadIdx.x;
    const int64_t ri = ty0 - 1 + (re >> 1), rj = (re & 1) ? tx0 + TX : tx0 - 1;
    if (re < 2 * (TY + 2)) {
        if (ri >= y0 && ri <= y1 && rj >= x0 && rj <= x1) rs = __fmul_rn(at2(K, ri, rj), at2(L1, ri, rj));
        if (ri >= ry0 && ri <= ry1 && rj >= rx0 && rj <= rx1) ru = at2(U, ri, rj);
    }
#pragma unroll
    for (int s2 = 0; s2 < NS; ++s2) {
        const int e = threadIdx.x + s2 * DT;
        if (e >= (TY + 2) * VQ) break;
        const int li = e / VQ, q = e % VQ;
        const int64_t i = ty0 - 1 + li, j = tx0 + 4 * q;
        const bool rsb = i >= y0 && i <= y1;
        float4 sv, uu = uv[s2];
        sv.x = sel(rsb && j >= x0 && j <= x1, __fmul_rn(kv[s2].x, lv[s2].x));
        sv.y = sel(rsb && j + 1 >= x0 && j + 1 <= x1, __fmul_rn(kv[s2].y, lv[s2].y));
        sv.z = sel(rsb && j + 2 >= x0 && j + 2 <= x1, __fmul_rn(kv[s2].z, lv[s2].z));
        sv.w = sel(rsb && j + 3 >= x0 && j + 3 <= x1, __fmul_rn(kv[s2].w, lv[s2].w));
        uu.x = sel(j >= rx0 && j <= rx1, uu.x);
        uu.y = sel(j + 1 >= rx0 && j + 1 <= rx1, uu.y);
        uu.z = sel(j + 2 >= rx0 && j + 2 <= rx1, uu.z);
        uu.w = sel(j + 3 >= rx0 && j + 3 <= rx1, uu.w);
        *(float4 *)&ss[li][4 + 4 * q] = sv;
        *(float4 *)&su[li][4 + 4 * q] = uu;
    }
    if (re < 2 * (TY + 2)) {
        const int c = (re & 1) ? 4 + TX : 3;
        ss[re >> 1][c] = rs;
        su[re >> 1][c] = ru;
    }
    __syncthreads();
#pragma unroll
    for (int c2 = 0; c2 < NC; ++c2) {
        const int e = threadIdx.x + c2 * DT;
        const int64_t i = ty0 + e / VQ, j = tx0 + 4 * (e % VQ);
        gc[c2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i >= y0 && i <= y1 && j + 3 >= x0 && j <= x1) gc[c2] = ld4v(G, i, j);
    }
#pragma unroll
    for (int c2 = 0; c2 < NC; ++c2) {
        const int e = threadIdx.x + c2 * DT;
        const int li = e / VQ + 1, q = e % VQ;
        const int64_t i = ty0 + li - 1, j = tx0 + 4 * q;
        if (i > ry1 || j > rx1 || j + 3 < rx0) continue;
        const int c = 4 + 4 * q;
        const bool row_sb = i >= y0 && i <= y1;
        const bool grp_sb = row_sb && j + 3 >= x0 && j <= x1;
        const float l1[4] = {l1c[c2].x, l1c[c2].y, l1c[c2].z, l1c[c2].w};
        float g[4] = {gc[c2].x, gc[c2].y, gc[c2].z, gc[c2].w};
        float o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const bool in = row_sb && j + m >= x0 && j + m <= x1;
            float acc = 0.f;
            if (in) {
                acc = __fsub_rn(l1[m], __fmul_rn(4.0f, ss[li][c + m]));
                const float cc = su[li][c + m];
                g[m] = __fadd_rn(g[m], __fmul_rn(l1[m], lap5(cc, su[li - 1][c + m], su[li + 1][c + m],
                                                              su[li][c + m - 1], su[li][c + m + 1])));
            }
            acc = __fadd_rn(acc, ss[li - 1][c + m]);
            acc = __fadd_rn(acc, ss[li + 1][c + m]);
            acc = __fadd_rn(acc, ss[li][c + m - 1]);
            acc = __fadd_rn(acc, ss[li][c + m + 1]);
            o[m] = acc;
        }
        float *dst = (float *)L0.base + i * L0.s[0] + j;
        if (j >= rx0 && j + 3 <= rx1) {
            *(float4 *)dst = make_float4(o[0], o[1], o[2], o[3]);
        } else {
            for (int m = 0; m < 4; ++m)
                if (j + m >= rx0 && j + m <= rx1) dst[m] = o[m];
        }
        if (grp_sb) {
            float *gd = (float *)G.base + i * G.s[0] + j;
            if (j >= x0 && j + 3 <= x1) {
                *(float4 *)gd = make_float4(g[0], g[1], g[2], g[3]);
            } else {
                for (int m = 0; m < 4; ++m)
                    if (j + m >= x0 && j + m <= x1) gd[m] = g[m];
            }
        }
    }
}

// Staged adjoint: the same tile and arithmetic as diffusion_adj_vec_kernel,
// but every input group goes global -> shared with cp.async (16 bytes,
// cached in L2 only) instead of through registers, so a CTA holds few
// registers and three CTAs fit on an SM with all their loads in flight.
// Shared tiles (TY+2 rows x VP columns; group q of a row, global columns
// tx0+4q .. tx0+4q+3, sits at shared columns 4+4q, q = -1 .. VQ covering the
// ring columns 3 and 4+TX): K (then s = K*L1 in place), L1, u_t and G.
// A group is copied when it meets the region its array may be read in (the
// same test as the register kernel, so the copied bytes lie in the chunk's
// padded rows); otherwise the copy zero-fills it.  Columns of a copied group
// that lie outside the region are cleared in shared memory before use.
constexpr int AQ = VQ + 2;                    // groups per staged row, ring groups included
constexpr int ATILE = (TY + 2) * VP;          // floats per staged tile
constexpr int ASMEM = 4 * ATILE * 4;          // dynamic shared memory of the kernel
constexpr int AT = DT;                        // threads per CTA
constexpr int ACTA = 3;                       // CTAs per SM the kernel is built for

__global__ void __launch_bounds__(AT, ACTA) diffusion_adj_async_kernel(const ExecTask *__restrict__ tasks,
                                                                      ExecParams p) {
    extern __shared__ __align__(16) float asmem[];
    float *sK = asmem, *sL = asmem + ATILE, *sU = asmem + 2 * ATILE, *sG = asmem + 3 * ATILE;
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    const int64_t rx0 = max(x0 - 1, (int64_t)0), ry0 = max(y0 - 1, (int64_t)0);
    const int64_t rx1 = min(x1 + 1, NX - 1), ry1 = min(y1 + 1, NY - 1);
    const int64_t ax0 = rx0 & ~(int64_t)3;  // tiles start on 4-aligned columns
    int64_t ty0, tx0;
    tile_of(blockIdx.x - t.cta_begin, ax0, rx1, ry0, &ty0, &tx0);
    const DView L1 = t.v[0], K = t.v[1], U = t.v[2], G = t.v[3], L0 = t.v[4];
    const void *nowhere = p.err;  // source of zero-filling copies (nothing is read)
    for (int e = threadIdx.x; e < (TY + 2) * AQ; e += AT) {
        const int li = e / AQ, qq = e % AQ - 1;
        const int64_t i = ty0 - 1 + li, j = tx0 + 4 * qq;
        const int o = li * VP + 4 + 4 * qq;
        const bool sb = i >= y0 && i <= y1 && j + 3 >= x0 && j <= x1;       // meets the superblock
        const bool ur = i >= ry0 && i <= ry1 && j + 3 >= rx0 && j <= rx1;   // meets U's region
        cp_async16(sK + o, sb ? (const void *)((const float *)K.base + i * K.s[0] + j) : nowhere, sb);
        cp_async16(sL + o, sb ? (const void *)((const float *)L1.base + i * L1.s[0] + j) : nowhere, sb);
        cp_async16(sU + o, ur ? (const void *)((const float *)U.base + i * U.s[0] + j) : nowhere, ur);
        if (li >= 1 && li <= TY)
            cp_async16(sG + o, sb ? (const void *)((const float *)G.base + i * G.s[0] + j) : nowhere, sb);
    }
    cp_async_wait_all();
    __syncthreads();
    // s = K * L1 on the superblock's cells, 0 elsewhere; u_t outside its region is 0
    for (int e = threadIdx.x; e < (TY + 2) * AQ; e += AT) {
        const int li = e / AQ, qq = e % AQ - 1;
        const int64_t i = ty0 - 1 + li, j = tx0 + 4 * qq;
        const int o = li * VP + 4 + 4 * qq;
        const bool rsb = i >= y0 && i <= y1;
        float4 k4 = *(float4 *)(sK + o);
        const float4 l4 = *(const float4 *)(sL + o);
        k4.x = sel(rsb && j >= x0 && j <= x1, __fmul_rn(k4.x, l4.x));
        k4.y = sel(rsb && j + 1 >= x0 && j + 1 <= x1, __fmul_rn(k4.y, l4.y));
        k4.z = sel(rsb && j + 2 >= x0 && j + 2 <= x1, __fmul_rn(k4.z, l4.z));
        k4.w = sel(rsb && j + 3 >= x0 && j + 3 <= x1, __fmul_rn(k4.w, l4.w));
        *(float4 *)(sK + o) = k4;
        if (j < rx0 || j + 3 > rx1) {
            float4 u4 = *(float4 *)(sU + o);
            u4.x = sel(j >= rx0 && j <= rx1, u4.x);
            u4.y = sel(j + 1 >= rx0 && j + 1 <= rx1, u4.y);
            u4.z = sel(j + 2 >= rx0 && j + 2 <= rx1, u4.z);
            u4.w = sel(j + 3 >= rx0 && j + 3 <= rx1, u4.w);
            *(float4 *)(sU + o) = u4;
        }
    }
    __syncthreads();
    auto ss = [&](int li, int c) { return sK[li * VP + c]; };
    auto su = [&](int li, int c) { return sU[li * VP + c]; };
    for (int e = threadIdx.x; e < TY * VQ; e += AT) {
        const int li = e / VQ + 1, q = e % VQ;
        const int64_t i = ty0 + li - 1, j = tx0 + 4 * q;
        if (i > ry1 || j > rx1 || j + 3 < rx0) continue;
        const int c = 4 + 4 * q;
        const bool row_sb = i >= y0 && i <= y1;
        const bool grp_sb = row_sb && j + 3 >= x0 && j <= x1;
        const float4 l14 = *(const float4 *)(sL + li * VP + c), g4 = *(const float4 *)(sG + li * VP + c);
        const float l1[4] = {l14.x, l14.y, l14.z, l14.w};
        float g[4] = {g4.x, g4.y, g4.z, g4.w};
        float o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const bool in = row_sb && j + m >= x0 && j + m <= x1;
            float acc = 0.f;
            if (in) {
                acc = __fsub_rn(l1[m], __fmul_rn(4.0f, ss(li, c + m)));
                const float cc = su(li, c + m);
                g[m] = __fadd_rn(g[m], __fmul_rn(l1[m], lap5(cc, su(li - 1, c + m), su(li + 1, c + m),
                                                              su(li, c + m - 1), su(li, c + m + 1))));
            }
            acc = __fadd_rn(acc, ss(li - 1, c + m));
            acc = __fadd_rn(acc, ss(li + 1, c + m));
            acc = __fadd_rn(acc, ss(li, c + m - 1));
            acc = __fadd_rn(acc, ss(li, c + m + 1));
            o[m] = acc;
        }
        float *dst = (float *)L0.base + i * L0.s[0] + j;
        if (j >= rx0 && j + 3 <= rx1) {
            *(float4 *)dst = make_float4(o[0], o[1], o[2], o[3]);
        } else {
            for (int m = 0; m < 4; ++m)
                if (j + m >= rx0 && j + m <= rx1) dst[m] = o[m];
        }
        if (grp_sb) {
            float *gd = (float *)G.base + i * G.s[0] + j;
            if (j >= x0 && j + 3 <= x1) {
                *(float4 *)gd = make_float4(g[0], g[1], g[2], g[3]);
            } else {
                for (int m = 0; m < 4; ++m)
                    if (j + m >= x0 && j + m <= x1) gd[m] = g[m];
            }
        }
    }
}

bool views_vec_ok(const ExecTask *t, int n, int nviews) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < nviews; ++a) {
            const DView &v = t[i].v[a];
            if (v.s[1] != 1 || (v.s[0] % 4) != 0 || (v.base % 16) != 0) return false;
        }
    return true;
}

}  // namespace

namespace k {

uint32_t prepare_diffusion(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    bool vec = views_vec_ok(t, n, 3);
    for (int i = 0; i < n; ++i)
        if (t[i].t_lo[0] % 4 != 0) vec = false;
    p.variant = vec ? 1 : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = (w > 0 && h > 0) ? (uint32_t)(((w + TX - 1) / TX) * ((h + TY - 1) / TY)) : 0;
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_diffusion(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 1)
        diffusion_fwd_vec_kernel<false><<<ctas, DT, 0, st>>>(dev, p);
    else
        diffusion_fwd_scalar_kernel<false><<<ctas, DT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

// The Laplacian alone (G = L U): the forward kernel without its coefficient.
uint32_t prepare_laplace(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    bool vec = views_vec_ok(t, n, 2);
    for (int i = 0; i < n; ++i)
        if (t[i].t_lo[0] % 4 != 0) vec = false;
    p.variant = vec ? 1 : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = (w > 0 && h > 0) ? (uint32_t)(((w + TX - 1) / TX) * ((h + TY - 1) / TY)) : 0;
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_laplace(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 1)
        diffusion_fwd_vec_kernel<true><<<ctas, DT, 0, st>>>(dev, p);
    else
        diffusion_fwd_scalar_kernel<true><<<ctas, DT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

uint32_t prepare_diffusion_adj(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const bool vec = views_vec_ok(t, n, 5);
    // variant 2: staged through shared memory with cp.async; 1: registers; 0: scalar
    p.variant = vec ? (p.no_staged ? 1 : 2) : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t x0 = t[i].t_lo[0], y0 = t[i].t_lo[1];
        int64_t x1 = std::min(t[i].t_hi[0], NX - 1), y1 = std::min(t[i].t_hi[1], NY - 1);
        uint32_t c = 0;
        if (x1 >= x0 && y1 >= y0) {
            int64_t bx0 = std::max<int64_t>(x0 - 1, 0);
            if (vec) bx0 &= ~(int64_t)3;
            int64_t w = std::min(x1 + 1, NX - 1) - bx0 + 1;
            int64_t h = std::min(y1 + 1, NY - 1) - std::max<int64_t>(y0 - 1, 0) + 1;
            c = (uint32_t)(((w + TX - 1) / TX) * ((h + TY - 1) / TY));
        }
        t[i].cta_begin = total;
        t[i].cta_count = c;
        total += c;
    }
    return total;
}

cudaError_t launch_diffusion_adj(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    if (p.variant == 2) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(diffusion_adj_async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 ASMEM);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        diffusion_adj_async_kernel<<<ctas, AT, ASMEM, st>>>(dev, p);
        return cudaGetLastError();
    }
    if (p.variant == 1)
        diffusion_adj_vec_kernel<<<ctas, DT, 0, st>>>(dev, p);
    else
        diffusion_adj_scalar_kernel<<<ctas, DT, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
