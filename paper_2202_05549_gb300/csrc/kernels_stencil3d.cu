// 3-D 7-point Jacobi built-in:
//   "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]"
//   V = ((((((U + U[k-1]) + U[k+1]) + U[i-1]) + U[i+1]) + U[j-1]) + U[j+1]) / 7
// zero outside the domain, __fadd_rn in that fixed order, then a correctly
// rounded division by 7 (div_const_rn).
// Three kernels compute it: the staged kernel (TMA plane ring, below) for
// tasks whose columns start 16-byte aligned; the register-strip kernel when no
// tensor map can be built for a launch; the scalar kernel for tasks whose
// columns do not start 16-byte aligned.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "div_const.cuh"
#include "kernels.cuh"
#include "task_lookup.cuh"
#include "tma.cuh"

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

// Staged kernel.  A work unit is a tile of TH rows x TW columns of one task,
// over a range of at most ZSEG planes [za, zb].  Thread 0 streams the tile's
// planes za-1 .. zb+1 into a ring of NS shared-memory slots with 3-D TMA
// loads.  Each box is BW x BH x 1: the tile plus one row above and below and
// TXH columns on each side (TXH = 4 keeps the box's first column 16-byte
// aligned).  Loads run up to NS-3 planes ahead of the plane being computed,
// across unit boundaries.  The tensor map spans the chunk's stored box; a
// stencil read leaves that box only across the domain edge, where TMA's zero
// fill is the boundary value.  Columns stored in front of the chunk box (row
// padding) are loaded but feed no output.  Warp w computes rows 4w .. 4w+3 of
// the tile, 4 columns per lane, and keeps planes k-1, k and k+1 of those rows
// in registers while it walks along k: one plane step reads 6 float4 of shared
// memory per lane (plane k+1's four rows, plane k's rows above and below) and
// two scalars in lanes 0 and 31 (the columns beside the tile).
constexpr int TW = 128, TH = 32, TXH = 4;
constexpr int BW = TW + 2 * TXH, BH = TH + 2;
constexpr int NS = 5;      // plane slots
constexpr int ZSEG = 16;   // planes per work unit (16: 0.958 of HBM at 1024^3; 32: 0.92, 64: 0.89)
constexpr int TT = 256;    // threads per CTA: 8 warps x 4 rows
constexpr int TCTA = 2;    // CTAs per SM
constexpr uint32_t PLANE_BYTES = BW * BH * 4;                  // bytes one box load writes
constexpr int SLOT = (int)((PLANE_BYTES + 1023) / 1024 * 1024) / 4;  // floats per slot (1024-byte aligned slots)
constexpr int TMA_SMEM = NS * SLOT * 4 + NS * 8 + 1024;
constexpr int J3_MAX_MAPS = 48;
static_assert(TH == 4 * (TT / 32), "a warp computes 4 rows");
static_assert(TW == 4 * 32, "a lane computes 4 columns");
static_assert((TXH * 4) % 16 == 0, "box columns must start 16-byte aligned");
static_assert(NS >= 4, "planes k-1, k, k+1 and one load in flight");

struct J3Maps {
    CUtensorMap m[J3_MAX_MAPS];
};

struct J3Unit {
    int64_t x0, y0, za, zb;  // tile origin and plane range (global)
    int64_t x1, y1;          // last output column and row of the task (clipped)
    int32_t cx, cy, cz;      // tensor coordinates of the box of plane za-1
    int32_t mi;              // tensor map of the task's U chunk
    uint64_t vrow;           // byte address of V(za, y0 + 4w, x0 + 4 lane) for this thread
    int64_t vs0, vs1;        // V strides in bytes (plane, row)
};

__device__ __forceinline__ void j3_unit(const ExecTask *tasks, const ExecParams &p, uint32_t u, int warp, int lane,
                                        J3Unit &d) {
    const ExecTask &t = tasks[task_of(tasks, p, u)];
    uint32_t l = u - t.cta_begin;
    const uint32_t gx = (uint32_t)t.aux[1], gy = (uint32_t)t.aux[2];
    const uint32_t tx = l % gx;
    l /= gx;
    const uint32_t ty = l % gy, tz = l / gy;
    d.x0 = t.t_lo[0] + (int64_t)tx * TW;
    d.y0 = t.t_lo[1] + (int64_t)ty * TH;
    d.za = t.t_lo[2] + (int64_t)tz * ZSEG;
    d.zb = min(d.za + ZSEG - 1, min(t.t_hi[2], p.shape[0][0] - 1));
    d.x1 = min(t.t_hi[0], p.shape[0][2] - 1);
    d.y1 = min(t.t_hi[1], p.shape[0][1] - 1);
    const DView &U = t.v[0], &V = t.v[1];
    d.cx = (int32_t)(d.x0 - TXH - U.org[2]);
    d.cy = (int32_t)(d.y0 - 1 - U.org[1]);
    d.cz = (int32_t)(d.za - 1 - U.org[0]);
    d.mi = t.aux[0];
    d.vs0 = V.s[0] * 4;
    d.vs1 = V.s[1] * 4;
    d.vrow = V.base + (uint64_t)((d.za * V.s[0] + (d.y0 + 4 * warp) * V.s[1] + d.x0 + 4 * lane) * 4);
}

__device__ __forceinline__ float4 lds4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

__global__ void __launch_bounds__(TT, TCTA)
    jacobi3d_tma_kernel(const ExecTask *__restrict__ tasks, ExecParams p, const __grid_constant__ J3Maps maps,
                        uint32_t units) {
    extern __shared__ uint8_t smem_raw[];
    float *ring = (float *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(ring + NS * SLOT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) tma::mbar_init(&full[s], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    // producer state (thread 0): load n goes to slot n % NS once load n - NS
    // has been consumed by every thread
    uint32_t pu = blockIdx.x, issued = 0;
    int32_t pk = 0, pn = 0;  // next plane of unit pu (0 = za-1) and its plane count
    J3Unit pd;
    if (tid == 0 && pu < units) {
        j3_unit(tasks, p, pu, 0, 0, pd);
        pn = (int32_t)(pd.zb - pd.za + 3);
    }
    auto produce = [&](uint32_t freed) {
        if (issued < freed + NS && pu < units) tma::fence_proxy_async_smem();
        while (issued < freed + NS && pu < units) {
            const uint32_t s = issued % NS;
            tma::mbar_expect_tx(&full[s], PLANE_BYTES);
            tma::load_3d(ring + s * SLOT, &maps.m[pd.mi], pd.cx, pd.cy, pd.cz + pk, &full[s]);
            ++issued;
            if (++pk == pn) {
                pu += gridDim.x;
                pk = 0;
                if (pu < units) {
                    j3_unit(tasks, p, pu, 0, 0, pd);
                    pn = (int32_t)(pd.zb - pd.za + 3);
                }
            }
        }
    };
    if (tid == 0) produce(0);

    auto slot = [&](uint32_t n) { return ring + (n % NS) * SLOT; };
    auto ready = [&](uint32_t n) { return tma::mbar_wait(&full[n % NS], (n / NS) & 1u, p.err, 0x6710u); };
    const int col = TXH + 4 * lane;                    // shared-memory column of this lane's first output
    const int hcol = lane == 0 ? TXH - 1 : TXH + TW;  // the column beside the tile (lanes 0 and 31)
    const int r0 = 4 * warp + 1;                       // shared-memory row of this warp's first output
    uint32_t consumed = 0;
    bool failed = false;
    for (uint32_t u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        J3Unit d;
        j3_unit(tasks, p, u, warp, lane, d);
        const uint32_t base = consumed;
        const int nz = (int)(d.zb - d.za + 1);
        bool ok = ready(base);
        ok = ready(base + 1) && ok;
        ok = ready(base + 2) && ok;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        float4 zm[4], c[4];
        {
            const float *P = slot(base), *Q = slot(base + 1);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                zm[m] = lds4(P + (r0 + m) * BW + col);
                c[m] = lds4(Q + (r0 + m) * BW + col);
            }
        }
        const int64_t j0 = d.x0 + 4 * lane;
        const int64_t ilast = d.y1 - (d.y0 + 4 * warp);  // rows m <= ilast are inside the task
        const bool colin = j0 <= d.x1;
        const int nfull = (int)min(d.x1 - j0 + 1, (int64_t)4);
        uint64_t vk = d.vrow;
        for (int kk = 0; kk < nz; ++kk) {
            const float *P0 = slot(base + kk + 1), *P1 = slot(base + kk + 2);  // planes k and k+1
            float4 zp[4];
            float xo[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                zp[m] = lds4(P1 + (r0 + m) * BW + col);
                xo[m] = P0[(r0 + m) * BW + hcol];
            }
            const float4 above = lds4(P0 + (r0 - 1) * BW + col), below = lds4(P0 + (r0 + 4) * BW + col);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 mid = c[m], up = m == 0 ? above : c[m - 1], dn = m == 3 ? below : c[m + 1];
                const float4 lo = zm[m], hi = zp[m];
                const float w_in = __shfl_up_sync(0xffffffffu, mid.w, 1);
                const float e_in = __shfl_down_sync(0xffffffffu, mid.x, 1);
                const float w = lane == 0 ? xo[m] : w_in;
                const float e = lane == 31 ? xo[m] : e_in;
                if (colin && m <= ilast) {
                    float4 o;
                    o.x = j7(mid.x, lo.x, hi.x, up.x, dn.x, w, mid.y);
                    o.y = j7(mid.y, lo.y, hi.y, up.y, dn.y, mid.x, mid.z);
                    o.z = j7(mid.z, lo.z, hi.z, up.z, dn.z, mid.y, mid.w);
                    o.w = j7(mid.w, lo.w, hi.w, up.w, dn.w, mid.z, e);
                    float *dst = (float *)(vk + (uint64_t)(m * d.vs1));
                    if (nfull == 4) {
                        *(float4 *)dst = o;
                    } else {
                        dst[0] = o.x;
                        if (nfull > 1) dst[1] = o.y;
                        if (nfull > 2) dst[2] = o.z;
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                zm[m] = c[m];
                c[m] = zp[m];
            }
            vk += (uint64_t)d.vs0;
            const bool next_ok = kk + 1 < nz ? ready(base + kk + 3) : true;
            // every thread is done with plane k-1 (and, after the last plane, with the unit)
            if (__syncthreads_or(!next_ok)) {
                failed = true;
                break;
            }
            if (tid == 0) produce(kk + 1 < nz ? base + kk + 1 : base + nz + 2);
        }
        consumed = base + nz + 2;
    }
    if (failed && tid == 0) {
        // a wait expired: let the loads still in flight land before the CTA's
        // shared memory is released
        for (uint32_t n = issued > (uint32_t)NS ? issued - NS : 0; n < issued; ++n)
            tma::mbar_drain(&full[n % NS], (n / NS) & 1u);
    }
}

J3Maps g_j3maps;        // built by prepare, consumed by the launch that follows it
uint32_t g_j3units = 0;
int g_j3sms = 0;

// 3-D f32 map over the stored box of a chunk view: x from org[2] (a multiple
// of 4), y and z from org[1] and org[0], up to hi; box BW x BH x 1.
bool j3_make_map(CUtensorMap *m, const DView &U) {
    tma::EncodeTiledFn fn = tma::encode_tiled();
    if (!fn) return false;
    const uint64_t start = U.base + (uint64_t)((U.org[0] * U.s[0] + U.org[1] * U.s[1] + U.org[2]) * 4);
    cuuint64_t dims[3] = {(cuuint64_t)(U.hi[2] - U.org[2] + 1), (cuuint64_t)(U.hi[1] - U.org[1] + 1),
                          (cuuint64_t)(U.hi[0] - U.org[0] + 1)};
    cuuint64_t strides[2] = {(cuuint64_t)U.s[1] * 4, (cuuint64_t)U.s[0] * 4};
    cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)BH, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)(uintptr_t)start, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Plans the staged kernel for a launch: one map per distinct U chunk, work
// units per task.  Returns the CTA count, or 0 when the launch does not
// qualify (columns or chunks not 16-byte aligned, too many chunks, offsets
// beyond 32 bits).
uint32_t prepare_jacobi3d_tma(ExecTask *t, int n, const ExecParams &p) {
    const int64_t NZ = p.shape[0][0], NY = p.shape[0][1], NX = p.shape[0][2];
    std::vector<uint64_t> starts;
    const int64_t lim = (int64_t)1 << 30;
    for (int i = 0; i < n; ++i) {
        const DView &U = t[i].v[0];
        if (t[i].t_lo[0] % 4 != 0 || U.org[2] % 4 != 0) return 0;
        for (int a = 0; a < 3; ++a)
            if (U.hi[a] - U.org[a] >= lim || U.org[a] >= lim || U.org[a] < 0) return 0;
        if (U.s[1] * 4 >= ((int64_t)1 << 40) || U.s[0] * 4 >= ((int64_t)1 << 40)) return 0;
    }
    // one map per distinct chunk (decided before any map is encoded)
    std::vector<int> first;  // task that introduces each map
    for (int i = 0; i < n; ++i) {
        const DView &U = t[i].v[0];
        const uint64_t st = U.base + (uint64_t)((U.org[0] * U.s[0] + U.org[1] * U.s[1] + U.org[2]) * 4);
        int mi = -1;
        for (size_t j = 0; j < starts.size() && mi < 0; ++j)
            if (starts[j] == st) mi = (int)j;
        if (mi < 0) {
            if ((int)starts.size() == J3_MAX_MAPS) return 0;
            mi = (int)starts.size();
            starts.push_back(st);
            first.push_back(i);
        }
        t[i].aux[0] = mi;
    }
    for (size_t j = 0; j < first.size(); ++j)
        if (!j3_make_map(&g_j3maps.m[j], t[first[j]].v[0])) return 0;
    uint64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        const int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        const int64_t dd = std::min(t[i].t_hi[2], NZ - 1) - t[i].t_lo[2] + 1;
        uint64_t c = 0;
        if (w > 0 && h > 0 && dd > 0) {
            t[i].aux[1] = (int32_t)((w + TW - 1) / TW);
            t[i].aux[2] = (int32_t)((h + TH - 1) / TH);
            c = (uint64_t)t[i].aux[1] * (uint64_t)t[i].aux[2] * (uint64_t)((dd + ZSEG - 1) / ZSEG);
        } else {
            t[i].aux[1] = t[i].aux[2] = 1;
        }
        t[i].cta_begin = (uint32_t)total;
        t[i].cta_count = (uint32_t)c;
        total += c;
        if (total >= 0xFFFFFFF0ull) return 0;
    }
    if (!g_j3sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_j3sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_j3sms <= 0) g_j3sms = 148;
    }
    g_j3units = (uint32_t)total;
    return (uint32_t)std::min<uint64_t>(total, (uint64_t)g_j3sms * TCTA);
}

}  // namespace

namespace k {

uint32_t prepare_jacobi3d(ExecTask *t, int n, ExecParams &p) {
    const int64_t NZ = p.shape[0][0], NY = p.shape[0][1], NX = p.shape[0][2];
    bool vec = true;
    for (int i = 0; i < n && vec; ++i)
        for (int a = 0; a < 2; ++a)
            if (t[i].v[a].s[2] != 1 || t[i].v[a].s[1] % 4 != 0 || t[i].v[a].s[0] % 4 != 0 ||
                t[i].v[a].base % 16 != 0)
                vec = false;
    if (vec && !p.no_staged) {
        const uint32_t ctas = prepare_jacobi3d_tma(t, n, p);
        if (ctas) {
            p.variant = 2;
            return ctas;
        }
    }
    vec = true;
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
    if (p.variant == 2) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(jacobi3d_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TMA_SMEM);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        jacobi3d_tma_kernel<<<ctas, TT, TMA_SMEM, st>>>(dev, p, g_j3maps, g_j3units);
    } else if (p.variant == 1)
        jacobi3d_vec_kernel<<<ctas, J3W * 32, 0, st>>>(dev, p);
    else
        jacobi3d_scalar_kernel<<<ctas, ST, 0, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
