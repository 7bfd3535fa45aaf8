// Stencil built-ins, written in the paper's convention (Sec. 3.5): the body
// is a device function of the virtual (global) index and of views whose
// base already has the chunk offset subtracted (DView), so the same code
// runs on any superblock of any chunking.
//
//   stencil1d (Listings 1-2):  out[i] = (in[i-1] + in[i] + in[i+1]) / 3.0
//   jacobi2d  (HotSpot-like 5-point stencil of Sec. 4.2):
//       V[i,j] = ((((U[i,j] + U[i-1,j]) + U[i+1,j]) + U[i,j-1]) + U[i,j+1]) / 5
// Out-of-domain reads are 0.  Sums use __fadd_rn and the division is
// correctly rounded (div_const_rn),
// so no FMA contraction changes the order: chunked and unchunked results are
// bit-identical, and equal to the CPU definition.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"
#include "task_lookup.cuh"
#include "stencil_body.cuh"

namespace lt {
namespace {

// ------------------------------------------------------------------ 1-D example
__device__ __forceinline__ void stencil1d_body(int64_t i, int64_t n, const DView &out, const DView &in) {
    const float *ip = (const float *)in.base;
    float left = i - 1 >= 0 ? ip[(i - 1) * in.s[0]] : 0.0f;
    float mid = ip[i * in.s[0]];
    float right = i + 1 < n ? ip[(i + 1) * in.s[0]] : 0.0f;
    float s = __fadd_rn(__fadd_rn(left, mid), right);
    ((float *)out.base)[i * out.s[0]] = __double2float_rn(__ddiv_rn((double)s, 3.0));
}

__global__ void __launch_bounds__(256) stencil1d_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    int64_t n = p.shape[0][0];
    int64_t i = t.t_lo[0] + (int64_t)(blockIdx.x - t.cta_begin) * blockDim.x + threadIdx.x;
    if (i > t.t_hi[0] || i >= n) return;
    stencil1d_body(i, n, t.v[0], t.v[1]);
}

// ------------------------------------------------------------------ 2-D Jacobi
constexpr int JWARPS = 4;    // warps per CTA, side by side along x
constexpr int JV = 8;        // rows per warp strip of the single-step kernel

// Vector variant: every lane owns 4 adjacent columns of a 128-column strip and
// sweeps R rows (jacobi_strip in stencil_body.cuh).  R = 8 keeps the kernel
// near 72 registers (7 CTAs of 128 threads per SM); the two halo rows each
// strip re-reads come from L2.  The CTA index is split with 32-bit
// arithmetic: a 64-bit division here costs registers and prologue latency in
// every CTA.
// Programmatic dependent launch: when p.pdl is set the kernel may start while
// the previous kernel on the stream is finishing.  Every CTA lets the next
// kernel launch at once (its CTAs take SM slots only as ours retire) and
// waits for the previous kernel's completion and memory before it touches
// array data; only the task table, which no kernel writes, is read before.
__device__ __forceinline__ void pdl_trigger_and_wait(const ExecParams &p) {
    if (p.pdl) {
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        asm volatile("griddepcontrol.wait;" ::: "memory");
    }
}

template <int R>
__global__ void __launch_bounds__(JWARPS * 32) jacobi2d_vec_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    if (blockIdx.x < p.rep_ctas) {  // write-through replica CTAs come first: their latency overlaps the strips
        pdl_trigger_and_wait(p);
        jacobi_replica_unit(tasks, p, blockIdx.x * JWARPS + (threadIdx.x >> 5), threadIdx.x & 31);
        return;
    }
    const uint32_t cta = blockIdx.x - p.rep_ctas;
    int ti = task_of(tasks, p, cta);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t xe = min(t.t_hi[0], NX - 1), ye = min(t.t_hi[1], NY - 1);  // last output column / row
    const uint32_t width = (uint32_t)(t.t_hi[0] - x0 + 1);
    const uint32_t gx = (width + JWARPS * JCOLS - 1) / (JWARPS * JCOLS);
    const uint32_t local = cta - t.cta_begin;
    const uint32_t tx = local % gx, ty = local / gx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t js = x0 + (int64_t)(tx * JWARPS + warp) * JCOLS;  // first column of this warp's strip
    const int64_t r0 = y0 + (int64_t)ty * R;
    pdl_trigger_and_wait(p);
    if (js > xe || r0 > ye) return;  // warp-uniform: nothing to write
    jacobi_strip<false, R>((const float *)t.v[0].base, t.v[0].s[0], (float *)t.v[1].base, t.v[1].s[0], NY, NX, js,
                           r0, xe, ye, lane);
}

// Scalar variant for unaligned tasks: one thread per output cell.
__global__ void __launch_bounds__(256) jacobi2d_scalar_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    if (blockIdx.x < p.rep_ctas) {  // write-through replica CTAs
        jacobi_replica_cell(tasks, p, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x);
        return;
    }
    const uint32_t cta = blockIdx.x - p.rep_ctas;
    int ti = task_of(tasks, p, cta);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t width = t.t_hi[0] - t.t_lo[0] + 1;
    const int64_t cell = (int64_t)(cta - t.cta_begin) * blockDim.x + threadIdx.x;
    const int64_t j = t.t_lo[0] + cell % width, i = t.t_lo[1] + cell / width;
    if (i > t.t_hi[1] || i >= NY || j >= NX) return;
    const DView U = t.v[0], V = t.v[1];
    const float *u = (const float *)U.base;
    auto at = [&](int64_t a, int64_t b) { return u[a * U.s[0] + b * U.s[1]]; };
    float c = at(i, j);
    float n = i > 0 ? at(i - 1, j) : 0.f;
    float s = i + 1 < NY ? at(i + 1, j) : 0.f;
    float w = j > 0 ? at(i, j - 1) : 0.f;
    float e = j + 1 < NX ? at(i, j + 1) : 0.f;
    ((float *)V.base)[i * V.s[0] + j * V.s[1]] = j5(c, n, s, w, e);
}

}  // namespace

namespace k {

uint32_t prepare_stencil1d(ExecTask *t, int n, ExecParams &p) {
    (void)p;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t len = t[i].t_hi[0] - t[i].t_lo[0] + 1;
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)((len + 255) / 256);
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_stencil1d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    stencil1d_kernel<<<ctas, 256, 0, st>>>(dev, p);
    return cudaGetLastError();
}

uint32_t prepare_jacobi2d(ExecTask *t, int n, ExecParams &p) {
    bool vec = true;
    for (int i = 0; i < n && vec; ++i) {
        if (t[i].t_lo[0] % 4 != 0) vec = false;
        for (int a = 0; a < 2; ++a)
            if (t[i].v[a].s[1] != 1 || (t[i].v[a].s[0] % 4) != 0 || (t[i].v[a].base % 16) != 0) vec = false;
    }
    // variant 1: strips of JV rows (vector); 0: one thread per cell (scalar)
    p.variant = vec ? 1 : 0;
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = t[i].t_hi[0] - t[i].t_lo[0] + 1, h = t[i].t_hi[1] - t[i].t_lo[1] + 1;
        uint64_t c = vec ? (uint64_t)((w + JWARPS * JCOLS - 1) / (JWARPS * JCOLS)) * (uint64_t)((h + JV - 1) / JV)
                         : (uint64_t)((w * h + 255) / 256);
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)c;
        total += (uint32_t)c;
    }
    return total;
}

// The grid is the write-through replica CTAs (one thread per replica cell)
// followed by the tasks' CTAs.
cudaError_t launch_jacobi2d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    const uint32_t threads = p.variant == 1 ? JWARPS * 32 : 256;
    // replica CTAs: warp units for the vector kernel, one thread per cell for the scalar one
    const uint64_t extra = p.variant == 1 ? (p.rep_cells ? ((uint64_t)p.nunits + JWARPS - 1) / JWARPS : 0)
                                          : (p.rep_cells + threads - 1) / threads;
    if ((uint64_t)ctas + extra > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    ExecParams q = p;
    q.rep_ctas = (uint32_t)extra;
    const uint32_t grid = ctas + (uint32_t)extra;
    if (p.variant == 1 && p.pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(threads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, jacobi2d_vec_kernel<JV>, dev, q);
    }
    q.pdl = 0;
    if (p.variant == 1)
        jacobi2d_vec_kernel<JV><<<grid, threads, 0, st>>>(dev, q);
    else
        jacobi2d_scalar_kernel<<<grid, threads, 0, st>>>(dev, q);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt

// ------------------------------------------------------------------ k steps per launch
// Temporal blocking: "global [i, j] => read U[i-k:i+k, j-k:j+k], write V[i, j]"
// computes k Jacobi iterations in one launch; every value it keeps equals the
// one the k sequential iterations compute (zero ghosts outside the array).
namespace lt {
namespace {

// Register pipeline (aligned tasks).  Each warp owns a 128-column window (4
// columns per lane) and streams down a segment of MH output rows.  Level l
// holds iteration l: at row step tr the warp loads row tr of the input
// (level 0), and each level l+1 produces row tr-l-1 from rows tr-l-2 ..
// tr-l of level l, which stay in registers (two previous rows per level and
// the row just produced), so every iteration of a row costs no memory
// access.  Horizontal neighbours come from the adjacent lanes; lanes 0 and 31
// see zeros beyond the window, which spoils one more column per level at
// each window edge, so windows overlap by 2*K4 columns (K4 = K rounded up to
// a multiple of 4, keeping float4 alignment) and each warp writes the middle
// 128 - 2*K4.  A segment reads MH + 2K rows; the rows and columns a level
// gets wrong near the segment's ends lie outside the cone of every value
// written.  Warps never wait for one another.
constexpr int MW = 1;     // warps per CTA (one: residency then follows registers alone)
constexpr int MH = 512;   // output rows per warp segment

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// One warp's segment: output rows [r0, r1], columns [c0, ce] (window
// [c0 - K4, c0 - K4 + 127]).  EDGE: the window reaches outside the readable
// region, so loads are guarded and cells outside the array are kept at zero
// (the ghosts); interior warps need neither check.  Lanes 0 and 31 take
// their own values for the missing neighbour: that spoils only window-edge
// columns, which are never written.
template <int K, bool EDGE>
__device__ __forceinline__ void multi_segment(const float *__restrict__ ub, int64_t su, float *__restrict__ vb,
                                              int64_t sv, int64_t NY, int64_t NX, int64_t r0, int64_t r1, int64_t c0,
                                              int64_t ce, int64_t rr0, int64_t rr1, int64_t rc0, int64_t rc1,
                                              int lane) {
    constexpr int K4 = (K + 3) / 4 * 4;
    const int64_t j0 = c0 - K4 + 4 * lane;  // this lane's first column
    bool ldc = true, k0 = true, k1 = true, k2 = true, k3 = true, d0 = true, d1 = true, d2 = true, d3 = true;
    if (EDGE) {
        ldc = j0 + 3 >= rc0 && j0 <= rc1;
        k0 = j0 >= rc0 && j0 <= rc1;
        k1 = j0 + 1 >= rc0 && j0 + 1 <= rc1;
        k2 = j0 + 2 >= rc0 && j0 + 2 <= rc1;
        k3 = j0 + 3 >= rc0 && j0 + 3 <= rc1;
        d0 = j0 >= 0 && j0 < NX;
        d1 = j0 + 1 >= 0 && j0 + 1 < NX;
        d2 = j0 + 2 >= 0 && j0 + 2 < NX;
        d3 = j0 + 3 >= 0 && j0 + 3 < NX;
    }
    auto load = [&](int64_t row) {
        float4 v = zero4();
        if (!EDGE || (ldc && row >= rr0 && row <= rr1)) {
            v = *(const float4 *)(ub + row * su + j0);
            if (EDGE) {
                v.x = k0 ? v.x : 0.f;
                v.y = k1 ? v.y : 0.f;
                v.z = k2 ? v.z : 0.f;
                v.w = k3 ? v.w : 0.f;
            }
        }
        return v;
    };
    float4 q1[K], q2[K];  // level l: rows tr-l-1 (q1) and tr-l-2 (q2)
#pragma unroll
    for (int l = 0; l < K; ++l) q1[l] = q2[l] = zero4();
    float4 nxt = load(r0 - K);
    for (int64_t tr = r0 - K; tr <= r1 + K; ++tr) {
        float4 cur = nxt;
        if (tr + 1 <= r1 + K) nxt = load(tr + 1);  // in flight while this row's levels compute
#pragma unroll
        for (int l = 0; l < K; ++l) {
            const float4 up = q2[l], mid = q1[l], dn = cur;
            const float wv = __shfl_up_sync(0xffffffffu, mid.w, 1);
            const float ev = __shfl_down_sync(0xffffffffu, mid.x, 1);
            float4 o = div4_const_rn<5>(make_float4(sum5(mid.x, up.x, dn.x, wv, mid.y),
                                                    sum5(mid.y, up.y, dn.y, mid.x, mid.z),
                                                    sum5(mid.z, up.z, dn.z, mid.y, mid.w),
                                                    sum5(mid.w, up.w, dn.w, mid.z, ev)));
            if (EDGE) {
                const int64_t r = tr - l - 1;
                const bool rin = r >= 0 && r < NY;
                o.x = (rin && d0) ? o.x : 0.f;
                o.y = (rin && d1) ? o.y : 0.f;
                o.z = (rin && d2) ? o.z : 0.f;
                o.w = (rin && d3) ? o.w : 0.f;
            }
            q2[l] = q1[l];
            q1[l] = cur;
            cur = o;
        }
        const int64_t r = tr - K;  // `cur` is row r of level K
        if (r >= r0) {
            float *dst = vb + r * sv + j0;
            if (j0 >= c0 && j0 + 3 <= ce) {
                *(float4 *)dst = cur;
            } else {
                if (j0 >= c0 && j0 <= ce) dst[0] = cur.x;
                if (j0 + 1 >= c0 && j0 + 1 <= ce) dst[1] = cur.y;
                if (j0 + 2 >= c0 && j0 + 2 <= ce) dst[2] = cur.z;
                if (j0 + 3 >= c0 && j0 + 3 <= ce) dst[3] = cur.w;
            }
        }
    }
}

template <int K>
__global__ void __launch_bounds__(MW * 32) jacobi2d_multi_reg_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    constexpr int K4 = (K + 3) / 4 * 4;
    constexpr int L = 128 - 2 * K4;  // output columns per warp
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    const uint32_t nsx = (uint32_t)((x1 - x0 + L) / L);
    const uint32_t w = (blockIdx.x - t.cta_begin) * MW + (threadIdx.x >> 5);
    const int64_t c0 = x0 + (int64_t)(w % nsx) * L;  // first output column of this warp
    const int64_t r0 = y0 + (int64_t)(w / nsx) * MH;  // first output row
    if (r0 > y1) return;                              // spare warps of the last CTA (warp-uniform)
    const int64_t r1 = min(r0 + MH - 1, y1), ce = min(c0 + L - 1, x1);
    // readable region (the annotation's, clipped to the array)
    const int64_t rr0 = max(y0 - K, (int64_t)0), rr1 = min(y1 + K, NY - 1);
    const int64_t rc0 = max(x0 - K, (int64_t)0), rc1 = min(x1 + K, NX - 1);
    const bool interior = c0 - K4 >= rc0 && c0 - K4 + 127 <= rc1 && r0 - K >= rr0 && r1 + K <= rr1;
    const float *ub = (const float *)t.v[0].base;
    float *vb = (float *)t.v[1].base;
    const int lane = threadIdx.x & 31;
    if (interior)
        multi_segment<K, false>(ub, t.v[0].s[0], vb, t.v[1].s[0], NY, NX, r0, r1, c0, ce, rr0, rr1, rc0, rc1, lane);
    else
        multi_segment<K, true>(ub, t.v[0].s[0], vb, t.v[1].s[0], NY, NX, r0, r1, c0, ce, rr0, rr1, rc0, rc1, lane);
}

// Shared-memory variant (unaligned tasks): each CTA loads its 32 x 128 tile
// plus a k-cell ring and updates a box that shrinks by one cell per step
// (step s is valid on tile +/- (k-s)).
constexpr int MTY = 32, MTX = 128, MT = 256;

__global__ void __launch_bounds__(MT) jacobi2d_multi_smem_kernel(const ExecTask *__restrict__ tasks, ExecParams p) {
    extern __shared__ float msm[];
    const int ti = task_of(tasks, p, blockIdx.x);
    const ExecTask &t = tasks[ti];
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int k = (int)p.i[0];
    const int64_t x0 = t.t_lo[0], y0 = t.t_lo[1];
    const int64_t x1 = min(t.t_hi[0], NX - 1), y1 = min(t.t_hi[1], NY - 1);
    if (x1 < x0 || y1 < y0) return;
    const uint32_t gx = (uint32_t)((x1 - x0 + MTX) / MTX);
    const uint32_t local = blockIdx.x - t.cta_begin;
    const int64_t ty0 = y0 + (int64_t)(local / gx) * MTY, tx0 = x0 + (int64_t)(local % gx) * MTX;
    const int H = MTY + 2 * k, W = MTX + 2 * k;
    float *A = msm, *B = msm + H * W;
    // readable region: superblock +/- k, clipped to the domain
    const int64_t rr0 = max(y0 - k, (int64_t)0), rr1 = min(y1 + k, NY - 1);
    const int64_t rc0 = max(x0 - k, (int64_t)0), rc1 = min(x1 + k, NX - 1);
    // local index ranges of in-domain cells (the zero ghosts lie outside them)
    const int dr0 = (int)max((int64_t)0, -(ty0 - k)), dr1 = (int)min((int64_t)H - 1, NY - 1 - (ty0 - k));
    const int dc0 = (int)max((int64_t)0, -(tx0 - k)), dc1 = (int)min((int64_t)W - 1, NX - 1 - (tx0 - k));
    const DView U = t.v[0], V = t.v[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int li = warp; li < H; li += MT / 32) {
        const int64_t i = ty0 - k + li;
        const bool rok = i >= rr0 && i <= rr1;
        const float *urow = (const float *)U.base + i * U.s[0];
        for (int lj = lane; lj < W; lj += 32) {
            const int64_t j = tx0 - k + lj;
            A[li * W + lj] = (rok && j >= rc0 && j <= rc1) ? urow[j * U.s[1]] : 0.f;
            B[li * W + lj] = 0.f;
        }
    }
    __syncthreads();
    for (int s = 1; s <= k; ++s) {
        // step s is valid on the tile +/- (k - s): local rows/cols [s, H-1-s], in the domain
        const int r0 = max(s, dr0), r1 = min(H - 1 - s, dr1);
        const int c0 = max(s, dc0), c1 = min(W - 1 - s, dc1);
        for (int li = r0 + warp; li <= r1; li += MT / 32) {
            const float *a = A + li * W;
            float *b = B + li * W;
            for (int lj = c0 + lane; lj <= c1; lj += 32) b[lj] = j5(a[lj], a[lj - W], a[lj + W], a[lj - 1], a[lj + 1]);
        }
        __syncthreads();
        float *tmp = A;
        A = B;
        B = tmp;
    }
    for (int r = warp; r < MTY; r += MT / 32) {
        const int64_t i = ty0 + r;
        if (i > y1) break;
        float *vrow = (float *)V.base + i * V.s[0];
        const float *a = A + (k + r) * W + k;
        for (int c = lane; c < MTX; c += 32) {
            const int64_t j = tx0 + c;
            if (j <= x1) vrow[j * V.s[1]] = a[c];
        }
    }
}

}  // namespace

namespace k {

uint32_t prepare_jacobi2d_multi(ExecTask *t, int n, ExecParams &p) {
    const int64_t NY = p.shape[0][0], NX = p.shape[0][1];
    const int64_t k = p.i[0];
    if (k < 1 || k > 16) return 0xFFFFFFFFu;
    // variant 1: register pipeline (16-byte aligned rows and columns); 0: shared memory
    bool reg = true;
    for (int i = 0; i < n && reg; ++i) {
        if (t[i].t_lo[0] % 4 != 0) reg = false;
        for (int a = 0; a < 2; ++a)
            if (t[i].v[a].s[1] != 1 || (t[i].v[a].s[0] % 4) != 0 || (t[i].v[a].base % 16) != 0) reg = false;
    }
    p.variant = reg ? 1 : 0;
    const int64_t L = 128 - 2 * ((k + 3) / 4 * 4);
    uint32_t total = 0;
    for (int i = 0; i < n; ++i) {
        int64_t w = std::min(t[i].t_hi[0], NX - 1) - t[i].t_lo[0] + 1;
        int64_t h = std::min(t[i].t_hi[1], NY - 1) - t[i].t_lo[1] + 1;
        uint64_t c = 0;
        if (w > 0 && h > 0)
            c = reg ? (uint64_t)((((w + L - 1) / L) * ((h + MH - 1) / MH) + MW - 1) / MW)
                    : (uint64_t)(((w + MTX - 1) / MTX) * ((h + MTY - 1) / MTY));
        t[i].cta_begin = total;
        t[i].cta_count = (uint32_t)c;
        total += t[i].cta_count;
    }
    return total;
}

cudaError_t launch_jacobi2d_multi(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    const int k = (int)p.i[0];
    if (p.variant == 1) {
        switch (k) {
#define LT_MULTI_CASE(K) \
    case K: jacobi2d_multi_reg_kernel<K><<<ctas, MW * 32, 0, st>>>(dev, p); break;
            LT_MULTI_CASE(1) LT_MULTI_CASE(2) LT_MULTI_CASE(3) LT_MULTI_CASE(4) LT_MULTI_CASE(5) LT_MULTI_CASE(6)
            LT_MULTI_CASE(7) LT_MULTI_CASE(8) LT_MULTI_CASE(9) LT_MULTI_CASE(10) LT_MULTI_CASE(11) LT_MULTI_CASE(12)
            LT_MULTI_CASE(13) LT_MULTI_CASE(14) LT_MULTI_CASE(15) LT_MULTI_CASE(16)
#undef LT_MULTI_CASE
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const size_t smem = 2 * (size_t)(MTY + 2 * k) * (MTX + 2 * k) * sizeof(float);
    static size_t set = 0;
    if (smem > 48 * 1024 && smem > set) {
        cudaError_t e = cudaFuncSetAttribute(jacobi2d_multi_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    jacobi2d_multi_smem_kernel<<<ctas, MT, smem, st>>>(dev, p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
