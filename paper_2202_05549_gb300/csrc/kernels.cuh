// Descriptors shared by the runtime (host) and the CUDA kernels.
//
// A DView is the paper's view type (Sec. 3.5, Listing 3): the chunk's base
// address with the chunk's global offset already subtracted, so a kernel
// indexes it with GLOBAL indices and pays nothing per access:
//     address(i0, i1, i2) = base + (i0*s0 + i1*s1 + i2*s2) * element_size
// (axis 0 is the slowest axis of the array).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lt {

struct DView {
    uint64_t base;   // byte address of global element (0,0,0) (may lie outside the allocation)
    int64_t s[3];    // element strides
    int64_t org[3];  // global index of the first stored element per axis
    int64_t hi[3];   // last valid global index per axis (the chunk box)
};

#define LT_MAX_ARRAYS 5

// A halo copy that an Execute kernel keeps current itself: the cells of the
// box [lo, hi] (global indices, axis 0 slowest), which task `task` writes,
// are also computed by extra CTAs of the same kernel, from that task's input
// views, and stored to `dst`, the view of another chunk whose halo holds a
// copy of them.  This replaces the copy step after the kernel.
struct ReplicaTarget {
    DView dst;
    int64_t lo[3], hi[3];
    uint64_t cell_begin;  // prefix sum of the box volumes over the launch's replicas
    int32_t task;
    int32_t pad;
};

// A warp's share of the write-through replicas (vector Jacobi kernel): 128
// columns of a one-row replica box whose row is 16-byte aligned in its
// chunk (row = 1, off = first column offset), or 32 cells of any other box
// (row = 0, off = first cell offset).
struct ReplicaUnit {
    uint32_t rep;
    uint32_t row : 1;
    uint32_t off : 31;
};

// One Execute task: a superblock's thread box and its argument views.
struct ExecTask {
    int64_t t_lo[3], t_hi[3];     // thread box (x, y, z), inclusive
    DView v[LT_MAX_ARRAYS];       // views, in array-parameter order
    uint32_t cta_begin;           // first CTA (or work tile) of this task in the launch
    uint32_t cta_count;
    int32_t aux[6];               // kernel-specific per-task values set by prepare_*
};

// Per-launch constants of an Execute kernel.
struct ExecParams {
    int64_t shape[LT_MAX_ARRAYS][3];  // global shapes of the array parameters
    int32_t nd[LT_MAX_ARRAYS];
    int64_t block[3];                 // launch block dims (x, y, z)
    double f[4];                      // value parameters (float)
    int64_t i[4];                     // value parameters (integer)
    uint32_t* err;                    // device error word (bounds checks)
    int32_t ntasks;
    int32_t variant;                  // kernel variant chosen by prepare_*
    int32_t red_op;                   // operator of the reduce(f) argument (0 + 1 * 2 min 3 max)
    int32_t uniform_ctas;             // if > 0: task i owns CTAs [i * uniform_ctas, (i + 1) * uniform_ctas)
    const ReplicaTarget *reps;        // write-through replicas of the launch (null if none) ...
    uint64_t rep_cells;               // ... their cells in total, one thread each in the grid's first CTAs
    uint32_t nreps;
    uint32_t rep_ctas;                // CTAs before the tasks' CTAs (set by the launch from rep_cells)
    int32_t no_staged;                // 1: prepare_* picks no TMA-staged kernel (context flag)
    int32_t pdl;                      // 1: launched as a programmatic dependent of the previous kernel
    const ReplicaUnit *runits;        // the replicas as warp units (vector Jacobi kernel)
    uint32_t nunits;
    uint32_t pad;
};

// Box copy (pack / unpack / replica update): copy the global box [lo, hi]
// from src to dst.
struct CopyPiece {
    DView src, dst;
    int64_t lo[3], hi[3];
    int32_t nd;
    int32_t esize;
    uint64_t unit_begin; // prefix sum of work units (see copy_piece_units)
};

// Work units of one copy piece: a unit is a run of whole rows (all axes but
// the innermost) of about LT_COPY_UNIT elements.  Within a row, when both
// sides are contiguous along the innermost axis and equally misaligned, the
// body moves as 16-byte vectors between a scalar head and tail.
#define LT_COPY_UNIT 16384
__host__ __device__ inline int64_t copy_piece_width(const CopyPiece &p) {
    return p.hi[p.nd - 1] - p.lo[p.nd - 1] + 1;
}
__host__ __device__ inline int64_t copy_piece_rows(const CopyPiece &p) {
    int64_t r = 1;
    for (int d = 0; d + 1 < p.nd; ++d) r *= p.hi[d] - p.lo[d] + 1;
    return r;
}
// Narrow pieces (rows under 512 bytes: column halos) take units of 2048
// elements, so a column of a few thousand rows spreads over several CTAs.
#define LT_COPY_UNIT_NARROW 2048
__host__ __device__ inline int64_t copy_piece_rows_per_unit(const CopyPiece &p) {
    int64_t w = copy_piece_width(p);
    const int64_t unit = w * p.esize < 512 ? LT_COPY_UNIT_NARROW : LT_COPY_UNIT;
    int64_t r = unit / (w > 0 ? w : 1);
    return r < 1 ? 1 : r;
}
__host__ __device__ inline uint64_t copy_piece_units(const CopyPiece &p) {
    int64_t rpu = copy_piece_rows_per_unit(p);
    int64_t seg = copy_piece_width(p) > LT_COPY_UNIT ? (copy_piece_width(p) + LT_COPY_UNIT - 1) / LT_COPY_UNIT : 1;
    return (uint64_t)((copy_piece_rows(p) + rpu - 1) / rpu) * (uint64_t)seg;
}

// Reduce: dst[box] = src_0 (op) src_1 (op) ... in the listed order.
struct ReducePiece {
    DView dst;
    int64_t lo[3], hi[3];
    int32_t nd;
    int32_t op;
    int32_t dtype;
    int32_t nsrc;
    uint32_t src_begin;  // index into the source-view table
    uint32_t pad;
    uint64_t elem_begin; // prefix sum of elements
};

// Seeded fill of a box of one chunk (see lt_array_fill).
struct FillDesc {
    DView dst;
    int64_t lo[3], hi[3];
    int64_t gstride[3];  // row-major strides of the global array (for the counter)
    int32_t nd;
    int32_t kind;
    int32_t dtype;
    int32_t pad;
    uint64_t key;
    double value, scale;
};

// Batched persistent kernel: instance tables and the work queue.
// One part of a batched Jacobi instance: a superblock of its launch, whose
// cells it computes from the part's chunk of the input buffer into the
// part's chunk of the output buffer (the buffers swap every iteration).
struct BatchJacobi {
    uint64_t u, v;     // views (global index base) of the part's chunks of the two ping-pong buffers
    int64_t su, sv;    // row strides (elements)
    int64_t ny, nx;    // the instance's global shape
    int64_t y0, y1, x0, x1;  // output rows and columns of the part (inclusive, x0 % 4 == 0)
    uint32_t tiles;    // work items per iteration of the instance (all its parts' tiles and replica items)
    uint32_t done_off; // first completion counter of the instance (one per iteration)
};
// Halo replica of a chunked instance: cells [lo, hi] that part `part`
// computes are also stored into the halo of another chunk (du / dv: that
// chunk in either buffer), from the same input with the same operations.
struct BatchRep {
    uint64_t du, dv;
    int64_t sdu, sdv;
    int64_t lo[2], hi[2];  // rows, columns (inclusive)
    uint32_t part;
    uint32_t pad;
};
struct BatchHist {
    uint64_t x;   // u8 array (contiguous, 128-byte aligned)
    int64_t len;
    uint64_t h;   // 256 u32 bins (contiguous)
};
struct BatchItem {
    uint32_t kind_inst;  // kind << 30 | index: 0 Jacobi tile (of part `index`), 1 histogram slice,
                         // 2 Jacobi replica cells (of replica `index`)
    uint32_t iter;       // Jacobi iteration
    uint32_t row0;       // first row (tile), slice index (histogram) or first cell (replica)
    uint32_t nrows;      // rows (tile) or cells (replica)
    uint32_t col0;       // tile: first column offset from the part's first column (a multiple of 128)
    uint32_t ncols;      // tile: columns (0: to the part's last column)
};
struct BatchParams {
    const BatchItem *items;
    uint64_t nitems;
    const BatchJacobi *jac;
    const BatchHist *hist;
    const BatchRep *reps;
    uint32_t *head;   // queue head (zeroed before every run)
    uint32_t *done;   // completion counters (zeroed before every run)
    uint32_t *abort;  // set when a bounded wait expires
    uint32_t *err;
    int64_t hist_slice;
};

namespace k {

int batch_threads();
int batch_ctas_per_sm();  // resident CTAs of the persistent batch kernel per SM
cudaError_t launch_batch(const BatchParams &p, int ctas, cudaStream_t st);
cudaError_t launch_batch_zero_hist(const BatchHist *hist, int n, cudaStream_t st);

// All launchers return the CUDA error of the launch (cudaSuccess on success).
cudaError_t fill(const FillDesc &d, cudaStream_t st);
cudaError_t copy_pieces(const CopyPiece *dev, int n, uint64_t total_units, cudaStream_t st);
cudaError_t reduce_pieces(const ReducePiece *dev, const DView *srcs, int n, uint64_t total_elems, cudaStream_t st);

// Execute kernels of the built-ins.  prepare_* fills cta_begin / cta_count
// of every task (host side) and returns the total CTA count; launch_* runs
// all tasks of one launch in one kernel.
uint32_t prepare_stencil1d(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_stencil1d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_jacobi2d(ExecTask *t, int n, ExecParams &p);
uint32_t prepare_jacobi2d_multi(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_jacobi2d_multi(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_jacobi3d(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_jacobi3d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_diffusion(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_diffusion(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_laplace(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_laplace(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_ewise(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_ewise(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_muladd(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_muladd(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_diffusion_adj(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_diffusion_adj(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_rowreduce(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_rowreduce(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_kmeans_assign(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_kmeans_assign(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_kmeans_update(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_kmeans_update(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_hist256(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_hist256(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
uint32_t prepare_gemm_bf16(ExecTask *t, int n, ExecParams &p);
cudaError_t launch_gemm_bf16(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);
cudaError_t launch_jacobi2d(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st);

}  // namespace k
}  // namespace lt
