// Batched form of many independent annotated launches (an extension beyond
// the paper, which schedules each launch's superblocks separately): one
// persistent kernel pulls work items from a device-side queue.
//   kind 0  Jacobi tile: rows [row0, row0+nrows) of one instance, one
//           iteration (ping-pong between the instance's two buffers);
//   kind 1  histogram slice: bytes [slice*HS, (slice+1)*HS) of one array,
//           counted in shared memory and added to H with integer atomics
//           (the reduce(+) of Sec. 2.3 folded into one level);
//   kind 2  halo replica cells of a chunked instance: cells of one part's
//           output that other chunks hold in their halos, computed from the
//           part's input like its own cells and stored into those halos.
// A Jacobi instance is one or more parts (the superblocks of its launch, one
// chunk each); its tiles and replica items of one iteration count together.
// Items are queued iteration-major, so every item an item waits for was
// dequeued before it by a resident CTA: a tile of iteration t waits (bounded)
// until all tiles of iteration t-1 of its instance are done, and no wait can
// deadlock.  Loads of Jacobi inputs bypass L1 (other SMs wrote them earlier
// in the same kernel).  Every wait is bounded by %globaltimer; on expiry the
// kernel records an error and every CTA returns.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "stencil_body.cuh"

namespace lt {
namespace {

constexpr int BT = 256;  // threads per CTA (8 warps)
constexpr int BR = 8;    // rows per warp strip of a Jacobi tile
constexpr int BOCC = 3;  // CTAs per SM the kernel is built for (registers capped to fit)
constexpr unsigned long long BWAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long btimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(BT, BOCC) batch_kernel(BatchParams P) {
    __shared__ uint32_t s_item[2];  // this item and the next one, claimed while this one runs
    __shared__ int s_stop;
    __shared__ uint32_t sh[BT / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_item[0] = atomicAdd(P.head, 1u);
    for (uint32_t par = 0;; par ^= 1u) {
        if (tid == 0) {
            s_stop = s_item[par] >= P.nitems || ld_acquire(P.abort) != 0;
            // Claiming the next item early keeps the queue's order argument:
            // the earliest unfinished item is always one a CTA is running.
            if (!s_stop) s_item[par ^ 1u] = atomicAdd(P.head, 1u);
        }
        __syncthreads();
        if (s_stop) break;
        const BatchItem w = P.items[s_item[par]];
        const uint32_t kind = w.kind_inst >> 30, inst = w.kind_inst & 0x3FFFFFFFu;
        if (kind != 1) {
            const BatchJacobi J = P.jac[kind == 0 ? inst : P.reps[inst].part];
            if (w.iter > 0) {
                if (tid == 0) {
                    const uint32_t *cnt = P.done + J.done_off + w.iter - 1;
                    unsigned long long t0 = btimer();
                    while (ld_acquire(cnt) < J.tiles) {
                        if (ld_acquire(P.abort) != 0 || btimer() - t0 > BWAIT_NS) {
                            atomicCAS(P.err, 0u, 0x6801u);
                            atomicExch(P.abort, 1u);
                            s_stop = 1;
                            break;
                        }
                    }
                }
                __syncthreads();
                if (s_stop) break;
            }
            const bool even = (w.iter & 1u) == 0;
            const float *src = (const float *)(even ? J.u : J.v);
            const int64_t ss = even ? J.su : J.sv;
            const int64_t ny = J.ny, nx = J.nx;
            if (kind == 0) {
                float *dst = (float *)(even ? J.v : J.u);
                const int64_t sd = even ? J.sv : J.su;
                const int64_t ye = min((int64_t)(w.row0 + w.nrows) - 1, J.y1);
                const int64_t xa = J.x0 + (int64_t)w.col0;
                const int64_t xe = w.ncols ? min(xa + (int64_t)w.ncols - 1, J.x1) : J.x1;
                const uint32_t sx = (uint32_t)((xe - xa + JCOLS) / JCOLS), sy = (w.nrows + BR - 1) / BR;
                // strip s = cy * sx + cx, s = warp, warp + 8, ...; (cx, cy) advance
                // without a division per strip (32-bit: tiles are small)
                uint32_t cx = warp % sx, cy = warp / sx;
                for (uint32_t s = warp; s < sx * sy; s += BT / 32) {
                    const int64_t js = xa + (int64_t)cx * JCOLS, r0 = (int64_t)w.row0 + (int64_t)cy * BR;
                    if (r0 <= ye) jacobi_strip<true, BR>(src, ss, dst, sd, ny, nx, js, r0, xe, ye, lane);
                    for (cx += BT / 32; cx >= sx; cx -= sx) ++cy;
                }
            } else {
                // replica cells: the same five-point sum and division as the strips
                const BatchRep R = P.reps[inst];
                float *dst = (float *)(even ? R.dv : R.du);
                const int64_t sd = even ? R.sdv : R.sdu;
                const int64_t wdt = R.hi[1] - R.lo[1] + 1;
                for (uint32_t e = tid; e < w.nrows; e += BT) {
                    const int64_t l = (int64_t)w.row0 + e, i = R.lo[0] + l / wdt, j = R.lo[1] + l % wdt;
                    const float *up = src + i * ss + j;
                    const float c = ld1<true>(up);
                    const float n = i > 0 ? ld1<true>(up - ss) : 0.f;
                    const float so = i + 1 < ny ? ld1<true>(up + ss) : 0.f;
                    const float we = j > 0 ? ld1<true>(up - 1) : 0.f;
                    const float ea = j + 1 < nx ? ld1<true>(up + 1) : 0.f;
                    dst[i * sd + j] = j5(c, n, so, we, ea);
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) atomicAdd(P.done + J.done_off + w.iter, 1u);
        } else {
            const BatchHist H = P.hist[inst];
            for (int i = tid; i < (BT / 32) * 256; i += BT) (&sh[0][0])[i] = 0;
            __syncthreads();
            const int64_t lo = (int64_t)w.row0 * P.hist_slice;
            const int64_t hi = min(lo + (int64_t)P.hist_slice, H.len);
            const uint8_t *x = (const uint8_t *)H.x;
            uint32_t *h = sh[warp];
            // H.x is 128-byte aligned and slices are multiples of 16 bytes
            const int64_t nv = (hi - lo) / 16;
            const uint4 *v = (const uint4 *)(x + lo);
            for (int64_t i = tid; i < nv; i += BT) {
                uint4 q = __ldg(v + i);
                uint32_t ws[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) {
                    atomicAdd(&h[ws[k2] & 255u], 1u);
                    atomicAdd(&h[(ws[k2] >> 8) & 255u], 1u);
                    atomicAdd(&h[(ws[k2] >> 16) & 255u], 1u);
                    atomicAdd(&h[ws[k2] >> 24], 1u);
                }
            }
            for (int64_t i = lo + nv * 16 + tid; i < hi; i += BT) atomicAdd(&h[x[i]], 1u);
            __syncthreads();
            uint32_t *out = (uint32_t *)H.h;
            for (int bin = tid; bin < 256; bin += BT) {
                uint32_t s = 0;
#pragma unroll
                for (int k2 = 0; k2 < BT / 32; ++k2) s += sh[k2][bin];
                if (s) atomicAdd(&out[bin], s);
            }
        }
        __syncthreads();
    }
}

__global__ void batch_zero_hist_kernel(const BatchHist *__restrict__ hist, int n) {
    for (int h = blockIdx.x; h < n; h += gridDim.x) {
        uint32_t *out = (uint32_t *)hist[h].h;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) out[b] = 0u;
    }
}

}  // namespace

namespace k {

int batch_threads() { return BT; }

int batch_ctas_per_sm() {
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel, BT, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

cudaError_t launch_batch_zero_hist(const BatchHist *hist, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    batch_zero_hist_kernel<<<n < 1024 ? n : 1024, 256, 0, st>>>(hist, n);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchParams &p, int ctas, cudaStream_t st) {
    batch_kernel<<<ctas, BT, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
