// Data-movement kernels of the engine: seeded fill, box copy (pack, unpack,
// replica update; Sec. 2.4 "Execution Planner") and the ordered reduction of
// per-superblock partials (reduce(f) of Sec. 2.3, first level of the
// hierarchical reduction of Sec. 2.4).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "tma.cuh"
#include "copy_staged.cuh"

namespace lt {
namespace {

// SplitMix64 output mix (Steele, Lea & Flood 2014)
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_elem(uint64_t key, uint64_t g) {
    return sm64_mix(key + (g + 1) * 0x9E3779B97F4A7C15ULL);
}

__device__ __forceinline__ float u01_f32(uint64_t x) { return (float)(x >> 40) * 0x1p-24f; }

__device__ __forceinline__ unsigned short f32_to_bf16_rne(float f) {
    uint32_t b = __float_as_uint(f);
    uint32_t lsb = (b >> 16) & 1u;
    return (unsigned short)((b + 0x7FFFu + lsb) >> 16);
}

__global__ void fill_kernel(FillDesc d) {
    int nd = d.nd;
    int inner = nd - 1;
    int64_t w = d.hi[inner] - d.lo[inner] + 1;
    int64_t rows = 1;
    for (int k = 0; k < inner; ++k) rows *= d.hi[k] - d.lo[k] + 1;
    const int64_t SEG = 8192;
    int64_t segs = (w + SEG - 1) / SEG;
    for (int64_t unit = blockIdx.x; unit < rows * segs; unit += gridDim.x) {
        int64_t r = unit / segs, seg = unit % segs;
        int64_t c0 = seg * SEG, c1 = c0 + SEG < w ? c0 + SEG : w;
        int64_t idx[3] = {0, 0, 0};
        int64_t rr = r;
        for (int k = inner - 1; k >= 0; --k) {
            int64_t e = d.hi[k] - d.lo[k] + 1;
            idx[k] = d.lo[k] + rr % e;
            rr /= e;
        }
        int64_t g0 = 0, a0 = 0;
        for (int k = 0; k < inner; ++k) {
            g0 += idx[k] * d.gstride[k];
            a0 += idx[k] * d.dst.s[k];
        }
        for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            int64_t col = d.lo[inner] + c;
            uint64_t g = (uint64_t)(g0 + col * d.gstride[inner]);
            uint64_t addr_el = (uint64_t)(a0 + col * d.dst.s[inner]);
            uint64_t x = sm64_elem(d.key, g);
            switch (d.dtype) {
                case 0: {  // f32
                    float v;
                    if (d.kind == 0)
                        v = 0.0f;
                    else if (d.kind == 1)
                        v = (float)d.value;
                    else if (d.kind == 2)
                        v = u01_f32(x);
                    else {  // kappa = 0.05 + 0.15 u in fp64, no contraction
                        double u = (double)u01_f32(x);
                        v = __double2float_rn(__dadd_rn(0.05, __dmul_rn(0.15, u)));
                    }
                    ((float *)d.dst.base)[addr_el] = v;
                    break;
                }
                case 1: {  // bf16
                    unsigned short h;
                    if (d.kind == 0)
                        h = 0;
                    else if (d.kind == 1)
                        h = f32_to_bf16_rne((float)d.value);
                    else {  // N(0,1)*scale by Box-Muller from counters 2g, 2g+1
                        uint64_t x1 = sm64_elem(d.key, 2 * g), x2 = sm64_elem(d.key, 2 * g + 1);
                        double u1 = ((double)(x1 >> 11) + 1.0) * 0x1p-53;
                        double u2 = (double)(x2 >> 11) * 0x1p-53;
                        double z = __dmul_rn(sqrt(-2.0 * log(u1)), cos(__dmul_rn(6.283185307179586, u2)));
                        h = f32_to_bf16_rne(__double2float_rn(__dmul_rn(z, d.scale)));
                    }
                    ((unsigned short *)d.dst.base)[addr_el] = h;
                    break;
                }
                case 2: {  // u8
                    unsigned char v = d.kind == 5 ? (unsigned char)(x >> 56)
                                                  : (d.kind == 1 ? (unsigned char)d.value : (unsigned char)0);
                    ((unsigned char *)d.dst.base)[addr_el] = v;
                    break;
                }
                case 4: {  // f64
                    ((double *)d.dst.base)[addr_el] = d.kind == 1 ? d.value : 0.0;
                    break;
                }
                default: {  // u32
                    uint32_t v = d.kind == 1 ? (uint32_t)d.value : 0u;
                    ((uint32_t *)d.dst.base)[addr_el] = v;
                }
            }
        }
    }
}

// The piece holding work unit u: the last piece whose unit_begin <= u.  The
// whole warp searches together: each round the 32 lanes test 32 evenly
// spaced pieces of the remaining range at once and a ballot keeps the
// segment after the last one at or below u, so a table of n pieces takes
// ceil(log32 n) dependent loads instead of log2 n (a copy of a few hundred
// pieces was measured to spend most of its time in the binary search).
// Every lane of the warp must call it with the same u.
__device__ __forceinline__ int find_piece_u(const CopyPiece *p, int n, uint64_t u) {
    const int lane = threadIdx.x & 31;
    int lo = 0, cnt = n;
    while (cnt > 1) {
        const int step = (cnt + 31) >> 5;
        const int idx = lo + lane * step;
        const bool le = lane * step < cnt && p[idx].unit_begin <= u;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, le);
        const int last = 31 - __clz(m);  // lane 0 always qualifies: p[lo].unit_begin <= u
        lo += last * step;
        cnt = min(step, cnt - last * step);
    }
    return lo;
}

__device__ __forceinline__ void copy_elem(const char *s, char *d, int esize) {
    switch (esize) {
        case 1: *d = *s; break;
        case 2: *(unsigned short *)d = *(const unsigned short *)s; break;
        case 4: *(uint32_t *)d = *(const uint32_t *)s; break;
        default: *(uint64_t *)d = *(const uint64_t *)s;
    }
}

// One CTA per work unit (a run of rows, or a segment of one long row, of
// about LT_COPY_UNIT elements); the piece is found by binary search and read
// in place (no local copy of the record).
__device__ __forceinline__ void copy_unit(const CopyPiece *__restrict__ pieces, const int pi, const uint64_t u) {
    const CopyPiece &p = pieces[pi];
    const int inner = p.nd - 1;
    const int64_t w = copy_piece_width(p), rows = copy_piece_rows(p);
    const int64_t rpu = copy_piece_rows_per_unit(p);
    const int64_t nseg = w > LT_COPY_UNIT ? (w + LT_COPY_UNIT - 1) / LT_COPY_UNIT : 1;
    const int64_t lu = (int64_t)(u - p.unit_begin);
    const int64_t r0 = (lu / nseg) * rpu, seg = lu % nseg;
    const int64_t r1 = min(r0 + rpu, rows);
    const int64_t c0 = seg * LT_COPY_UNIT, c1 = nseg > 1 ? min(c0 + LT_COPY_UNIT, w) : w;
    const int64_t e1 = p.nd == 3 ? p.hi[1] - p.lo[1] + 1 : 1;
    const int es = p.esize;
    const bool contig = p.src.s[inner] == 1 && p.dst.s[inner] == 1;
    if ((c1 - c0) * es < 512) {
        // narrow rows: spread the unit's elements (rows x columns) over the threads
        const uint32_t ncol = (uint32_t)(c1 - c0), nel = (uint32_t)((r1 - r0) * (c1 - c0));
        if (p.nd == 2) {  // 2-D: one element per thread and step, 32-bit index arithmetic
            const char *sb = (const char *)(p.src.base + (uint64_t)(((p.lo[0] + r0) * p.src.s[0] +
                                                                     (p.lo[1] + c0) * p.src.s[1]) * es));
            char *db = (char *)(p.dst.base + (uint64_t)(((p.lo[0] + r0) * p.dst.s[0] + (p.lo[1] + c0) * p.dst.s[1]) * es));
            const int64_t sr = p.src.s[0] * es, sc = p.src.s[1] * es, dr = p.dst.s[0] * es, dc = p.dst.s[1] * es;
            if (es == 4 || es == 8) {
                // up to eight loads in flight per thread before the stores (a
                // one-column halo of 2048 rows is eight strided elements per thread)
                for (uint32_t e0 = threadIdx.x; e0 < nel; e0 += 8 * blockDim.x) {
                    uint64_t v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t e = e0 + (uint32_t)k * blockDim.x;
                        if (e < nel) {
                            const uint32_t r = ncol == 1 ? e : e / ncol, col = ncol == 1 ? 0u : e - r * ncol;
                            const char *sa = sb + r * sr + col * sc;
                            v[k] = es == 4 ? (uint64_t)__ldcg((const unsigned int *)sa)
                                           : (uint64_t)__ldcg((const unsigned long long *)sa);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t e = e0 + (uint32_t)k * blockDim.x;
                        if (e < nel) {
                            const uint32_t r = ncol == 1 ? e : e / ncol, col = ncol == 1 ? 0u : e - r * ncol;
                            char *da = db + r * dr + col * dc;
                            if (es == 4)
                                *(unsigned int *)da = (unsigned int)v[k];
                            else
                                *(unsigned long long *)da = (unsigned long long)v[k];
                        }
                    }
                }
                return;
            }
            for (uint32_t e = threadIdx.x; e < nel; e += blockDim.x) {
                const uint32_t r = ncol == 1 ? e : e / ncol, col = ncol == 1 ? 0u : e - r * ncol;
                copy_elem(sb + r * sr + col * sc, db + r * dr + col * dc, es);
            }
            return;
        }
        for (uint32_t e = threadIdx.x; e < nel; e += blockDim.x) {
            const int64_t r = r0 + e / ncol, col = p.lo[inner] + c0 + e % ncol;
            int64_t idx[3] = {0, 0, 0};
            if (p.nd == 3) {
                idx[0] = p.lo[0] + r / e1;
                idx[1] = p.lo[1] + r % e1;
            } else if (p.nd == 2) {
                idx[0] = p.lo[0] + r;
            }
            idx[inner] = col;
            int64_t os = 0, od = 0;
            for (int d = 0; d < p.nd; ++d) {
                os += idx[d] * p.src.s[d];
                od += idx[d] * p.dst.s[d];
            }
            copy_elem((const char *)(p.src.base + (uint64_t)(os * es)), (char *)(p.dst.base + (uint64_t)(od * es)),
                      es);
        }
        return;
    }
    // Rows of equal misalignment in both (row pitches multiples of 16 bytes):
    // the unit's 16-byte vectors are numbered across its rows and every
    // thread keeps eight loads in flight before its stores, so short rows
    // (a 1024-column tile row is 256 vectors, one per thread) no longer
    // leave one load per thread in flight.
    if (contig && p.nd == 2 && ((p.src.s[0] * es) & 15) == 0 && ((p.dst.s[0] * es) & 15) == 0) {
        const int64_t col0 = p.lo[1] + c0, ncol = c1 - c0;
        const char *sb = (const char *)(p.src.base + (uint64_t)((p.lo[0] + r0) * p.src.s[0] * es + col0 * es));
        char *db = (char *)(p.dst.base + (uint64_t)((p.lo[0] + r0) * p.dst.s[0] * es + col0 * es));
        if (((uintptr_t)sb & 15) == ((uintptr_t)db & 15)) {
            const int64_t sp = p.src.s[0] * es, dp = p.dst.s[0] * es;
            int64_t head = (int64_t)(((16 - ((uintptr_t)sb & 15)) & 15) / es);
            if (head > ncol) head = ncol;
            const uint32_t nv = (uint32_t)((ncol - head) * es / 16);
            const int64_t tail0 = head + (int64_t)nv * 16 / es;
            const uint32_t nr = (uint32_t)(r1 - r0);
            // scalar heads and tails of every row
            const uint32_t ns = (uint32_t)(head + (ncol - tail0));
            for (uint32_t e = threadIdx.x; e < nr * ns; e += blockDim.x) {
                const uint32_t r = e / ns, k = e % ns;
                const int64_t col = k < (uint32_t)head ? (int64_t)k : tail0 + (int64_t)(k - (uint32_t)head);
                copy_elem(sb + r * sp + col * es, db + r * dp + col * es, es);
            }
            if (nv) {
                const uint32_t total = nr * nv;
                const uint32_t minv = (uint32_t)(0xFFFFFFFFull / nv);  // row = idx / nv by multiply and one fix-up
                const char *sv = sb + head * es;
                char *dv = db + head * es;
                for (uint32_t b = threadIdx.x; b < total; b += 8u * blockDim.x) {
                    uint4 v[8];
                    int64_t doff[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t i = b + (uint32_t)k * blockDim.x;
                        doff[k] = -1;
                        if (i < total) {
                            uint32_t r = __umulhi(i, minv);
                            if ((r + 1) * nv <= i) ++r;
                            const uint32_t c = i - r * nv;
                            v[k] = __ldcg((const uint4 *)(sv + r * sp) + c);
                            doff[k] = r * dp + (int64_t)c * 16;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (doff[k] >= 0) *(uint4 *)(dv + doff[k]) = v[k];
                }
            }
            return;
        }
    }
    for (int64_t r = r0; r < r1; ++r) {
        int64_t idx[3] = {0, 0, 0};
        if (p.nd == 3) {
            idx[0] = p.lo[0] + r / e1;
            idx[1] = p.lo[1] + r % e1;
        } else if (p.nd == 2) {
            idx[0] = p.lo[0] + r;
        }
        int64_t os = 0, od = 0;
        for (int d = 0; d < inner; ++d) {
            os += idx[d] * p.src.s[d];
            od += idx[d] * p.dst.s[d];
        }
        const int64_t col0 = p.lo[inner] + c0, ncol = c1 - c0;
        const char *sb = (const char *)(p.src.base + (uint64_t)((os + col0 * p.src.s[inner]) * es));
        char *db = (char *)(p.dst.base + (uint64_t)((od + col0 * p.dst.s[inner]) * es));
        if (contig && ((uintptr_t)sb & 15) == ((uintptr_t)db & 15)) {
            int64_t head = (int64_t)(((16 - ((uintptr_t)sb & 15)) & 15) / es);
            if (head > ncol) head = ncol;
            const int64_t nv = (ncol - head) * es / 16;
            const int64_t tail0 = head + nv * 16 / es;
            for (int64_t i = threadIdx.x; i < head; i += blockDim.x) copy_elem(sb + i * es, db + i * es, es);
            const uint4 *sv = (const uint4 *)(sb + head * es);
            uint4 *dv = (uint4 *)(db + head * es);
            // four 16-byte loads in flight per thread before their stores
            for (int64_t b = 0; b < nv; b += 4 * (int64_t)blockDim.x) {
                uint4 v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t i = b + k * (int64_t)blockDim.x + threadIdx.x;
                    if (i < nv) v[k] = __ldcg(sv + i);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t i = b + k * (int64_t)blockDim.x + threadIdx.x;
                    if (i < nv) dv[i] = v[k];
                }
            }
            for (int64_t i = tail0 + threadIdx.x; i < ncol; i += blockDim.x) copy_elem(sb + i * es, db + i * es, es);
        } else {
            const int64_t ss = p.src.s[inner] * es, ds = p.dst.s[inner] * es;
            for (int64_t i = threadIdx.x; i < ncol; i += blockDim.x) copy_elem(sb + i * ss, db + i * ds, es);
        }
    }
}

__global__ void __launch_bounds__(256, 3) copy_kernel(const CopyPiece *__restrict__ pieces, int n) {
    copy_unit(pieces, find_piece_u(pieces, n, blockIdx.x), blockIdx.x);
}

// Staged variant: a unit of whole rows whose body (the 16-byte aligned part
// of every row, equally aligned in source and destination) fits the stage
// moves through shared memory with bulk asynchronous copies (TMA, no tensor
// map): one thread issues a bulk load per row into the stage, completing on
// an mbarrier, then a bulk store per row out of it; the other threads copy
// the rows' unaligned heads and tails meanwhile.  Other units take the
// register path.  The wait is bounded: on expiry the kernel records 0x6730,
// lets its loads land (bounded) and returns.
constexpr int BULK_STAGE = 64 * 1024;

__device__ __forceinline__ void bulk_load_row(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tma::smem_u32(smem)),
        "l"(gmem), "r"(bytes), "r"(tma::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_store_row(void *gmem, const void *smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem),
                 "r"(tma::smem_u32(smem)), "r"(bytes)
                 : "memory");
}

__global__ void __launch_bounds__(256, 3) copy_bulk_kernel(const CopyPiece *__restrict__ pieces, int n, uint32_t *err) {
    extern __shared__ __align__(128) unsigned char stage[];
    __shared__ __align__(8) uint64_t bar;
    const uint64_t u = blockIdx.x;
    const int pi = find_piece_u(pieces, n, u);
    const CopyPiece &p = pieces[pi];
    const int es = p.esize;
    bool bulk = p.nd == 2 && p.src.s[1] == 1 && p.dst.s[1] == 1 && ((p.src.s[0] * es) & 15) == 0 &&
                ((p.dst.s[0] * es) & 15) == 0;
    int64_t r0 = 0, r1 = 0, head = 0, tail0 = 0, ncol = 0;
    const char *sb = nullptr;
    char *db = nullptr;
    uint32_t rowbytes = 0;
    if (bulk) {
        const int64_t w = copy_piece_width(p), rows = copy_piece_rows(p), rpu = copy_piece_rows_per_unit(p);
        bulk = w <= LT_COPY_UNIT && w * es >= 512;  // whole rows in the unit, not a narrow piece
        if (bulk) {
            const int64_t lu = (int64_t)(u - p.unit_begin);
            r0 = lu * rpu;
            r1 = min(r0 + rpu, rows);
            ncol = w;
            sb = (const char *)(p.src.base + (uint64_t)(((p.lo[0] + r0) * p.src.s[0] + p.lo[1]) * es));
            db = (char *)(p.dst.base + (uint64_t)(((p.lo[0] + r0) * p.dst.s[0] + p.lo[1]) * es));
            bulk = ((uintptr_t)sb & 15) == ((uintptr_t)db & 15);
            head = (int64_t)(((16 - ((uintptr_t)sb & 15)) & 15) / es);
            if (head > ncol) head = ncol;
            rowbytes = (uint32_t)((ncol - head) * es / 16 * 16);
            tail0 = head + rowbytes / es;
            bulk = bulk && rowbytes > 0 && (r1 - r0) * (int64_t)rowbytes <= BULK_STAGE;
        }
    }
    if (!bulk) {
        copy_unit(pieces, pi, u);
        return;
    }
    const int64_t sp = p.src.s[0] * es, dp = p.dst.s[0] * es;
    const uint32_t nr = (uint32_t)(r1 - r0);
    if (threadIdx.x == 0) {
        tma::mbar_init(&bar, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        tma::mbar_expect_tx(&bar, nr * rowbytes);
        for (uint32_t r = 0; r < nr; ++r) bulk_load_row(stage + r * rowbytes, sb + r * sp + head * es, rowbytes, &bar);
    }
    // the unaligned heads and tails of the rows, by the other threads
    const uint32_t ns = (uint32_t)(head + (ncol - tail0));
    for (uint32_t e = threadIdx.x; e < nr * ns; e += blockDim.x) {
        const uint32_t r = e / ns, k = e % ns;
        const int64_t col = k < (uint32_t)head ? (int64_t)k : tail0 + (int64_t)(k - (uint32_t)head);
        copy_elem(sb + r * sp + col * es, db + r * dp + col * es, es);
    }
    if (threadIdx.x == 0) {
        ok = tma::mbar_wait(&bar, 0, err, 0x6730u);
        if (ok) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (uint32_t r = 0; r < nr; ++r) bulk_store_row(db + r * dp + head * es, stage + r * rowbytes, rowbytes);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            // the stage must stay valid until the stores have read it
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        } else {
            tma::mbar_drain(&bar, 0);  // let the loads in flight land before the CTA leaves
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int find_rpiece(const ReducePiece *p, int n, uint64_t e) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (p[mid].elem_begin <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T red_apply(int op, T a, T b) {
    switch (op) {
        case 0: return a + b;
        case 1: return a * b;
        case 2: return b < a ? b : a;
        default: return b > a ? b : a;
    }
}

template <typename T>
__device__ void reduce_one(const ReducePiece &p, const DView *srcs, const int64_t idx[3]) {
    int64_t od = 0;
    for (int d = 0; d < p.nd; ++d) od += idx[d] * p.dst.s[d];
    T acc = T(0);
    for (int k = 0; k < p.nsrc; ++k) {
        const DView &v = srcs[p.src_begin + k];
        int64_t os = 0;
        for (int d = 0; d < p.nd; ++d) os += idx[d] * v.s[d];
        T x = ((const T *)v.base)[os];
        acc = k == 0 ? x : red_apply<T>(p.op, acc, x);
    }
    ((T *)p.dst.base)[od] = acc;
}

__global__ void __launch_bounds__(256) reduce_kernel(const ReducePiece *__restrict__ pieces,
                                                     const DView *__restrict__ srcs, int n, uint64_t total) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        int pi = find_rpiece(pieces, n, e);
        const ReducePiece &p = pieces[pi];
        uint64_t l = e - p.elem_begin;
        int64_t ext[3] = {1, 1, 1};
        for (int d = 0; d < p.nd; ++d) ext[d] = p.hi[d] - p.lo[d] + 1;
        int64_t idx[3] = {0, 0, 0};
        for (int d = p.nd - 1; d >= 0; --d) {
            idx[d] = p.lo[d] + (int64_t)(l % (uint64_t)ext[d]);
            l /= (uint64_t)ext[d];
        }
        if (p.dtype == 0)
            reduce_one<float>(p, srcs, idx);
        else if (p.dtype == 3)
            reduce_one<uint32_t>(p, srcs, idx);
        else if (p.dtype == 2)
            reduce_one<unsigned char>(p, srcs, idx);
        else if (p.dtype == 4)
            reduce_one<double>(p, srcs, idx);
    }
}

}  // namespace

namespace k {

cudaError_t fill(const FillDesc &d, cudaStream_t st) {
    int64_t rows = 1;
    for (int k2 = 0; k2 < d.nd - 1; ++k2) rows *= d.hi[k2] - d.lo[k2] + 1;
    int64_t w = d.hi[d.nd - 1] - d.lo[d.nd - 1] + 1;
    int64_t units = rows * ((w + 8191) / 8192);
    int64_t grid = units < 152 * 64 ? units : 152 * 64;
    fill_kernel<<<(unsigned)grid, 256, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t copy_pieces(const CopyPiece *dev, int n, uint64_t total_units, cudaStream_t st) {
    if (!n || !total_units) return cudaSuccess;
    if (total_units > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    copy_kernel<<<(unsigned)total_units, 256, 0, st>>>(dev, n);
    return cudaGetLastError();
}

cudaError_t copy_pieces_staged(const CopyPiece *dev, int n, uint64_t total_units, uint32_t *err, cudaStream_t st) {
    if (!n || !total_units) return cudaSuccess;
    if (total_units > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(copy_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BULK_STAGE);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    copy_bulk_kernel<<<(unsigned)total_units, 256, BULK_STAGE, st>>>(dev, n, err);
    return cudaGetLastError();
}

cudaError_t reduce_pieces(const ReducePiece *dev, const DView *srcs, int n, uint64_t total_elems, cudaStream_t st) {
    if (!n || !total_elems) return cudaSuccess;
    uint64_t blocks = (total_elems + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(dev, srcs, n, total_elems);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
