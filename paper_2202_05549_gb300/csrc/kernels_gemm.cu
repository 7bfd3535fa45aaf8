// BF16 GEMM built-in on the 5th-generation tensor cores (tcgen05), for the
// annotated launch "global [i, j] => read A[i, :], read B[:, j], write C[i, j]"
// (the naive matrix-multiplication annotation of Sec. 2.3; GEMM workload of
// Sec. 4.2).  C = A B with bf16 inputs and f32 accumulation and output.
//
// One persistent kernel runs every superblock (output tile chunk) of a
// launch.  Each CTA owns one SM and walks output tiles of 256 x 256, each
// computed as two M = 128 halves that share the B operand of a stage:
//   warp 0      TMA producer: A (256 x 64) and B (256 x 64) K-slices, 64 KB
//               per stage, into a 3-stage shared-memory ring, 128-byte
//               swizzled;
//   warp 1      MMA issuer: per K-step of 16, two tcgen05.mma kind::f16
//               (M=128, N=256), one per M-half, into a single TMEM
//               accumulator of 2 x 256 = 512 columns; commits to mbarriers
//               that free ring stages and publish the accumulator;
//   warps 2-5   epilogue: tcgen05.ld of both halves (each warp reads its
//               32-lane quarter), masked f32 stores to the C chunk, then
//               release of the accumulator.
// With one accumulator the MMA warp waits for the epilogue of a tile before
// it starts the next one; at the K of the GEMM workload (65536) that wait is
// a small fraction of a tile, at small K it is visible.
// A must be stored row-major and B column-major (both K-contiguous), which
// the column-major chunk order of the distribution provides.  Ragged M, N
// and K are handled by TMA zero fill and masked stores.
// Every mbarrier wait is bounded (%globaltimer, 2 s): on expiry the kernel
// records an error, lets its own copies and MMAs finish (bounded), frees
// TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace lt {
namespace {

// Tile BM x BN: MH M-halves of UM = 128 rows (one tcgen05.mma each, both
// reading the same B stage), so a stage's B bytes serve MH MMAs.  The
// accumulators of a tile take MH x BN TMEM columns; NACC tiles fit in the
// 512 columns.  At 256 x 256 that is one (a shape with NACC = 2 would let
// the epilogue of one tile overlap the MMAs of the next).
constexpr int MH = 2, UM = 128;
// BK = 64: 128-byte stage rows, 128-byte swizzle, 3 stages of 64 KB.  (BK =
// 32 with 64-byte swizzle fits 7 stages of 32 KB in 224 KB, but its 64-byte
// TMA rows raised L2 throughput from 41 % to 66 % of peak and lowered the
// tensor pipe's active time from 84 % to 76 %: 11 % slower at 16384^3.)
constexpr int BM = MH * UM, BN = 256, BK = 64, UMMA_K = 16;
constexpr int SW_BYTES = BK * 2;  // bytes of one K-row of a stage = the swizzle span
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 512;
constexpr int NACC = TMEM_COLS / (MH * BN);
static_assert(NACC >= 1 && STAGES >= 2, "tile shape does not fit TMEM or shared memory");
static_assert(SW_BYTES == 128 || SW_BYTES == 64, "one K-row of a stage must be a 128- or 64-byte swizzle span");
constexpr int MAX_MAPS = 15;
constexpr int GROUP_M = 16;  // tile raster: 16 M-tiles share each B panel
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;

struct GemmParams {
    CUtensorMap amap[MAX_MAPS];
    CUtensorMap bmap[MAX_MAPS];
    uint64_t total_tiles;
    int64_t K;
    int64_t M, N;
    uint32_t *err;
    int32_t ntasks;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done;
}

// Bounded wait; returns false (and raises the abort flag) on expiry or if
// another role already aborted.
__device__ __noinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint32_t *err,
                                       uint32_t code) {
    unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            if (err) atomicCAS(err, 0u, code);
            return false;
        }
    }
}

// Wait used while cleaning up after an abort: bounded, never raises.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity) && gtimer() - t0 < WAIT_NS / 4) {
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t c0, int32_t c1,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// K-major operand in shared memory, swizzled rows of SW_BYTES (the swizzle
// span): 8-row groups 8 x SW_BYTES apart (stride byte offset), descriptor
// version 1, layout type 2 (128-byte swizzle) or 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)((8 * SW_BYTES) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(SW_BYTES == 128 ? 2 : 4) << 61;
    return d;
}

// Instruction descriptor, kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N = BN = 256, M = UM = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(UM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TileInfo {
    int task;
    int64_t m0, n0, m_last, n_last;
};

__device__ __forceinline__ TileInfo decode_tile(const ExecTask *__restrict__ tasks, int ntasks, uint64_t g,
                                                int64_t M, int64_t N) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((uint64_t)tasks[mid].cta_begin <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ExecTask &t = tasks[lo];
    int64_t r0 = t.t_lo[1], r1 = min(t.t_hi[1], M - 1);
    int64_t c0 = t.t_lo[0], c1 = min(t.t_hi[0], N - 1);
    int64_t tiles_m = (r1 - r0 + BM) / BM, tiles_n = (c1 - c0 + BN) / BN;
    int64_t l = (int64_t)(g - t.cta_begin);
    int64_t per_group = GROUP_M * tiles_n;
    int64_t grp = l / per_group, first_m = grp * GROUP_M;
    int64_t gm = min((int64_t)GROUP_M, tiles_m - first_m);
    int64_t within = l % per_group;
    int64_t tm = first_m + within % gm, tn = within / gm;
    TileInfo ti;
    ti.task = lo;
    ti.m0 = r0 + tm * BM;
    ti.n0 = c0 + tn * BN;
    ti.m_last = r1;
    ti.n_last = c1;
    return ti;
}

__global__ void __launch_bounds__(THREADS, 1) gemm_bf16_kernel(const ExecTask *__restrict__ tasks,
                                                               const __grid_constant__ GemmParams P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + NACC;
    uint32_t *tmem_slot = (uint32_t *)(acc_empty + NACC);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t nk = (P.K + BK - 1) / BK;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0, armed_parity = 0;  // bit s: stage armed; parity of its last arm
            bool ok = true;
            for (uint64_t g = blockIdx.x; g < P.total_tiles && ok; g += gridDim.x) {
                TileInfo ti = decode_tile(tasks, P.ntasks, g, P.M, P.N);
                const ExecTask &t = tasks[ti.task];
                const CUtensorMap *am = &P.amap[t.aux[0]];
                const CUtensorMap *bm = &P.bmap[t.aux[1]];
                int32_t arow = (int32_t)(ti.m0 - t.v[0].org[0]);
                int32_t bcol = (int32_t)(ti.n0 - t.v[1].org[1]);
                int32_t ak0 = (int32_t)(0 - t.v[0].org[1]);
                int32_t bk0 = (int32_t)(0 - t.v[1].org[0]);
                for (int64_t kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, P.err, 0x6701)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[stage], STAGE_BYTES);
                    uint8_t *sa = smem + stage * STAGE_BYTES;
                    tma_load_2d(sa, am, ak0 + (int32_t)(kb * BK), arow, &full[stage]);
                    tma_load_2d(sa + A_BYTES, bm, bk0 + (int32_t)(kb * BK), bcol, &full[stage]);
                    armed |= 1u << stage;
                    armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (!ok)  // let our own copies land before the CTA exits
                for (int s = 0; s < STAGES; ++s)
                    if (armed & (1u << s)) mbar_drain(&full[s], (armed_parity >> s) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (uint64_t g = blockIdx.x; g < P.total_tiles && ok; g += gridDim.x) {
                if (!mbar_wait(&acc_empty[acc], acc_phase ^ 1, abort_flag, P.err, 0x6702)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * MH * BN);
                for (int64_t kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(&full[stage], phase, abort_flag, P.err, 0x6703)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
                    const uint64_t ad = sw_desc(sa), bd = sw_desc(sa + A_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / UMMA_K; ++k) {
                        const uint64_t koff = (uint64_t)((k * UMMA_K * 2) >> 4);
#pragma unroll
                        for (int h = 0; h < MH; ++h)  // M-half h: A rows h*UM.., accumulator columns h*BN..
                            umma(d_tmem + (uint32_t)(h * BN), ad + (uint64_t)((h * UM * BK * 2) >> 4) + koff,
                                 bd + koff, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    umma_commit(&empty[stage]);  // frees the stage once these MMAs have read it
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(&acc_full[acc]);
                if (++acc == NACC) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (!ok) {  // let issued MMAs finish before TMEM is freed
                umma_commit(&acc_full[acc]);
                mbar_drain(&acc_full[acc], acc_phase);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5, 128 threads)
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        int acc = 0;
        uint32_t acc_phase = 0;
        for (uint64_t g = blockIdx.x; g < P.total_tiles; g += gridDim.x) {
            TileInfo ti = decode_tile(tasks, P.ntasks, g, P.M, P.N);
            if (!mbar_wait(&acc_full[acc], acc_phase, abort_flag, P.err, 0x6704)) break;
            tc_fence_after();
            const ExecTask &t = tasks[ti.task];
            const DView cv = t.v[2];
#pragma unroll 1
            for (int hc = 0; hc < MH * (BN / 32); ++hc) {
            const int h = hc / (BN / 32), c = hc % (BN / 32);
            const int64_t row = ti.m0 + h * UM + q * 32 + lane;
            float *crow = (float *)(cv.base + (uint64_t)(row * cv.s[0] * 4));
            {
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * MH * BN + h * BN + c * 32), v);
                const int64_t col = ti.n0 + c * 32;
                if (row <= ti.m_last && col <= ti.n_last) {
                    if (col + 31 <= ti.n_last && cv.s[1] == 1) {
                        float4 *dst = (float4 *)(crow + col);
#pragma unroll
                        for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (col + i <= ti.n_last) crow[(col + i) * cv.s[1]] = v[i];
                    }
                }
            }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[acc]);
            if (++acc == NACC) {
                acc = 0;
                acc_phase ^= 1;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D K-major bf16 operand map over one chunk: inner extent k_valid, outer
// extent rows_valid, row pitch in bytes, box BK x box_rows, SW_BYTES swizzle.
bool make_map(CUtensorMap *m, uint64_t base, uint64_t k_valid, uint64_t rows_valid, uint64_t pitch_bytes,
              uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {k_valid, rows_valid};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)(uintptr_t)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, SW_BYTES == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

GemmParams g_params;  // built by prepare, consumed by the launch that follows it
int g_num_sms = 0;

}  // namespace

namespace k {

uint32_t prepare_gemm_bf16(ExecTask *t, int n, ExecParams &p) {
    std::memset(&g_params, 0, sizeof(g_params));
    const int64_t M = p.shape[2][0], N = p.shape[2][1], K = p.shape[0][1];
    std::vector<uint64_t> abase, bbase;
    uint64_t tiles = 0;
    p.variant = 0;
    for (int i = 0; i < n; ++i) {
        const DView &A = t[i].v[0], &B = t[i].v[1];
        // A row-major (K contiguous), B column-major (K contiguous)
        if (A.s[1] != 1 || B.s[0] != 1) {
            p.variant = -1;
            return 0xFFFFFFFFu;
        }
        uint64_t a0 = A.base + (uint64_t)((A.org[0] * A.s[0] + A.org[1]) * 2);
        uint64_t b0 = B.base + (uint64_t)((B.org[0] + B.org[1] * B.s[1]) * 2);
        int ai = -1, bi = -1;
        for (size_t j = 0; j < abase.size(); ++j)
            if (abase[j] == a0) ai = (int)j;
        for (size_t j = 0; j < bbase.size(); ++j)
            if (bbase[j] == b0) bi = (int)j;
        if (ai < 0) {
            if ((int)abase.size() == MAX_MAPS) {
                p.variant = -2;
                return 0xFFFFFFFFu;
            }
            ai = (int)abase.size();
            abase.push_back(a0);
            if (!make_map(&g_params.amap[ai], a0, (uint64_t)(A.hi[1] - A.org[1] + 1), (uint64_t)(A.hi[0] - A.org[0] + 1),
                          (uint64_t)A.s[0] * 2, BM)) {
                p.variant = -3;
                return 0xFFFFFFFFu;
            }
        }
        if (bi < 0) {
            if ((int)bbase.size() == MAX_MAPS) {
                p.variant = -2;
                return 0xFFFFFFFFu;
            }
            bi = (int)bbase.size();
            bbase.push_back(b0);
            if (!make_map(&g_params.bmap[bi], b0, (uint64_t)(B.hi[0] - B.org[0] + 1), (uint64_t)(B.hi[1] - B.org[1] + 1),
                          (uint64_t)B.s[1] * 2, BN)) {
                p.variant = -3;
                return 0xFFFFFFFFu;
            }
        }
        t[i].aux[0] = ai;
        t[i].aux[1] = bi;
        int64_t r0 = t[i].t_lo[1], r1 = std::min(t[i].t_hi[1], M - 1);
        int64_t c0 = t[i].t_lo[0], c1 = std::min(t[i].t_hi[0], N - 1);
        uint64_t nt = (r1 >= r0 && c1 >= c0) ? (uint64_t)((r1 - r0 + BM) / BM) * (uint64_t)((c1 - c0 + BN) / BN) : 0;
        t[i].cta_begin = (uint32_t)tiles;
        t[i].cta_count = (uint32_t)nt;
        tiles += nt;
    }
    g_params.total_tiles = tiles;
    g_params.K = K;
    g_params.M = M;
    g_params.N = N;
    g_params.err = p.err;
    g_params.ntasks = n;
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    uint64_t ctas = tiles < (uint64_t)g_num_sms ? tiles : (uint64_t)g_num_sms;
    return (uint32_t)ctas;
}

cudaError_t launch_gemm_bf16(const ExecTask *dev, uint32_t ctas, const ExecParams &p, cudaStream_t st) {
    (void)p;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gemm_bf16_kernel<<<ctas, THREADS, SMEM_BYTES, st>>>(dev, g_params);
    return cudaGetLastError();
}

}  // namespace k
}  // namespace lt
