/*
 * lightning.h -- C ABI of the single-GPU annotated-launch engine.
 *
 * The model follows the Lightning paper (arXiv 2202.05549):
 *   - a kernel launch is cut into superblocks, rectangular disjoint sub-grids
 *     of thread blocks (Sec. 2.1 "Distributed Kernel Launches");
 *   - arrays are 1-3-D, made of rectangular chunks defined by a
 *     distribution policy; chunks may overlap in halo cells whose replicas
 *     the runtime keeps coherent (Sec. 2.2 "Multi-Dimensional Distributed
 *     Arrays");
 *   - a data annotation gives each thread's affine read / write / readwrite /
 *     reduce(f) region; the access region of a superblock is the dense box of
 *     elements its threads touch (Sec. 2.3 "Data Annotations");
 *   - a planner turns each launch into tasks (Execute, Copy, Create/Delete of
 *     temporary chunks, Reduce) and adds dependencies on earlier launches for
 *     read-write / write-write / write-read conflicts on chunks (Sec. 2.4
 *     "Execution Planner");
 *   - a memory manager stages chunks in GPU memory from pre-allocated pools and
 *     evicts least-recently-used chunks to pinned host memory
 *     (Sec. 3.4 "Memory Management");
 *   - the kernel runs on an offset sub-grid with views whose base pointer has
 *     the chunk offset subtracted once (Sec. 3.5, Listing 3).
 * Everything runs on one GPU in one process.  There is no transport, no
 * worker process and no collective.
 *
 * Conventions for every call:
 *   - Each returns an lt_status: LT_OK (0) or a negative LT_ERR_* code.  No C++
 *     exception crosses the ABI.  lt_last_error() returns a message for the
 *     calling thread's most recent failure.
 *   - Pointers are host pointers unless the parameter says "device".
 *   - Objects (contexts, arrays, kernels) are owned by the library.  They are
 *     released by the matching *_destroy call; destroying a context releases
 *     everything created in it.
 *   - A context is not thread-safe: calls on one context must not overlap.
 *   - After an LT_ERR_CUDA the context is poisoned: every further call
 *     except lt_ctx_destroy returns LT_ERR_BUSY.  LT_ERR_TIMEOUT (a bounded
 *     device-side wait expired; the kernel returned early) leaves the context
 *     usable; the results of the work since the previous synchronize are
 *     undefined.
 */
#ifndef LIGHTNING_H
#define LIGHTNING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int32_t lt_status;
#define LT_OK 0
#define LT_ERR_INVALID_ARG (-1)  /* bad argument, shape, handle or dtype */
#define LT_ERR_PARSE (-2)        /* annotation text does not parse */
#define LT_ERR_OOM_DEVICE (-3)   /* HBM budget or device pool too small */
#define LT_ERR_OOM_HOST (-4)     /* pinned host pool too small */
#define LT_ERR_CUDA (-5)         /* a CUDA call failed; context poisoned */
#define LT_ERR_TIMEOUT (-6)      /* a bounded device-side wait expired */
#define LT_ERR_BUSY (-7)         /* context poisoned by an earlier error */
#define LT_ERR_UNSUPPORTED (-8)  /* valid request this build does not do */
#define LT_ERR_DEVICE_CHECK (-9) /* a kernel recorded a bounds violation */
#define LT_ERR_COMPILE (-10)      /* runtime compilation of a user kernel failed */

/* ---- element types (Sec. 2.2: arrays hold a primitive type) ------------- */
typedef enum {
    LT_F32 = 0,
    LT_BF16 = 1,
    LT_U8 = 2,
    LT_U32 = 3,
    LT_F64 = 4
} lt_dtype;

/* ---- distributions (Sec. 2.2; StencilDist / row-wise / column-wise /
 * tiled of Fig. 2 and the host code of Sec. 3.6) --------------------------
 * chunk[d]: extent of one chunk along axis d (axis 0 is the slowest, i.e.
 * rows of a 2-D array); 0 means the whole axis.  ROWS splits axis 0 only,
 * COLS axis 1 only, TILES every axis, BLOCK makes one chunk.  halo[d] widens
 * every chunk by that many cells on both sides along axis d (clipped to the
 * array), so neighbouring chunks overlap in replicated halo cells.
 * order: LT_ORDER_ROW stores each chunk row-major (last axis contiguous);
 * LT_ORDER_COL (2-D only) stores each chunk column-major (axis 0
 * contiguous).  The storage layout never changes results. */
typedef enum {
    LT_DIST_BLOCK = 0,
    LT_DIST_ROWS = 1,
    LT_DIST_COLS = 2,
    LT_DIST_TILES = 3
} lt_dist_kind;

typedef enum { LT_ORDER_ROW = 0, LT_ORDER_COL = 1 } lt_order;

typedef struct {
    int32_t kind;      /* lt_dist_kind */
    int32_t order;     /* lt_order */
    int64_t chunk[3];  /* chunk extent per axis, 0 = whole axis */
    int64_t halo[3];   /* halo width per axis */
} lt_dist;

/* ---- context ------------------------------------------------------------- */
/* hbm_budget_bytes: size of the device chunk pool (0 = 90% of free HBM).
 * host_pool_bytes: size of the pinned host pool that evicted chunks move to
 *   (0 = none: nothing may spill).
 * staging_cap_bytes: at most this many bytes of tasks may be enqueued ahead
 *   of the GPU before lt_launch waits (Sec. 3.4's staging throttle, 2 GB in
 *   the paper; 0 = 2 GiB).
 * flags: LT_FLAG_TIMING records CUDA events around every kernel and copy
 *   (read with lt_stats); LT_FLAG_DRYRUN runs planner, dependency tracker and
 *   memory manager without any device (no CUDA call is made; nothing is
 *   computed; lt_array_read/write/fill only update bookkeeping), for tests of
 *   the host logic; LT_FLAG_FIXED_SWEEP visits superblocks in index order
 *   every launch (default: the order alternates between launches, so the
 *   chunks used last are reused first); LT_FLAG_NO_STAGED makes the stencil
 *   built-ins use their register kernels instead of the TMA-staged ones, and
 *   packs, write-backs and replica updates copy through registers instead of
 *   through shared memory with bulk asynchronous copies (same results; for
 *   comparing the two); LT_FLAG_NO_LINK_QUARANTINE turns off
 *   the quarantine of slow host-pool ranges (every fetch and eviction of at
 *   least 256 MiB is timed; one that ran at less than half the fastest copy
 *   in its direction takes its host range out of the pool, up to a quarter
 *   of the pool: parts of large pinned allocations were measured to copy
 *   2-20x slower than the rest);
 *   LT_FLAG_NO_PDL launches every kernel in the plain stream order (default:
 *   a 2-D Jacobi launch that runs entirely in device memory, without copy
 *   steps, starts as a programmatic dependent of the kernel before it, so its
 *   CTAs launch while that kernel finishes);
 *   LT_FLAG_NO_FUSED_REPLICAS updates the halo replicas that a source kernel
 *   (lt_kernel_register_source) writes with a copy kernel after it (default:
 *   the wrapper's CTAs copy them after a grid-wide barrier in the same
 *   launch, which is then a cooperative launch); LT_FLAG_TEST_REPLICA_STALL
 *   (tests only) makes that barrier wait for one CTA more than the launch
 *   has, so its bounded wait (2 s) expires: the replicas are left as they
 *   were and lt_synchronize reports LT_ERR_TIMEOUT. */
#define LT_FLAG_TIMING 1
#define LT_FLAG_DRYRUN 2
#define LT_FLAG_FIXED_SWEEP 4
#define LT_FLAG_NO_STAGED 8
#define LT_FLAG_NO_LINK_QUARANTINE 16
#define LT_FLAG_NO_PDL 32
#define LT_FLAG_NO_FUSED_REPLICAS 64
#define LT_FLAG_TEST_REPLICA_STALL 128

typedef struct {
    size_t hbm_budget_bytes;
    size_t host_pool_bytes;
    size_t staging_cap_bytes;
    int32_t device;
    int32_t flags;
} lt_config;

typedef struct lt_ctx lt_ctx;
typedef struct lt_array lt_array;
typedef struct lt_kernel lt_kernel;

/* Create a context on `device`: allocates the HBM pool and the pinned host
 * pool up front (allocation is expensive, Sec. 3.4) and three streams
 * (compute, host-to-device, device-to-host).  *out is set on success. */
lt_status lt_ctx_create(const lt_config *cfg, lt_ctx **out);
/* Waits for all work, then frees every object of the context. */
lt_status lt_ctx_destroy(lt_ctx *ctx);
/* Message of the calling thread's last failure ("" if none).  Valid until
 * the thread's next lt_* call. */
const char *lt_last_error(void);

/* ---- arrays (Sec. 2.2; context.ones / context.zeros of Sec. 3.6) -------- */
/* Create an ndim (1..3) array of `shape` elements distributed by `dist`.
 * Its contents start as zero (chunks materialise lazily). */
lt_status lt_array_create(lt_ctx *ctx, lt_dtype dtype, int32_t ndim, const int64_t shape[3],
                          const lt_dist *dist, lt_array **out);

/* Zero-copy import of caller-owned DEVICE memory (for instance a CUDA
 * tensor) as a one-chunk array (no paper counterpart; the paper's arrays are
 * always library-owned).  ptr: device address of element 0; strides:
 * element strides per axis, the innermost 1.  The library reads and writes
 * that memory in place; it never moves, evicts or frees it.  The caller's
 * pending work on the memory must be complete before this call, and after
 * lt_synchronize the memory holds the results of every launch so far.
 * lt_array_destroy returns once no queued work uses the memory; the caller
 * may free it then.  Errors: LT_ERR_INVALID_ARG (null pointer, bad ndim,
 * non-positive strides, innermost stride not 1). */
lt_status lt_array_wrap_device(lt_ctx *ctx, lt_dtype dtype, int32_t ndim, const int64_t shape[3],
                               const int64_t strides[3], void *ptr, lt_array **out);
lt_status lt_array_destroy(lt_ctx *ctx, lt_array *arr);

/* Declare that the array's current contents will not be read again (for
 * instance the stale buffer of a ping-pong pair once the result is in the
 * other).  Its chunks are then dropped instead of written back when memory
 * is needed: once the launch that is still pending, if any, has finished
 * with each of them.  Reading the array before writing it again gives
 * unspecified values; any write (launch, lt_array_write, lt_array_fill)
 * makes the written chunks live again.  No counterpart in the paper: its
 * runtime learns that data is dead only from a later launch that overwrites
 * it (one launch of lookahead here), so a run's last launch must write back
 * an input it will never read again.  Errors: LT_ERR_INVALID_ARG. */
lt_status lt_array_discard(lt_ctx *ctx, lt_array *arr);

/* Copy the whole array from / to a dense row-major host buffer of exactly
 * `bytes` bytes.  Synchronous: waits for all earlier work; the buffer is
 * borrowed only during the call. */
lt_status lt_array_write(lt_ctx *ctx, lt_array *arr, const void *host, size_t bytes);
lt_status lt_array_read(lt_ctx *ctx, lt_array *arr, void *host, size_t bytes);
/* The same without waiting (an extension: the paper's arrays are filled and
 * read synchronously).  Each chunk's copy is enqueued as an operation on a
 * copy stream (H2D for writes, D2H for reads) behind the operations that
 * last produced or used the chunk, so the copies overlap kernels and copies
 * of the other direction, and later launches wait only for the chunks they
 * use.  The buffer must stay valid and must not be touched by the caller
 * until lt_synchronize (or another synchronous call) returns; pinned host
 * memory is needed for the copies to run asynchronously.  Several calls on
 * the same buffer are ordered where their host regions overlap: a write of
 * a chunk reads its whole box (halo included) from the buffer, a read writes
 * the chunk's owned box into it.  Column-major arrays, and reads of arrays
 * with chunks outside device memory, take the synchronous path.  Errors as
 * for lt_array_write / lt_array_read. */
lt_status lt_array_write_async(lt_ctx *ctx, lt_array *arr, const void *host, size_t bytes);
lt_status lt_array_read_async(lt_ctx *ctx, lt_array *arr, void *host, size_t bytes);
/* The same with a dense row-major DEVICE buffer of the context's device
 * (for instance a CUDA tensor).  Row-major chunks only
 * (LT_ERR_UNSUPPORTED otherwise).  Synchronous. */
lt_status lt_array_write_device(lt_ctx *ctx, lt_array *arr, const void *dev, size_t bytes);
lt_status lt_array_read_device(lt_ctx *ctx, lt_array *arr, void *dev, size_t bytes);
/* Copy the box lo..hi (inclusive, per axis) of the array into a dense
 * row-major host buffer of exactly (box volume * element size) bytes.
 * Synchronous; reads each element from the chunk that owns it. */
lt_status lt_array_read_box(lt_ctx *ctx, lt_array *arr, const int64_t lo[3], const int64_t hi[3], void *host,
                            size_t bytes);

/* Fill every element from its global row-major index g with a seeded
 * counter-based generator (SplitMix64, Steele, Lea & Flood 2014): element g
 * takes output x = mix(key + (g+1)*0x9E3779B97F4A7C15), key = first output
 * of SplitMix64 seeded with (seed ^ (stream << 32)).
 *   LT_INIT_ZERO, LT_INIT_CONST (value): constants;
 *   LT_INIT_UNIFORM: f32 (x >> 40) * 2^-24 in [0,1);
 *   LT_INIT_KAPPA: f32 of 0.05 + 0.15 * u (u as above, in fp64);
 *   LT_INIT_NORMAL_BF16: bf16 of N(0,1)*scale by Box-Muller from counters
 *     2g and 2g+1, rounded to f32 then to bf16 (RNE);
 *   LT_INIT_U8: u8 x >> 56.
 * Asynchronous (ordered like a launch that writes the whole array). */
typedef enum {
    LT_INIT_ZERO = 0,
    LT_INIT_CONST = 1,
    LT_INIT_UNIFORM = 2,
    LT_INIT_KAPPA = 3,
    LT_INIT_NORMAL_BF16 = 4,
    LT_INIT_U8 = 5
} lt_init_kind;

typedef struct {
    int32_t kind;
    uint64_t seed;
    uint64_t stream;
    double value;
    double scale;
} lt_init;

lt_status lt_array_fill(lt_ctx *ctx, lt_array *arr, const lt_init *init);

/* Number of chunks, and the box of chunk `index`: lo/hi inclusive per axis
 * (the halo included) and where it currently lives (0 none, 1 device,
 * 2 host). */
lt_status lt_array_num_chunks(lt_ctx *ctx, const lt_array *arr, int64_t *n);
lt_status lt_array_chunk_info(lt_ctx *ctx, const lt_array *arr, int64_t index, int64_t lo[3],
                              int64_t hi[3], int32_t *location);

/* ---- kernels (Sec. 3.5-3.6: CudaKernelDef ... .param_value / .param_array
 * / .annotate / .compile) -------------------------------------------------
 * The kernel bodies are built in, compiled ahead of time for sm_103a; each
 * one is written in the paper's convention (a device function of the
 * virtual block index and of array views).  The annotation is parsed and
 * checked here: it must name every array parameter once, and its regions
 * must contain the accesses the built-in actually makes.
 *
 * Annotation grammar (Sec. 2.3):
 *   annotation := bindings "=>" stmt ("," stmt)*
 *   bindings   := binding ("," binding)*
 *   binding    := ("global" | "block" | "local") (var | "[" var ("," var)* "]")
 *   stmt       := mode name "[" index ("," index)* "]"
 *   mode       := "read" | "write" | "readwrite" | "reduce(" ("+"|"*"|"min"|"max") ")"
 *   index      := affine | [affine] ":" [affine]     (bounds inclusive)
 *   affine     := integer linear combination of bound variables plus a constant
 * A bracketed list binds its LAST variable to the x grid dimension, the one
 * before to y, then z (so "global [i, j]" gives j = x, the contiguous axis of
 * a row-major array); a single variable binds x.  Omitted slice bounds are
 * the array's first / last index. */
typedef enum {
    LT_K_PLAN_ONLY = 0,      /* no body: any annotation, any arrays; plans and dry-run launches only */
    LT_K_STENCIL1D = 1,      /* out[i] = (in[i-1]+in[i]+in[i+1])/3.0 (Listing 1), f32 */
    LT_K_JACOBI2D = 2,       /* V = ((((U+Un)+Us)+Uw)+Ue)/5, zero ghosts, f32 */
    LT_K_JACOBI3D = 3,       /* 7-point analogue, /7 */
    LT_K_GEMM_BF16 = 4,      /* C[i,j] = sum_k A[i,k] B[k,j]; bf16 in, f32 accumulate/out */
    LT_K_HIST256 = 5,        /* reduce(+) H[:] of one count per u8 element */
    LT_K_DIFFUSION2D = 6,    /* u1 = u + K*(Lu), f32 */
    LT_K_DIFFUSION2D_ADJ = 7, /* adjoint step: reduce(+) of the transposed stencil */
    LT_K_ROWREDUCE = 8,       /* "read A[i, j], reduce(f) S[i]" (Sec. 2.3), f32, f in + * min max */
    LT_K_JACOBI2D_MULTI = 9,  /* k Jacobi iterations per launch (value parameter k, 1..16), reads U[i-k:i+k, j-k:j+k] */
    LT_K_KMEANS_ASSIGN = 10,  /* K-Means (Sec. 4): X (f32, 4 features per record, flat), C (f32, k x 4, flat),
                               * reduce(+) S (f64, k x 5: feature sums and count per centre); value parameter
                               * k (1..64); "global i => read X[4*i:4*i+3], read C[:], reduce(+) S[:]" */
    LT_K_KMEANS_UPDATE = 11,  /* new centres: C2[4j+f] = f32(S[5j+f] / S[5j+4]), or C[4j+f] when the count
                               * is 0; "global j => read S[5*j:5*j+4], read C[4*j:4*j+3], write C2[4*j:4*j+3]" */
    LT_K_LAPLACE2D = 12,      /* G = L U: ((((U[i-1,j] + U[i+1,j]) + U[i,j-1]) + U[i,j+1]) - 4 U[i,j]), zero ghosts, f32;
                               * "global [i, j] => read U[i-1:i+1, j-1:j+1], write G[i, j]" */
    LT_K_EWISE2D = 13,        /* C = A + B (value parameter op = 0) or C = A * B (op = 1), f32;
                               * "global [i, j] => read A[i, j], read B[i, j], write C[i, j]" */
    LT_K_MULADD2D = 14,       /* C = C + A * B, f32; "global [i, j] => read A[i, j], read B[i, j], readwrite C[i, j]"
                               * (LAPLACE2D, EWISE2D and MULADD2D are the steps of the diffusion and of its adjoint
                               * as separate launches: the unfused form the fused adjoint is measured against) */
    LT_K_USER = 100           /* (kernels from lt_kernel_register_source) */
} lt_builtin;

typedef struct {
    const char *name;
    int32_t is_array; /* 1: array parameter (param_array), 0: value (param_value) */
    int32_t dtype;    /* lt_dtype of the array, or of the value (LT_F32 / LT_U32) */
} lt_param;

lt_status lt_kernel_register(lt_ctx *ctx, int32_t builtin, const char *annotation, const lt_param *params,
                             int32_t nparams, lt_kernel **out);
lt_status lt_kernel_destroy(lt_ctx *ctx, lt_kernel *k);

/* Register a kernel from CUDA source, compiled at run time (Sec. 3.5,
 * Listings 2-3).  `source` defines
 *     __device__ void <name>(dim3 virtBlockIdx, <one parameter per params[i]>)
 * value parameters arrive as int64_t (integer dtypes) or double (LT_F32);
 * array parameters as lightning::Vector<T> / Matrix<T> / Tensor<T> for 1, 2
 * or 3 indices in the annotation, indexed with global indices (v[i],
 * m(i, j) or m[i][j], t(k, i, j)); T is float, unsigned short (bf16 bits),
 * unsigned char or unsigned int.  lightning::div_rn<C>(float) and
 * lightning::div4_rn<C>(float4) divide by a small integer constant C with
 * IEEE rounding (equal to x / C) in a few instructions, as the built-in
 * stencils do.  Use virtBlockIdx instead of blockIdx and
 * gridDim; blockDim and threadIdx are those of the launch.  The library
 * generates the wrapper kernel that maps physical to virtual blocks and
 * builds the views (the chunk offset subtracted once).  The wrapper is
 * persistent: each CTA calls the function for several virtual blocks in turn,
 * with a __syncthreads() before each call, so shared memory is not shared
 * between two virtual blocks' calls.  When the launch writes an array whose
 * chunks keep halo replicas, the wrapper's CTAs update those replicas
 * themselves after all virtual blocks are done (a grid-wide barrier with a
 * bounded wait; the launch is then cooperative, and the function must not
 * end its block early with a trap or leave CTAs that never return); with
 * LT_FLAG_NO_FUSED_REPLICAS a copy kernel after the launch does it.  T may
 * also be double (LT_F64).  The library compiles both with NVRTC for sm_103a
 * (IEEE arithmetic, no FMA contraction) and loads them.  The annotation is
 * trusted: the kernel must not touch elements outside it.  At most 5 array,
 * 4 integer and 4 float parameters.  Errors: LT_ERR_PARSE, LT_ERR_COMPILE
 * (the compiler log is in lt_last_error()), LT_ERR_UNSUPPORTED (no NVRTC).
 * In LT_FLAG_DRYRUN contexts the source is compiled but not loaded. */
lt_status lt_kernel_register_source(lt_ctx *ctx, const char *source, const char *name, const char *annotation,
                                    const lt_param *params, int32_t nparams, lt_kernel **out);

/* ---- launches (Sec. 2.1, Sec. 2.4; kernel.launch of Sec. 3.6) ------------
 * grid: number of threads along x, y, z (like launch(n, 16, ...) in the
 * host code of Sec. 3.6); block: threads per block.  workdist.superblock:
 * threads per superblock along x, y, z (BlockDist), rounded up to whole
 * blocks; 0 = the whole grid.  args[i] matches params[i] of the kernel.
 * The launch is planned, enqueued and returns without waiting for the GPU
 * (Sec. 2.4: plan construction overlaps execution).  It may block only when
 * the staging throttle is reached. */
typedef struct {
    uint64_t x, y, z;
} lt_dim3;

typedef struct {
    int64_t superblock[3];
} lt_workdist;

typedef struct {
    lt_array *array; /* for array parameters */
    double f;        /* for value parameters of type LT_F32 */
    int64_t i;       /* for value parameters of type LT_U32 / integers */
} lt_arg;

lt_status lt_launch(lt_ctx *ctx, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
                    const lt_arg *args, int32_t nargs);

/* ---- batched launches (an extension beyond the paper) --------------------
 * One descriptor is one launch, issued `repeat` times; between repeats the
 * first two array arguments swap (ping-pong), so {JACOBI2D, args {U, V},
 * repeat 8} means U->V, V->U, ... eight launches.  lt_launch_batch(descs, n)
 * has the meaning of issuing every descriptor's launches in order with
 * lt_launch.  When every descriptor is a JACOBI2D or HIST256 launch over
 * single-chunk arrays and no array appears in two descriptors, the whole
 * batch runs as ONE persistent kernel fed by a device-side work queue
 * (items ordered iteration-major; a tile waits, bounded, for the previous
 * iteration of its instance), captured once in a CUDA graph and replayed
 * while the same arrays stay at the same addresses.  Its tile height and
 * histogram slice come from an autotuner that times candidates on the first
 * iteration of the batch (which writes only data the real run overwrites)
 * and caches the choice per batch shape.  Otherwise, or with
 * LT_BATCH_PLAIN, the launches are issued one by one (the plain form).
 * The fused form checks every descriptor's annotation as lt_launch does,
 * once: a call whose descriptors equal the last checked batch (kernels,
 * grids, blocks, superblocks, arguments and repeats) skips the checks.
 * Asynchronous like lt_launch; the descriptors are read during the call. */
typedef struct {
    lt_kernel *kernel;
    lt_dim3 grid, block;
    lt_workdist wd;
    const lt_arg *args;
    int32_t nargs;
    int32_t repeat;
} lt_launch_desc;

#define LT_BATCH_PLAIN 1    /* issue the launches one by one */
#define LT_BATCH_NO_GRAPH 2 /* fused kernel, launched directly (no graph capture) */
#define LT_BATCH_RETUNE 4   /* run the autotuner again for this batch shape */
/* Test hook: omit the first iteration's work items of every Jacobi launch
 * with repeat >= 2, so the later items' bounded waits (2 s) expire and
 * lt_synchronize reports LT_ERR_TIMEOUT without any fault.  Not cached. */
#define LT_BATCH_TEST_STALL 256
/* Test hook: skip the autotuner and use work items of 32 rows by 1024
 * columns (so the column split of wide parts is exercised).  Not cached. */
#define LT_BATCH_TEST_TILE_COLS 512

lt_status lt_launch_batch(lt_ctx *ctx, const lt_launch_desc *descs, int32_t n, int32_t flags);

/* Blocks until every enqueued task has finished (context.synchronize() of
 * Sec. 3.6).  Reports device-side error words (bounds checks, timeouts). */
lt_status lt_synchronize(lt_ctx *ctx);

/* Device-side timing of everything enqueued between the two calls, across
 * the context's three streams.  lt_timer_start records a CUDA event on the
 * compute stream and makes both copy streams wait for it; lt_timer_stop
 * makes the compute stream wait for both copy streams, records a second
 * event, waits for it on the host and returns the elapsed milliseconds. */
lt_status lt_timer_start(lt_ctx *ctx);
lt_status lt_timer_stop(lt_ctx *ctx, double *ms);

/* Turns the per-operation CUDA events of LT_FLAG_TIMING on (1) or off (0)
 * for the operations enqueued from now on (the pending launch is enqueued
 * first).  The events cost a few microseconds of GPU time per operation, so
 * a caller can time a run with them off and measure kernels with them on. */
lt_status lt_op_timing(lt_ctx *ctx, int32_t on);

/* ---- statistics and plan inspection -------------------------------------- */
typedef struct {
    uint64_t launches;        /* lt_launch calls */
    uint64_t tasks_execute;   /* Execute tasks (superblocks run) */
    uint64_t tasks_copy;      /* Copy tasks: pack, unpack, replica updates */
    uint64_t tasks_reduce;    /* Reduce tasks */
    uint64_t deps;            /* dependency edges added between tasks */
    uint64_t fetches;         /* chunk host -> device transfers */
    uint64_t evictions;       /* chunk device -> host transfers */
    uint64_t dead_skips;      /* transfers skipped because the data was dead */
    uint64_t bytes_h2d;       /* host -> device bytes */
    uint64_t bytes_d2h;       /* device -> host bytes */
    uint64_t bytes_d2d;       /* device -> device copy bytes (pack/unpack/replica) */
    uint64_t kernels;         /* kernels launched by the library */
    uint64_t hbm_in_use;      /* bytes of the HBM pool in use now */
    uint64_t hbm_peak;        /* high-water mark of hbm_in_use */
    uint64_t host_in_use;     /* bytes of the host pool in use now */
    /* with LT_FLAG_TIMING, measured with CUDA events on the launching stream
     * (valid after lt_synchronize): */
    double ms_execute;        /* sum of Execute kernel durations */
    uint64_t n_execute_kernels;
    double ms_copy_kernels;   /* pack/unpack/replica/reduce kernels */
    uint64_t n_copy_kernels;
    double ms_h2d;            /* sum of host->device copy durations */
    double ms_d2h;            /* sum of device->host copy durations */
    double ms_fill;           /* fill kernels */
    uint64_t batches_fused;   /* lt_launch_batch calls run as one persistent kernel */
    uint64_t batches_plain;   /* lt_launch_batch calls issued launch by launch */
    uint64_t graph_replays;   /* fused batches replayed from a cached CUDA graph */
    int64_t tuned_tile_rows;  /* autotuner choice of the last fused batch */
    int64_t tuned_hist_slice;
    uint64_t tables_resident; /* descriptor tables reused on the device without a copy */
    uint64_t plans_reused;    /* launches whose plan came from the kernel's plan cache */
    uint64_t reduce_inplace;  /* reduce partials accumulated in their destination chunk (no copy) */
    uint64_t bytes_replica_wt; /* halo-replica bytes the Execute kernels wrote themselves (no copy step) */
    /* with LT_FLAG_TIMING, from the start and end events of the timed
     * operations, per synchronize (valid after lt_synchronize): */
    double ms_span;           /* first operation's start to the last one's end, summed over synchronizes */
    double ms_link_busy;      /* time a host<->device chunk copy (fetch or eviction) was running */
    double ms_link_both;      /* time copies in both directions were running at once */
    double ms_exec_hidden;    /* Execute kernel time during which a host<->device copy was running */
    uint64_t host_withheld_bytes; /* host pool bytes withheld as slow to copy (quarantine), now */
    uint64_t host_quarantined;    /* copies that put their host range in quarantine */
    int64_t tuned_tile_cols;      /* autotuner choice of the last fused batch: tile columns (0: a part's width) */
} lt_stats;

lt_status lt_stats_get(lt_ctx *ctx, lt_stats *out);
lt_status lt_stats_reset(lt_ctx *ctx);

/* Plan a launch without enqueueing it and write a JSON description into
 * buf (NUL-terminated, truncated to cap bytes; *needed receives the full
 * length): superblocks, each argument's access region, the chunk decision
 * (direct / pack / temp-write / reduce) and the replica copies.  Host-only;
 * valid in LT_FLAG_DRYRUN contexts. */
lt_status lt_plan_explain(lt_ctx *ctx, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
                          const lt_arg *args, int32_t nargs, char *buf, size_t cap, size_t *needed);

/* JSON log of the tasks enqueued since the last reset: kind, superblock,
 * chunks, predecessor task ids, memory actions (fetch / evict / dead);
 * execute tasks add the kernel variant the built-in chose for the launch
 * ("variant") and the CTA count.  Kept only while `enable` is 1
 * (lt_debug_log_enable), for tests. */
lt_status lt_debug_log_enable(lt_ctx *ctx, int32_t enable);
lt_status lt_debug_log(lt_ctx *ctx, char *buf, size_t cap, size_t *needed);
/* JSON list of the operations timed with LT_FLAG_TIMING events while the log
 * is enabled, collected at each lt_synchronize: task id (as in lt_debug_log),
 * stream (0 compute, 1 host-to-device, 2 device-to-host), category (0 Execute
 * kernel, 1 copy kernel, 2 fetch, 3 eviction, 4 fill), start and end in
 * milliseconds.  Times within one synchronize share an origin; each later
 * synchronize's times start after the previous ones.  Same buffer rules as
 * lt_debug_log. */
lt_status lt_debug_timeline(lt_ctx *ctx, char *buf, size_t cap, size_t *needed);

/* ---- allocation-free Jacobi step -------------------------------------------
 * The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory (code running under another framework's allocator
 * or memory budget, or a process that must not grow its device footprint
 * after start-up).  It computes one 2-D 5-point Jacobi step
 *     V[i,j] = ((((U[i,j] + U[i-1,j]) + U[i+1,j]) + U[i,j-1]) + U[i,j+1]) / 5
 * (zero outside the ny x nx grid), bit-identical to lt_launch of
 * LT_K_JACOBI2D, by the same pack-then-execute sequence as an annotated
 * launch over tiles without halo: each tile_rows x tile_cols tile's read
 * region (the tile plus a one-cell ring) is gathered into scratch and the
 * tile is computed from that copy.
 *   U, V: distinct DEVICE pointers to row-major f32 grids with leading
 *         dimensions ld_u, ld_v >= nx (elements); the caller owns both.
 *   stream: a cudaStream_t (NULL = the legacy default stream); the call is
 *         asynchronous on it and returns once everything is enqueued.
 * Scratch: a file-scope device array of LT_NOALLOC_SCRATCH_BYTES (64 MiB),
 * present on every device that loads the library until the process exits.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  Tiles are processed in batches that fit the scratch; a tile
 * whose packed region exceeds it is rejected with LT_ERR_INVALID_ARG.
 * Every call shares the scratch and leaves the last call's contents in it:
 * calls that overlap on the GPU race, calls ordered on one stream do not.
 * Every call looks up the scratch's device address on the current device
 * (cudaGetSymbolAddress); the first call on a device also loads the module
 * there, so make that first call before any stream capture.  The descriptor
 * tables are uploaded from a host buffer that lives only for the call: on a
 * stream that is capturing the call returns LT_ERR_UNSUPPORTED and enqueues
 * nothing.
 * Errors: LT_ERR_INVALID_ARG (bad pointers or sizes), LT_ERR_UNSUPPORTED
 * (the stream is capturing), LT_ERR_CUDA (a CUDA call failed);
 * lt_last_error() gives the message. */
#define LT_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
lt_status lt_jacobi2d_packed_noalloc(const float *U, float *V, int64_t ny, int64_t nx, int64_t ld_u, int64_t ld_v,
                                     int64_t tile_rows, int64_t tile_cols, void *stream);

/* ---- self-test of the stencils' constant divisions (no paper counterpart) --
 * The Jacobi built-ins divide their sums by 5 (2-D) and 7 (3-D) with a
 * correctly rounded three-instruction sequence (Markstein's correction step)
 * instead of a full IEEE division.  This call runs that sequence on `device`
 * for all 2^32 float bit patterns and counts the inputs where it differs
 * from the IEEE quotient (any two NaNs count as equal) into *mismatches
 * (0 expected); it runs the four-wide form (one range test for four
 * quotients) the same way, each pattern in each of the four positions.  divisor: 5 or 7.  Synchronous; allocates 8 bytes of device
 * memory for the count.  Errors: LT_ERR_INVALID_ARG (other divisor, null
 * output), LT_ERR_CUDA (a CUDA call failed). */
lt_status lt_selftest_div_const(int32_t device, int32_t divisor, uint64_t *mismatches);

#ifdef __cplusplus
}
#endif
#endif /* LIGHTNING_H */
