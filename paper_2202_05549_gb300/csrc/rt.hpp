// Internal types and functions of the runtime, shared by its translation
// units (not part of the C ABI):
//   rt_streams.cpp  error messages, fences on the three streams, per-operation
//                   timing, the descriptor upload ring and resident tables
//   rt_memory.cpp   chunk views, the HBM and pinned-host arenas, eviction,
//                   fetches and host transfers, dead-data tracking
//   rt_launch.cpp   plan cache, lookahead and the launch executor (lt_launch)
//   rt_batch.cpp    fused batches, their CUDA graphs and the autotuner
//   rt_api.cpp      the rest of the C ABI: contexts, arrays, kernels, stats
//
// Runtime of the single-GPU annotated-launch engine: context, stream-ordered
// fences, pooled memory with LRU spilling, the launch executor and the C ABI.
//
// Scheduling model (Sec. 3.3 "Scheduling", Sec. 3.4 "Memory Management"),
// re-designed for one GPU: the planner runs on the calling thread and turns
// each launch into operations on three CUDA streams (compute, host->device,
// device->host).  Every chunk carries two fence sets: `ready` (operations
// that produced its current contents) and `busy` (operations that read or
// wrote the memory it occupies).  A task waits on the fences its accesses
// conflict with (read-after-write, write-after-read, write-after-write), so
// the dependency DAG of Sec. 2.4 is realised as CUDA event waits between the
// three in-order streams, and lt_launch returns before the GPU runs it.
// Memory decisions (which chunk to evict, where a fetch lands) are made at
// enqueue time in program order; freed memory keeps the fences of its last
// users, so reuse never races with them.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "core.hpp"
#include "kernels.cuh"
#include "lightning.h"
#include "userkernel.hpp"

namespace lt {
namespace rt {

enum { S_COMP = 0, S_H2D = 1, S_D2H = 2, NSTREAM = 3 };
enum { LOC_NONE = 0, LOC_DEV = 1, LOC_HOST = 2 };
const int RING = 1024;
const size_t ALIGN = 1024;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Allocation size class: requests are rounded up to 1/128 of their power of
// two (under 1% waste), so chunks of nearly equal size (a band with one halo
// row fewer) fit each other's holes and the pool does not fragment.
inline size_t size_class(size_t sz) {
    if (sz == 0) sz = 1;
    size_t g = ALIGN;
    if (sz > ((size_t)1 << 17)) {
        int lg = 63 - __builtin_clzll((unsigned long long)sz);
        g = (size_t)1 << (lg - 7);
    }
    return align_up(sz, g);
}

struct FenceSet {
    uint64_t q[NSTREAM] = {0, 0, 0};
    void add(int s, uint64_t v) {
        if (v > q[s]) q[s] = v;
    }
    void merge(const FenceSet &o) {
        for (int s = 0; s < NSTREAM; ++s) add(s, o.q[s]);
    }
    static FenceSet one(int s, uint64_t v) {
        FenceSet f;
        f.add(s, v);
        return f;
    }
};

// Pool of one pre-allocated region; best-fit, coalescing on demand.  Each
// free block remembers the fences of the operations that last used its memory
// and when it was released.  Freed blocks stay separate, each with its own
// fences, and among equally good fits the block released longest ago is
// reused first: the copy that freed the newest block is likely still running,
// and reusing its memory would order the next copy behind it (for instance a
// device-to-host eviction behind the host-to-device fetch that just released
// a host block, which serialises the two directions of the link).  Only when
// no single free block is large enough are adjacent blocks merged (and their
// fences with them).
struct Arena {
    struct Free {
        size_t size;
        FenceSet f;
        uint64_t tick;
    };
    size_t cap = 0;
    char *base = nullptr;
    std::map<size_t, Free> free_;
    size_t used = 0, peak = 0;
    uint64_t tick = 0;
    // Oldest-first instead of best-fit: the host pool, whose requests are all
    // chunk-sized evictions, takes the block freed longest ago (untouched
    // space first), whose last users are most likely done.  Best-fit there
    // picked the slot a fetch had just emptied over untouched space, so the
    // eviction waited for that fetch and the two copy directions ran in turn.
    bool oldest_first = false;

    void init(size_t c, char *b) {
        cap = c / ALIGN * ALIGN;
        base = b;
        free_.clear();
        if (cap) free_[0] = {cap, FenceSet(), 0};
        used = peak = 0;
    }
    bool take(size_t sz, size_t *off, FenceSet *f) {
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second.size < sz) continue;
            if (best == free_.end() ||
                (oldest_first ? it->second.tick < best->second.tick
                              : it->second.size < best->second.size ||
                                    (it->second.size == best->second.size && it->second.tick < best->second.tick)))
                best = it;
        }
        if (best == free_.end()) return false;
        *off = best->first;
        *f = best->second.f;
        size_t rem = best->second.size - sz;
        Free keep = best->second;
        free_.erase(best);
        if (rem) free_[*off + sz] = {rem, keep.f, keep.tick};
        used += sz;
        peak = std::max(peak, used);
        return true;
    }
    void coalesce() {
        for (auto it = free_.begin(); it != free_.end();) {
            auto nx = std::next(it);
            if (nx != free_.end() && it->first + it->second.size == nx->first) {
                it->second.size += nx->second.size;
                it->second.f.merge(nx->second.f);
                it->second.tick = std::max(it->second.tick, nx->second.tick);
                free_.erase(nx);
            } else {
                it = nx;
            }
        }
    }
    bool alloc(size_t sz, size_t *off, FenceSet *f) {
        sz = size_class(sz);
        if (take(sz, off, f)) return true;
        coalesce();
        return take(sz, off, f);
    }
    // Quarantine: ranges taken out of the free space for good.  A range is
    // withheld where it is free now and, for the parts in use, when their
    // block is released.
    std::vector<std::pair<size_t, size_t>> bad;  // [begin, end)
    struct Held {
        size_t off, size;
        FenceSet f;  // the fences of the range's last users
        uint64_t tick;
    };
    std::vector<Held> held;  // the ranges taken out of the free space
    size_t withheld = 0;
    // Give every withheld range back (a slow pool beats no pool) and forget
    // the bad ranges.
    void release_quarantine() {
        for (const Held &h : held) free_[h.off] = {h.size, h.f, h.tick};
        held.clear();
        bad.clear();
        withheld = 0;
    }
    void withhold_free(size_t b, size_t e) {
        for (auto it = free_.begin(); it != free_.end();) {
            const size_t fb = it->first, fe = fb + it->second.size;
            const size_t lo = std::max(fb, b), hi = std::min(fe, e);
            if (lo >= hi) {
                ++it;
                continue;
            }
            Free keep = it->second;
            it = free_.erase(it);
            if (lo > fb) free_[fb] = {lo - fb, keep.f, keep.tick};
            if (fe > hi) free_[hi] = {fe - hi, keep.f, keep.tick};
            held.push_back({lo, hi - lo, keep.f, keep.tick});
            withheld += hi - lo;
            it = free_.upper_bound(lo);
        }
    }
    void quarantine(size_t off, size_t len) {
        bad.push_back({off, off + len});
        withhold_free(off, off + len);
    }
    void release(size_t off, size_t sz, const FenceSet &f) {
        sz = size_class(sz);
        used -= sz;
        free_[off] = {sz, f, ++tick};
        for (const auto &r : bad)
            if (r.first < off + sz && r.second > off) withhold_free(std::max(r.first, off), std::min(r.second, off + sz));
    }
};

struct CState {
    int loc = LOC_NONE;
    size_t off = 0;     // offset from the device pool's base (external chunks: their address, minus that base)
    bool ext = false;   // storage owned by the caller (lt_array_wrap_device): always resident, never freed
    FenceSet ready, busy;
    uint64_t lru = 0;
    int pin = 0;
    int64_t dead_launch = -1;       // launch whose first touch may skip the fetch
    int64_t next_dead_launch = -1;  // launch after which the next launch overwrites it unread
    int64_t last_use_launch = -1;   // launch and group of its last use in that launch
    int64_t last_use_group = -1;
    int64_t last_write_launch = -1;  // last launch that wrote it
    bool discarded = false;          // contents declared dead (lt_array_discard) and not written since
    // the last asynchronous copies between this chunk and a host buffer
    // (lt_array_write_async reads the chunk's box from the buffer,
    // lt_array_read_async writes the chunk's owned box into it)
    FenceSet host_write, host_read;
};


struct BuiltinDef {
    int id;
    const char *canon;
    int narr;
    int dtype[LT_MAX_ARRAYS];
    int nd[LT_MAX_ARRAYS];
    uint32_t (*prepare)(ExecTask *, int, ExecParams &);
    cudaError_t (*launch)(const ExecTask *, uint32_t, const ExecParams &, cudaStream_t);
    bool reduce_zero = true;  // reduce partials must start at the identity (else the kernel writes every cell)
    bool any_reduce_op = false;  // the reduce argument may use any of + * min max
    int write_through = -1;      // array slot whose halo replicas the kernel writes itself (ExecTask.rep_*)
    bool pdl = false;            // the launch function supports programmatic dependent launch (ExecParams.pdl)
};


extern const BuiltinDef kBuiltins[];
extern const size_t kNumBuiltins;
std::string canon_text(const BuiltinDef *d, int64_t kval);
const BuiltinDef *find_builtin(int id);

}  // namespace rt
}  // namespace lt

using namespace lt;
using namespace lt::rt;

struct lt_array {
    ArrayGeom g;
    std::vector<CState> cs;
    int64_t id = 0;
};

// A launch plan and what follows from the plan alone.  Launches of the same
// shape (kernel, grid, block, superblock, step count, and array arguments of
// the same geometry with the same aliasing) share one, so an iterative loop
// that swaps its arrays plans once.
struct PlanBundle {
    LaunchPlan plan;
    std::vector<std::pair<int, int64_t>> dead;  // (parameter, chunk) the launch overwrites without reading
};

struct CachedPlan {
    std::shared_ptr<const PlanBundle> b;
    uint64_t last_use = 0;
};

struct PlanKeyHash {
    size_t operator()(const std::vector<int64_t> &v) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (int64_t x : v) h = (h ^ (uint64_t)x) * 0x100000001B3ull + (h >> 29);
        return (size_t)h;
    }
};

struct lt_kernel {
    // plans of the most recently used launch shapes (at most PLAN_CACHE), by key
    std::unordered_map<std::vector<int64_t>, CachedPlan, PlanKeyHash> plans;
    uint64_t plan_tick = 0;
    const BuiltinDef *def = nullptr;
    std::unique_ptr<BuiltinDef> own_def;     // user kernels: their own signature
    cudaLibrary_t ulib = nullptr;            // user kernels: loaded NVRTC cubin
    cudaKernel_t ufn = nullptr;
    std::map<int, int> uocc;                 // user kernels: resident CTAs per SM by block size
    Annotation ann, canon;
    std::vector<lt_param> params;
    std::vector<std::string> names;
    std::vector<int> stmt_of_param;  // annotation statement of each parameter (-1 = value)
    std::vector<int> slot_of_param;  // array slot of each parameter (-1 = value)
    std::vector<int> canon_stmt;     // canonical statement of each array slot
};

struct TimedOp {
    int cat;
    cudaEvent_t a, b;
    int64_t task = -1;
    int stream = 0;
};

// A planned launch waiting for the next one (one launch of lookahead).
struct PendingLaunch {
    lt_kernel *k = nullptr;
    std::shared_ptr<const PlanBundle> b;
    std::vector<lt_array *> parr;
    ExecParams ep{};
};

// A fused batch: device tables, tuned shape and (optionally) its CUDA graph.
struct BatchCache {
    std::vector<uint64_t> key;
    size_t off = 0, bytes = 0;  // device block in the HBM pool holding the tables
    BatchParams bp{};
    const BatchHist *dev_hist = nullptr;
    int nhist = 0;
    size_t counters_off = 0, counters_bytes = 0;
    int ctas = 0;
    cudaGraphExec_t exec = nullptr;
};

// The fused form of a batch of launches (rt_batch.cpp).
struct BatchShape {
    struct Jac {
        lt_array *u, *v;
        int repeat;
        std::shared_ptr<const PlanBundle> plan;  // the launch's plan: superblocks over direct chunks
    };
    struct Hist {
        lt_array *x, *h;
    };
    std::vector<Jac> jac;
    std::vector<Hist> hist;
};

struct UploadUse {
    size_t off, end;
    uint64_t seq;
};

struct lt_ctx {
    lt_config cfg{};
    bool dry = false;
    bool no_staged = false;  // LT_FLAG_NO_STAGED
    bool no_pdl = false;     // LT_FLAG_NO_PDL
    int sm_count = 1;        // streaming multiprocessors of the device
    // Host-link copies being timed (quarantine of slow host-pool ranges).
    struct LinkProbe {
        cudaEvent_t a, b;
        size_t host_off, bytes;
        int dir;  // 0 fetch, 1 eviction
    };
    std::vector<LinkProbe> link_probes;
    std::vector<cudaEvent_t> link_ev_pool;
    double link_best[2] = {0, 0};  // fastest copy seen per direction (bytes per ms)
    bool no_quarantine = false;     // LT_FLAG_NO_LINK_QUARANTINE
    bool poisoned = false;
    cudaStream_t st[NSTREAM] = {nullptr, nullptr, nullptr};
    uint64_t seq[NSTREAM] = {0, 0, 0};
    std::vector<cudaEvent_t> ev[NSTREAM];
    std::vector<uint64_t> evseq[NSTREAM];
    std::vector<int64_t> evtask[NSTREAM];
    // Deferred fences: an operation may end without recording its event (so
    // that two kernels follow each other directly on the stream and the
    // second can use programmatic dependent launch).  Per ring slot: the
    // deferred sequence number, its task, and the sequence number whose event
    // covers it (0: none yet; ~0: known complete).  `deferred` lists the ones
    // no event covers yet.
    std::vector<uint64_t> dfseq[NSTREAM], dfcov[NSTREAM];
    std::vector<int64_t> dftask[NSTREAM];
    std::vector<uint64_t> deferred[NSTREAM];
    Arena dev, host;
    char *dev_base = nullptr;
    char *host_base = nullptr;
    // descriptor upload ring
    char *up_host = nullptr, *up_dev = nullptr;
    size_t up_cap = 0, up_head = 0;
    std::deque<UploadUse> up_inflight;
    // resident descriptor tables (after the ring in both allocations)
    struct TableSlot {
        std::vector<char> bytes;  // host copy of the slot's contents (empty: free)
        uint64_t last_use = 0;
        cudaEvent_t staged = nullptr;  // recorded after the copy that filled the slot
    };
    std::vector<TableSlot> tslots;
    uint64_t tslot_tick = 0;
    uint32_t *err_word = nullptr;  // device error word
    uint32_t *err_host = nullptr;  // pinned host copy of the error word, read back in stream order by sync_all
    // Grid barrier of source kernels that update their replicas themselves:
    // a device counter every CTA of such a launch increments once, and the
    // host's running total of those increments (a launch waits for the total
    // after its own CTAs have arrived).
    unsigned long long *ubar = nullptr;
    uint64_t ubar_total = 0;
    bool no_fused_replicas = false;   // LT_FLAG_NO_FUSED_REPLICAS
    bool test_replica_stall = false;  // LT_FLAG_TEST_REPLICA_STALL
    std::vector<std::unique_ptr<lt_array>> arrays;       // creation order (iteration order)
    std::unordered_set<const lt_array *> array_set;      // membership: handles are checked on every call
    std::vector<uint64_t> batch_checked;  // the last fused batch whose launches passed prepare_plan
    std::shared_ptr<BatchShape> batch_shape;  // and its fused form
    std::vector<std::unique_ptr<lt_kernel>> kernels;
    uint64_t clock = 0;
    int64_t launch_id = 0;
    int64_t task_id = 0;
    int64_t next_array_id = 1;
    lt_stats stats{};
    bool log_on = false;
    std::ostringstream log;
    std::ostringstream tlog;  // start and end times of timed operations (while the log is on)
    int tlog_n = 0;
    double tlog_base = 0;
    int log_n = 0;
    std::vector<TimedOp> timed;
    std::vector<cudaEvent_t> tev_pool;
    std::unique_ptr<PendingLaunch> pending;
    std::unique_ptr<BatchCache> batch;
    std::map<std::pair<int64_t, int64_t>, std::array<int, 3>> tuned;  // batch shape -> (tile rows, cols, slice)
    int64_t cur_group = 0;
    cudaEvent_t timer[2] = {nullptr, nullptr};
    cudaEvent_t timer_join[2] = {nullptr, nullptr};
    // current operation (between op_begin and op_end)
    int cur_stream = 0;
    int64_t cur_task = -1;
    std::vector<int64_t> cur_deps;
};

#define CK(ctx, expr)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            (ctx)->poisoned = true;                                                            \
            return fail(LT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));      \
        }                                                                                      \
    } while (0)

namespace lt {
namespace rt {

lt_status fail(lt_status st, const std::string &msg);
const char *last_error_text();
lt_status link_copy_timed(lt_ctx *c, int dir, void *dst, const void *src, size_t n, size_t host_off);
lt_status link_poll(lt_ctx *c);

// fences and timing (rt_streams.cpp)
lt_status op_begin(lt_ctx *c, int s, const char *kind);
lt_status op_wait(lt_ctx *c, const FenceSet &f);
lt_status op_end(lt_ctx *c, uint64_t *out_seq, const std::string &extra = "", bool defer = false);
cudaEvent_t fence_event(lt_ctx *c, int t, uint64_t q, int64_t *task, bool flush);
lt_status host_wait(lt_ctx *c, int s, uint64_t q);
cudaEvent_t tev_get(lt_ctx *c);
lt_status timeline_overlap(lt_ctx *c);
lt_status collect_timing(lt_ctx *c);
lt_status sync_all(lt_ctx *c);
lt_status check_ctx(lt_ctx *c);
lt_array *find_array(lt_ctx *c, const lt_array *a);
lt_kernel *find_kernel(lt_ctx *c, const lt_kernel *k);
int32_t uniform_cta_count(const std::vector<ExecTask> &tasks);

constexpr int TSLOTS = 32;
constexpr size_t TSLOT_BYTES = (size_t)64 << 10;
constexpr size_t NO_RING = ~(size_t)0;  // ring offset of a table served by a resident slot
lt_status upload_resident(lt_ctx *c, const void *src, size_t n, void **dev_ptr, bool *done);
lt_status upload(lt_ctx *c, const void *src, size_t n, void **dev_ptr, size_t *ring_off);
void upload_done(lt_ctx *c, size_t off, size_t n, uint64_t seq);

enum { CAT_EXEC = 0, CAT_COPYK = 1, CAT_H2D = 2, CAT_D2H = 3, CAT_FILL = 4 };

struct TimeScope {
    lt_ctx *c;
    int cat;
    cudaEvent_t a = nullptr;
    TimeScope(lt_ctx *ctx, int category) : c(ctx), cat(category) {
        if (!c->dry && (c->cfg.flags & LT_FLAG_TIMING)) {
            a = tev_get(c);
            if (a) cudaEventRecord(a, c->st[c->cur_stream]);
        }
    }
    void end() {
        if (!a) return;
        cudaEvent_t b = tev_get(c);
        if (b) {
            cudaEventRecord(b, c->st[c->cur_stream]);
            c->timed.push_back({cat, a, b, c->cur_task, c->cur_stream});
        }
        a = nullptr;
    }
    ~TimeScope() { end(); }
};

// memory (rt_memory.cpp)
char *dptr(const lt_ctx *c, uint64_t off);
DView view_of(lt_ctx *c, const ArrayGeom &g, const ChunkGeom &cg, size_t off);
bool droppable(const lt_ctx *c, const CState &s);
bool pick_victim(lt_ctx *c, lt_array **va, int64_t *vc);
lt_status dev_alloc(lt_ctx *c, size_t bytes, size_t *off, FenceSet *f, bool soft = false);
lt_status evict(lt_ctx *c, lt_array *a, int64_t ci);
lt_status ensure_dev(lt_ctx *c, lt_array *a, int64_t ci, bool need_data, bool soft = false);
lt_status xfer_chunk(lt_ctx *c, lt_array *a, int64_t ci, const Box &box, char *hb, bool to_dev,
                     bool other_is_device = false, int stream = S_COMP, bool wait = true);
void xfer_chunk_host(lt_ctx *c, lt_array *a, int64_t ci, const Box &box, char *hb, bool to_chunk);
std::vector<std::pair<lt_array *, int64_t>> dead_chunks(const LaunchPlan &plan, const std::vector<lt_array *> &parr);
std::vector<std::pair<int, int64_t>> dead_by_param(const LaunchPlan &plan, const std::vector<lt_array *> &parr);
void mark_dead(lt_ctx *c, const PlanBundle &b, const std::vector<lt_array *> &parr);

// launches (rt_launch.cpp)
lt_status prepare_plan(lt_ctx *c, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
                       const lt_arg *args, int32_t nargs, std::shared_ptr<const PlanBundle> *out,
                       std::vector<lt_array *> *parr);
lt_status emit_launch(lt_ctx *c, PendingLaunch &pl, const std::vector<std::pair<lt_array *, int64_t>> *next_dead);
bool pending_writes(lt_ctx *c, const lt_array *a);
lt_status flush_pending(lt_ctx *c);

}  // namespace rt
}  // namespace lt
