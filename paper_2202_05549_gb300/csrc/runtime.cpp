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
#include <cuda_runtime.h>

#include <algorithm>
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

using namespace lt;

static thread_local std::string g_err;

static lt_status fail(lt_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

extern "C" const char *lt_last_error(void) { return g_err.c_str(); }

lt_status lt::set_last_error(lt_status st, const std::string &msg) { return fail(st, msg); }

namespace {

enum { S_COMP = 0, S_H2D = 1, S_D2H = 2, NSTREAM = 3 };
enum { LOC_NONE = 0, LOC_DEV = 1, LOC_HOST = 2 };
const int RING = 1024;
const size_t ALIGN = 1024;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Allocation size class: requests are rounded up to 1/128 of their power of
// two (under 1% waste), so chunks of nearly equal size (a band with one halo
// row fewer) fit each other's holes and the pool does not fragment.
size_t size_class(size_t sz) {
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
    void release(size_t off, size_t sz, const FenceSet &f) {
        sz = size_class(sz);
        used -= sz;
        free_[off] = {sz, f, ++tick};
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
};

const BuiltinDef kBuiltins[] = {
    {LT_K_PLAN_ONLY, nullptr, 0, {0}, {0}, nullptr, nullptr},
    {LT_K_STENCIL1D, "global i => write A0[i], read A1[i-1:i+1]", 2, {LT_F32, LT_F32}, {1, 1},
     k::prepare_stencil1d, k::launch_stencil1d},
    {LT_K_JACOBI2D, "global [i, j] => read A0[i-1:i+1, j-1:j+1], write A1[i, j]", 2, {LT_F32, LT_F32}, {2, 2},
     k::prepare_jacobi2d, k::launch_jacobi2d, true, false, 1},
    {LT_K_JACOBI3D, "global [k, i, j] => read A0[k-1:k+1, i-1:i+1, j-1:j+1], write A1[k, i, j]", 2,
     {LT_F32, LT_F32}, {3, 3}, k::prepare_jacobi3d, k::launch_jacobi3d},
    {LT_K_HIST256, "global i => read A0[i], reduce(+) A1[:]", 2, {LT_U8, LT_U32}, {1, 1}, k::prepare_hist256,
     k::launch_hist256},
    {LT_K_DIFFUSION2D, "global [i, j] => read A0[i-1:i+1, j-1:j+1], read A1[i, j], write A2[i, j]", 3,
     {LT_F32, LT_F32, LT_F32}, {2, 2, 2}, k::prepare_diffusion, k::launch_diffusion},
    {LT_K_DIFFUSION2D_ADJ,
     "global [i, j] => read A0[i, j], read A1[i, j], read A2[i-1:i+1, j-1:j+1], readwrite A3[i, j], "
     "reduce(+) A4[i-1:i+1, j-1:j+1]",
     5, {LT_F32, LT_F32, LT_F32, LT_F32, LT_F32}, {2, 2, 2, 2, 2}, k::prepare_diffusion_adj, k::launch_diffusion_adj,
     false},
    {LT_K_JACOBI2D_MULTI, "global [i, j] => read A0[i-{K}:i+{K}, j-{K}:j+{K}], write A1[i, j]", 2,
     {LT_F32, LT_F32}, {2, 2}, k::prepare_jacobi2d_multi, k::launch_jacobi2d_multi},
    {LT_K_ROWREDUCE, "global [i, j] => read A0[i, j], reduce(+) A1[i]", 2, {LT_F32, LT_F32}, {2, 1},
     k::prepare_rowreduce, k::launch_rowreduce, false, true},
    {LT_K_KMEANS_ASSIGN, "global i => read A0[4*i:4*i+3], read A1[:], reduce(+) A2[:]", 3, {LT_F32, LT_F32, LT_F64},
     {1, 1, 1}, k::prepare_kmeans_assign, k::launch_kmeans_assign},
    {LT_K_KMEANS_UPDATE, "global i => read A0[5*i:5*i+4], read A1[4*i:4*i+3], write A2[4*i:4*i+3]", 3,
     {LT_F64, LT_F32, LT_F32}, {1, 1, 1}, k::prepare_kmeans_update, k::launch_kmeans_update},
    {LT_K_GEMM_BF16, "global [i, j] => read A0[i, :], read A1[:, j], write A2[i, j]", 3, {LT_BF16, LT_BF16, LT_F32},
     {2, 2, 2}, k::prepare_gemm_bf16, k::launch_gemm_bf16},
};

// Canonical annotation of a built-in; "{K}" stands for the launch's first
// integer value parameter (the step count of the multi-step stencil).
std::string canon_text(const BuiltinDef *d, int64_t kval) {
    std::string s = d->canon ? d->canon : "";
    const std::string key = "{K}";
    for (size_t pos = s.find(key); pos != std::string::npos; pos = s.find(key))
        s.replace(pos, key.size(), std::to_string(kval));
    return s;
}

const BuiltinDef *find_builtin(int id) {
    for (const auto &b : kBuiltins)
        if (b.id == id) return &b;
    return nullptr;
}

}  // namespace

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

struct UploadUse {
    size_t off, end;
    uint64_t seq;
};

struct lt_ctx {
    lt_config cfg{};
    bool dry = false;
    bool no_staged = false;  // LT_FLAG_NO_STAGED
    bool poisoned = false;
    cudaStream_t st[NSTREAM] = {nullptr, nullptr, nullptr};
    uint64_t seq[NSTREAM] = {0, 0, 0};
    std::vector<cudaEvent_t> ev[NSTREAM];
    std::vector<uint64_t> evseq[NSTREAM];
    std::vector<int64_t> evtask[NSTREAM];
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
    std::vector<std::unique_ptr<lt_array>> arrays;       // creation order (iteration order)
    std::unordered_set<const lt_array *> array_set;      // membership: handles are checked on every call
    std::vector<uint64_t> batch_checked;  // the last fused batch whose launches passed prepare_plan
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
    std::map<std::pair<int64_t, int64_t>, std::pair<int, int>> tuned;  // batch shape -> (tile rows, slice)
    int64_t cur_group = 0;
    cudaEvent_t timer[2] = {nullptr, nullptr};
    cudaEvent_t timer_join[2] = {nullptr, nullptr};
    // current operation (between op_begin and op_end)
    int cur_stream = 0;
    int64_t cur_task = -1;
    std::vector<int64_t> cur_deps;
};

namespace {

#define CK(ctx, expr)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            (ctx)->poisoned = true;                                                            \
            return fail(LT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));      \
        }                                                                                      \
    } while (0)

// ---------------------------------------------------------------- fences
lt_status op_begin(lt_ctx *c, int s, const char *kind) {
    c->cur_stream = s;
    c->cur_task = ++c->task_id;
    c->cur_deps.clear();
    if (c->log_on) {
        c->log << (c->log_n++ ? "," : "") << "{\"id\":" << c->cur_task << ",\"kind\":\"" << kind
               << "\",\"stream\":" << s << ",\"launch\":" << c->launch_id;
    }
    return LT_OK;
}

lt_status op_wait(lt_ctx *c, const FenceSet &f) {
    int s = c->cur_stream;
    for (int t = 0; t < NSTREAM; ++t) {
        uint64_t q = f.q[t];
        if (!q) continue;
        int slot = (int)(q % RING);
        bool live = c->evseq[t][slot] == q;
        if (live) {
            int64_t pt = c->evtask[t][slot];
            if (pt >= 0 && std::find(c->cur_deps.begin(), c->cur_deps.end(), pt) == c->cur_deps.end()) {
                c->cur_deps.push_back(pt);
                c->stats.deps++;
            }
        }
        if (t == s || c->dry || !live) continue;
        CK(c, cudaStreamWaitEvent(c->st[s], c->ev[t][slot], 0));
    }
    return LT_OK;
}

// Finish the current operation: record its fence on its stream.
lt_status op_end(lt_ctx *c, uint64_t *out_seq, const std::string &extra = "") {
    int s = c->cur_stream;
    uint64_t q = ++c->seq[s];
    int slot = (int)(q % RING);
    if (!c->dry) {
        if (c->evseq[s][slot] != 0) CK(c, cudaEventSynchronize(c->ev[s][slot]));  // bounded run-ahead
        CK(c, cudaEventRecord(c->ev[s][slot], c->st[s]));
    }
    c->evseq[s][slot] = q;
    c->evtask[s][slot] = c->cur_task;
    if (c->log_on) {
        c->log << ",\"deps\":[";
        for (size_t i = 0; i < c->cur_deps.size(); ++i) c->log << (i ? "," : "") << c->cur_deps[i];
        c->log << "]" << extra << "}";
    }
    *out_seq = q;
    return LT_OK;
}

lt_status host_wait(lt_ctx *c, int s, uint64_t q) {
    if (c->dry || !q) return LT_OK;
    int slot = (int)(q % RING);
    if (c->evseq[s][slot] == q) CK(c, cudaEventSynchronize(c->ev[s][slot]));
    return LT_OK;
}

// timing events around one operation (LT_FLAG_TIMING)
cudaEvent_t tev_get(lt_ctx *c) {
    if (!c->tev_pool.empty()) {
        cudaEvent_t e = c->tev_pool.back();
        c->tev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

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

// Overlap of the timed operations collected at one synchronize (all streams
// were idle before the first of them): the time the host link carried a
// copy, the time it carried copies in both directions at once, and the
// Execute-kernel time during which a copy ran (kernel time hidden under the
// link).  Times are relative to the first operation's start event.
lt_status timeline_overlap(lt_ctx *c) {
    if (c->timed.empty()) return LT_OK;
    struct Edge {
        float t;
        int cat;
        int d;
    };
    std::vector<Edge> ev;
    ev.reserve(c->timed.size() * 2);
    float lo = 0, hi = 0;
    for (size_t i = 0; i < c->timed.size(); ++i) {
        const TimedOp &t = c->timed[i];
        float t0 = 0, t1 = 0;
        if (i) CK(c, cudaEventElapsedTime(&t0, c->timed[0].a, t.a));
        CK(c, cudaEventElapsedTime(&t1, c->timed[0].a, t.b));
        if (t1 < t0) t1 = t0;
        if (c->log_on) {
            c->tlog << (c->tlog_n++ ? "," : "") << "{\"id\":" << t.task << ",\"stream\":" << t.stream
                    << ",\"cat\":" << t.cat << ",\"t0\":" << c->tlog_base + t0 << ",\"t1\":" << c->tlog_base + t1
                    << "}";
        }
        lo = i ? std::min(lo, t0) : t0;
        hi = i ? std::max(hi, t1) : t1;
        if (t.cat != CAT_EXEC && t.cat != CAT_H2D && t.cat != CAT_D2H) continue;
        ev.push_back({t0, t.cat, +1});
        ev.push_back({t1, t.cat, -1});
    }
    std::sort(ev.begin(), ev.end(), [](const Edge &x, const Edge &y) { return x.t < y.t || (x.t == y.t && x.d < y.d); });
    int n[5] = {0, 0, 0, 0, 0};
    for (size_t i = 0; i < ev.size(); ++i) {
        if (i) {
            double dt = (double)ev[i].t - (double)ev[i - 1].t;
            if (dt > 0) {
                const bool h = n[CAT_H2D] > 0, d = n[CAT_D2H] > 0;
                if (h || d) c->stats.ms_link_busy += dt;
                if (h && d) c->stats.ms_link_both += dt;
                if (n[CAT_EXEC] > 0 && (h || d)) c->stats.ms_exec_hidden += dt;
            }
        }
        n[ev[i].cat] += ev[i].d;
    }
    c->stats.ms_span += (double)hi - (double)lo;
    c->tlog_base += (double)hi + 1.0;  // the next synchronize's operations start after these
    return LT_OK;
}

lt_status collect_timing(lt_ctx *c) {
    lt_status ov = timeline_overlap(c);
    if (ov) return ov;
    for (auto &t : c->timed) {
        float ms = 0;
        CK(c, cudaEventElapsedTime(&ms, t.a, t.b));
        switch (t.cat) {
            case CAT_EXEC:
                c->stats.ms_execute += ms;
                c->stats.n_execute_kernels++;
                break;
            case CAT_COPYK:
                c->stats.ms_copy_kernels += ms;
                c->stats.n_copy_kernels++;
                break;
            case CAT_H2D: c->stats.ms_h2d += ms; break;
            case CAT_D2H: c->stats.ms_d2h += ms; break;
            default: c->stats.ms_fill += ms;
        }
        c->tev_pool.push_back(t.a);
        c->tev_pool.push_back(t.b);
    }
    c->timed.clear();
    return LT_OK;
}

// ---------------------------------------------------------------- views
// Device address of pool offset `off`.  Unsigned arithmetic, so offsets of
// external chunks (their address minus the pool base, modulo 2^64) come back
// exactly.
char *dptr(const lt_ctx *c, uint64_t off) { return (char *)(uintptr_t)((uint64_t)(uintptr_t)c->dev_base + off); }

DView view_of(lt_ctx *c, const ArrayGeom &g, const ChunkGeom &cg, size_t off) {
    DView v;
    uint64_t p = (uint64_t)(uintptr_t)dptr(c, off);
    int64_t o = 0;
    for (int d = 0; d < 3; ++d) {
        v.s[d] = d < g.nd ? cg.stride[d] : 0;
        o += (d < g.nd ? cg.s_origin[d] : 0) * v.s[d];
    }
    v.base = p - (uint64_t)(o * (int64_t)g.esize());
    for (int d = 0; d < 3; ++d) {
        v.org[d] = d < g.nd ? cg.s_origin[d] : 0;
        v.hi[d] = d < g.nd ? cg.box.hi[d] : 0;
    }
    return v;
}

// ---------------------------------------------------------------- memory manager
lt_status evict(lt_ctx *c, lt_array *a, int64_t ci);

// Pick the least-recently-used unpinned resident chunk.
// Can chunk state s be evicted without writing it back?  Its contents are
// overwritten unread in this launch (not yet touched by it), or in the next
// launch and this launch has used it for the last time.
bool droppable(const lt_ctx *c, const CState &s) {
    if (s.dead_launch == c->launch_id) return true;
    if (s.discarded) return s.last_use_launch != c->launch_id || s.last_use_group < c->cur_group;
    return s.next_dead_launch == c->launch_id &&
           (s.last_use_launch != c->launch_id || s.last_use_group < c->cur_group);
}

// Victim for eviction, in this order:
//   0. a droppable chunk (no transfer), least recently used first;
//   1. a chunk this launch does not use again and did not write, then one it
//      wrote (its output is the likely input of the next launch), least
//      recently used first within each;
//   2. a chunk this launch still needs: the one it needs last (the planner
//      knows each chunk's last group in the launch; a chunk that the launch
//      uses once is needed exactly then, so this is Belady's choice).
// Plain LRU writes back bands the launch has just written while dead bands
// hold their memory, and in a launch over more data than fits it evicts the
// inputs it has not read yet (their last use was the previous launch) only to
// fetch them again.
bool pick_victim(lt_ctx *c, lt_array **va, int64_t *vc) {
    int best_cls = 4;
    uint64_t best_key = 0;
    *va = nullptr;
    for (auto &ap : c->arrays) {
        lt_array *a = ap.get();
        for (size_t i = 0; i < a->cs.size(); ++i) {
            const CState &s = a->cs[i];
            if (s.loc != LOC_DEV || s.pin != 0) continue;
            int cls;
            uint64_t key;  // smaller is the better victim within a class
            if (droppable(c, s)) {
                cls = 0;
                key = s.lru;
            } else if (s.last_use_launch != c->launch_id || s.last_use_group < c->cur_group) {
                cls = s.last_write_launch == c->launch_id ? 2 : 1;
                key = s.lru;
            } else {
                cls = 3;
                key = UINT64_MAX - (uint64_t)s.last_use_group;
            }
            if (cls < best_cls || (cls == best_cls && key < best_key)) {
                best_cls = cls;
                best_key = key;
                *va = a;
                *vc = (int64_t)i;
            }
        }
    }
    return *va != nullptr;
}

// soft: report a full budget as LT_ERR_OOM_DEVICE without recording an error
// (a prefetch that does not fit is skipped, not failed)
lt_status dev_alloc(lt_ctx *c, size_t bytes, size_t *off, FenceSet *f, bool soft = false) {
    for (;;) {
        if (c->dev.alloc(bytes, off, f)) return LT_OK;
        lt_array *va;
        int64_t vc;
        if (!pick_victim(c, &va, &vc)) {
            if (soft) return LT_ERR_OOM_DEVICE;
            return fail(LT_ERR_OOM_DEVICE, "HBM budget too small: no evictable chunk left for a request of " +
                                               std::to_string(bytes) + " bytes");
        }
        lt_status st = evict(c, va, vc);
        if (st) return st;
    }
}

lt_status evict(lt_ctx *c, lt_array *a, int64_t ci) {
    CState &s = a->cs[(size_t)ci];
    const ChunkGeom &cg = a->g.chunks[(size_t)ci];
    if (droppable(c, s)) {
        // contents are overwritten unread in this launch, or in the next one
        // after their last use here: drop them instead of writing them back
        FenceSet f = s.busy;
        f.merge(s.ready);
        c->dev.release(s.off, cg.bytes, f);
        s.loc = LOC_NONE;
        s.ready = FenceSet();
        s.busy = FenceSet();
        c->stats.dead_skips++;
        return LT_OK;
    }
    size_t hoff;
    FenceSet hf;
    if (!c->host.alloc(cg.bytes, &hoff, &hf))
        return fail(LT_ERR_OOM_HOST, "pinned host pool too small to evict a chunk of " + std::to_string(cg.bytes) +
                                         " bytes (host pool " + std::to_string(c->host.cap) + " bytes)");
    op_begin(c, S_D2H, "evict");
    FenceSet w = s.ready;
    w.merge(hf);
    lt_status st = op_wait(c, w);
    if (st) return st;
    if (!c->dry) {
        TimeScope ts(c, CAT_D2H);
        CK(c, cudaMemcpyAsync(c->host_base + hoff, dptr(c, s.off), cg.bytes, cudaMemcpyDeviceToHost,
                              c->st[S_D2H]));
    }
    uint64_t q;
    std::ostringstream ex;
    ex << ",\"array\":" << a->id << ",\"chunk\":" << ci << ",\"bytes\":" << cg.bytes;
    st = op_end(c, &q, ex.str());
    if (st) return st;
    FenceSet rel = s.busy;
    rel.merge(s.ready);
    rel.add(S_D2H, q);
    c->dev.release(s.off, cg.bytes, rel);
    s.loc = LOC_HOST;
    s.off = hoff;
    s.ready = FenceSet::one(S_D2H, q);
    s.busy = FenceSet::one(S_D2H, q);
    c->stats.evictions++;
    c->stats.bytes_d2h += cg.bytes;
    return LT_OK;
}

// Materialise chunk ci of a in device memory.  need_data: its current
// contents must be preserved (fetched from host, or zero if never written).
lt_status ensure_dev(lt_ctx *c, lt_array *a, int64_t ci, bool need_data, bool soft = false) {
    CState &s = a->cs[(size_t)ci];
    const ChunkGeom &cg = a->g.chunks[(size_t)ci];
    s.lru = ++c->clock;
    if (s.loc == LOC_DEV) {
        s.dead_launch = -1;  // first touch in this launch done
        return LT_OK;
    }
    s.pin++;
    size_t off;
    FenceSet bf;
    lt_status st = dev_alloc(c, cg.bytes, &off, &bf, soft);
    s.pin--;
    if (st) return st;
    if (s.dead_launch == c->launch_id) need_data = false;
    s.dead_launch = -1;  // first touch in this launch done
    if (s.loc == LOC_HOST) {
        if (need_data) {
            op_begin(c, S_H2D, "fetch");
            FenceSet w = s.ready;
            w.merge(bf);
            st = op_wait(c, w);
            if (st) return st;
            if (!c->dry) {
                TimeScope ts(c, CAT_H2D);
                CK(c, cudaMemcpyAsync(dptr(c, off), c->host_base + s.off, cg.bytes, cudaMemcpyHostToDevice,
                                      c->st[S_H2D]));
            }
            uint64_t q;
            std::ostringstream ex;
            ex << ",\"array\":" << a->id << ",\"chunk\":" << ci << ",\"bytes\":" << cg.bytes;
            st = op_end(c, &q, ex.str());
            if (st) return st;
            FenceSet rel = s.busy;
            rel.merge(s.ready);
            rel.add(S_H2D, q);
            c->host.release(s.off, cg.bytes, rel);
            s.ready = FenceSet::one(S_H2D, q);
            s.busy = FenceSet::one(S_H2D, q);
            c->stats.fetches++;
            c->stats.bytes_h2d += cg.bytes;
        } else {
            FenceSet rel = s.busy;
            rel.merge(s.ready);
            c->host.release(s.off, cg.bytes, rel);
            s.ready = FenceSet();
            s.busy = bf;
            c->stats.dead_skips++;
        }
    } else {  // never materialised: contents are zero
        if (need_data) {
            op_begin(c, S_COMP, "zero");
            st = op_wait(c, bf);
            if (st) return st;
            if (!c->dry) CK(c, cudaMemsetAsync(dptr(c, off), 0, cg.bytes, c->st[S_COMP]));
            uint64_t q;
            st = op_end(c, &q);
            if (st) return st;
            s.ready = FenceSet::one(S_COMP, q);
            s.busy = FenceSet::one(S_COMP, q);
        } else {
            s.ready = FenceSet();
            s.busy = bf;
        }
    }
    s.loc = LOC_DEV;
    s.off = off;
    return LT_OK;
}

// Upload a descriptor table for the next compute-stream kernel.
// Descriptor tables that repeat (iterative launches over resident chunks
// plan the same tasks, views and copy pieces every time) stay on the device:
// a table whose bytes equal a resident slot is used in place, with no
// host-to-device copy.  Every kernel that reads a table runs on the compute
// stream, as does the copy that refills a slot, so stream order keeps a
// slot's earlier readers ahead of its new contents; the slot's event keeps
// its pinned staging bytes until that copy has run.
constexpr int TSLOTS = 32;
constexpr size_t TSLOT_BYTES = (size_t)64 << 10;
constexpr size_t NO_RING = ~(size_t)0;  // ring offset of a table served by a resident slot

lt_status upload_resident(lt_ctx *c, const void *src, size_t n, void **dev_ptr, bool *done) {
    *done = false;
    if (n == 0 || n > TSLOT_BYTES || c->tslots.empty()) return LT_OK;
    int lru = 0;
    for (int i = 0; i < (int)c->tslots.size(); ++i) {
        auto &t = c->tslots[(size_t)i];
        if (t.bytes.size() == n && std::memcmp(t.bytes.data(), src, n) == 0) {
            t.last_use = ++c->tslot_tick;
            *dev_ptr = c->up_dev + c->up_cap + (size_t)i * TSLOT_BYTES;
            *done = true;
            c->stats.tables_resident++;
            return LT_OK;
        }
        if (t.last_use < c->tslots[(size_t)lru].last_use) lru = i;
    }
    auto &t = c->tslots[(size_t)lru];
    char *h = c->up_host + c->up_cap + (size_t)lru * TSLOT_BYTES;
    char *d = c->up_dev + c->up_cap + (size_t)lru * TSLOT_BYTES;
    if (!t.bytes.empty()) CK(c, cudaEventSynchronize(t.staged));  // its last copy has read the staging bytes
    t.bytes.assign((const char *)src, (const char *)src + n);
    std::memcpy(h, src, n);
    CK(c, cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, c->st[S_COMP]));
    CK(c, cudaEventRecord(t.staged, c->st[S_COMP]));
    t.last_use = ++c->tslot_tick;
    *dev_ptr = d;
    *done = true;
    return LT_OK;
}

lt_status upload(lt_ctx *c, const void *src, size_t n, void **dev_ptr, size_t *ring_off) {
    if (c->dry) {
        *dev_ptr = nullptr;
        *ring_off = NO_RING;
        return LT_OK;
    }
    bool done = false;
    lt_status rs = upload_resident(c, src, n, dev_ptr, &done);
    if (rs) return rs;
    if (done) {
        *ring_off = NO_RING;
        return LT_OK;
    }
    size_t sz = align_up(n ? n : 1, 256);
    if (sz > c->up_cap) return fail(LT_ERR_UNSUPPORTED, "descriptor table larger than the upload ring");
    if (c->up_head + sz > c->up_cap) c->up_head = 0;
    size_t off = c->up_head;
    for (auto it = c->up_inflight.begin(); it != c->up_inflight.end();) {
        if (it->off < off + sz && it->end > off) {
            lt_status st = host_wait(c, S_COMP, it->seq);
            if (st) return st;
            it = c->up_inflight.erase(it);
        } else {
            ++it;
        }
    }
    std::memcpy(c->up_host + off, src, n);
    CK(c, cudaMemcpyAsync(c->up_dev + off, c->up_host + off, n, cudaMemcpyHostToDevice, c->st[S_COMP]));
    c->up_head = off + sz;
    *dev_ptr = c->up_dev + off;
    *ring_off = off;
    return LT_OK;
}

void upload_done(lt_ctx *c, size_t off, size_t n, uint64_t seq) {
    if (c->dry || off == NO_RING) return;
    c->up_inflight.push_back({off, off + align_up(n ? n : 1, 256), seq});
}

lt_status check_ctx(lt_ctx *c) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    if (c->poisoned) return fail(LT_ERR_BUSY, "context poisoned by an earlier CUDA error or timeout");
    return LT_OK;
}

lt_array *find_array(lt_ctx *c, const lt_array *a) {
    return c->array_set.count(a) ? const_cast<lt_array *>(a) : nullptr;
}

lt_kernel *find_kernel(lt_ctx *c, const lt_kernel *k) {
    for (auto &p : c->kernels)
        if (p.get() == k) return p.get();
    return nullptr;
}

// The CTA count shared by every task when task i owns CTAs [i*n, (i+1)*n),
// else 0.  Kernels then find their task by one division (task_of).
int32_t uniform_cta_count(const std::vector<ExecTask> &tasks) {
    if (tasks.empty()) return 0;
    const uint32_t n = tasks[0].cta_count;
    if (n == 0 || n > (uint32_t)INT32_MAX) return 0;
    for (size_t i = 0; i < tasks.size(); ++i)
        if (tasks[i].cta_count != n || (uint64_t)tasks[i].cta_begin != (uint64_t)i * n) return 0;
    return (int32_t)n;
}

lt_status sync_all(lt_ctx *c) {
    if (c->dry) return LT_OK;
    for (int s = 0; s < NSTREAM; ++s) CK(c, cudaStreamSynchronize(c->st[s]));
    uint32_t e = 0;
    CK(c, cudaMemcpy(&e, c->err_word, 4, cudaMemcpyDeviceToHost));
    if (e) {
        CK(c, cudaMemset(c->err_word, 0, 4));
        return fail(e >= 0x6700 && e < 0x6900 ? LT_ERR_TIMEOUT : LT_ERR_DEVICE_CHECK,
                    "a kernel recorded an error (code " + std::to_string(e) +
                        "; 0x67xx / 0x68xx = a bounded wait expired and the kernel returned)");
    }
    return collect_timing(c);
}

// ---------------------------------------------------------------- host transfers
// Copy between the dense row-major host buffer `hb` (whole array) and the
// part `box` of chunk ci that lives in device memory.
lt_status xfer_chunk(lt_ctx *c, lt_array *a, int64_t ci, const Box &box, char *hb, bool to_dev,
                     bool other_is_device = false) {
    const ArrayGeom &g = a->g;
    const ChunkGeom &cg = g.chunks[(size_t)ci];
    CState &s = a->cs[(size_t)ci];
    size_t es = g.esize();
    int64_t gs[3] = {1, 1, 1};
    for (int d = g.nd - 2; d >= 0; --d) gs[d] = gs[d + 1] * g.shape[d + 1];
    char *dev = dptr(c, s.off);
    auto dev_addr = [&](int64_t i0, int64_t i1, int64_t i2) {
        int64_t idx[3] = {i0, i1, i2};
        int64_t o = 0;
        for (int d = 0; d < g.nd; ++d) o += (idx[d] - cg.s_origin[d]) * cg.stride[d];
        return dev + o * (int64_t)es;
    };
    auto host_addr = [&](int64_t i0, int64_t i1, int64_t i2) {
        int64_t idx[3] = {i0, i1, i2};
        int64_t o = 0;
        for (int d = 0; d < g.nd; ++d) o += idx[d] * gs[d];
        return hb + o * (int64_t)es;
    };
    cudaStream_t st = c->st[S_COMP];
    const bool chunk_on_host = s.loc == LOC_HOST;
    char *cbase = chunk_on_host ? c->host_base + s.off : dev;
    if (other_is_device || chunk_on_host) {
        // generic copy through unified addressing: chunk (HBM pool or pinned
        // host pool) <-> a device buffer
        auto caddr = [&](int64_t i0, int64_t i1, int64_t i2) {
            int64_t idx[3] = {i0, i1, i2};
            int64_t o = 0;
            for (int d = 0; d < g.nd; ++d) o += (idx[d] - cg.s_origin[d]) * cg.stride[d];
            return cbase + o * (int64_t)es;
        };
        int nd = g.nd;
        int64_t n0 = nd == 3 ? box.extent(0) : 1;
        for (int64_t z = 0; z < n0; ++z) {
            size_t width, rows, cp, hp;
            char *cptr, *hptr;
            if (nd == 1) {
                width = (size_t)box.extent(0) * es;
                rows = 1;
                cp = hp = width;
                cptr = caddr(box.lo[0], 0, 0);
                hptr = host_addr(box.lo[0], 0, 0);
            } else if (nd == 2) {
                width = (size_t)box.extent(1) * es;
                rows = (size_t)box.extent(0);
                cp = (size_t)cg.stride[0] * es;
                hp = (size_t)gs[0] * es;
                cptr = caddr(box.lo[0], box.lo[1], 0);
                hptr = host_addr(box.lo[0], box.lo[1], 0);
            } else {
                int64_t i0 = box.lo[0] + z;
                width = (size_t)box.extent(2) * es;
                rows = (size_t)box.extent(1);
                cp = (size_t)cg.stride[1] * es;
                hp = (size_t)gs[1] * es;
                cptr = caddr(i0, box.lo[1], box.lo[2]);
                hptr = host_addr(i0, box.lo[1], box.lo[2]);
            }
            if (to_dev)
                CK(c, cudaMemcpy2DAsync(cptr, cp, hptr, hp, width, rows, cudaMemcpyDefault, st));
            else
                CK(c, cudaMemcpy2DAsync(hptr, hp, cptr, cp, width, rows, cudaMemcpyDefault, st));
        }
        CK(c, cudaStreamSynchronize(st));
        return LT_OK;
    }
    if (g.dist.order == LT_ORDER_COL) {
        // column-major chunk: transpose on the host through a staging vector
        int64_t R = box.extent(0), Cn = box.extent(1);
        std::vector<char> tmp((size_t)(R * Cn) * es);
        if (to_dev) {
            for (int64_t j = 0; j < Cn; ++j)
                for (int64_t i = 0; i < R; ++i)
                    std::memcpy(&tmp[(size_t)(j * R + i) * es], host_addr(box.lo[0] + i, box.lo[1] + j, 0), es);
            CK(c, cudaMemcpy2DAsync(dev_addr(box.lo[0], box.lo[1], 0), (size_t)cg.stride[1] * es, tmp.data(),
                                    (size_t)R * es, (size_t)R * es, (size_t)Cn, cudaMemcpyHostToDevice, st));
            CK(c, cudaStreamSynchronize(st));
        } else {
            CK(c, cudaMemcpy2DAsync(tmp.data(), (size_t)R * es, dev_addr(box.lo[0], box.lo[1], 0),
                                    (size_t)cg.stride[1] * es, (size_t)R * es, (size_t)Cn, cudaMemcpyDeviceToHost,
                                    st));
            CK(c, cudaStreamSynchronize(st));
            for (int64_t j = 0; j < Cn; ++j)
                for (int64_t i = 0; i < R; ++i)
                    std::memcpy(host_addr(box.lo[0] + i, box.lo[1] + j, 0), &tmp[(size_t)(j * R + i) * es], es);
        }
        return LT_OK;
    }
    int nd = g.nd;
    int64_t n0 = nd == 3 ? box.extent(0) : 1;
    for (int64_t z = 0; z < n0; ++z) {
        int64_t i0 = nd == 3 ? box.lo[0] + z : (nd == 2 ? box.lo[0] : box.lo[0]);
        size_t width, rows, dpitch, hpitch;
        char *dp, *hp;
        if (nd == 1) {
            width = (size_t)box.extent(0) * es;
            rows = 1;
            dpitch = hpitch = width;
            dp = dev_addr(box.lo[0], 0, 0);
            hp = host_addr(box.lo[0], 0, 0);
        } else if (nd == 2) {
            width = (size_t)box.extent(1) * es;
            rows = (size_t)box.extent(0);
            dpitch = (size_t)cg.stride[0] * es;
            hpitch = (size_t)gs[0] * es;
            dp = dev_addr(box.lo[0], box.lo[1], 0);
            hp = host_addr(box.lo[0], box.lo[1], 0);
        } else {
            width = (size_t)box.extent(2) * es;
            rows = (size_t)box.extent(1);
            dpitch = (size_t)cg.stride[1] * es;
            hpitch = (size_t)gs[1] * es;
            dp = dev_addr(i0, box.lo[1], box.lo[2]);
            hp = host_addr(i0, box.lo[1], box.lo[2]);
        }
        if (to_dev)
            CK(c, cudaMemcpy2DAsync(dp, dpitch, hp, hpitch, width, rows, cudaMemcpyHostToDevice, st));
        else
            CK(c, cudaMemcpy2DAsync(hp, hpitch, dp, dpitch, width, rows, cudaMemcpyDeviceToHost, st));
    }
    CK(c, cudaStreamSynchronize(st));
    return LT_OK;
}

// Same for a chunk resident in the pinned host pool (plain CPU copy).
void xfer_chunk_host(lt_ctx *c, lt_array *a, int64_t ci, const Box &box, char *hb, bool to_chunk) {
    const ArrayGeom &g = a->g;
    const ChunkGeom &cg = g.chunks[(size_t)ci];
    size_t es = g.esize();
    char *base = c->host_base + a->cs[(size_t)ci].off;
    int64_t gs[3] = {1, 1, 1};
    for (int d = g.nd - 2; d >= 0; --d) gs[d] = gs[d + 1] * g.shape[d + 1];
    int64_t e0 = box.extent(0), e1 = g.nd > 1 ? box.extent(1) : 1, e2 = g.nd > 2 ? box.extent(2) : 1;
    if (cg.stride[g.nd - 1] == 1) {
        // the innermost axis is contiguous in both: one memcpy per run
        const int64_t run = g.nd == 1 ? e0 : (g.nd == 2 ? e1 : e2);
        const int64_t outer0 = g.nd == 1 ? 1 : e0, outer1 = g.nd == 3 ? e1 : 1;
        for (int64_t x = 0; x < outer0; ++x)
            for (int64_t y = 0; y < outer1; ++y) {
                int64_t idx[3] = {box.lo[0], box.lo[1], box.lo[2]};
                if (g.nd >= 2) idx[0] += x;
                if (g.nd == 3) idx[1] += y;
                int64_t co = 0, ho = 0;
                for (int d = 0; d < g.nd; ++d) {
                    co += (idx[d] - cg.s_origin[d]) * cg.stride[d];
                    ho += idx[d] * gs[d];
                }
                if (to_chunk)
                    std::memcpy(base + co * (int64_t)es, hb + ho * (int64_t)es, (size_t)run * es);
                else
                    std::memcpy(hb + ho * (int64_t)es, base + co * (int64_t)es, (size_t)run * es);
            }
        return;
    }
    for (int64_t x = 0; x < e0; ++x)
        for (int64_t y = 0; y < e1; ++y)
            for (int64_t z = 0; z < e2; ++z) {
                int64_t idx[3] = {box.lo[0] + x, box.lo[1] + y, box.lo[2] + z};
                int64_t co = 0, ho = 0;
                for (int d = 0; d < g.nd; ++d) {
                    co += (idx[d] - cg.s_origin[d]) * cg.stride[d];
                    ho += idx[d] * gs[d];
                }
                if (to_chunk)
                    std::memcpy(base + co * (int64_t)es, hb + ho * (int64_t)es, es);
                else
                    std::memcpy(hb + ho * (int64_t)es, base + co * (int64_t)es, es);
            }
}

// ---------------------------------------------------------------- launches
struct ArgUse {
    lt_array *a;
    int64_t chunk;
    bool write;
};

struct TempAlloc {
    size_t off, bytes;
    ChunkGeom geom;
};

// Chunks whose contents a launch fully overwrites without reading them.
std::vector<std::pair<lt_array *, int64_t>> dead_chunks(const LaunchPlan &plan, const std::vector<lt_array *> &parr) {
    std::vector<std::pair<lt_array *, int64_t>> out;
    std::vector<lt_array *> uniq;
    for (lt_array *a : parr)
        if (a && std::find(uniq.begin(), uniq.end(), a) == uniq.end()) uniq.push_back(a);
    for (lt_array *a : uniq) {
        std::vector<Box> wr, rd;
        for (const auto &sb : plan.sbs)
            for (const auto &ap : sb.args) {
                if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE || parr[(size_t)ap.param] != a) continue;
                if (ap.mode == MODE_WRITE || ap.mode == MODE_REDUCE)
                    wr.push_back(ap.region);
                else
                    rd.push_back(ap.region);
            }
        if (wr.empty()) continue;
        for (size_t ci = 0; ci < a->g.chunks.size(); ++ci) {
            const Box &cb = a->g.chunks[ci].box;
            bool read = false;
            for (const Box &r : rd)
                if (!cb.intersect(r).empty()) {
                    read = true;
                    break;
                }
            if (read) continue;
            std::vector<Box> parts;
            for (const Box &w : wr)
                if (!cb.intersect(w).empty()) parts.push_back(w);
            if (!parts.empty() && box_covered(cb, parts)) out.push_back({a, (int64_t)ci});
        }
    }
    return out;
}

// The same, as (parameter, chunk): parameter = the first one naming the array.
std::vector<std::pair<int, int64_t>> dead_by_param(const LaunchPlan &plan, const std::vector<lt_array *> &parr) {
    std::vector<std::pair<int, int64_t>> out;
    for (auto &d : dead_chunks(plan, parr)) {
        int p = 0;
        while (parr[(size_t)p] != d.first) ++p;
        out.push_back({p, d.second});
    }
    return out;
}

// Mark the chunks this launch overwrites unread (no fetch on first touch).
void mark_dead(lt_ctx *c, const PlanBundle &b, const std::vector<lt_array *> &parr) {
    for (auto &d : b.dead) parr[(size_t)d.first]->cs[(size_t)d.second].dead_launch = c->launch_id;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

static lt_status flush_pending(lt_ctx *c);
static bool pending_writes(lt_ctx *c, const lt_array *a);

lt_status lt_ctx_create(const lt_config *cfg, lt_ctx **out) {
    if (!cfg || !out) return fail(LT_ERR_INVALID_ARG, "null argument");
    auto c = std::make_unique<lt_ctx>();
    c->cfg = *cfg;
    c->dry = (cfg->flags & LT_FLAG_DRYRUN) != 0;
    c->no_staged = (cfg->flags & LT_FLAG_NO_STAGED) != 0;
    for (int s = 0; s < NSTREAM; ++s) {
        c->ev[s].assign(RING, nullptr);
        c->evseq[s].assign(RING, 0);
        c->evtask[s].assign(RING, -1);
    }
    size_t budget = cfg->hbm_budget_bytes;
    if (c->dry) {
        if (!budget) budget = (size_t)1 << 34;
        c->dev.init(budget, nullptr);
        c->host.init(cfg->host_pool_bytes, nullptr);
        c->host.oldest_first = true;
        *out = c.release();
        return LT_OK;
    }
    lt_ctx *cp = c.get();
    CK(cp, cudaSetDevice(cfg->device));
    int major = 0, minor = 0;
    CK(cp, cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, cfg->device));
    CK(cp, cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, cfg->device));
    if (major * 10 + minor != 103)
        return fail(LT_ERR_UNSUPPORTED, "this library is built for sm_103a (GB300) only; device is sm_" +
                                            std::to_string(major) + std::to_string(minor));
    for (int s = 0; s < NSTREAM; ++s) {
        CK(cp, cudaStreamCreateWithFlags(&c->st[s], cudaStreamNonBlocking));
        for (int i = 0; i < RING; ++i) CK(cp, cudaEventCreateWithFlags(&c->ev[s][i], cudaEventDisableTiming));
    }
    size_t fr = 0, tot = 0;
    CK(cp, cudaMemGetInfo(&fr, &tot));
    if (!budget) budget = fr / 10 * 9;
    budget = budget / ALIGN * ALIGN;
    if (budget > fr) return fail(LT_ERR_OOM_DEVICE, "HBM budget exceeds free device memory");
    if (cudaMalloc((void **)&c->dev_base, budget) != cudaSuccess) {
        cudaGetLastError();
        return fail(LT_ERR_OOM_DEVICE, "cudaMalloc of the HBM pool failed");
    }
    c->dev.init(budget, c->dev_base);
    if (cfg->host_pool_bytes) {
        if (cudaHostAlloc((void **)&c->host_base, cfg->host_pool_bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->dev_base);
            return fail(LT_ERR_OOM_HOST, "cudaHostAlloc of the pinned host pool failed");
        }
    }
    c->host.init(cfg->host_pool_bytes, c->host_base);
    c->host.oldest_first = true;
    c->up_cap = (size_t)32 << 20;
    CK(cp, cudaHostAlloc((void **)&c->up_host, c->up_cap + TSLOTS * TSLOT_BYTES, cudaHostAllocDefault));
    CK(cp, cudaMalloc((void **)&c->up_dev, c->up_cap + TSLOTS * TSLOT_BYTES));
    c->tslots.resize(TSLOTS);
    for (auto &t : c->tslots) CK(cp, cudaEventCreateWithFlags(&t.staged, cudaEventDisableTiming));
    CK(cp, cudaMalloc((void **)&c->err_word, 16));
    CK(cp, cudaMemset(c->err_word, 0, 16));
    *out = c.release();
    return LT_OK;
}

lt_status lt_ctx_destroy(lt_ctx *c) {
    if (!c) return LT_OK;
    if (!c->poisoned) flush_pending(c);
    if (!c->dry) {
        for (int s = 0; s < NSTREAM; ++s)
            if (c->st[s]) cudaStreamSynchronize(c->st[s]);
        for (auto &t : c->timed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto e : c->tev_pool) cudaEventDestroy(e);
        for (int i = 0; i < 2; ++i) {
            if (c->timer[i]) cudaEventDestroy(c->timer[i]);
            if (c->timer_join[i]) cudaEventDestroy(c->timer_join[i]);
        }
        for (int s = 0; s < NSTREAM; ++s) {
            for (auto e : c->ev[s])
                if (e) cudaEventDestroy(e);
            if (c->st[s]) cudaStreamDestroy(c->st[s]);
        }
        if (c->batch && c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
        if (c->dev_base) cudaFree(c->dev_base);
        if (c->host_base) cudaFreeHost(c->host_base);
        for (auto &t : c->tslots)
            if (t.staged) cudaEventDestroy(t.staged);
        if (c->up_host) cudaFreeHost(c->up_host);
        if (c->up_dev) cudaFree(c->up_dev);
        if (c->err_word) cudaFree(c->err_word);
    }
    delete c;
    return LT_OK;
}

lt_status lt_array_create(lt_ctx *c, lt_dtype dtype, int32_t ndim, const int64_t shape[3], const lt_dist *dist,
                          lt_array **out) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if (!shape || !dist || !out) return fail(LT_ERR_INVALID_ARG, "null argument");
    auto a = std::make_unique<lt_array>();
    std::string err;
    if (!make_geometry((int)dtype, ndim, shape, *dist, &a->g, &err)) return fail(LT_ERR_INVALID_ARG, err);
    for (const auto &cg : a->g.chunks)
        if (cg.bytes > c->dev.cap)
            return fail(LT_ERR_OOM_DEVICE, "a chunk (" + std::to_string(cg.bytes) + " bytes) exceeds the HBM budget");
    a->cs.resize(a->g.chunks.size());
    a->id = c->next_array_id++;
    *out = a.get();
    c->array_set.insert(a.get());
    c->arrays.push_back(std::move(a));
    return LT_OK;
}

lt_status lt_array_wrap_device(lt_ctx *c, lt_dtype dtype, int32_t ndim, const int64_t shape[3],
                               const int64_t strides[3], void *ptr, lt_array **out) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if (!shape || !strides || !out || (!ptr && !c->dry)) return fail(LT_ERR_INVALID_ARG, "null argument");
    if (ndim < 1 || ndim > 3) return fail(LT_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
    if (strides[ndim - 1] != 1) return fail(LT_ERR_INVALID_ARG, "the innermost stride must be 1");
    lt_dist whole{};
    whole.kind = LT_DIST_BLOCK;
    auto a = std::make_unique<lt_array>();
    std::string err;
    if (!make_geometry((int)dtype, ndim, shape, whole, &a->g, &err)) return fail(LT_ERR_INVALID_ARG, err);
    ChunkGeom &cg = a->g.chunks[0];
    int64_t span = 1;  // elements from the first to one past the last
    for (int d = 0; d < ndim; ++d) {
        if (strides[d] < 1) return fail(LT_ERR_INVALID_ARG, "strides must be positive");
        cg.s_origin[d] = 0;
        cg.stride[d] = strides[d];
        span += (shape[d] - 1) * strides[d];
    }
    cg.bytes = (size_t)span * a->g.esize();
    a->cs.resize(1);
    CState &cs = a->cs[0];
    cs.loc = LOC_DEV;
    cs.ext = true;
    cs.pin = 1;  // never a victim
    cs.off = (size_t)((uint64_t)(uintptr_t)ptr - (uint64_t)(uintptr_t)c->dev_base);
    a->id = c->next_array_id++;
    *out = a.get();
    c->array_set.insert(a.get());
    c->arrays.push_back(std::move(a));
    return LT_OK;
}

lt_status lt_array_destroy(lt_ctx *c, lt_array *arr) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    lt_array *a = find_array(c, arr);
    if (!a) return fail(LT_ERR_INVALID_ARG, "unknown array");
    for (size_t i = 0; i < a->cs.size(); ++i) {
        CState &s = a->cs[i];
        FenceSet f = s.busy;
        f.merge(s.ready);
        if (s.ext) {  // the caller's memory: return once no queued work uses it
            for (int t = 0; t < NSTREAM; ++t)
                if ((st = host_wait(c, t, f.q[t]))) return st;
            s.loc = LOC_NONE;
            continue;
        }
        if (s.loc == LOC_DEV) c->dev.release(s.off, a->g.chunks[i].bytes, f);
        if (s.loc == LOC_HOST) c->host.release(s.off, a->g.chunks[i].bytes, f);
        s.loc = LOC_NONE;
    }
    c->array_set.erase(a);
    for (auto it = c->arrays.begin(); it != c->arrays.end(); ++it)
        if (it->get() == a) {
            c->arrays.erase(it);
            break;
        }
    return LT_OK;
}

static size_t array_bytes(const lt_array *a) {
    size_t n = a->g.esize();
    for (int d = 0; d < a->g.nd; ++d) n *= (size_t)a->g.shape[d];
    return n;
}

lt_status lt_array_write(lt_ctx *c, lt_array *arr, const void *host, size_t bytes) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    lt_array *a = find_array(c, arr);
    if (!a || (!host && !c->dry)) return fail(LT_ERR_INVALID_ARG, "unknown array or null buffer");
    if (bytes != array_bytes(a)) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the array");
    if ((st = sync_all(c))) return st;
    ++c->launch_id;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
            a->cs[ci].dead_launch = c->launch_id;
            a->cs[ci].discarded = false;
        }
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        CState &s = a->cs[ci];
        if (s.loc == LOC_HOST && !c->dry) {
            // rewrite in place in the host pool once earlier copies are done
            if ((st = sync_all(c))) return st;
            xfer_chunk_host(c, a, (int64_t)ci, a->g.chunks[ci].box, (char *)host, true);
            s.dead_launch = -1;
            continue;
        }
        s.pin++;
        st = ensure_dev(c, a, (int64_t)ci, false);
        s.pin--;
        if (st) return st;
        op_begin(c, S_COMP, "write");
        FenceSet w = s.ready;
        w.merge(s.busy);
        if ((st = op_wait(c, w))) return st;
        if (!c->dry) {
            for (int s2 = 0; s2 < NSTREAM; ++s2) CK(c, cudaStreamSynchronize(c->st[s2]));
            if ((st = xfer_chunk(c, a, (int64_t)ci, a->g.chunks[ci].box, (char *)host, true))) return st;
        }
        uint64_t q;
        if ((st = op_end(c, &q))) return st;
        s.ready = FenceSet::one(S_COMP, q);
        s.busy = FenceSet::one(S_COMP, q);
        c->stats.bytes_h2d += a->g.chunks[ci].box.volume() * a->g.esize();
    }
    return sync_all(c);
}

lt_status lt_array_read(lt_ctx *c, lt_array *arr, void *host, size_t bytes) {
    lt_status st = check_ctx(c);
    if (st) return st;
    // a read needs the pending launch enqueued only if that launch writes the array
    if (pending_writes(c, arr) && (st = flush_pending(c))) return st;
    lt_array *a = find_array(c, arr);
    if (!a || (!host && !c->dry)) return fail(LT_ERR_INVALID_ARG, "unknown array or null buffer");
    if (bytes != array_bytes(a)) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the array");
    if ((st = sync_all(c))) return st;
    if (c->dry) return LT_OK;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        const CState &s = a->cs[ci];
        const Box &ob = a->g.chunks[ci].owned;
        if (s.loc == LOC_DEV) {
            if ((st = xfer_chunk(c, a, (int64_t)ci, ob, (char *)host, false))) return st;
        } else if (s.loc == LOC_HOST) {
            xfer_chunk_host(c, a, (int64_t)ci, ob, (char *)host, false);
        } else {
            // never written: zero
            std::vector<char> z(a->g.esize(), 0);
            int64_t gs[3] = {1, 1, 1};
            for (int d = a->g.nd - 2; d >= 0; --d) gs[d] = gs[d + 1] * a->g.shape[d + 1];
            int64_t e0 = ob.extent(0), e1 = a->g.nd > 1 ? ob.extent(1) : 1, e2 = a->g.nd > 2 ? ob.extent(2) : 1;
            for (int64_t x = 0; x < e0; ++x)
                for (int64_t y = 0; y < e1; ++y) {
                    int64_t idx[3] = {ob.lo[0] + x, ob.lo[1] + y, ob.lo[2]};
                    int64_t ho = 0;
                    for (int d = 0; d < a->g.nd; ++d) ho += idx[d] * gs[d];
                    std::memset((char *)host + ho * (int64_t)a->g.esize(), 0, (size_t)e2 * a->g.esize());
                }
        }
    }
    return LT_OK;
}

static lt_status array_copy_device(lt_ctx *c, lt_array *arr, void *dev, size_t bytes, bool to_array) {
    lt_status st = check_ctx(c);
    if (st) return st;
    lt_array *a = find_array(c, arr);
    if (!a || !dev) return fail(LT_ERR_INVALID_ARG, "unknown array or null buffer");
    if (bytes != array_bytes(a)) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the array");
    if (a->g.dist.order == LT_ORDER_COL) return fail(LT_ERR_UNSUPPORTED, "device copies need row-major chunks");
    if (c->dry) return fail(LT_ERR_UNSUPPORTED, "device copies need a device");
    if ((st = flush_pending(c))) return st;
    if ((st = sync_all(c))) return st;
    if (to_array) {
        ++c->launch_id;
        for (size_t ci = 0; ci < a->cs.size(); ++ci) {
            a->cs[ci].dead_launch = c->launch_id;
            a->cs[ci].discarded = false;
        }
    }
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        CState &s = a->cs[ci];
        const ChunkGeom &cg = a->g.chunks[ci];
        if (!to_array && s.loc == LOC_NONE) {
            // never written: zero the owned part of the destination
            int64_t gs0 = a->g.nd > 1 ? a->g.shape[a->g.nd - 1] : 1;
            (void)gs0;
            if ((st = ensure_dev(c, a, (int64_t)ci, true))) return st;
            if ((st = sync_all(c))) return st;
        }
        if (to_array && s.loc != LOC_HOST) {
            s.pin++;
            st = ensure_dev(c, a, (int64_t)ci, false);
            s.pin--;
            if (st) return st;
            if ((st = sync_all(c))) return st;
        }
        s.dead_launch = -1;
        if ((st = xfer_chunk(c, a, (int64_t)ci, to_array ? cg.box : cg.owned, (char *)dev, to_array, true))) return st;
        if (to_array) {
            s.ready = FenceSet();
            s.busy = FenceSet();
        }
    }
    return LT_OK;
}

lt_status lt_array_write_device(lt_ctx *c, lt_array *arr, const void *dev, size_t bytes) {
    return array_copy_device(c, arr, const_cast<void *>(dev), bytes, true);
}

lt_status lt_array_read_device(lt_ctx *c, lt_array *arr, void *dev, size_t bytes) {
    return array_copy_device(c, arr, dev, bytes, false);
}

lt_status lt_array_read_box(lt_ctx *c, lt_array *arr, const int64_t lo[3], const int64_t hi[3], void *host,
                            size_t bytes) {
    lt_status st = check_ctx(c);
    if (st) return st;
    // a read needs the pending launch enqueued only if that launch writes the array
    if (pending_writes(c, arr) && (st = flush_pending(c))) return st;
    lt_array *a = find_array(c, arr);
    if (!a || !lo || !hi || (!host && !c->dry)) return fail(LT_ERR_INVALID_ARG, "bad argument");
    Box want;
    want.nd = a->g.nd;
    for (int d = 0; d < a->g.nd; ++d) {
        want.lo[d] = lo[d];
        want.hi[d] = hi[d];
        if (lo[d] < 0 || hi[d] >= a->g.shape[d] || lo[d] > hi[d]) return fail(LT_ERR_INVALID_ARG, "box outside the array");
    }
    if (bytes != (size_t)want.volume() * a->g.esize()) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the box");
    if ((st = sync_all(c))) return st;
    if (c->dry) return LT_OK;
    // stage through a dense buffer shaped like the whole array's index space
    // restricted to the box: address(idx) = host + row-major offset in the box
    size_t es = a->g.esize();
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        Box ob = a->g.chunks[ci].owned.intersect(want);
        if (ob.empty()) continue;
        const CState &s = a->cs[ci];
        const ChunkGeom &cg = a->g.chunks[ci];
        int64_t bs[3] = {1, 1, 1};
        for (int d = a->g.nd - 2; d >= 0; --d) bs[d] = bs[d + 1] * want.extent(d + 1);
        int64_t e0 = ob.extent(0), e1 = a->g.nd > 1 ? ob.extent(1) : 1;
        int inner = a->g.nd - 1;
        int64_t w = ob.extent(inner);
        for (int64_t x = 0; x < (a->g.nd == 3 ? e0 : 1); ++x)
            for (int64_t y = 0; y < (a->g.nd >= 2 ? (a->g.nd == 3 ? e1 : e0) : 1); ++y) {
                int64_t idx[3] = {0, 0, 0};
                if (a->g.nd == 3) {
                    idx[0] = ob.lo[0] + x;
                    idx[1] = ob.lo[1] + y;
                } else if (a->g.nd == 2) {
                    idx[0] = ob.lo[0] + y;
                }
                idx[inner] = ob.lo[inner];
                int64_t ho = 0, co = 0;
                for (int d = 0; d < a->g.nd; ++d) {
                    ho += (idx[d] - want.lo[d]) * bs[d];
                    co += (idx[d] - cg.s_origin[d]) * cg.stride[d];
                }
                char *dst = (char *)host + ho * (int64_t)es;
                int64_t cstride = cg.stride[inner];
                if (s.loc == LOC_DEV) {
                    const char *src = dptr(c, s.off + co * (int64_t)es);
                    if (cstride == 1)
                        CK(c, cudaMemcpyAsync(dst, src, (size_t)w * es, cudaMemcpyDeviceToHost, c->st[S_COMP]));
                    else
                        CK(c, cudaMemcpy2DAsync(dst, es, src, (size_t)cstride * es, es, (size_t)w,
                                                cudaMemcpyDeviceToHost, c->st[S_COMP]));
                } else if (s.loc == LOC_HOST) {
                    const char *src = c->host_base + s.off + co * (int64_t)es;
                    for (int64_t k = 0; k < w; ++k) std::memcpy(dst + k * (int64_t)es, src + k * cstride * (int64_t)es, es);
                } else {
                    std::memset(dst, 0, (size_t)w * es);
                }
            }
    }
    CK(c, cudaStreamSynchronize(c->st[S_COMP]));
    return LT_OK;
}

lt_status lt_array_fill(lt_ctx *c, lt_array *arr, const lt_init *init) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    lt_array *a = find_array(c, arr);
    if (!a || !init) return fail(LT_ERR_INVALID_ARG, "unknown array or null init");
    int kind = init->kind;
    int dt = a->g.dtype;
    bool ok = kind == LT_INIT_ZERO || kind == LT_INIT_CONST || (kind == LT_INIT_UNIFORM && dt == LT_F32) ||
              (kind == LT_INIT_KAPPA && dt == LT_F32) || (kind == LT_INIT_NORMAL_BF16 && dt == LT_BF16) ||
              (kind == LT_INIT_U8 && dt == LT_U8);
    if (!ok) return fail(LT_ERR_INVALID_ARG, "fill kind does not match the array dtype");
    ++c->launch_id;
    c->stats.launches++;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
            a->cs[ci].dead_launch = c->launch_id;
            a->cs[ci].discarded = false;
        }
    uint64_t key;
    {
        uint64_t s0 = init->seed ^ (init->stream << 32);
        s0 += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s0;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        key = z ^ (z >> 31);
    }
    bool rev = !(c->cfg.flags & LT_FLAG_FIXED_SWEEP) && (c->launch_id & 1);
    size_t n = a->cs.size();
    for (size_t kk = 0; kk < n; ++kk) {
        size_t ci = rev ? n - 1 - kk : kk;
        CState &s = a->cs[ci];
        const ChunkGeom &cg = a->g.chunks[ci];
        s.pin++;
        st = ensure_dev(c, a, (int64_t)ci, false);
        s.pin--;
        if (st) return st;
        op_begin(c, S_COMP, "fill");
        FenceSet w = s.ready;
        w.merge(s.busy);
        if ((st = op_wait(c, w))) return st;
        if (!c->dry) {
            FillDesc d{};
            d.dst = view_of(c, a->g, cg, s.off);
            d.nd = a->g.nd;
            for (int dd = 0; dd < 3; ++dd) {
                d.lo[dd] = dd < a->g.nd ? cg.box.lo[dd] : 0;
                d.hi[dd] = dd < a->g.nd ? cg.box.hi[dd] : 0;
            }
            int64_t gs = 1;
            for (int dd = a->g.nd - 1; dd >= 0; --dd) {
                d.gstride[dd] = gs;
                gs *= a->g.shape[dd];
            }
            d.kind = kind;
            d.dtype = dt;
            d.key = key;
            d.value = init->value;
            d.scale = init->scale;
            TimeScope ts(c, CAT_FILL);
            CK(c, k::fill(d, c->st[S_COMP]));
            c->stats.kernels++;
        }
        uint64_t q;
        std::ostringstream ex;
        ex << ",\"array\":" << a->id << ",\"chunk\":" << ci;
        if ((st = op_end(c, &q, ex.str()))) return st;
        s.ready = FenceSet::one(S_COMP, q);
        s.busy = FenceSet::one(S_COMP, q);
    }
    return LT_OK;
}

lt_status lt_array_num_chunks(lt_ctx *c, const lt_array *arr, int64_t *n) {
    if (!c || !n) return fail(LT_ERR_INVALID_ARG, "null argument");
    lt_array *a = find_array(c, arr);
    if (!a) return fail(LT_ERR_INVALID_ARG, "unknown array");
    *n = (int64_t)a->cs.size();
    return LT_OK;
}

lt_status lt_array_chunk_info(lt_ctx *c, const lt_array *arr, int64_t index, int64_t lo[3], int64_t hi[3],
                              int32_t *location) {
    if (!c || !lo || !hi || !location) return fail(LT_ERR_INVALID_ARG, "null argument");
    lt_array *a = find_array(c, arr);
    if (!a || index < 0 || index >= (int64_t)a->cs.size()) return fail(LT_ERR_INVALID_ARG, "bad array or index");
    const ChunkGeom &cg = a->g.chunks[(size_t)index];
    for (int d = 0; d < 3; ++d) {
        lo[d] = d < a->g.nd ? cg.box.lo[d] : 0;
        hi[d] = d < a->g.nd ? cg.box.hi[d] : 0;
    }
    *location = a->cs[(size_t)index].loc;
    return LT_OK;
}

lt_status lt_kernel_register(lt_ctx *c, int32_t builtin, const char *annotation, const lt_param *params,
                             int32_t nparams, lt_kernel **out) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if (!annotation || (!params && nparams) || !out || nparams < 0 || nparams > 16)
        return fail(LT_ERR_INVALID_ARG, "bad kernel registration arguments");
    const BuiltinDef *def = find_builtin(builtin);
    if (!def) return fail(LT_ERR_UNSUPPORTED, "unknown built-in kernel id " + std::to_string(builtin));
    auto k = std::make_unique<lt_kernel>();
    k->def = def;
    std::string err;
    if (!parse_annotation(annotation, &k->ann, &err)) return fail(LT_ERR_PARSE, "annotation: " + err);
    bool plan_only = def->canon == nullptr;
    if (!plan_only && !parse_annotation(canon_text(def, 1), &k->canon, &err))
        return fail(LT_ERR_PARSE, "internal canonical: " + err);
    int slot = 0;
    for (int p = 0; p < nparams; ++p) {
        if (!params[p].name) return fail(LT_ERR_INVALID_ARG, "parameter without a name");
        k->params.push_back(params[p]);
        k->names.push_back(params[p].name);
        if (!params[p].is_array) {
            k->stmt_of_param.push_back(-1);
            k->slot_of_param.push_back(-1);
            continue;
        }
        int si = -1;
        for (size_t s = 0; s < k->ann.stmts.size(); ++s)
            if (k->ann.stmts[s].array == params[p].name) si = (int)s;
        if (si < 0) return fail(LT_ERR_INVALID_ARG, std::string("array parameter '") + params[p].name +
                                                       "' is not named in the annotation");
        if (!plan_only) {
            if (slot >= def->narr) return fail(LT_ERR_INVALID_ARG, "too many array parameters for this built-in");
            if (params[p].dtype != def->dtype[slot])
                return fail(LT_ERR_INVALID_ARG,
                            std::string("dtype of '") + params[p].name + "' does not match the built-in");
            if ((int)k->ann.stmts[(size_t)si].idx.size() != def->nd[slot])
                return fail(LT_ERR_INVALID_ARG, std::string("'") + params[p].name + "' is indexed with the wrong rank");
        } else if (slot >= LT_MAX_ARRAYS) {
            return fail(LT_ERR_INVALID_ARG, "too many array parameters");
        }
        k->stmt_of_param.push_back(si);
        k->slot_of_param.push_back(slot);
        slot++;
    }
    if (!plan_only && slot != def->narr)
        return fail(LT_ERR_INVALID_ARG, "the built-in needs " + std::to_string(def->narr) + " array parameters");
    for (const auto &s : k->ann.stmts) {
        bool found = false;
        for (const auto &nm : k->names)
            if (nm == s.array) found = true;
        if (!found) return fail(LT_ERR_INVALID_ARG, "annotation names unknown array '" + s.array + "'");
    }
    // canonical statement of each slot, and mode compatibility
    k->canon_stmt.assign((size_t)std::max(def->narr, slot), -1);
    for (size_t p = 0; p < k->params.size() && !plan_only; ++p) {
        int sl = k->slot_of_param[p];
        if (sl < 0) continue;
        std::string nm = "A" + std::to_string(sl);
        for (size_t s = 0; s < k->canon.stmts.size(); ++s)
            if (k->canon.stmts[s].array == nm) k->canon_stmt[(size_t)sl] = (int)s;
        const Stmt &cs = k->canon.stmts[(size_t)k->canon_stmt[(size_t)sl]];
        const Stmt &us = k->ann.stmts[(size_t)k->stmt_of_param[p]];
        bool ok;
        switch (cs.mode) {
            case MODE_READ: ok = us.mode == MODE_READ || us.mode == MODE_READWRITE; break;
            case MODE_WRITE: ok = us.mode == MODE_WRITE || us.mode == MODE_READWRITE; break;
            case MODE_READWRITE: ok = us.mode == MODE_READWRITE; break;
            default: ok = us.mode == MODE_REDUCE && (us.op == cs.op || def->any_reduce_op);
        }
        if (!ok)
            return fail(LT_ERR_INVALID_ARG, "access mode of '" + us.array + "' does not allow what the kernel does");
    }
    *out = k.get();
    c->kernels.push_back(std::move(k));
    return LT_OK;
}

lt_status lt_kernel_register_source(lt_ctx *c, const char *source, const char *name, const char *annotation,
                                    const lt_param *params, int32_t nparams, lt_kernel **out) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if (!source || !name || !annotation || (!params && nparams) || !out || nparams < 0 || nparams > 13)
        return fail(LT_ERR_INVALID_ARG, "bad source-kernel registration arguments");
    for (const char *q = name; *q; ++q)
        if (!(std::isalnum((unsigned char)*q) || *q == '_')) return fail(LT_ERR_INVALID_ARG, "bad kernel name");
    auto k = std::make_unique<lt_kernel>();
    std::string err;
    if (!parse_annotation(annotation, &k->ann, &err)) return fail(LT_ERR_PARSE, "annotation: " + err);
    auto def = std::make_unique<BuiltinDef>();
    def->id = LT_K_USER;
    def->canon = nullptr;
    def->narr = 0;
    def->prepare = k::prepare_user;
    def->launch = nullptr;
    def->reduce_zero = true;
    std::vector<UserParam> ups;
    int nf = 0, ni = 0;
    for (int p = 0; p < nparams; ++p) {
        if (!params[p].name) return fail(LT_ERR_INVALID_ARG, "parameter without a name");
        k->params.push_back(params[p]);
        k->names.push_back(params[p].name);
        UserParam up;
        up.is_array = params[p].is_array != 0;
        up.dtype = params[p].dtype;
        if (!up.is_array) {
            if (params[p].dtype == LT_F32 ? ++nf > 4 : ++ni > 4)
                return fail(LT_ERR_INVALID_ARG, "at most 4 integer and 4 float value parameters");
            k->stmt_of_param.push_back(-1);
            k->slot_of_param.push_back(-1);
            ups.push_back(up);
            continue;
        }
        int si = -1;
        for (size_t s2 = 0; s2 < k->ann.stmts.size(); ++s2)
            if (k->ann.stmts[s2].array == params[p].name) si = (int)s2;
        if (si < 0)
            return fail(LT_ERR_INVALID_ARG, std::string("array parameter '") + params[p].name +
                                                "' is not named in the annotation");
        if (def->narr >= LT_MAX_ARRAYS) return fail(LT_ERR_INVALID_ARG, "at most 5 array parameters");
        if (dtype_size(params[p].dtype) == 0) return fail(LT_ERR_INVALID_ARG, "unknown dtype");
        up.rank = (int)k->ann.stmts[(size_t)si].idx.size();
        def->dtype[def->narr] = params[p].dtype;
        def->nd[def->narr] = up.rank;
        k->stmt_of_param.push_back(si);
        k->slot_of_param.push_back(def->narr);
        def->narr++;
        ups.push_back(up);
    }
    for (const auto &s2 : k->ann.stmts) {
        bool found = false;
        for (const auto &nm : k->names)
            if (nm == s2.array) found = true;
        if (!found) return fail(LT_ERR_INVALID_ARG, "annotation names unknown array '" + s2.array + "'");
    }
    std::string src = user_wrapper_source(source, name, ups);
    std::vector<char> cubin;
    std::string log;
    st = compile_user_kernel(src, &cubin, &log);
    if (st) return fail(st, "runtime compilation failed:\n" + log);
    if (!c->dry) {
        CK(c, cudaLibraryLoadData(&k->ulib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
        CK(c, cudaLibraryGetKernel(&k->ufn, k->ulib, "lt_user_wrapper"));
    }
    k->def = def.get();
    k->own_def = std::move(def);
    *out = k.get();
    c->kernels.push_back(std::move(k));
    return LT_OK;
}

lt_status lt_kernel_destroy(lt_ctx *c, lt_kernel *kk) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    if (c->pending && c->pending->k == kk && !c->poisoned) {
        lt_status st = flush_pending(c);
        if (st) return st;
    }
    for (auto it = c->kernels.begin(); it != c->kernels.end(); ++it)
        if (it->get() == kk) {
            if (kk->ulib && !c->dry) {
                for (int s2 = 0; s2 < NSTREAM; ++s2) cudaStreamSynchronize(c->st[s2]);
                cudaLibraryUnload(kk->ulib);
            }
            c->kernels.erase(it);
            c->batch_checked.clear();  // a new kernel may reuse the address
            return LT_OK;
        }
    return fail(LT_ERR_INVALID_ARG, "unknown kernel");
}

constexpr size_t PLAN_CACHE = 4096;

static lt_status prepare_plan(lt_ctx *c, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
                              const lt_arg *args, int32_t nargs, std::shared_ptr<const PlanBundle> *out,
                              std::vector<lt_array *> *parr) {
    if (!k || !find_kernel(c, k)) return fail(LT_ERR_INVALID_ARG, "unknown kernel");
    if (nargs != (int32_t)k->params.size() || (nargs && !args))
        return fail(LT_ERR_INVALID_ARG, "argument count does not match the kernel's parameters");
    std::vector<PlanArray> pa((size_t)nargs);
    parr->assign((size_t)nargs, nullptr);
    for (int p = 0; p < nargs; ++p) {
        if (!k->params[(size_t)p].is_array) continue;
        lt_array *a = find_array(c, args[p].array);
        if (!a) return fail(LT_ERR_INVALID_ARG, "argument " + std::to_string(p) + " is not an array of this context");
        if (a->g.dtype != k->params[(size_t)p].dtype)
            return fail(LT_ERR_INVALID_ARG, "argument " + std::to_string(p) + " has the wrong dtype");
        if (a->g.nd != (int)k->ann.stmts[(size_t)k->stmt_of_param[(size_t)p]].idx.size())
            return fail(LT_ERR_INVALID_ARG, "argument " + std::to_string(p) + " has the wrong rank");
        pa[(size_t)p].geom = &a->g;
        (*parr)[(size_t)p] = a;
    }
    if (k->def->id == LT_K_GEMM_BF16) {
        // the tensor-core operands must be K-contiguous: A row-major, B column-major chunks
        lt_array *A = nullptr, *B = nullptr;
        for (int p = 0; p < nargs; ++p) {
            if (k->slot_of_param[(size_t)p] == 0) A = (*parr)[(size_t)p];
            if (k->slot_of_param[(size_t)p] == 1) B = (*parr)[(size_t)p];
        }
        if (!A || !B || A->g.dist.order != LT_ORDER_ROW || B->g.dist.order != LT_ORDER_COL)
            return fail(LT_ERR_UNSUPPORTED, "the BF16 GEMM needs A with row-major chunks and B with column-major "
                                            "chunks (LT_ORDER_COL)");
    }
    uint64_t g3[3] = {grid.x, grid.y, grid.z}, b3[3] = {block.x, block.y, block.z};
    int64_t sb3[3] = {0, 0, 0};
    if (wd)
        for (int d = 0; d < 3; ++d) sb3[d] = wd->superblock[d];
    const bool has_k = k->def->canon && std::strstr(k->def->canon, "{K}") != nullptr;
    int64_t kval = 0;
    if (has_k) {
        bool found = false;
        for (int p = 0; p < nargs && !found; ++p)
            if (!k->params[(size_t)p].is_array && k->params[(size_t)p].dtype != LT_F32) {
                kval = args[p].i;
                found = true;
            }
        if (!found || kval < 1 || kval > 16)
            return fail(LT_ERR_INVALID_ARG, "this built-in needs an integer step count between 1 and 16");
    }
    // plan cache: everything the plan depends on
    std::vector<int64_t> key = {(int64_t)g3[0], (int64_t)g3[1], (int64_t)g3[2], (int64_t)b3[0], (int64_t)b3[1],
                                (int64_t)b3[2], sb3[0], sb3[1], sb3[2], kval, nargs};
    for (int p = 0; p < nargs; ++p) {
        const lt_array *a = (*parr)[(size_t)p];
        if (!a) {
            key.push_back(-1);
            continue;
        }
        int alias = p;
        for (int q = 0; q < p; ++q)
            if ((*parr)[(size_t)q] == a) {
                alias = q;
                break;
            }
        const ArrayGeom &g = a->g;
        key.insert(key.end(), {(int64_t)alias, (int64_t)g.dtype, (int64_t)g.nd, g.shape[0], g.shape[1], g.shape[2],
                               (int64_t)g.dist.kind, (int64_t)g.dist.order, g.dist.chunk[0], g.dist.chunk[1],
                               g.dist.chunk[2], g.dist.halo[0], g.dist.halo[1], g.dist.halo[2]});
    }
    auto hit = k->plans.find(key);
    if (hit != k->plans.end()) {
        hit->second.last_use = ++k->plan_tick;
        *out = hit->second.b;
        c->stats.plans_reused++;
        return LT_OK;
    }
    auto bundle = std::make_shared<PlanBundle>();
    LaunchPlan *plan = &bundle->plan;
    std::string err;
    if (!plan_launch(k->ann, k->stmt_of_param, pa, g3, b3, sb3, plan, &err)) return fail(LT_ERR_INVALID_ARG, err);
    // the annotation must contain every access the built-in makes
    int64_t B[3];
    for (int d = 0; d < 3; ++d) B[d] = (int64_t)(b3[d] ? b3[d] : 1);
    std::vector<int64_t> vlo, vhi;
    Annotation canon_launch;
    const Annotation *canon = &k->canon;
    if (has_k) {
        std::string err2;
        if (!parse_annotation(canon_text(k->def, kval), &canon_launch, &err2))
            return fail(LT_ERR_PARSE, "internal canonical: " + err2);
        canon = &canon_launch;
    }
    for (const auto &sb : plan->sbs) {
        if (!k->def->canon) break;
        var_ranges(*canon, sb.threads, B, &vlo, &vhi);
        for (const auto &ap : sb.args) {
            if (ap.kind == ARG_VALUE) continue;
            int sl = k->slot_of_param[(size_t)ap.param];
            const Stmt &cs = canon->stmts[(size_t)k->canon_stmt[(size_t)sl]];
            Box need = eval_region(cs, vlo, vhi, (*parr)[(size_t)ap.param]->g.shape);
            if (!need.empty() && !ap.region.contains(need))
                return fail(LT_ERR_INVALID_ARG, "the annotation's region for '" +
                                                    k->names[(size_t)ap.param] +
                                                    "' does not contain what the kernel accesses");
        }
    }
    bundle->dead = dead_by_param(*plan, *parr);
    if (k->plans.size() >= PLAN_CACHE) {  // full: drop the least recently used shape
        auto lru = k->plans.begin();
        for (auto it = k->plans.begin(); it != k->plans.end(); ++it)
            if (it->second.last_use < lru->second.last_use) lru = it;
        k->plans.erase(lru);
    }
    CachedPlan ce;
    ce.b = bundle;
    ce.last_use = ++k->plan_tick;
    k->plans.emplace(std::move(key), std::move(ce));
    *out = std::move(bundle);
    return LT_OK;
}

lt_status lt_plan_explain(lt_ctx *c, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
                          const lt_arg *args, int32_t nargs, char *buf, size_t cap, size_t *needed) {
    lt_status st = check_ctx(c);
    if (st) return st;
    std::shared_ptr<const PlanBundle> b;
    std::vector<lt_array *> parr;
    if ((st = prepare_plan(c, k, grid, block, wd, args, nargs, &b, &parr))) return st;
    std::string js = plan_to_json(b->plan);
    if (needed) *needed = js.size() + 1;
    if (buf && cap) {
        size_t n = std::min(cap - 1, js.size());
        std::memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return LT_OK;
}

static lt_status emit_launch(lt_ctx *c, PendingLaunch &pl,
                             const std::vector<std::pair<lt_array *, int64_t>> *next_dead);

// Does the pending launch write array a?
static bool pending_writes(lt_ctx *c, const lt_array *a) {
    if (!c->pending) return false;
    const lt_kernel *k = c->pending->k;
    for (size_t p = 0; p < c->pending->parr.size(); ++p)
        if (c->pending->parr[p] == a && k->ann.stmts[(size_t)k->stmt_of_param[p]].mode != MODE_READ) return true;
    return false;
}

// Enqueue the pending launch, if any, without lookahead.
static lt_status flush_pending(lt_ctx *c) {
    if (!c->pending) return LT_OK;
    std::unique_ptr<PendingLaunch> p = std::move(c->pending);
    return emit_launch(c, *p, nullptr);
}

// Does the launch use only chunks already in device memory, with no
// temporaries (packs, temp writes, reduce partials)?
static bool runs_in_place(const lt_ctx *c, const PendingLaunch &pl) {
    if (c->dry) return false;  // dry runs keep the lookahead, whose decisions the tests inspect
    for (const auto &sb : pl.b->plan.sbs)
        for (const auto &ap : sb.args) {
            if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE) continue;
            if (ap.kind != ARG_DIRECT) return false;
            const lt_array *a = pl.parr[(size_t)ap.param];
            if (a->cs[(size_t)ap.chunk].loc != LOC_DEV) return false;
            for (const auto &pc : ap.replicas)
                if (a->cs[(size_t)pc.chunk].loc != LOC_DEV) return false;
        }
    return true;
}

lt_status lt_launch(lt_ctx *c, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd, const lt_arg *args,
                    int32_t nargs) {
    lt_status st = check_ctx(c);
    if (st) return st;
    auto pl = std::make_unique<PendingLaunch>();
    if ((st = prepare_plan(c, k, grid, block, wd, args, nargs, &pl->b, &pl->parr))) return st;
    if (!k->def->launch && !k->ufn && !c->dry && k->def->id != LT_K_USER)
        return fail(LT_ERR_UNSUPPORTED, "a plan-only kernel can be launched only in a dry-run context");
    if (k->def->id == LT_K_USER &&
        (uint64_t)(block.x ? block.x : 1) * (block.y ? block.y : 1) * (block.z ? block.z : 1) > 1024)
        return fail(LT_ERR_INVALID_ARG, "a source kernel's block holds at most 1024 threads");
    pl->k = k;
    ExecParams &ep = pl->ep;
    const std::vector<lt_array *> &parr = pl->parr;
    for (size_t p = 0; p < parr.size(); ++p) {
        int sl = k->slot_of_param[p];
        if (sl < 0) continue;
        for (int d = 0; d < 3; ++d) ep.shape[sl][d] = parr[p]->g.shape[d];
        ep.nd[sl] = parr[p]->g.nd;
    }
    {
        int nf = 0, ni = 0;
        for (size_t p = 0; p < parr.size(); ++p) {
            if (k->params[p].is_array) continue;
            if (k->params[p].dtype == LT_F32 && nf < 4) ep.f[nf++] = args[p].f;
            if (k->params[p].dtype != LT_F32 && ni < 4) ep.i[ni++] = args[p].i;
        }
    }
    ep.block[0] = (int64_t)(block.x ? block.x : 1);
    ep.block[1] = (int64_t)(block.y ? block.y : 1);
    ep.block[2] = (int64_t)(block.z ? block.z : 1);
    ep.err = c->err_word;
    ep.no_staged = c->no_staged ? 1 : 0;
    for (size_t p = 0; p < parr.size(); ++p)
        if (k->stmt_of_param[p] >= 0 && k->ann.stmts[(size_t)k->stmt_of_param[p]].mode == MODE_REDUCE)
            ep.red_op = k->ann.stmts[(size_t)k->stmt_of_param[p]].op;
    // one launch of lookahead: the previous launch is enqueued now, knowing
    // which chunks this one overwrites without reading them
    if (c->pending) {
        std::vector<std::pair<lt_array *, int64_t>> nd;
        for (auto &d : pl->b->dead) nd.push_back({pl->parr[(size_t)d.first], d.second});
        std::unique_ptr<PendingLaunch> prev = std::move(c->pending);
        if ((st = emit_launch(c, *prev, &nd))) return st;
    }
    // A launch that touches only resident chunks and needs no temporaries
    // will evict nothing, so the next launch's plan cannot change what it
    // does: it is enqueued at once instead of waiting for that plan, and the
    // GPU does not idle while the host plans the next launch.
    if (runs_in_place(c, *pl)) return emit_launch(c, *pl, nullptr);
    c->pending = std::move(pl);
    return LT_OK;
}

static lt_status emit_launch(lt_ctx *c, PendingLaunch &pl,
                             const std::vector<std::pair<lt_array *, int64_t>> *next_dead) {
    lt_status st = LT_OK;
    lt_kernel *k = pl.k;
    const LaunchPlan &plan = pl.b->plan;
    const std::vector<lt_array *> &parr = pl.parr;
    ExecParams &ep = pl.ep;
    ++c->launch_id;
    c->stats.launches++;
    mark_dead(c, *pl.b, parr);
    if (next_dead)
        for (auto &d : *next_dead) d.first->cs[(size_t)d.second].next_dead_launch = c->launch_id;
    const BuiltinDef *def = k->def;

    // footprint: every distinct chunk and temporary of the launch
    size_t foot = 0;
    {
        std::vector<std::pair<lt_array *, int64_t>> seen;
        auto touch = [&](lt_array *a, int64_t ci) {
            for (auto &s : seen)
                if (s.first == a && s.second == ci) return;
            seen.push_back({a, ci});
            foot += align_up(a->g.chunks[(size_t)ci].bytes, ALIGN);
        };
        for (const auto &sb : plan.sbs)
            for (const auto &ap : sb.args) {
                if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE) continue;
                lt_array *a = parr[(size_t)ap.param];
                if (ap.kind == ARG_DIRECT) touch(a, ap.chunk);
                for (auto &pc : ap.pieces) touch(a, pc.chunk);
                for (auto &pc : ap.replicas) touch(a, pc.chunk);
                if (ap.kind != ARG_DIRECT) foot += align_up(temp_geometry(a->g, ap.region).bytes, ALIGN);
            }
    }
    bool batched = foot <= c->dev.cap / 20 * 19;
    size_t nsb = plan.sbs.size();
    std::vector<size_t> order(nsb);
    bool rev = !(c->cfg.flags & LT_FLAG_FIXED_SWEEP) && (c->launch_id & 1);
    for (size_t i = 0; i < nsb; ++i) order[i] = rev ? nsb - 1 - i : i;

    // reduce partials.  A superblock whose reduce region is exactly the box
    // of a chunk of the destination array (an array no other argument of the
    // launch names; a chunk no earlier superblock took) accumulates in that
    // chunk itself: the cells only it contributes to are then final where
    // they lie, and the combine touches the shared ones only.  The other
    // partials share one temporary block.
    std::vector<std::vector<ChunkGeom>> red_geom(nsb);
    std::vector<std::vector<size_t>> red_off(nsb);
    std::vector<std::vector<int64_t>> red_chunk(nsb);  // chunk holding the partial, -1 = temporary
    std::vector<std::pair<lt_array *, int64_t>> red_inplace;
    size_t red_bytes = 0;
    for (size_t s = 0; s < nsb; ++s)
        for (const auto &ap : plan.sbs[s].args)
            if (ap.kind == ARG_REDUCE) {
                lt_array *a = parr[(size_t)ap.param];
                int64_t ic = -1;
                if (std::count(parr.begin(), parr.end(), a) == 1)
                    for (const auto &pc : ap.pieces) {
                        const Box &cb = a->g.chunks[(size_t)pc.chunk].box;
                        if (cb.contains(ap.region) && ap.region.contains(cb) &&
                            std::find(red_inplace.begin(), red_inplace.end(), std::make_pair(a, pc.chunk)) ==
                                red_inplace.end()) {
                            ic = pc.chunk;
                            break;
                        }
                    }
                red_chunk[s].push_back(ic);
                if (ic >= 0) {
                    c->stats.reduce_inplace++;
                    red_inplace.push_back({a, ic});
                    red_geom[s].push_back(a->g.chunks[(size_t)ic]);
                    red_off[s].push_back(0);
                    continue;
                }
                ChunkGeom g = temp_geometry(a->g, ap.region);
                red_geom[s].push_back(g);
                red_off[s].push_back(red_bytes);
                red_bytes += align_up(g.bytes, 256);
            }
    size_t red_base = 0;
    FenceSet red_fence;
    const bool any_red = red_bytes || !red_inplace.empty();
    if (red_bytes && (st = dev_alloc(c, red_bytes, &red_base, &red_fence))) return st;
    for (auto &ip : red_inplace) {
        ip.first->cs[(size_t)ip.second].pin++;
        ip.first->cs[(size_t)ip.second].discarded = false;  // the launch writes its partial there
    }
    for (auto &ip : red_inplace) {
        // the launch overwrites the chunk's region: its old contents are not needed
        if ((st = ensure_dev(c, ip.first, ip.second, false))) return st;
        CState &cs = ip.first->cs[(size_t)ip.second];
        red_fence.merge(cs.ready);
        red_fence.merge(cs.busy);
    }
    if (any_red && def->reduce_zero) {
        op_begin(c, S_COMP, "reduce_init");
        if ((st = op_wait(c, red_fence))) return st;
        if (!c->dry) {
            if (red_bytes) CK(c, cudaMemsetAsync(dptr(c, red_base), 0, red_bytes, c->st[S_COMP]));
            for (auto &ip : red_inplace)
                CK(c, cudaMemsetAsync(dptr(c, ip.first->cs[(size_t)ip.second].off), 0,
                                      ip.first->g.chunks[(size_t)ip.second].bytes, c->st[S_COMP]));
        }
        uint64_t q;
        if ((st = op_end(c, &q))) return st;
        red_fence = FenceSet::one(S_COMP, q);
    }
    // the view of superblock s's ri-th reduce partial
    auto red_view = [&](size_t s, size_t ri, lt_array *a) {
        const int64_t ic = red_chunk[s][ri];
        if (ic >= 0) return view_of(c, a->g, a->g.chunks[(size_t)ic], a->cs[(size_t)ic].off);
        return view_of(c, a->g, red_geom[s][ri], red_base + red_off[s][ri]);
    };

    // process superblocks in groups: all at once when the launch fits in
    // the HBM budget, else one at a time (streaming through host memory)
    size_t gsz = batched ? nsb : 1;
    // last group that uses each chunk (evicting before it must write back)
    for (size_t g0 = 0, gi = 0; g0 < nsb; g0 += gsz, ++gi) {
        size_t g1 = std::min(nsb, g0 + gsz);
        for (size_t oi = g0; oi < g1; ++oi)
            for (const auto &ap : plan.sbs[order[oi]].args) {
                if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE) continue;
                lt_array *a = parr[(size_t)ap.param];
                int64_t grp = ap.kind == ARG_REDUCE ? (int64_t)((nsb + gsz - 1) / gsz) : (int64_t)gi;
                auto mark = [&](int64_t ci) {
                    CState &cs = a->cs[(size_t)ci];
                    if (cs.last_use_launch != c->launch_id || cs.last_use_group < grp) cs.last_use_group = grp;
                    cs.last_use_launch = c->launch_id;
                };
                if (ap.kind == ARG_DIRECT) mark(ap.chunk);
                for (auto &pc : ap.pieces) mark(pc.chunk);
                for (auto &pc : ap.replicas) mark(pc.chunk);
            }
    }
    // the chunks the superblocks [g0, g1) of this launch use
    auto collect_uses = [&](size_t g0, size_t g1) {
        std::vector<ArgUse> uses;
        auto add_use = [&](lt_array *a, int64_t ci, bool w) {
            for (auto &u : uses)
                if (u.a == a && u.chunk == ci) {
                    u.write = u.write || w;
                    return;
                }
            uses.push_back({a, ci, w});
        };
        for (size_t oi = g0; oi < g1; ++oi) {
            const auto &sb = plan.sbs[order[oi]];
            for (const auto &ap : sb.args) {
                if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE || ap.kind == ARG_REDUCE) continue;
                lt_array *a = parr[(size_t)ap.param];
                bool w = ap.mode != MODE_READ;
                if (ap.kind == ARG_DIRECT) add_use(a, ap.chunk, w);
                if (ap.kind == ARG_PACK)
                    for (auto &pc : ap.pieces) add_use(a, pc.chunk, false);
                if (ap.kind == ARG_TEMPW)
                    for (auto &pc : ap.pieces) add_use(a, pc.chunk, true);
                for (auto &pc : ap.replicas) add_use(a, pc.chunk, ap.kind == ARG_DIRECT);
            }
        }
        return uses;
    };
    // Streaming: the next group's chunks are fetched (or allocated) while
    // this group runs, so host-to-device copies overlap its kernels and the
    // evictions that make room; `ahead` keeps them pinned until their group.
    // Pinning them early also takes them out of the eviction choices, which
    // costs more transfers than the overlap saves when the budget holds only
    // a few groups (measured: with 3 groups' worth it lost 4 %, with 6 it
    // gained 2 %), so it runs ahead only with at least 4 groups' worth.
    std::vector<ArgUse> ahead;
    auto unpin_ahead = [&]() {
        for (auto &u : ahead) u.a->cs[(size_t)u.chunk].pin--;
        ahead.clear();
    };
    c->cur_group = 0;
    for (size_t g0 = 0; g0 < nsb; g0 += gsz, ++c->cur_group) {
        size_t g1 = std::min(nsb, g0 + gsz);
        std::vector<ArgUse> uses = collect_uses(g0, g1);
        for (auto &u : uses) {
            u.a->cs[(size_t)u.chunk].pin++;
            if (u.write) {
                u.a->cs[(size_t)u.chunk].last_write_launch = c->launch_id;
                u.a->cs[(size_t)u.chunk].discarded = false;
            }
        }
        unpin_ahead();  // now pinned as this group's uses
        for (auto &u : uses) {
            // a chunk whose region is only partly written must keep its data
            st = ensure_dev(c, u.a, u.chunk, true);
            if (st) {
                for (auto &v : uses) v.a->cs[(size_t)v.chunk].pin--;
                return st;
            }
        }
        size_t group_bytes = 0;
        for (auto &u : uses) group_bytes += align_up(u.a->g.chunks[(size_t)u.chunk].bytes, ALIGN);
        if (!batched && g1 < nsb && c->dev.cap >= 4 * group_bytes) {
            ahead = collect_uses(g1, std::min(nsb, g1 + gsz));
            for (auto &u : ahead) u.a->cs[(size_t)u.chunk].pin++;
            for (auto &u : ahead) {
                st = ensure_dev(c, u.a, u.chunk, true, /*soft=*/true);
                if (st == LT_ERR_OOM_DEVICE) break;  // no room to run ahead: fetch when the group starts
                if (st) {
                    unpin_ahead();
                    for (auto &v : uses) v.a->cs[(size_t)v.chunk].pin--;
                    return st;
                }
            }
            st = LT_OK;
        }
        // temporaries for pack / temp-write
        std::vector<TempAlloc> temps;
        std::vector<std::vector<int>> temp_of(g1 - g0);
        FenceSet temp_fences;
        for (size_t oi = g0; oi < g1; ++oi) {
            const auto &sb = plan.sbs[order[oi]];
            temp_of[oi - g0].assign(sb.args.size(), -1);
            for (size_t ai = 0; ai < sb.args.size(); ++ai) {
                const auto &ap = sb.args[ai];
                if (ap.kind != ARG_PACK && ap.kind != ARG_TEMPW) continue;
                TempAlloc t;
                t.geom = temp_geometry(parr[(size_t)ap.param]->g, ap.region);
                t.bytes = t.geom.bytes;
                FenceSet f;
                st = dev_alloc(c, t.bytes, &t.off, &f);
                if (st) {
                    for (auto &v : uses) v.a->cs[(size_t)v.chunk].pin--;
                    return st;
                }
                temp_fences.merge(f);
                temp_of[oi - g0][ai] = (int)temps.size();
                temps.push_back(t);
            }
        }
        // --- pack (read regions spanning several chunks; readwrite temps)
        std::vector<CopyPiece> packs;
        FenceSet pack_wait = temp_fences;
        for (size_t oi = g0; oi < g1; ++oi) {
            const auto &sb = plan.sbs[order[oi]];
            for (size_t ai = 0; ai < sb.args.size(); ++ai) {
                const auto &ap = sb.args[ai];
                const std::vector<Piece> *src = nullptr;
                if (ap.kind == ARG_PACK) src = &ap.pieces;
                if (ap.kind == ARG_TEMPW && ap.mode == MODE_READWRITE) src = &ap.replicas;
                if (!src) continue;
                lt_array *a = parr[(size_t)ap.param];
                const TempAlloc &t = temps[(size_t)temp_of[oi - g0][ai]];
                for (const auto &pc : *src) {
                    CopyPiece cp{};
                    const CState &cs = a->cs[(size_t)pc.chunk];
                    cp.src = view_of(c, a->g, a->g.chunks[(size_t)pc.chunk], cs.off);
                    cp.dst = view_of(c, a->g, t.geom, t.off);
                    cp.nd = a->g.nd;
                    cp.esize = (int32_t)a->g.esize();
                    for (int d = 0; d < 3; ++d) {
                        cp.lo[d] = d < a->g.nd ? pc.box.lo[d] : 0;
                        cp.hi[d] = d < a->g.nd ? pc.box.hi[d] : 0;
                    }
                    packs.push_back(cp);
                    pack_wait.merge(cs.ready);
                    c->stats.bytes_d2d += (uint64_t)pc.box.volume() * a->g.esize();
                }
            }
        }
        FenceSet temp_ready;
        if (!packs.empty()) {
            uint64_t rows = 0;
            for (auto &p : packs) {
                p.unit_begin = rows;
                rows += copy_piece_units(p);
            }
            op_begin(c, S_COMP, "pack");
            if ((st = op_wait(c, pack_wait))) return st;
            void *dptr;
            size_t roff;
            if ((st = upload(c, packs.data(), packs.size() * sizeof(CopyPiece), &dptr, &roff))) return st;
            if (!c->dry) {
                TimeScope ts(c, CAT_COPYK);
                CK(c, k::copy_pieces((const CopyPiece *)dptr, (int)packs.size(), rows, c->st[S_COMP]));
                c->stats.kernels++;
            }
            uint64_t q;
            if ((st = op_end(c, &q))) return st;
            upload_done(c, roff, packs.size() * sizeof(CopyPiece), q);
            c->stats.tasks_copy++;
            temp_ready.add(S_COMP, q);
            for (size_t oi = g0; oi < g1; ++oi)
                for (const auto &ap : plan.sbs[order[oi]].args) {
                    const std::vector<Piece> *src = nullptr;
                    if (ap.kind == ARG_PACK) src = &ap.pieces;
                    if (ap.kind == ARG_TEMPW && ap.mode == MODE_READWRITE) src = &ap.replicas;
                    if (!src) continue;
                    for (const auto &pc : *src) parr[(size_t)ap.param]->cs[(size_t)pc.chunk].busy.add(S_COMP, q);
                }
        }
        // --- execute (all superblocks of the group in one kernel)
        // A kernel that keeps halo replicas itself (write_through) writes the
        // replicas of a write-only argument no other parameter aliases; its
        // tasks carry the replica boxes and no copy step follows for them.
        auto writes_through = [&](const ArgPlan &ap, int sl) {
            if (k->ufn || def->write_through < 0 || sl != def->write_through) return false;
            if (ap.kind != ARG_DIRECT || ap.mode != MODE_WRITE || ap.replicas.empty()) return false;
            for (size_t j = 0; j < parr.size(); ++j)
                if ((int)j != ap.param && parr[j] == parr[(size_t)ap.param]) return false;
            return true;
        };
        std::vector<ExecTask> tasks;
        std::vector<ReplicaTarget> reps;
        uint64_t rep_cells = 0;
        std::vector<CState *> wt_chunks;  // replica chunks the execute kernel writes
        FenceSet ex_wait = temp_fences;
        ex_wait.merge(temp_ready);
        ex_wait.merge(red_fence);
        for (size_t oi = g0; oi < g1; ++oi) {
            size_t s = order[oi];
            const auto &sb = plan.sbs[s];
            ExecTask t{};
            for (int d = 0; d < 3; ++d) {
                t.t_lo[d] = sb.threads.lo[d];
                t.t_hi[d] = sb.threads.hi[d];
            }
            size_t ri = 0;
            for (size_t ai = 0; ai < sb.args.size(); ++ai) {
                const auto &ap = sb.args[ai];
                int sl = k->slot_of_param[(size_t)ap.param];
                if (sl < 0) continue;
                lt_array *a = parr[(size_t)ap.param];
                if (ap.kind == ARG_DIRECT) {
                    CState &cs = a->cs[(size_t)ap.chunk];
                    t.v[sl] = view_of(c, a->g, a->g.chunks[(size_t)ap.chunk], cs.off);
                    ex_wait.merge(cs.ready);
                    if (ap.mode != MODE_READ) ex_wait.merge(cs.busy);
                    if (writes_through(ap, sl)) {
                        for (const auto &pc : ap.replicas) {
                            CState &dcs = a->cs[(size_t)pc.chunk];
                            ReplicaTarget r{};
                            r.dst = view_of(c, a->g, a->g.chunks[(size_t)pc.chunk], dcs.off);
                            for (int d = 0; d < 3; ++d) {
                                r.lo[d] = d < a->g.nd ? pc.box.lo[d] : 0;
                                r.hi[d] = d < a->g.nd ? pc.box.hi[d] : 0;
                            }
                            r.task = (int32_t)tasks.size();
                            r.cell_begin = rep_cells;
                            rep_cells += (uint64_t)pc.box.volume();
                            reps.push_back(r);
                            ex_wait.merge(dcs.ready);
                            ex_wait.merge(dcs.busy);
                            wt_chunks.push_back(&dcs);
                            c->stats.bytes_replica_wt += (uint64_t)pc.box.volume() * a->g.esize();
                        }
                    }
                } else if (ap.kind == ARG_PACK || ap.kind == ARG_TEMPW) {
                    const TempAlloc &tm = temps[(size_t)temp_of[oi - g0][ai]];
                    t.v[sl] = view_of(c, a->g, tm.geom, tm.off);
                } else if (ap.kind == ARG_REDUCE) {
                    t.v[sl] = red_view(s, ri, a);
                    ri++;
                }
            }
            tasks.push_back(t);
        }
        uint64_t exq = 0;
        {
            op_begin(c, S_COMP, "execute");
            if ((st = op_wait(c, ex_wait))) return st;
            ep.ntasks = (int32_t)tasks.size();
            ep.uniform_ctas = 0;
            uint32_t ctas = def->prepare ? def->prepare(tasks.data(), (int)tasks.size(), ep) : 0;
            if (ctas != 0xFFFFFFFFu) ep.uniform_ctas = uniform_cta_count(tasks);
            if (ctas == 0xFFFFFFFFu)
                return fail(LT_ERR_UNSUPPORTED,
                            "this kernel cannot run this launch (code " + std::to_string(ep.variant) +
                                "): the GEMM needs A row-major and B column-major chunks, at most 15 distinct "
                                "chunks of each per launch; the multi-step stencil 1 <= k <= 16; K-Means "
                                "1 <= k <= 64 and arrays of 4k / 5k elements; a source kernel virtual block "
                                "indices below 2^32");
            // one table: the tasks, then their replica targets
            const size_t tbytes = tasks.size() * sizeof(ExecTask), rbytes = reps.size() * sizeof(ReplicaTarget);
            std::vector<char> table(tbytes + rbytes);
            std::memcpy(table.data(), tasks.data(), tbytes);
            if (rbytes) std::memcpy(table.data() + tbytes, reps.data(), rbytes);
            void *dptr;
            size_t roff;
            if ((st = upload(c, table.data(), table.size(), &dptr, &roff))) return st;
            ep.reps = (rbytes && dptr) ? (const ReplicaTarget *)((const char *)dptr + tbytes) : nullptr;
            ep.nreps = (uint32_t)reps.size();
            ep.rep_cells = ep.reps ? rep_cells : 0;
            if (!c->dry && ctas) {
                TimeScope ts(c, CAT_EXEC);
                if (k->ufn) {
                    const ExecTask *tp = (const ExecTask *)dptr;
                    void *kargs[] = {(void *)&tp, (void *)&ep};
                    dim3 blk((unsigned)ep.block[0], (unsigned)ep.block[1], (unsigned)ep.block[2]);
                    CK(c, cudaLaunchKernel((const void *)k->ufn, dim3(ctas), blk, kargs, 0, c->st[S_COMP]));
                } else {
                    CK(c, def->launch((const ExecTask *)dptr, ctas, ep, c->st[S_COMP]));
                }
                c->stats.kernels++;
            }
            std::string extra;
            if (c->log_on) {
                std::ostringstream ex;
                ex << ",\"superblocks\":[";
                for (size_t oi = g0; oi < g1; ++oi) ex << (oi > g0 ? "," : "") << plan.sbs[order[oi]].index;
                ex << "],\"variant\":" << ep.variant << ",\"ctas\":" << ctas << ",\"replicas\":" << reps.size();
                extra = ex.str();
            }
            if ((st = op_end(c, &exq, extra))) return st;
            upload_done(c, roff, table.size(), exq);
            for (CState *d : wt_chunks) {
                d->ready = FenceSet::one(S_COMP, exq);
                d->busy.add(S_COMP, exq);
            }
            c->stats.tasks_execute += tasks.size();
            for (auto &u : uses) {
                CState &cs = u.a->cs[(size_t)u.chunk];
                cs.busy.add(S_COMP, exq);
            }
            for (size_t oi = g0; oi < g1; ++oi)
                for (const auto &ap : plan.sbs[order[oi]].args)
                    if (ap.kind == ARG_DIRECT && ap.mode != MODE_READ) {
                        CState &cs = parr[(size_t)ap.param]->cs[(size_t)ap.chunk];
                        cs.ready = FenceSet::one(S_COMP, exq);
                    }
            red_fence.add(S_COMP, exq);
        }
        // --- replica updates and temp scatters (unpack)
        std::vector<CopyPiece> outs;
        FenceSet out_wait;
        out_wait.add(S_COMP, exq);
        for (size_t oi = g0; oi < g1; ++oi) {
            const auto &sb = plan.sbs[order[oi]];
            for (size_t ai = 0; ai < sb.args.size(); ++ai) {
                const auto &ap = sb.args[ai];
                lt_array *a = ap.param >= 0 && ap.kind != ARG_VALUE ? parr[(size_t)ap.param] : nullptr;
                if (ap.kind == ARG_DIRECT && ap.mode != MODE_READ &&
                    !writes_through(ap, k->slot_of_param[(size_t)ap.param])) {
                    for (const auto &pc : ap.replicas) {
                        CopyPiece cp{};
                        cp.src = view_of(c, a->g, a->g.chunks[(size_t)ap.chunk], a->cs[(size_t)ap.chunk].off);
                        CState &dcs = a->cs[(size_t)pc.chunk];
                        cp.dst = view_of(c, a->g, a->g.chunks[(size_t)pc.chunk], dcs.off);
                        cp.nd = a->g.nd;
                        cp.esize = (int32_t)a->g.esize();
                        for (int d = 0; d < 3; ++d) {
                            cp.lo[d] = d < a->g.nd ? pc.box.lo[d] : 0;
                            cp.hi[d] = d < a->g.nd ? pc.box.hi[d] : 0;
                        }
                        out_wait.merge(dcs.ready);
                        out_wait.merge(dcs.busy);
                        outs.push_back(cp);
                        c->stats.bytes_d2d += (uint64_t)pc.box.volume() * a->g.esize();
                    }
                } else if (ap.kind == ARG_TEMPW) {
                    const TempAlloc &tm = temps[(size_t)temp_of[oi - g0][ai]];
                    for (const auto &pc : ap.pieces) {
                        CopyPiece cp{};
                        cp.src = view_of(c, a->g, tm.geom, tm.off);
                        CState &dcs = a->cs[(size_t)pc.chunk];
                        cp.dst = view_of(c, a->g, a->g.chunks[(size_t)pc.chunk], dcs.off);
                        cp.nd = a->g.nd;
                        cp.esize = (int32_t)a->g.esize();
                        for (int d = 0; d < 3; ++d) {
                            cp.lo[d] = d < a->g.nd ? pc.box.lo[d] : 0;
                            cp.hi[d] = d < a->g.nd ? pc.box.hi[d] : 0;
                        }
                        out_wait.merge(dcs.ready);
                        out_wait.merge(dcs.busy);
                        outs.push_back(cp);
                        c->stats.bytes_d2d += (uint64_t)pc.box.volume() * a->g.esize();
                    }
                }
            }
        }
        uint64_t outq = 0;
        if (!outs.empty()) {
            uint64_t rows = 0;
            for (auto &p : outs) {
                p.unit_begin = rows;
                rows += copy_piece_units(p);
            }
            op_begin(c, S_COMP, "unpack");
            if ((st = op_wait(c, out_wait))) return st;
            void *dptr;
            size_t roff;
            if ((st = upload(c, outs.data(), outs.size() * sizeof(CopyPiece), &dptr, &roff))) return st;
            if (!c->dry) {
                TimeScope ts(c, CAT_COPYK);
                CK(c, k::copy_pieces((const CopyPiece *)dptr, (int)outs.size(), rows, c->st[S_COMP]));
                c->stats.kernels++;
            }
            if ((st = op_end(c, &outq))) return st;
            upload_done(c, roff, outs.size() * sizeof(CopyPiece), outq);
            c->stats.tasks_copy++;
            for (size_t oi = g0; oi < g1; ++oi)
                for (const auto &ap : plan.sbs[order[oi]].args) {
                    if (ap.kind == ARG_VALUE) continue;
                    lt_array *a = parr[(size_t)ap.param];
                    if (ap.kind == ARG_DIRECT && ap.mode != MODE_READ &&
                        !writes_through(ap, k->slot_of_param[(size_t)ap.param])) {
                        a->cs[(size_t)ap.chunk].busy.add(S_COMP, outq);
                        for (const auto &pc : ap.replicas) {
                            CState &d = a->cs[(size_t)pc.chunk];
                            d.ready = FenceSet::one(S_COMP, outq);
                            d.busy.add(S_COMP, outq);
                        }
                    } else if (ap.kind == ARG_TEMPW) {
                        for (const auto &pc : ap.pieces) {
                            CState &d = a->cs[(size_t)pc.chunk];
                            d.ready = FenceSet::one(S_COMP, outq);
                            d.busy.add(S_COMP, outq);
                        }
                    }
                }
        }
        // release temporaries and pins
        FenceSet rel;
        rel.add(S_COMP, outq ? outq : exq);
        for (auto &t : temps) c->dev.release(t.off, t.bytes, rel);
        for (auto &u : uses) u.a->cs[(size_t)u.chunk].pin--;
    }

    // --- reduce: combine the per-superblock partials in superblock order
    c->cur_group = (int64_t)((nsb + gsz - 1) / gsz);
    if (any_red) {
        std::vector<ReducePiece> rp;
        std::vector<CopyPiece> rcopies;
        std::vector<DView> srcs;
        FenceSet rw = red_fence;
        // With partials in place, a cell several superblocks share is reduced
        // into scratch first and copied to its chunks after: no kernel writes
        // a cell another piece may still read.
        const bool two_phase = !red_inplace.empty();
        struct ScratchPiece {
            size_t rp;  // reduce piece writing the scratch block
            lt_array *a;
            int64_t chunk;
            Box box;
            ChunkGeom geom;
            size_t off;
        };
        std::vector<ScratchPiece> scratch;
        size_t scratch_bytes = 0;
        // per destination chunk, the (superblock, box) contributions
        struct Contrib {
            size_t sb, ri;
            Box box;
        };
        std::map<std::pair<lt_array *, int64_t>, std::vector<Contrib>> per;
        std::vector<std::pair<lt_array *, int64_t>> dest_order;
        int red_op = RED_ADD;
        for (size_t s = 0; s < nsb; ++s) {
            size_t ri = 0;
            for (const auto &ap : plan.sbs[s].args) {
                if (ap.kind != ARG_REDUCE) continue;
                red_op = ap.op;
                lt_array *a = parr[(size_t)ap.param];
                for (const auto &pc : ap.pieces) {
                    auto key = std::make_pair(a, pc.chunk);
                    if (!per.count(key)) dest_order.push_back(key);
                    per[key].push_back({s, ri, pc.box});
                }
                ri++;
            }
        }
        std::vector<std::pair<lt_array *, int64_t>> dests = dest_order;
        for (auto &d : dests) {
            d.first->cs[(size_t)d.second].pin++;
            d.first->cs[(size_t)d.second].discarded = false;  // the reduce writes it
        }
        for (auto &d : dests) {
            if ((st = ensure_dev(c, d.first, d.second, true))) {
                for (auto &e : dests) e.first->cs[(size_t)e.second].pin--;
                return st;
            }
        }
        for (auto &d : dests) {
            lt_array *a = d.first;
            const ChunkGeom &cg = a->g.chunks[(size_t)d.second];
            CState &cs = a->cs[(size_t)d.second];
            rw.merge(cs.ready);
            rw.merge(cs.busy);
            const auto &cl = per[d];
            // coordinate compression of the contribution boxes
            std::vector<int64_t> cuts[3];
            for (int dd = 0; dd < a->g.nd; ++dd) {
                for (const auto &cb : cl) {
                    cuts[dd].push_back(cb.box.lo[dd]);
                    cuts[dd].push_back(cb.box.hi[dd] + 1);
                }
                std::sort(cuts[dd].begin(), cuts[dd].end());
                cuts[dd].erase(std::unique(cuts[dd].begin(), cuts[dd].end()), cuts[dd].end());
            }
            for (int dd = a->g.nd; dd < 3; ++dd) cuts[dd] = {0, 1};
            for (size_t x = 0; x + 1 < cuts[0].size(); ++x)
                for (size_t y = 0; y + 1 < cuts[1].size(); ++y)
                    for (size_t z = 0; z + 1 < cuts[2].size(); ++z) {
                        Box cell;
                        cell.nd = a->g.nd;
                        size_t ix[3] = {x, y, z};
                        for (int dd = 0; dd < a->g.nd; ++dd) {
                            cell.lo[dd] = cuts[dd][ix[dd]];
                            cell.hi[dd] = cuts[dd][ix[dd] + 1] - 1;
                        }
                        ReducePiece p{};
                        p.src_begin = (uint32_t)srcs.size();
                        const Contrib *only = nullptr;
                        for (const auto &cb : cl)
                            if (cb.box.contains(cell)) {
                                srcs.push_back(red_view(cb.sb, cb.ri, a));
                                p.nsrc++;
                                only = &cb;
                            }
                        if (!p.nsrc) continue;
                        if (p.nsrc == 1 && red_chunk[only->sb][only->ri] == d.second) {
                            srcs.pop_back();  // the partial lies in this chunk already
                            continue;
                        }
                        if (p.nsrc == 1) {  // a single contribution: a plain copy
                            CopyPiece cp{};
                            cp.src = srcs.back();
                            srcs.pop_back();
                            cp.dst = view_of(c, a->g, cg, cs.off);
                            cp.nd = a->g.nd;
                            cp.esize = (int32_t)a->g.esize();
                            for (int dd = 0; dd < 3; ++dd) {
                                cp.lo[dd] = dd < a->g.nd ? cell.lo[dd] : 0;
                                cp.hi[dd] = dd < a->g.nd ? cell.hi[dd] : 0;
                            }
                            rcopies.push_back(cp);
                            continue;
                        }
                        p.dst = view_of(c, a->g, cg, cs.off);
                        p.nd = a->g.nd;
                        p.op = red_op;
                        p.dtype = a->g.dtype;
                        for (int dd = 0; dd < 3; ++dd) {
                            p.lo[dd] = dd < a->g.nd ? cell.lo[dd] : 0;
                            p.hi[dd] = dd < a->g.nd ? cell.hi[dd] : 0;
                        }
                        if (two_phase) {
                            ScratchPiece sp;
                            sp.rp = rp.size();
                            sp.a = a;
                            sp.chunk = d.second;
                            sp.box = cell;
                            sp.geom = temp_geometry(a->g, cell);
                            sp.off = scratch_bytes;
                            scratch_bytes += align_up(sp.geom.bytes, 256);
                            scratch.push_back(sp);
                        }
                        rp.push_back(p);
                    }
        }
        size_t scratch_base = 0;
        if (scratch_bytes) {
            FenceSet sf;
            if ((st = dev_alloc(c, scratch_bytes, &scratch_base, &sf))) return st;
            rw.merge(sf);
            for (auto &sp : scratch) {  // reduce into scratch, then copy the scratch block to the chunk
                const DView sv = view_of(c, sp.a->g, sp.geom, scratch_base + sp.off);
                rp[sp.rp].dst = sv;
                CopyPiece cp{};
                cp.src = sv;
                cp.dst = view_of(c, sp.a->g, sp.a->g.chunks[(size_t)sp.chunk], sp.a->cs[(size_t)sp.chunk].off);
                cp.nd = sp.a->g.nd;
                cp.esize = (int32_t)sp.a->g.esize();
                for (int dd = 0; dd < 3; ++dd) {
                    cp.lo[dd] = dd < sp.a->g.nd ? sp.box.lo[dd] : 0;
                    cp.hi[dd] = dd < sp.a->g.nd ? sp.box.hi[dd] : 0;
                }
                rcopies.push_back(cp);
            }
        }
        uint64_t elems = 0;
        for (auto &p : rp) {
            p.elem_begin = elems;
            uint64_t e = 1;
            for (int d = 0; d < p.nd; ++d) e *= (uint64_t)(p.hi[d] - p.lo[d] + 1);
            elems += e;
        }
        op_begin(c, S_COMP, "reduce");
        if ((st = op_wait(c, rw))) return st;
        void *dp1, *dp2;
        size_t ro1, ro2;
        if ((st = upload(c, rp.data(), rp.size() * sizeof(ReducePiece), &dp1, &ro1))) return st;
        if ((st = upload(c, srcs.data(), srcs.size() * sizeof(DView), &dp2, &ro2))) return st;
        void *dp3;
        size_t ro3;
        uint64_t cunits = 0;
        for (auto &p : rcopies) {
            p.unit_begin = cunits;
            cunits += copy_piece_units(p);
        }
        if ((st = upload(c, rcopies.data(), rcopies.size() * sizeof(CopyPiece), &dp3, &ro3))) return st;
        if (!c->dry && !rp.empty()) {
            TimeScope ts(c, CAT_COPYK);
            CK(c, k::reduce_pieces((const ReducePiece *)dp1, (const DView *)dp2, (int)rp.size(), elems,
                                   c->st[S_COMP]));
            c->stats.kernels++;
        }
        if (!c->dry && !rcopies.empty()) {
            TimeScope ts(c, CAT_COPYK);
            CK(c, k::copy_pieces((const CopyPiece *)dp3, (int)rcopies.size(), cunits, c->st[S_COMP]));
            c->stats.kernels++;
        }
        uint64_t q;
        if ((st = op_end(c, &q))) return st;
        upload_done(c, ro1, rp.size() * sizeof(ReducePiece), q);
        upload_done(c, ro2, srcs.size() * sizeof(DView), q);
        upload_done(c, ro3, rcopies.size() * sizeof(CopyPiece), q);
        c->stats.tasks_reduce++;
        for (auto &d : dests) {
            CState &cs = d.first->cs[(size_t)d.second];
            cs.ready = FenceSet::one(S_COMP, q);
            cs.busy.add(S_COMP, q);
            cs.pin--;
        }
        for (auto &ip : red_inplace) {
            CState &cs = ip.first->cs[(size_t)ip.second];
            cs.ready = FenceSet::one(S_COMP, q);
            cs.busy.add(S_COMP, q);
            cs.pin--;
        }
        if (red_bytes) c->dev.release(red_base, red_bytes, FenceSet::one(S_COMP, q));
        if (scratch_bytes) c->dev.release(scratch_base, scratch_bytes, FenceSet::one(S_COMP, q));
    }
    return LT_OK;
}

// ---------------------------------------------------------------- batches
struct BatchShape {
    struct Jac {
        lt_array *u, *v;
        int repeat;
    };
    struct Hist {
        lt_array *x, *h;
    };
    std::vector<Jac> jac;
    std::vector<Hist> hist;
};

// Tables of one fused batch for tile height th and histogram slice hs;
// `iters_cap` > 0 limits every instance to that many iterations (tuning).
static void batch_tables(lt_ctx *c, const BatchShape &bs, int th, int hs, int iters_cap,
                         std::vector<BatchJacobi> *jac, std::vector<BatchHist> *hist, std::vector<BatchItem> *items,
                         size_t *ncounters, bool stall = false) {
    jac->clear();
    hist->clear();
    items->clear();
    uint32_t done = 0;
    int rmax = 0;
    for (size_t q = 0; q < bs.jac.size(); ++q) {
        const auto &J = bs.jac[q];
        const ArrayGeom &g = J.u->g;
        const ChunkGeom &cu = g.chunks[0], &cv = J.v->g.chunks[0];
        BatchJacobi b{};
        b.u = (uint64_t)(uintptr_t)(dptr(c, J.u->cs[0].off));
        b.v = (uint64_t)(uintptr_t)(dptr(c, J.v->cs[0].off));
        b.su = cu.stride[0];
        b.sv = cv.stride[0];
        b.ny = g.shape[0];
        b.nx = g.shape[1];
        b.tiles = (uint32_t)((g.shape[0] + th - 1) / th);
        b.done_off = done;
        int r = iters_cap > 0 ? std::min(iters_cap, J.repeat) : J.repeat;
        done += (uint32_t)r;
        rmax = std::max(rmax, r);
        jac->push_back(b);
    }
    for (size_t h = 0; h < bs.hist.size(); ++h) {
        BatchHist b{};
        b.x = (uint64_t)(uintptr_t)(dptr(c, bs.hist[h].x->cs[0].off));
        b.len = bs.hist[h].x->g.shape[0];
        b.h = (uint64_t)(uintptr_t)(dptr(c, bs.hist[h].h->cs[0].off));
        hist->push_back(b);
        int64_t ns = (b.len + hs - 1) / hs;
        for (int64_t k = 0; k < ns; ++k) items->push_back({(1u << 30) | (uint32_t)h, 0u, (uint32_t)k, 0u});
    }
    for (int t = 0; t < rmax; ++t)
        for (size_t q = 0; q < bs.jac.size(); ++q) {
            int r = iters_cap > 0 ? std::min(iters_cap, bs.jac[q].repeat) : bs.jac[q].repeat;
            if (t >= r) continue;
            if (stall && t == 0 && r >= 2) continue;  // test hook: iteration 1 then waits forever (bounded)
            const BatchJacobi &b = (*jac)[q];
            for (uint32_t k = 0; k < b.tiles; ++k)
                items->push_back({(uint32_t)q, (uint32_t)t, k * (uint32_t)th,
                                  (uint32_t)std::min<int64_t>(th, b.ny - (int64_t)k * th)});
        }
    *ncounters = (size_t)done + 2;  // + queue head + abort flag
}

// Upload the tables into a fresh device block; fills cache fields.
static lt_status batch_upload(lt_ctx *c, BatchCache *bc, const std::vector<BatchJacobi> &jac,
                              const std::vector<BatchHist> &hist, const std::vector<BatchItem> &items,
                              size_t ncounters) {
    size_t o_jac = 0, o_hist = align_up(jac.size() * sizeof(BatchJacobi), 256);
    size_t o_items = o_hist + align_up(hist.size() * sizeof(BatchHist), 256);
    size_t o_cnt = o_items + align_up(items.size() * sizeof(BatchItem), 256);
    size_t total = o_cnt + align_up(ncounters * 4, 256);
    FenceSet f;
    lt_status st = dev_alloc(c, total, &bc->off, &f);
    if (st) return st;
    bc->bytes = total;
    if ((st = sync_all(c))) return st;  // the block's previous users are done
    char *base = dptr(c, bc->off);
    if (!jac.empty()) CK(c, cudaMemcpy(base + o_jac, jac.data(), jac.size() * sizeof(BatchJacobi), cudaMemcpyHostToDevice));
    if (!hist.empty()) CK(c, cudaMemcpy(base + o_hist, hist.data(), hist.size() * sizeof(BatchHist), cudaMemcpyHostToDevice));
    if (!items.empty())
        CK(c, cudaMemcpy(base + o_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    BatchParams &bp = bc->bp;
    bp.items = (const BatchItem *)(base + o_items);
    bp.nitems = items.size();
    bp.jac = (const BatchJacobi *)(base + o_jac);
    bp.hist = (const BatchHist *)(base + o_hist);
    bp.head = (uint32_t *)(base + o_cnt);
    bp.abort = (uint32_t *)(base + o_cnt + 4);
    bp.done = (uint32_t *)(base + o_cnt + 8);
    bp.err = c->err_word;
    bc->dev_hist = bp.hist;
    bc->nhist = (int)hist.size();
    bc->counters_off = o_cnt;
    bc->counters_bytes = ncounters * 4;
    return LT_OK;
}

// The work of one run on stream st: zero counters and histograms, run the queue.
static cudaError_t batch_enqueue(lt_ctx *c, const BatchCache &bc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(dptr(c, bc.off + bc.counters_off), 0, bc.counters_bytes, st);
    if (e == cudaSuccess) e = k::launch_batch_zero_hist(bc.dev_hist, bc.nhist, st);
    if (e == cudaSuccess && bc.bp.nitems) e = k::launch_batch(bc.bp, bc.ctas, st);
    return e;
}

static lt_status batch_plain(lt_ctx *c, const lt_launch_desc *d, int32_t n) {
    lt_status st;
    for (int32_t i = 0; i < n; ++i) {
        std::vector<lt_arg> a(d[i].args, d[i].args + d[i].nargs);
        std::vector<int> arr;
        lt_kernel *k = d[i].kernel;
        for (int32_t p = 0; p < d[i].nargs; ++p)
            if (k->params[(size_t)p].is_array) arr.push_back(p);
        for (int32_t r = 0; r < d[i].repeat; ++r) {
            if ((st = lt_launch(c, k, d[i].grid, d[i].block, &d[i].wd, a.data(), d[i].nargs))) return st;
            if (arr.size() >= 2) std::swap(a[(size_t)arr[0]].array, a[(size_t)arr[1]].array);
        }
    }
    c->stats.batches_plain++;
    return LT_OK;
}

lt_status lt_launch_batch(lt_ctx *c, const lt_launch_desc *d, int32_t n, int32_t flags) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if (n < 0 || (n && !d)) return fail(LT_ERR_INVALID_ARG, "bad batch");
    for (int32_t i = 0; i < n; ++i) {
        if (!d[i].kernel || !find_kernel(c, d[i].kernel) || d[i].repeat < 1 ||
            d[i].nargs != (int32_t)d[i].kernel->params.size() || (d[i].nargs && !d[i].args))
            return fail(LT_ERR_INVALID_ARG, "bad launch descriptor " + std::to_string(i));
    }
    // eligibility of the fused form
    BatchShape bs;
    bool fused = !(flags & LT_BATCH_PLAIN) && !c->dry && n > 0;
    std::unordered_set<const lt_array *> seen;
    for (int32_t i = 0; i < n && fused; ++i) {
        lt_kernel *k = d[i].kernel;
        std::vector<lt_array *> arrs;
        for (int32_t p = 0; p < d[i].nargs; ++p)
            if (k->params[(size_t)p].is_array) arrs.push_back(find_array(c, d[i].args[p].array));
        for (lt_array *a : arrs) {
            if (!a || a->cs.size() != 1 || !seen.insert(a).second) fused = false;
        }
        if (!fused) break;
        if (k->def->id == LT_K_JACOBI2D && arrs.size() == 2 && arrs[0] != arrs[1] &&
            arrs[0]->g.shape[0] == arrs[1]->g.shape[0] && arrs[0]->g.shape[1] == arrs[1]->g.shape[1] &&
            d[i].grid.x >= (uint64_t)arrs[0]->g.shape[1] && d[i].grid.y >= (uint64_t)arrs[0]->g.shape[0])
            bs.jac.push_back({arrs[0], arrs[1], d[i].repeat});
        else if (k->def->id == LT_K_HIST256 && arrs.size() == 2 && arrs[1]->g.shape[0] == 256 && d[i].repeat == 1 &&
                 d[i].grid.x >= (uint64_t)arrs[0]->g.shape[0])
            bs.hist.push_back({arrs[0], arrs[1]});
        else
            fused = false;
    }
    if (!fused) return batch_plain(c, d, n);
    // The plain form validates annotations per launch; the fused form checks
    // each launch once and skips the check while the batch repeats exactly
    // (same kernels, grids, blocks, superblocks, arguments and repeats; array
    // ids are never reused).
    std::vector<uint64_t> chk;
    chk.reserve((size_t)n * 16);
    for (int32_t i = 0; i < n; ++i) {
        const lt_launch_desc &e = d[i];
        chk.insert(chk.end(), {(uint64_t)(uintptr_t)e.kernel, e.grid.x, e.grid.y, e.grid.z, e.block.x, e.block.y,
                               e.block.z, (uint64_t)e.wd.superblock[0], (uint64_t)e.wd.superblock[1],
                               (uint64_t)e.wd.superblock[2], (uint64_t)e.repeat, (uint64_t)e.nargs});
        for (int32_t p = 0; p < e.nargs; ++p) {
            uint64_t fb;
            std::memcpy(&fb, &e.args[p].f, sizeof fb);
            const lt_array *a = e.kernel->params[(size_t)p].is_array ? find_array(c, e.args[p].array) : nullptr;
            chk.insert(chk.end(), {a ? (uint64_t)a->id : ~0ull, fb, (uint64_t)e.args[p].i});
        }
    }
    if (chk != c->batch_checked) {
        c->batch_checked.clear();
        for (int32_t i = 0; i < n; ++i) {
            std::shared_ptr<const PlanBundle> b;
            std::vector<lt_array *> parr;
            if ((st = prepare_plan(c, d[i].kernel, d[i].grid, d[i].block, &d[i].wd, d[i].args, d[i].nargs, &b, &parr)))
                return st;
        }
        c->batch_checked = std::move(chk);
    }
    if ((st = flush_pending(c))) return st;
    ++c->launch_id;
    c->stats.launches++;
    // stage: outputs (V, H) are overwritten unread; inputs keep their data
    std::vector<std::pair<lt_array *, bool>> uses;  // (array, written)
    for (auto &J : bs.jac) {
        uses.push_back({J.u, true});
        uses.push_back({J.v, true});
        J.v->cs[0].dead_launch = c->launch_id;
        J.u->cs[0].discarded = false;  // both buffers of an instance are written (ping-pong)
        J.v->cs[0].discarded = false;
    }
    for (auto &H : bs.hist) {
        uses.push_back({H.x, false});
        uses.push_back({H.h, true});
        H.h->cs[0].dead_launch = c->launch_id;
        H.h->cs[0].discarded = false;
    }
    for (auto &u : uses) u.first->cs[0].pin++;
    auto unpin = [&]() {
        for (auto &u : uses) u.first->cs[0].pin--;
    };
    for (auto &u : uses)
        if ((st = ensure_dev(c, u.first, 0, true))) {
            unpin();
            return st;
        }
    // cache key: arrays, their device offsets and repeats
    std::vector<uint64_t> key;
    for (auto &J : bs.jac) key.insert(key.end(), {(uint64_t)J.u->id, J.u->cs[0].off, (uint64_t)J.v->id, J.v->cs[0].off,
                                                  (uint64_t)J.repeat});
    key.push_back(~0ull);
    for (auto &H : bs.hist) key.insert(key.end(), {(uint64_t)H.x->id, H.x->cs[0].off, (uint64_t)H.h->id, H.h->cs[0].off});
    const bool stall = (flags & LT_BATCH_TEST_STALL) != 0;
    if (stall) key.push_back(0x57A11ull);  // never matches a real batch
    bool use_graph = !(flags & LT_BATCH_NO_GRAPH) && !stall;
    std::pair<int64_t, int64_t> shape_key = {(int64_t)bs.jac.size(), (int64_t)bs.hist.size()};
    if (!c->batch || c->batch->key != key || (flags & LT_BATCH_RETUNE) || (use_graph && !c->batch->exec)) {
        if (c->batch) {
            if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
            c->dev.release(c->batch->off, c->batch->bytes, FenceSet::one(S_COMP, c->seq[S_COMP]));
            c->batch.reset();
        }
        int sms = 0, dev = 0;
        CK(c, cudaGetDevice(&dev));
        CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        std::vector<BatchJacobi> jac;
        std::vector<BatchHist> hist;
        std::vector<BatchItem> items;
        size_t ncnt = 0;
        // autotuner: time every candidate on the first iteration of the batch
        // (it writes only V and H, which the real run overwrites)
        if (stall && !c->tuned.count(shape_key)) c->tuned[shape_key] = {32, 256 << 10};
        if (!c->tuned.count(shape_key) || (flags & LT_BATCH_RETUNE)) {
            if ((st = sync_all(c))) {
                unpin();
                return st;
            }
            const int ths[] = {16, 32, 64, 128};
            const int hss[] = {64 << 10, 256 << 10, 1 << 20};
            float best = 1e30f;
            std::pair<int, int> pick = {32, 256 << 10};
            cudaEvent_t e0, e1;
            CK(c, cudaEventCreate(&e0));
            CK(c, cudaEventCreate(&e1));
            for (int th : ths)
                for (int hs : hss) {
                    if (bs.hist.empty() && hs != hss[0]) continue;
                    if (bs.jac.empty() && th != ths[0]) continue;
                    batch_tables(c, bs, th, hs, 1, &jac, &hist, &items, &ncnt);
                    BatchCache tc;
                    if ((st = batch_upload(c, &tc, jac, hist, items, ncnt))) {
                        unpin();
                        return st;
                    }
                    tc.bp.hist_slice = hs;
                    tc.ctas = sms * k::batch_ctas_per_sm();
                    CK(c, cudaEventRecord(e0, c->st[S_COMP]));
                    CK(c, batch_enqueue(c, tc, c->st[S_COMP]));
                    CK(c, cudaEventRecord(e1, c->st[S_COMP]));
                    CK(c, cudaEventSynchronize(e1));
                    float ms = 0;
                    CK(c, cudaEventElapsedTime(&ms, e0, e1));
                    c->stats.kernels += 2;
                    if (ms < best) {
                        best = ms;
                        pick = {th, hs};
                    }
                    c->dev.release(tc.off, tc.bytes, FenceSet());
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if ((st = sync_all(c))) {
                unpin();
                return st;
            }
            c->tuned[shape_key] = pick;
        }
        auto tp = c->tuned[shape_key];
        auto bc = std::make_unique<BatchCache>();
        bc->key = key;
        batch_tables(c, bs, tp.first, tp.second, 0, &jac, &hist, &items, &ncnt, stall);
        if ((st = batch_upload(c, bc.get(), jac, hist, items, ncnt))) {
            unpin();
            return st;
        }
        bc->bp.hist_slice = tp.second;
        bc->ctas = sms * k::batch_ctas_per_sm();
        if (use_graph) {
            cudaGraph_t graph = nullptr;
            CK(c, cudaStreamBeginCapture(c->st[S_COMP], cudaStreamCaptureModeThreadLocal));
            cudaError_t e = batch_enqueue(c, *bc, c->st[S_COMP]);
            cudaError_t e2 = cudaStreamEndCapture(c->st[S_COMP], &graph);
            CK(c, e);
            CK(c, e2);
            cudaError_t e3 = cudaGraphInstantiate(&bc->exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(c, e3);
        }
        c->batch = std::move(bc);
    } else if (use_graph) {
        c->stats.graph_replays++;
    }
    c->stats.tuned_tile_rows = c->tuned[shape_key].first;
    c->stats.tuned_hist_slice = c->tuned[shape_key].second;
    // run: wait for every staged chunk, then the graph (or the kernels)
    op_begin(c, S_COMP, "batch");
    FenceSet w;
    for (auto &u : uses) {
        w.merge(u.first->cs[0].ready);
        w.merge(u.first->cs[0].busy);
    }
    if ((st = op_wait(c, w))) {
        unpin();
        return st;
    }
    {
        TimeScope ts(c, CAT_EXEC);
        if (use_graph)
            CK(c, cudaGraphLaunch(c->batch->exec, c->st[S_COMP]));
        else
            CK(c, batch_enqueue(c, *c->batch, c->st[S_COMP]));
    }
    c->stats.kernels += 2;
    uint64_t q;
    if ((st = op_end(c, &q))) {
        unpin();
        return st;
    }
    for (auto &u : uses) {
        CState &cs = u.first->cs[0];
        if (u.second) cs.ready = FenceSet::one(S_COMP, q);
        cs.busy.add(S_COMP, q);
    }
    unpin();
    c->stats.batches_fused++;
    size_t tasks = 0;
    for (auto &J : bs.jac) tasks += (size_t)J.repeat;
    c->stats.tasks_execute += tasks + bs.hist.size();
    return LT_OK;
}

lt_status lt_synchronize(lt_ctx *c) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    return sync_all(c);
}

lt_status lt_array_discard(lt_ctx *c, lt_array *arr) {
    lt_status st = check_ctx(c);
    if (st) return st;
    lt_array *a = find_array(c, arr);
    if (!a) return fail(LT_ERR_INVALID_ARG, "unknown array");
    // No flush: the pending launch (if any) still reads the array; its chunks
    // become droppable as that launch finishes with each of them.
    for (auto &s : a->cs)
        if (!s.ext) s.discarded = true;
    return LT_OK;
}

lt_status lt_op_timing(lt_ctx *c, int32_t on) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    if (on)
        c->cfg.flags |= LT_FLAG_TIMING;
    else
        c->cfg.flags &= ~(int32_t)LT_FLAG_TIMING;
    return LT_OK;
}

lt_status lt_timer_start(lt_ctx *c) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    if (c->dry) return LT_OK;
    for (int i = 0; i < 2; ++i) {
        if (!c->timer[i]) CK(c, cudaEventCreate(&c->timer[i]));
        if (!c->timer_join[i]) CK(c, cudaEventCreateWithFlags(&c->timer_join[i], cudaEventDisableTiming));
    }
    CK(c, cudaEventRecord(c->timer[0], c->st[S_COMP]));
    CK(c, cudaStreamWaitEvent(c->st[S_H2D], c->timer[0], 0));
    CK(c, cudaStreamWaitEvent(c->st[S_D2H], c->timer[0], 0));
    return LT_OK;
}

lt_status lt_timer_stop(lt_ctx *c, double *ms) {
    lt_status st = check_ctx(c);
    if (st) return st;
    if ((st = flush_pending(c))) return st;
    if (!ms) return fail(LT_ERR_INVALID_ARG, "null output");
    *ms = 0.0;
    if (c->dry) return LT_OK;
    if (!c->timer[0]) return fail(LT_ERR_INVALID_ARG, "lt_timer_stop without lt_timer_start");
    CK(c, cudaEventRecord(c->timer_join[0], c->st[S_H2D]));
    CK(c, cudaEventRecord(c->timer_join[1], c->st[S_D2H]));
    CK(c, cudaStreamWaitEvent(c->st[S_COMP], c->timer_join[0], 0));
    CK(c, cudaStreamWaitEvent(c->st[S_COMP], c->timer_join[1], 0));
    CK(c, cudaEventRecord(c->timer[1], c->st[S_COMP]));
    CK(c, cudaEventSynchronize(c->timer[1]));
    float f = 0.f;
    CK(c, cudaEventElapsedTime(&f, c->timer[0], c->timer[1]));
    *ms = f;
    return LT_OK;
}

lt_status lt_stats_get(lt_ctx *c, lt_stats *out) {
    if (!c || !out) return fail(LT_ERR_INVALID_ARG, "null argument");
    if (!c->poisoned) {
        lt_status st = flush_pending(c);
        if (st) return st;
    }
    c->stats.hbm_in_use = c->dev.used;
    c->stats.hbm_peak = c->dev.peak;
    c->stats.host_in_use = c->host.used;
    *out = c->stats;
    return LT_OK;
}

lt_status lt_stats_reset(lt_ctx *c) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    c->stats = lt_stats{};
    c->dev.peak = c->dev.used;
    return LT_OK;
}

lt_status lt_debug_log_enable(lt_ctx *c, int32_t enable) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    c->log_on = enable != 0;
    c->log.str("");
    c->log.clear();
    c->log_n = 0;
    c->tlog.str("");
    c->tlog.clear();
    c->tlog_n = 0;
    c->tlog_base = 0;
    return LT_OK;
}

lt_status lt_debug_timeline(lt_ctx *c, char *buf, size_t cap, size_t *needed) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    std::string js = "[" + c->tlog.str() + "]";
    if (needed) *needed = js.size() + 1;
    if (buf && cap) {
        size_t n = std::min(cap - 1, js.size());
        std::memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return LT_OK;
}

lt_status lt_debug_log(lt_ctx *c, char *buf, size_t cap, size_t *needed) {
    if (!c) return fail(LT_ERR_INVALID_ARG, "null context");
    if (!c->poisoned) {
        lt_status st = flush_pending(c);
        if (st) return st;
    }
    std::string js = "[" + c->log.str() + "]";
    if (needed) *needed = js.size() + 1;
    if (buf && cap) {
        size_t n = std::min(cap - 1, js.size());
        std::memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return LT_OK;
}

}  // extern "C"
