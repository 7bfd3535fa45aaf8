// Runtime: error messages, stream-ordered fences, per-operation timing and
// the descriptor-table upload ring (see rt.hpp for the file map).
#include "rt.hpp"

namespace lt {
namespace rt {

static thread_local std::string g_err;

lt_status fail(lt_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

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

// The event that marks fence (t, q) complete, or null when the operation is
// known to be complete (its event slot was reused, which the bounded run-ahead
// allows only after that event completed, or a synchronize passed it).  A
// deferred fence maps to the event of a later operation on the same stream;
// if none has been recorded yet and `flush` is set, one is recorded now (it
// fires after everything enqueued on stream t so far: a later point than the
// fence, which is safe).  *task: the operation's task id (for the log).
cudaEvent_t fence_event(lt_ctx *c, int t, uint64_t q, int64_t *task, bool flush) {
    const int slot = (int)(q % RING);
    *task = -1;
    if (c->evseq[t][slot] == q) {
        *task = c->evtask[t][slot];
        return c->ev[t][slot];
    }
    if (c->dfseq[t][slot] != q) return nullptr;
    *task = c->dftask[t][slot];
    uint64_t cov = c->dfcov[t][slot];
    if (cov == ~(uint64_t)0) return nullptr;
    if (cov == 0) {
        if (!flush || c->dry) return nullptr;
        // cover every deferred fence of stream t with one event in the ring
        // slot of the newest of them (a slot its own deferral left unused)
        const uint64_t last = c->deferred[t].back();
        const int ls = (int)(last % RING);
        if (c->evseq[t][ls] != 0 && cudaEventSynchronize(c->ev[t][ls]) != cudaSuccess) return nullptr;
        if (cudaEventRecord(c->ev[t][ls], c->st[t]) != cudaSuccess) return nullptr;
        c->evseq[t][ls] = last;
        c->evtask[t][ls] = c->dftask[t][ls];
        for (uint64_t d : c->deferred[t]) c->dfcov[t][d % RING] = last;
        c->deferred[t].clear();
        cov = last;
    }
    const int cs = (int)(cov % RING);
    return c->evseq[t][cs] == cov ? c->ev[t][cs] : nullptr;
}

lt_status op_wait(lt_ctx *c, const FenceSet &f) {
    int s = c->cur_stream;
    for (int t = 0; t < NSTREAM; ++t) {
        uint64_t q = f.q[t];
        if (!q) continue;
        int64_t pt = -1;
        // a fence on the waiting stream itself needs no event (stream order)
        cudaEvent_t e = fence_event(c, t, q, &pt, t != s);
        if (pt >= 0 && (e || t == s || c->dry) &&
            std::find(c->cur_deps.begin(), c->cur_deps.end(), pt) == c->cur_deps.end()) {
            c->cur_deps.push_back(pt);
            c->stats.deps++;
        }
        if (t == s || c->dry || !e) continue;
        CK(c, cudaStreamWaitEvent(c->st[s], e, 0));
    }
    return LT_OK;
}

// Finish the current operation: record its fence on its stream.  defer: do
// not record an event now (see lt_ctx::deferred); a later operation's event,
// or one recorded when something waits for this fence, stands for it.
lt_status op_end(lt_ctx *c, uint64_t *out_seq, const std::string &extra, bool defer) {
    int s = c->cur_stream;
    uint64_t q = ++c->seq[s];
    int slot = (int)(q % RING);
    if (c->dry) defer = false;  // dry runs keep the plain bookkeeping the host-logic tests inspect
    if (defer && c->deferred[s].size() >= RING / 2) defer = false;
    if (defer) {
        c->dfseq[s][slot] = q;
        c->dfcov[s][slot] = 0;
        c->dftask[s][slot] = c->cur_task;
        c->deferred[s].push_back(q);
    } else {
        if (!c->dry) {
            if (c->evseq[s][slot] != 0) CK(c, cudaEventSynchronize(c->ev[s][slot]));  // bounded run-ahead
            CK(c, cudaEventRecord(c->ev[s][slot], c->st[s]));
        }
        c->evseq[s][slot] = q;
        c->evtask[s][slot] = c->cur_task;
        for (uint64_t d : c->deferred[s]) c->dfcov[s][d % RING] = q;  // this event fires after them
        c->deferred[s].clear();
    }
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
    int64_t task;
    cudaEvent_t e = fence_event(c, s, q, &task, true);
    if (e) CK(c, cudaEventSynchronize(e));
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

// Upload a descriptor table for the next compute-stream kernel.
// Descriptor tables that repeat (iterative launches over resident chunks
// plan the same tasks, views and copy pieces every time) stay on the device:
// a table whose bytes equal a resident slot is used in place, with no
// host-to-device copy.  Every kernel that reads a table runs on the compute
// stream, as does the copy that refills a slot, so stream order keeps a
// slot's earlier readers ahead of its new contents; the slot's event keeps
// its pinned staging bytes until that copy has run.

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
    // Every kernel that can record an error runs on the compute stream, so a
    // copy of the error word queued there behind them lands in pinned host
    // memory by the time that stream is idle: no separate round trip.
    CK(c, cudaMemcpyAsync(c->err_host, c->err_word, 4, cudaMemcpyDeviceToHost, c->st[S_COMP]));
    for (int s = 0; s < NSTREAM; ++s) CK(c, cudaStreamSynchronize(c->st[s]));
    if (lt_status lp = link_poll(c)) return lp;
    for (int s = 0; s < NSTREAM; ++s) {  // every deferred fence is complete now
        for (uint64_t d : c->deferred[s]) c->dfcov[s][d % RING] = ~(uint64_t)0;
        c->deferred[s].clear();
    }
    const uint32_t e = *(volatile uint32_t *)c->err_host;
    if (e) {
        CK(c, cudaMemset(c->err_word, 0, 4));
        return fail(e >= 0x6700 && e < 0x6900 ? LT_ERR_TIMEOUT : LT_ERR_DEVICE_CHECK,
                    "a kernel recorded an error (code " + std::to_string(e) +
                        "; 0x67xx / 0x68xx = a bounded wait expired and the kernel returned)");
    }
    return collect_timing(c);
}

}  // namespace rt
}  // namespace lt

const char *lt::rt::last_error_text() { return g_err.c_str(); }
extern "C" const char *lt_last_error(void) { return lt::rt::last_error_text(); }

lt_status lt::set_last_error(lt_status st, const std::string &msg) { return lt::rt::fail(st, msg); }
