// Runtime: chunk views, the HBM and pinned-host pools, eviction by class and
// Belady's choice, fetches, host transfers of array contents, and the
// tracking of chunks a launch overwrites unread (see rt.hpp).
#include "rt.hpp"

namespace lt {
namespace rt {

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

// Quarantine of slow host-pool ranges.  On the GB300 machines measured, a few
// 4 GiB stretches of a large pinned allocation copied to and from the GPU 2
// to 20 times slower than the rest, for the whole life of the process (not in
// the first process after the box started; which stretches differed from one
// process to the next, mostly at the start and the end of the allocation; a
// copy timed right after the allocation did not show it).  One such chunk in
// a streaming launch stalls the pipeline for hundreds of milliseconds.  So
// every fetch and eviction of at least 256 MiB is timed with two events; a
// copy that ran at less than half the fastest copy seen in its direction
// marks its host range bad, and the host pool withholds bad ranges from
// allocation (at once where they are free, else when their block is
// released), up to a quarter of the pool (lt_stats.host_withheld_bytes).
lt_status link_copy_timed(lt_ctx *c, int dir, void *dst, const void *src, size_t n, size_t host_off) {
    cudaStream_t st = c->st[dir == 0 ? S_H2D : S_D2H];
    const cudaMemcpyKind kind = dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    const bool probe = !c->no_quarantine && n >= ((size_t)256 << 20);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (probe) {
        for (auto &e : ev) {
            if (!c->link_ev_pool.empty()) {
                e = c->link_ev_pool.back();
                c->link_ev_pool.pop_back();
            } else {
                CK(c, cudaEventCreate(&e));
            }
        }
        CK(c, cudaEventRecord(ev[0], st));
    }
    CK(c, cudaMemcpyAsync(dst, src, n, kind, st));
    if (probe) {
        CK(c, cudaEventRecord(ev[1], st));
        c->link_probes.push_back({ev[0], ev[1], host_off, n, dir});
    }
    return LT_OK;
}

// Rate the timed copies that have finished; quarantine the slow ones' ranges.
lt_status link_poll(lt_ctx *c) {
    if (c->dry || c->link_probes.empty()) return LT_OK;
    std::vector<lt_ctx::LinkProbe> keep;
    std::vector<lt_ctx::LinkProbe> done;
    for (auto &pr : c->link_probes) {
        cudaError_t q = cudaEventQuery(pr.b);
        if (q == cudaErrorNotReady) {
            keep.push_back(pr);
            continue;
        }
        CK(c, q);
        done.push_back(pr);
    }
    c->link_probes.swap(keep);
    for (auto &pr : done) {
        float ms = 0;
        CK(c, cudaEventElapsedTime(&ms, pr.a, pr.b));
        c->link_ev_pool.push_back(pr.a);
        c->link_ev_pool.push_back(pr.b);
        const double rate = (double)pr.bytes / std::max(ms, 1e-3f);
        double &best = c->link_best[pr.dir];
        if (rate > best) best = rate;
        if (rate < 0.5 * best && c->host.withheld + pr.bytes <= c->host.cap / 4) {
            c->host.quarantine(pr.host_off, pr.bytes);
            c->stats.host_quarantined++;
        }
    }
    return LT_OK;
}

// ---------------------------------------------------------------- memory manager

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
lt_status dev_alloc(lt_ctx *c, size_t bytes, size_t *off, FenceSet *f, bool soft) {
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
    bool ok = c->host.alloc(cg.bytes, &hoff, &hf);
    if (!ok && c->host.withheld) {  // quarantine only while the pool can spare it
        c->host.release_quarantine();
        ok = c->host.alloc(cg.bytes, &hoff, &hf);
    }
    if (!ok)
        return fail(LT_ERR_OOM_HOST, "pinned host pool too small to evict a chunk of " + std::to_string(cg.bytes) +
                                         " bytes (host pool " + std::to_string(c->host.cap) + " bytes)");
    op_begin(c, S_D2H, "evict");
    FenceSet w = s.ready;
    w.merge(hf);
    lt_status st = op_wait(c, w);
    if (st) return st;
    if (!c->dry) {
        TimeScope ts(c, CAT_D2H);
        if ((st = link_poll(c))) return st;
        if ((st = link_copy_timed(c, 1, c->host_base + hoff, dptr(c, s.off), cg.bytes, hoff))) return st;
    }
    uint64_t q;
    std::ostringstream ex;
    ex << ",\"array\":" << a->id << ",\"chunk\":" << ci << ",\"bytes\":" << cg.bytes << ",\"host_off\":" << hoff
       << ",\"dev_off\":" << s.off;
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
lt_status ensure_dev(lt_ctx *c, lt_array *a, int64_t ci, bool need_data, bool soft) {
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
                if ((st = link_poll(c))) return st;
                if ((st = link_copy_timed(c, 0, dptr(c, off), c->host_base + s.off, cg.bytes, s.off))) return st;
            }
            uint64_t q;
            std::ostringstream ex;
            ex << ",\"array\":" << a->id << ",\"chunk\":" << ci << ",\"bytes\":" << cg.bytes
               << ",\"host_off\":" << s.off << ",\"dev_off\":" << off;
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
// ---------------------------------------------------------------- host transfers
// Copy between the dense row-major host buffer `hb` (whole array) and the
// part `box` of chunk ci that lives in device memory.
lt_status xfer_chunk(lt_ctx *c, lt_array *a, int64_t ci, const Box &box, char *hb, bool to_dev,
                     bool other_is_device, int stream, bool wait) {
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
    cudaStream_t st = c->st[stream];
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
        if (wait) CK(c, cudaStreamSynchronize(st));
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
    if (wait) CK(c, cudaStreamSynchronize(st));
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

}  // namespace rt
}  // namespace lt
