// Runtime: fused batches of launches (one persistent kernel over a device
// work queue), their CUDA graphs and the autotuner; see rt.hpp.
#include "rt.hpp"

extern "C" {

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


}  // extern "C"
