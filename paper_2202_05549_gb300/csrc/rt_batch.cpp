// Runtime: fused batches of launches (one persistent kernel over a device
// work queue), their CUDA graphs and the autotuner; see rt.hpp.
#include "rt.hpp"

extern "C" {

// ---------------------------------------------------------------- batches
// Tables of one fused batch for tiles of th rows by tw columns (0: the
// part's width) and histogram slice hs; `iters_cap` > 0 limits every
// instance to that many iterations (tuning).
// A Jacobi instance becomes one part per superblock of its launch (one chunk
// of each buffer) and one replica table entry per halo box its parts keep
// current; both buffers share the distribution, so the same chunks serve
// when they swap roles.
static void batch_tables(lt_ctx *c, const BatchShape &bs, int th, int tw, int hs, int iters_cap,
                         std::vector<BatchJacobi> *jac, std::vector<BatchHist> *hist, std::vector<BatchRep> *reps,
                         std::vector<BatchItem> *items, size_t *ncounters, bool stall = false) {
    jac->clear();
    hist->clear();
    reps->clear();
    items->clear();
    constexpr uint32_t REP_CELLS = 2048;  // replica cells per work item
    struct Inst {
        uint32_t part0, nparts, rep0, nreps, per_iter;
        int repeat;
    };
    std::vector<Inst> inst;
    uint32_t done = 0;
    int rmax = 0;
    for (size_t q = 0; q < bs.jac.size(); ++q) {
        const auto &J = bs.jac[q];
        const ArrayGeom &g = J.u->g;
        Inst in{(uint32_t)jac->size(), 0, (uint32_t)reps->size(), 0, 0, 0};
        for (const auto &sb : J.plan->plan.sbs) {
            const ArgPlan *au = nullptr, *av = nullptr;
            for (const auto &ap : sb.args) {
                if (ap.kind != ARG_DIRECT) continue;
                if (ap.mode == MODE_READ) au = &ap; else av = &ap;
            }
            BatchJacobi b{};
            const int64_t cu = au->chunk, cv = av->chunk;
            b.u = view_of(c, g, g.chunks[(size_t)cu], J.u->cs[(size_t)cu].off).base;
            b.v = view_of(c, J.v->g, J.v->g.chunks[(size_t)cv], J.v->cs[(size_t)cv].off).base;
            b.su = g.chunks[(size_t)cu].stride[0];
            b.sv = J.v->g.chunks[(size_t)cv].stride[0];
            b.ny = g.shape[0];
            b.nx = g.shape[1];
            b.y0 = sb.threads.lo[1];
            b.y1 = std::min<int64_t>(sb.threads.hi[1], g.shape[0] - 1);
            b.x0 = sb.threads.lo[0];
            b.x1 = std::min<int64_t>(sb.threads.hi[0], g.shape[1] - 1);
            b.done_off = done;
            const uint32_t part = (uint32_t)jac->size();
            jac->push_back(b);
            in.nparts++;
            const int64_t pw = b.x1 - b.x0 + 1;
            in.per_iter += (uint32_t)((b.y1 - b.y0 + th) / th) * (uint32_t)(tw ? (pw + tw - 1) / tw : 1);
            for (const auto &pc : av->replicas) {
                BatchRep r{};
                const int64_t cj = pc.chunk;
                r.du = view_of(c, g, g.chunks[(size_t)cj], J.u->cs[(size_t)cj].off).base;
                r.dv = view_of(c, J.v->g, J.v->g.chunks[(size_t)cj], J.v->cs[(size_t)cj].off).base;
                r.sdu = g.chunks[(size_t)cj].stride[0];
                r.sdv = J.v->g.chunks[(size_t)cj].stride[0];
                for (int d = 0; d < 2; ++d) {
                    r.lo[d] = pc.box.lo[d];
                    r.hi[d] = pc.box.hi[d];
                }
                r.part = part;
                reps->push_back(r);
                in.nreps++;
                in.per_iter += (uint32_t)((pc.box.volume() + REP_CELLS - 1) / REP_CELLS);
            }
        }
        for (uint32_t i = 0; i < in.nparts; ++i) (*jac)[in.part0 + i].tiles = in.per_iter;
        in.repeat = iters_cap > 0 ? std::min(iters_cap, J.repeat) : J.repeat;
        done += (uint32_t)in.repeat;
        rmax = std::max(rmax, in.repeat);
        inst.push_back(in);
    }
    for (size_t h = 0; h < bs.hist.size(); ++h) {
        BatchHist b{};
        b.x = (uint64_t)(uintptr_t)(dptr(c, bs.hist[h].x->cs[0].off));
        b.len = bs.hist[h].x->g.shape[0];
        b.h = (uint64_t)(uintptr_t)(dptr(c, bs.hist[h].h->cs[0].off));
        hist->push_back(b);
        int64_t ns = (b.len + hs - 1) / hs;
        for (int64_t k = 0; k < ns; ++k) items->push_back({(1u << 30) | (uint32_t)h, 0u, (uint32_t)k, 0u, 0u, 0u});
    }
    for (int t = 0; t < rmax; ++t)
        for (const Inst &in : inst) {
            if (t >= in.repeat) continue;
            if (stall && t == 0 && in.repeat >= 2) continue;  // test hook: iteration 1 then waits forever (bounded)
            for (uint32_t p = in.part0; p < in.part0 + in.nparts; ++p) {
                const BatchJacobi &b = (*jac)[p];
                const int64_t pw = b.x1 - b.x0 + 1;
                for (int64_t r = b.y0; r <= b.y1; r += th)
                    for (int64_t c0 = 0; c0 < pw; c0 += tw ? tw : pw)
                        items->push_back({p, (uint32_t)t, (uint32_t)r, (uint32_t)std::min<int64_t>(th, b.y1 - r + 1),
                                          (uint32_t)c0, (uint32_t)(tw ? tw : 0)});
            }
            for (uint32_t ri = in.rep0; ri < in.rep0 + in.nreps; ++ri) {
                const BatchRep &r = (*reps)[ri];
                const uint64_t cells = (uint64_t)(r.hi[0] - r.lo[0] + 1) * (uint64_t)(r.hi[1] - r.lo[1] + 1);
                for (uint64_t e = 0; e < cells; e += REP_CELLS)
                    items->push_back({(2u << 30) | ri, (uint32_t)t, (uint32_t)e,
                                      (uint32_t)std::min<uint64_t>(REP_CELLS, cells - e), 0u, 0u});
            }
        }
    *ncounters = (size_t)done + 2;  // + queue head + abort flag
}

// Upload the tables into a fresh device block; fills cache fields.
static lt_status batch_upload(lt_ctx *c, BatchCache *bc, const std::vector<BatchJacobi> &jac,
                              const std::vector<BatchHist> &hist, const std::vector<BatchRep> &reps,
                              const std::vector<BatchItem> &items, size_t ncounters) {
    size_t o_jac = 0, o_hist = align_up(jac.size() * sizeof(BatchJacobi), 256);
    size_t o_reps = o_hist + align_up(hist.size() * sizeof(BatchHist), 256);
    size_t o_items = o_reps + align_up(reps.size() * sizeof(BatchRep), 256);
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
    if (!reps.empty()) CK(c, cudaMemcpy(base + o_reps, reps.data(), reps.size() * sizeof(BatchRep), cudaMemcpyHostToDevice));
    if (!items.empty())
        CK(c, cudaMemcpy(base + o_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    BatchParams &bp = bc->bp;
    bp.items = (const BatchItem *)(base + o_items);
    bp.nitems = items.size();
    bp.jac = (const BatchJacobi *)(base + o_jac);
    bp.hist = (const BatchHist *)(base + o_hist);
    bp.reps = (const BatchRep *)(base + o_reps);
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
    const bool repeat_batch = chk == c->batch_checked && c->batch_shape;
    if (!repeat_batch) {
        c->batch_checked.clear();
        c->batch_shape.reset();
        for (int32_t i = 0; i < n; ++i) {
            std::shared_ptr<const PlanBundle> b;
            std::vector<lt_array *> parr;
            if ((st = prepare_plan(c, d[i].kernel, d[i].grid, d[i].block, &d[i].wd, d[i].args, d[i].nargs, &b, &parr)))
                return st;
        }
    }
    if (repeat_batch && !(flags & LT_BATCH_PLAIN)) {
        // an identical batch: its shape (and plans) are those of the last call
    } else if (repeat_batch) {
        return batch_plain(c, d, n);
    } else {
        // eligibility of the fused form: Jacobi instances whose two buffers share
        // one distribution and whose every superblock reads and writes a single
        // chunk of each (halo replicas are kept by the batch kernel), superblocks
        // starting on a multiple of 4 columns; histograms of one-chunk arrays
        auto shape = std::make_shared<BatchShape>();
        BatchShape &bs = *shape;
        bool fused = !(flags & LT_BATCH_PLAIN) && !c->dry && n > 0;
        std::unordered_set<const lt_array *> seen;
        auto same_dist = [](const ArrayGeom &a, const ArrayGeom &b) {
            if (a.nd != b.nd || a.dist.kind != b.dist.kind || a.dist.order != b.dist.order) return false;
            for (int x = 0; x < 3; ++x)
                if (a.shape[x] != b.shape[x] || a.dist.chunk[x] != b.dist.chunk[x] || a.dist.halo[x] != b.dist.halo[x])
                    return false;
            return true;
        };
        for (int32_t i = 0; i < n && fused; ++i) {
            lt_kernel *k = d[i].kernel;
            std::vector<lt_array *> arrs;
            for (int32_t p = 0; p < d[i].nargs; ++p)
                if (k->params[(size_t)p].is_array) arrs.push_back(find_array(c, d[i].args[p].array));
            for (lt_array *a : arrs) {
                if (!a || !seen.insert(a).second) fused = false;
            }
            if (!fused) break;
            if (k->def->id == LT_K_JACOBI2D && arrs.size() == 2 && arrs[0] != arrs[1] && same_dist(arrs[0]->g, arrs[1]->g) &&
                arrs[0]->g.dist.order == LT_ORDER_ROW && d[i].grid.x >= (uint64_t)arrs[0]->g.shape[1] &&
                d[i].grid.y >= (uint64_t)arrs[0]->g.shape[0]) {
                std::shared_ptr<const PlanBundle> b;
                std::vector<lt_array *> parr;
                if ((st = prepare_plan(c, k, d[i].grid, d[i].block, &d[i].wd, d[i].args, d[i].nargs, &b, &parr))) return st;
                for (const auto &sb : b->plan.sbs) {
                    int direct = 0;
                    for (const auto &ap : sb.args) {
                        if (ap.kind == ARG_VALUE || ap.kind == ARG_NONE) continue;
                        if (ap.kind != ARG_DIRECT) fused = false;
                        direct++;
                    }
                    if (direct != 2 || sb.threads.lo[0] % 4 != 0) fused = false;
                }
                if (fused) bs.jac.push_back({arrs[0], arrs[1], d[i].repeat, b});
            } else if (k->def->id == LT_K_HIST256 && arrs.size() == 2 && arrs[0]->cs.size() == 1 &&
                       arrs[1]->cs.size() == 1 && arrs[1]->g.shape[0] == 256 && d[i].repeat == 1 &&
                       d[i].grid.x >= (uint64_t)arrs[0]->g.shape[0]) {
                bs.hist.push_back({arrs[0], arrs[1]});
            } else {
                fused = false;
            }
        }
        if (!fused) return batch_plain(c, d, n);
        c->batch_checked = std::move(chk);
        c->batch_shape = shape;
    }
    const BatchShape &bs = *c->batch_shape;

    if ((st = flush_pending(c))) return st;
    ++c->launch_id;
    c->stats.launches++;
    // stage every chunk: outputs (V, H) are overwritten unread (V's halos
    // by the replica items); inputs keep their data
    struct Use {
        lt_array *a;
        int64_t ci;
        bool written;
    };
    std::vector<Use> uses;
    for (auto &J : bs.jac) {
        for (int64_t ci = 0; ci < (int64_t)J.u->cs.size(); ++ci) {
            uses.push_back({J.u, ci, true});
            uses.push_back({J.v, ci, true});
            J.v->cs[(size_t)ci].dead_launch = c->launch_id;
            J.u->cs[(size_t)ci].discarded = false;  // both buffers of an instance are written (ping-pong)
            J.v->cs[(size_t)ci].discarded = false;
        }
    }
    for (auto &H : bs.hist) {
        uses.push_back({H.x, 0, false});
        uses.push_back({H.h, 0, true});
        H.h->cs[0].dead_launch = c->launch_id;
        H.h->cs[0].discarded = false;
    }
    for (auto &u : uses) u.a->cs[(size_t)u.ci].pin++;
    auto unpin = [&]() {
        for (auto &u : uses) u.a->cs[(size_t)u.ci].pin--;
    };
    for (auto &u : uses)
        if ((st = ensure_dev(c, u.a, u.ci, true))) {
            unpin();
            return st;
        }
    // cache key: arrays, the device offsets of their chunks, repeats and plans
    std::vector<uint64_t> key;
    for (auto &J : bs.jac) {
        key.insert(key.end(), {(uint64_t)J.u->id, (uint64_t)J.v->id, (uint64_t)J.repeat,
                               (uint64_t)(uintptr_t)J.plan.get()});
        for (size_t ci = 0; ci < J.u->cs.size(); ++ci) key.insert(key.end(), {J.u->cs[ci].off, J.v->cs[ci].off});
    }
    key.push_back(~0ull);
    for (auto &H : bs.hist) key.insert(key.end(), {(uint64_t)H.x->id, H.x->cs[0].off, (uint64_t)H.h->id, H.h->cs[0].off});
    const bool stall = (flags & LT_BATCH_TEST_STALL) != 0;
    const bool force_cols = (flags & LT_BATCH_TEST_TILE_COLS) != 0;
    if (stall) key.push_back(0x57A11ull);  // never matches a real batch
    if (force_cols) key.push_back(0xC015ull);
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
        std::vector<BatchRep> reps;
        std::vector<BatchItem> items;
        size_t ncnt = 0;
        // autotuner: time every candidate on the first iteration of the batch
        // (it writes only V and H, which the real run overwrites)
        if (stall && !c->tuned.count(shape_key)) c->tuned[shape_key] = {32, 0, 256 << 10};
        if (!c->tuned.count(shape_key) || (flags & LT_BATCH_RETUNE)) {
            if ((st = sync_all(c))) {
                unpin();
                return st;
            }
            // work-item shapes: tile rows, tile columns (0: a part's full width) and histogram slice
            const int ths[] = {16, 32, 64, 128};
            const int tws[] = {0, 1024};
            const int hss[] = {64 << 10, 256 << 10, 1 << 20};
            int64_t widest = 0;
            for (auto &J : bs.jac) widest = std::max(widest, J.u->g.shape[1]);
            float best = 1e30f;
            std::array<int, 3> pick = {32, 0, 256 << 10};
            cudaEvent_t e0, e1;
            CK(c, cudaEventCreate(&e0));
            CK(c, cudaEventCreate(&e1));
            for (int th : ths)
                for (int tw : tws)
                    for (int hs : hss) {
                        if (bs.hist.empty() && hs != hss[0]) continue;
                        if (bs.jac.empty() && (th != ths[0] || tw != tws[0])) continue;
                        if (tw && widest <= tw) continue;  // no part wider than the tile: same as full width
                        batch_tables(c, bs, th, tw, hs, 1, &jac, &hist, &reps, &items, &ncnt);
                        BatchCache tc;
                        if ((st = batch_upload(c, &tc, jac, hist, reps, items, ncnt))) {
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
                            pick = {th, tw, hs};
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
        if (force_cols) tp = {32, 1024, 256 << 10};
        auto bc = std::make_unique<BatchCache>();
        bc->key = key;
        batch_tables(c, bs, tp[0], tp[1], tp[2], 0, &jac, &hist, &reps, &items, &ncnt, stall);
        if ((st = batch_upload(c, bc.get(), jac, hist, reps, items, ncnt))) {
            unpin();
            return st;
        }
        bc->bp.hist_slice = tp[2];
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
    c->stats.tuned_tile_rows = force_cols ? 32 : c->tuned[shape_key][0];
    c->stats.tuned_tile_cols = force_cols ? 1024 : c->tuned[shape_key][1];
    c->stats.tuned_hist_slice = force_cols ? (256 << 10) : c->tuned[shape_key][2];
    // run: wait for every staged chunk, then the graph (or the kernels)
    op_begin(c, S_COMP, "batch");
    FenceSet w;
    for (auto &u : uses) {
        w.merge(u.a->cs[(size_t)u.ci].ready);
        w.merge(u.a->cs[(size_t)u.ci].busy);
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
        CState &cs = u.a->cs[(size_t)u.ci];
        if (u.written) cs.ready = FenceSet::one(S_COMP, q);
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
