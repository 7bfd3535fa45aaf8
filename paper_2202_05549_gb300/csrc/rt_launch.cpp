// Runtime: the plan cache, one launch of lookahead and the launch executor
// (groups of superblocks, temporaries, pack, execute, unpack, reduce,
// replica updates, streaming through the host pool); see rt.hpp.
#include "rt.hpp"
#include "copy_staged.cuh"

namespace lt {
namespace rt {

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


constexpr size_t PLAN_CACHE = 4096;

lt_status prepare_plan(lt_ctx *c, lt_kernel *k, lt_dim3 grid, lt_dim3 block, const lt_workdist *wd,
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

// Does the pending launch write array a?
bool pending_writes(lt_ctx *c, const lt_array *a) {
    if (!c->pending) return false;
    const lt_kernel *k = c->pending->k;
    for (size_t p = 0; p < c->pending->parr.size(); ++p)
        if (c->pending->parr[p] == a && k->ann.stmts[(size_t)k->stmt_of_param[p]].mode != MODE_READ) return true;
    return false;
}

// Enqueue the pending launch, if any, without lookahead.
lt_status flush_pending(lt_ctx *c) {
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

lt_status emit_launch(lt_ctx *c, PendingLaunch &pl,
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
                CK(c, c->no_staged ? k::copy_pieces((const CopyPiece *)dptr, (int)packs.size(), rows, c->st[S_COMP])
                                   : k::copy_pieces_staged((const CopyPiece *)dptr, (int)packs.size(), rows,
                                                           c->err_word, c->st[S_COMP]));
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
        // A source kernel copies the replicas of the arrays it writes itself,
        // after a grid-wide barrier at the end of its launch (no copy kernel
        // follows it for them).
        auto fused_replicas = [&](const ArgPlan &ap) {
            return k->own_def && !c->no_fused_replicas && ap.kind == ARG_DIRECT && ap.mode != MODE_READ &&
                   !ap.replicas.empty();
        };
        std::vector<CopyPiece> ucopies;  // replica boxes the source kernel's wrapper copies
        std::vector<uint32_t> uunits;    // their units of 32 elements: (box, first element) pairs
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
                    } else if (fused_replicas(ap)) {
                        for (const auto &pc : ap.replicas) {
                            CState &dcs = a->cs[(size_t)pc.chunk];
                            CopyPiece cp{};
                            cp.src = t.v[sl];
                            cp.dst = view_of(c, a->g, a->g.chunks[(size_t)pc.chunk], dcs.off);
                            cp.nd = a->g.nd;
                            cp.esize = (int32_t)a->g.esize();
                            for (int d = 0; d < 3; ++d) {
                                cp.lo[d] = d < a->g.nd ? pc.box.lo[d] : 0;
                                cp.hi[d] = d < a->g.nd ? pc.box.hi[d] : 0;
                            }
                            const uint64_t vol = (uint64_t)pc.box.volume();
                            if (vol > 0xFFFFFFE0ull)
                                return fail(LT_ERR_UNSUPPORTED, "a halo replica box of 2^32 elements or more");
                            for (uint64_t f = 0; f < vol; f += 32) {
                                uunits.push_back((uint32_t)ucopies.size());
                                uunits.push_back((uint32_t)f);
                            }
                            ucopies.push_back(cp);
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
            // A launch that runs in device memory with no copy step before or
            // after its kernel leaves the kernel next to the previous one on
            // the compute stream: it starts as a programmatic dependent of
            // that kernel and its fence event is deferred (an event between
            // the two kernels would serialise them).  Not with per-operation
            // timing (its events sit between the kernels anyway).
            const bool pdl = def->pdl && !c->no_pdl && batched && temps.empty() && packs.empty() &&
                             !(c->cfg.flags & LT_FLAG_TIMING);
            ep.pdl = pdl ? 1 : 0;
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
            // the replicas once more as warp units: 128 columns of an aligned one-row box, else 32 cells
            std::vector<ReplicaUnit> units;
            for (size_t ri = 0; ri < reps.size(); ++ri) {
                const ReplicaTarget &r = reps[ri];
                const int64_t w = r.hi[1] - r.lo[1] + 1, h = r.hi[0] - r.lo[0] + 1;
                const bool row = h == 1 && r.lo[1] % 4 == 0 && r.dst.s[1] == 1 && r.dst.s[0] % 4 == 0 &&
                                 (r.dst.base + (uint64_t)((r.lo[0] * r.dst.s[0] + r.lo[1]) * 4)) % 16 == 0;
                const int64_t n = row ? w : w * h, step = row ? 128 : 32;
                for (int64_t o = 0; o < n; o += step) {
                    ReplicaUnit u{};
                    u.rep = (uint32_t)ri;
                    u.row = row ? 1u : 0u;
                    u.off = (uint32_t)o;
                    units.push_back(u);
                }
            }
            const size_t tbytes = tasks.size() * sizeof(ExecTask), rbytes = reps.size() * sizeof(ReplicaTarget),
                         ubytes = units.size() * sizeof(ReplicaUnit), cbytes = ucopies.size() * sizeof(CopyPiece),
                         cubytes = uunits.size() * sizeof(uint32_t);
            std::vector<char> table(tbytes + rbytes + ubytes + cbytes + cubytes);
            std::memcpy(table.data(), tasks.data(), tbytes);
            if (rbytes) std::memcpy(table.data() + tbytes, reps.data(), rbytes);
            if (ubytes) std::memcpy(table.data() + tbytes + rbytes, units.data(), ubytes);
            if (cbytes) std::memcpy(table.data() + tbytes + rbytes + ubytes, ucopies.data(), cbytes);
            if (cubytes) std::memcpy(table.data() + tbytes + rbytes + ubytes + cbytes, uunits.data(), cubytes);
            void *dptr;
            size_t roff;
            if ((st = upload(c, table.data(), table.size(), &dptr, &roff))) return st;
            ep.reps = (rbytes && dptr) ? (const ReplicaTarget *)((const char *)dptr + tbytes) : nullptr;
            ep.nreps = (uint32_t)reps.size();
            ep.rep_cells = ep.reps ? rep_cells : 0;
            ep.runits = (ubytes && dptr) ? (const ReplicaUnit *)((const char *)dptr + tbytes + rbytes) : nullptr;
            ep.nunits = ep.runits ? (uint32_t)units.size() : 0;
            if (!c->dry && ctas) {
                TimeScope ts(c, CAT_EXEC);
                if (k->ufn) {
                    // the wrapper is persistent: as many CTAs as fit on the GPU at once, each looping over
                    // the launch's blocks, so short blocks do not pay one CTA launch each
                    const ExecTask *tp = (const ExecTask *)dptr;
                    unsigned nblocks = ctas;
                    const CopyPiece *ucp =
                        cbytes ? (const CopyPiece *)((const char *)dptr + tbytes + rbytes + ubytes) : nullptr;
                    const uint32_t *ucu =
                        cubytes ? (const uint32_t *)((const char *)dptr + tbytes + rbytes + ubytes + cbytes) : nullptr;
                    unsigned nucu = (unsigned)(uunits.size() / 2);
                    unsigned long long target = 0;
                    unsigned long long *bar = c->ubar;
                    void *kargs[] = {(void *)&tp, (void *)&ep, (void *)&nblocks, (void *)&ucp,
                                     (void *)&ucu, (void *)&nucu, (void *)&bar, (void *)&target};
                    dim3 blk((unsigned)ep.block[0], (unsigned)ep.block[1], (unsigned)ep.block[2]);
                    const int threads = (int)(blk.x * blk.y * blk.z);
                    auto occ = k->uocc.find(threads);
                    if (occ == k->uocc.end()) {
                        int per_sm = 0;
                        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k->ufn, threads, 0));
                        occ = k->uocc.emplace(threads, std::max(1, per_sm)).first;
                    }
                    const uint32_t grid = (uint32_t)std::min<uint64_t>(ctas, (uint64_t)occ->second * c->sm_count);
                    if (nucu) {
                        // every CTA arrives once; the barrier completes at the running total of arrivals
                        // (one more with the test flag, so that its bounded wait runs out)
                        target = c->ubar_total + grid + (c->test_replica_stall ? 1u : 0u);
                        cudaLaunchConfig_t cfg{};
                        cfg.gridDim = dim3(grid);
                        cfg.blockDim = blk;
                        cfg.dynamicSmemBytes = 0;
                        cfg.stream = c->st[S_COMP];
                        cudaLaunchAttribute attr[1];
                        attr[0].id = cudaLaunchAttributeCooperative;
                        attr[0].val.cooperative = 1;
                        cfg.attrs = attr;
                        cfg.numAttrs = 1;
                        CK(c, cudaLaunchKernelExC(&cfg, (const void *)k->ufn, kargs));
                        c->ubar_total += grid;  // counted once the launch is in the stream
                    } else {
                        CK(c, cudaLaunchKernel((const void *)k->ufn, dim3(grid), blk, kargs, 0, c->st[S_COMP]));
                    }
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
            if ((st = op_end(c, &exq, extra, pdl))) return st;
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
                    !writes_through(ap, k->slot_of_param[(size_t)ap.param]) && !fused_replicas(ap)) {
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
                CK(c, c->no_staged ? k::copy_pieces((const CopyPiece *)dptr, (int)outs.size(), rows, c->st[S_COMP])
                                   : k::copy_pieces_staged((const CopyPiece *)dptr, (int)outs.size(), rows,
                                                           c->err_word, c->st[S_COMP]));
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

}  // namespace rt
}  // namespace lt

extern "C" {

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

}  // extern "C"
