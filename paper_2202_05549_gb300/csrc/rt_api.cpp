// Runtime: the C ABI for contexts, arrays, kernel registration, synchronize,
// timers, statistics and the debug log, and the table of built-in kernels
// with their canonical annotations (see rt.hpp).
#include "rt.hpp"
#include "copy_staged.cuh"

namespace lt {
namespace rt {

const BuiltinDef kBuiltins[] = {
    {LT_K_PLAN_ONLY, nullptr, 0, {0}, {0}, nullptr, nullptr},
    {LT_K_STENCIL1D, "global i => write A0[i], read A1[i-1:i+1]", 2, {LT_F32, LT_F32}, {1, 1},
     k::prepare_stencil1d, k::launch_stencil1d},
    {LT_K_JACOBI2D, "global [i, j] => read A0[i-1:i+1, j-1:j+1], write A1[i, j]", 2, {LT_F32, LT_F32}, {2, 2},
     k::prepare_jacobi2d, k::launch_jacobi2d, true, false, 1, true},
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
    {LT_K_LAPLACE2D, "global [i, j] => read A0[i-1:i+1, j-1:j+1], write A1[i, j]", 2, {LT_F32, LT_F32}, {2, 2},
     k::prepare_laplace, k::launch_laplace},
    {LT_K_EWISE2D, "global [i, j] => read A0[i, j], read A1[i, j], write A2[i, j]", 3, {LT_F32, LT_F32, LT_F32},
     {2, 2, 2}, k::prepare_ewise, k::launch_ewise},
    {LT_K_MULADD2D, "global [i, j] => read A0[i, j], read A1[i, j], readwrite A2[i, j]", 3, {LT_F32, LT_F32, LT_F32},
     {2, 2, 2}, k::prepare_muladd, k::launch_muladd},
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

const size_t kNumBuiltins = sizeof(kBuiltins) / sizeof(kBuiltins[0]);

}  // namespace rt
}  // namespace lt

extern "C" {

lt_status lt_ctx_create(const lt_config *cfg, lt_ctx **out) {
    if (!cfg || !out) return fail(LT_ERR_INVALID_ARG, "null argument");
    auto c = std::make_unique<lt_ctx>();
    c->cfg = *cfg;
    c->dry = (cfg->flags & LT_FLAG_DRYRUN) != 0;
    c->no_staged = (cfg->flags & LT_FLAG_NO_STAGED) != 0;
    c->no_pdl = (cfg->flags & LT_FLAG_NO_PDL) != 0;
    c->no_quarantine = (cfg->flags & LT_FLAG_NO_LINK_QUARANTINE) != 0;
    c->no_fused_replicas = (cfg->flags & LT_FLAG_NO_FUSED_REPLICAS) != 0;
    c->test_replica_stall = (cfg->flags & LT_FLAG_TEST_REPLICA_STALL) != 0;
    for (int s = 0; s < NSTREAM; ++s) {
        c->ev[s].assign(RING, nullptr);
        c->evseq[s].assign(RING, 0);
        c->evtask[s].assign(RING, -1);
        c->dfseq[s].assign(RING, 0);
        c->dfcov[s].assign(RING, 0);
        c->dftask[s].assign(RING, -1);
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
    CK(cp, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, cfg->device));
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
    CK(cp, cudaHostAlloc((void **)&c->err_host, 64, cudaHostAllocDefault));
    *c->err_host = 0;
    CK(cp, cudaMalloc((void **)&c->ubar, sizeof(unsigned long long)));
    CK(cp, cudaMemset(c->ubar, 0, sizeof(unsigned long long)));
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
        for (auto &pr : c->link_probes) {
            cudaEventDestroy(pr.a);
            cudaEventDestroy(pr.b);
        }
        for (auto e : c->link_ev_pool) cudaEventDestroy(e);
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
        if (c->err_host) cudaFreeHost(c->err_host);
        if (c->ubar) cudaFree(c->ubar);
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

// Asynchronous host copies: each chunk's copy is an operation on a copy
// stream, ordered by the chunk's fences like a launch's, so copies overlap
// kernels and each other.  The host buffer is the caller's until the copies
// end (lt_synchronize): a write of one chunk reads its whole box (halo
// included) from the buffer, a read writes the chunk's owned box into it, so
// each such copy also waits for the earlier copies of the other direction
// whose host region overlaps its own.
static lt_status array_copy_async(lt_ctx *c, lt_array *arr, void *host, size_t bytes, bool to_array) {
    lt_status st = check_ctx(c);
    if (st) return st;
    lt_array *a = find_array(c, arr);
    if (!a || (!host && !c->dry)) return fail(LT_ERR_INVALID_ARG, "unknown array or null buffer");
    if (bytes != array_bytes(a)) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the array");
    if (a->g.dist.order == LT_ORDER_COL)
        return to_array ? lt_array_write(c, arr, host, bytes) : lt_array_read(c, arr, host, bytes);
    if (to_array) {
        if ((st = flush_pending(c))) return st;
        ++c->launch_id;
        for (auto &cs : a->cs) {
            cs.dead_launch = c->launch_id;
            cs.discarded = false;
        }
    } else {
        if (pending_writes(c, arr) && (st = flush_pending(c))) return st;
        // chunks that are not in device memory take the synchronous path
        for (const auto &cs : a->cs)
            if (cs.loc != LOC_DEV && !c->dry) return lt_array_read(c, arr, host, bytes);
    }
    const int sid = to_array ? S_H2D : S_D2H;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        CState &s = a->cs[ci];
        const ChunkGeom &cg = a->g.chunks[ci];
        if (to_array) {
            if (s.loc == LOC_HOST && !c->dry) {  // spilled: rewritten in place in the host pool
                if ((st = sync_all(c))) return st;
                xfer_chunk_host(c, a, (int64_t)ci, cg.box, (char *)host, true);
                s.dead_launch = -1;
                continue;
            }
            s.pin++;
            st = ensure_dev(c, a, (int64_t)ci, false);
            s.pin--;
            if (st) return st;
        }
        const Box &hbox = to_array ? cg.box : cg.owned;  // the host region this copy touches
        op_begin(c, sid, to_array ? "write" : "read");
        FenceSet w = s.ready;
        if (to_array) w.merge(s.busy);
        for (int64_t o : chunks_intersecting(a->g, hbox)) {
            const CState &os = a->cs[(size_t)o];
            w.merge(to_array ? os.host_read : os.host_write);
        }
        if ((st = op_wait(c, w))) return st;
        if (!c->dry && (st = xfer_chunk(c, a, (int64_t)ci, hbox, (char *)host, to_array, false, sid, false)))
            return st;
        uint64_t q;
        if ((st = op_end(c, &q))) return st;
        if (to_array) {
            s.ready = FenceSet::one(sid, q);
            s.busy = FenceSet::one(sid, q);
            s.host_write = FenceSet::one(sid, q);
            c->stats.bytes_h2d += cg.box.volume() * a->g.esize();
        } else {
            s.busy.add(sid, q);
            s.host_read = FenceSet::one(sid, q);
            c->stats.bytes_d2h += cg.owned.volume() * a->g.esize();
        }
    }
    return LT_OK;
}

// Copies between an array and a dense device buffer when every chunk can be
// in device memory at once: the chunks are pinned there and one box-copy
// kernel moves all of them (a strided cudaMemcpy2DAsync per chunk ran at
// about 1.8 TB/s between two device buffers).  LT_ERR_OOM_DEVICE, with
// nothing enqueued, when a chunk lies in the host pool or the chunks do not
// fit together; the caller then copies chunk by chunk.
static lt_status copy_device_kernel(lt_ctx *c, lt_array *a, void *dev, bool to_array) {
    for (const auto &cs : a->cs)
        if (cs.loc == LOC_HOST) return LT_ERR_OOM_DEVICE;
    lt_status st = LT_OK;
    size_t npin = 0;
    for (; npin < a->cs.size(); ++npin) {
        CState &s = a->cs[npin];
        s.pin++;
        // a chunk never written reads as zeros; a write needs the chunk's memory only
        if (s.loc != LOC_DEV && (st = ensure_dev(c, a, (int64_t)npin, !to_array, /*soft=*/true))) {
            ++npin;
            break;
        }
    }
    auto unpin = [&]() {
        for (size_t ci = 0; ci < npin; ++ci) a->cs[ci].pin--;
    };
    if (st) {
        unpin();
        return st;
    }
    const ArrayGeom &g = a->g;
    DView dense{};
    dense.base = (uint64_t)(uintptr_t)dev;
    int64_t gs[3] = {1, 1, 1};
    for (int d = g.nd - 2; d >= 0; --d) gs[d] = gs[d + 1] * g.shape[d + 1];
    for (int d = 0; d < 3; ++d) {
        dense.s[d] = d < g.nd ? gs[d] : 0;
        dense.hi[d] = d < g.nd ? g.shape[d] - 1 : 0;
    }
    std::vector<CopyPiece> pieces;
    FenceSet w;
    uint64_t units = 0;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        CState &s = a->cs[ci];
        const ChunkGeom &cg = g.chunks[ci];
        const Box &b = to_array ? cg.box : cg.owned;
        if (b.volume() == 0) continue;
        CopyPiece cp{};
        const DView cv = view_of(c, g, cg, s.off);
        cp.src = to_array ? dense : cv;
        cp.dst = to_array ? cv : dense;
        cp.nd = g.nd;
        cp.esize = (int32_t)g.esize();
        for (int d = 0; d < 3; ++d) {
            cp.lo[d] = d < g.nd ? b.lo[d] : 0;
            cp.hi[d] = d < g.nd ? b.hi[d] : 0;
        }
        cp.unit_begin = units;
        units += copy_piece_units(cp);
        pieces.push_back(cp);
        w.merge(s.ready);
        if (to_array) w.merge(s.busy);
        s.dead_launch = -1;
    }
    op_begin(c, S_COMP, to_array ? "write_device" : "read_device");
    void *dptr = nullptr;
    size_t roff = NO_RING;
    if ((st = op_wait(c, w)) || (!pieces.empty() && (st = upload(c, pieces.data(), pieces.size() * sizeof(CopyPiece),
                                                                 &dptr, &roff)))) {
        unpin();
        return st;
    }
    if (!pieces.empty()) {
        TimeScope ts(c, CAT_COPYK);
        const cudaError_t e = c->no_staged ? k::copy_pieces((const CopyPiece *)dptr, (int)pieces.size(), units,
                                                            c->st[S_COMP])
                                           : k::copy_pieces_staged((const CopyPiece *)dptr, (int)pieces.size(), units,
                                                                   c->err_word, c->st[S_COMP]);
        if (e != cudaSuccess) {
            unpin();
            CK(c, e);
        }
        c->stats.kernels++;
    }
    uint64_t q;
    if ((st = op_end(c, &q))) {
        unpin();
        return st;
    }
    upload_done(c, roff, pieces.size() * sizeof(CopyPiece), q);
    for (auto &s : a->cs) {
        if (to_array) {
            s.ready = FenceSet::one(S_COMP, q);
            s.busy = FenceSet::one(S_COMP, q);
        } else {
            s.busy.add(S_COMP, q);
        }
    }
    unpin();
    return sync_all(c);
}

// Copies between an array and a dense device buffer: each chunk's copy is an
// operation on the compute stream behind the operations on that chunk (as for
// the asynchronous host copies), and the call returns once all of them are
// done, so the buffer is the caller's again.
static lt_status array_copy_device(lt_ctx *c, lt_array *arr, void *dev, size_t bytes, bool to_array) {
    lt_status st = check_ctx(c);
    if (st) return st;
    lt_array *a = find_array(c, arr);
    if (!a || !dev) return fail(LT_ERR_INVALID_ARG, "unknown array or null buffer");
    if (bytes != array_bytes(a)) return fail(LT_ERR_INVALID_ARG, "buffer size does not match the array");
    if (a->g.dist.order == LT_ORDER_COL) return fail(LT_ERR_UNSUPPORTED, "device copies need row-major chunks");
    if (c->dry) return fail(LT_ERR_UNSUPPORTED, "device copies need a device");
    if ((st = flush_pending(c))) return st;
    if (to_array) {
        ++c->launch_id;
        for (auto &cs : a->cs) {
            cs.dead_launch = c->launch_id;
            cs.discarded = false;
        }
    }
    if ((st = copy_device_kernel(c, a, dev, to_array)) != LT_ERR_OOM_DEVICE) return st;
    for (size_t ci = 0; ci < a->cs.size(); ++ci) {
        CState &s = a->cs[ci];
        const ChunkGeom &cg = a->g.chunks[ci];
        // a chunk never written reads as zeros (zero-filled in device memory); a write
        // into a chunk that is not in the host pool needs it in device memory
        if ((!to_array && s.loc == LOC_NONE) || (to_array && s.loc != LOC_HOST)) {
            s.pin++;
            st = ensure_dev(c, a, (int64_t)ci, !to_array);
            s.pin--;
            if (st) return st;
        }
        s.dead_launch = -1;
        op_begin(c, S_COMP, to_array ? "write_device" : "read_device");
        FenceSet w = s.ready;
        if (to_array) w.merge(s.busy);
        if ((st = op_wait(c, w))) return st;
        if ((st = xfer_chunk(c, a, (int64_t)ci, to_array ? cg.box : cg.owned, (char *)dev, to_array, true, S_COMP,
                             false)))
            return st;
        uint64_t q;
        if ((st = op_end(c, &q))) return st;
        if (to_array) {
            s.ready = FenceSet::one(S_COMP, q);
            s.busy = FenceSet::one(S_COMP, q);
        } else {
            s.busy.add(S_COMP, q);
        }
    }
    return sync_all(c);
}

lt_status lt_array_write_async(lt_ctx *c, lt_array *arr, const void *host, size_t bytes) {
    return array_copy_async(c, arr, const_cast<void *>(host), bytes, true);
}

lt_status lt_array_read_async(lt_ctx *c, lt_array *arr, void *host, size_t bytes) {
    return array_copy_async(c, arr, host, bytes, false);
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
            const int nd = a->g.nd;
            const int64_t es = (int64_t)a->g.esize();
            if (kind == LT_INIT_ZERO && nd <= 2 && d.dst.s[nd - 1] == 1) {
                // zeros are all-zero bytes in every dtype: a strided memset of the box's rows
                const int64_t e0 = nd == 2 ? d.hi[0] - d.lo[0] + 1 : 1, e1 = d.hi[nd - 1] - d.lo[nd - 1] + 1;
                const int64_t first = nd == 2 ? d.lo[0] * d.dst.s[0] + d.lo[1] : d.lo[0];
                const size_t pitch = nd == 2 ? (size_t)(d.dst.s[0] * es) : (size_t)(e1 * es);
                CK(c, cudaMemset2DAsync((void *)(uintptr_t)(d.dst.base + (uint64_t)(first * es)), pitch, 0,
                                        (size_t)(e1 * es), (size_t)e0, c->st[S_COMP]));
            } else {
                CK(c, k::fill(d, c->st[S_COMP]));
                c->stats.kernels++;
            }
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
    c->stats.host_withheld_bytes = c->host.withheld;
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
