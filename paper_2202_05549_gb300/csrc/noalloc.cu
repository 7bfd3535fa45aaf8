// Allocation-free variant of the 2-D Jacobi pack path.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory budget or allocator, or a process that must not grow
// its device footprint after start-up.  This entry point gives them one
// Jacobi step with the same pack-then-execute sequence as an annotated
// launch over a distribution without halo (every tile's read region, tile
// plus a one-cell ring, is first gathered into scratch, then the tile is
// computed from that copy).  The scratch is the file-scope device array
// below instead of the engine's pool, so the call allocates nothing.
//
// The array exists once per device that loads the library and stays there
// until the process exits.  Every call on a device shares it, so calls that
// overlap on the GPU (different streams, no ordering between them) race;
// calls ordered on one stream do not.  Every call looks up the array's
// device address on the current device (cudaGetSymbolAddress, a few
// microseconds), so the address stays right after the device's context is
// torn down and made again.  The first call on a device also loads this
// module there; make that first call before any stream capture.  The
// descriptor tables are uploaded from a host buffer that lives only for the
// call, so a call on a stream that is capturing returns LT_ERR_UNSUPPORTED
// and enqueues nothing.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "core.hpp"
#include "kernels.cuh"
#include "lightning.h"

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;  // LT_NOALLOC_SCRATCH_BYTES
constexpr size_t kDescBytes = (size_t)1 << 20;      // descriptor tables at the front
constexpr size_t kPackBytes = kScratchBytes - kDescBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

lt_status nfail(lt_status s, const std::string &m) { return lt::set_last_error(s, m); }

// Device address of the scratch array on the current device.
lt_status scratch_ptr(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return nfail(LT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = (unsigned char *)p;
    return LT_OK;
}

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" lt_status lt_jacobi2d_packed_noalloc(const float *U, float *V, int64_t ny, int64_t nx, int64_t ld_u,
                                               int64_t ld_v, int64_t tile_rows, int64_t tile_cols, void *stream) {
    using namespace lt;
    if (!U || !V || (const void *)U == (const void *)V) return nfail(LT_ERR_INVALID_ARG, "U and V must be distinct device pointers");
    if (ny < 1 || nx < 1 || ld_u < nx || ld_v < nx || tile_rows < 1 || tile_cols < 1)
        return nfail(LT_ERR_INVALID_ARG, "need ny, nx, tile sizes >= 1 and leading dimensions >= nx");
    // largest packed tile: (tile_rows + 2) rows x columns padded to 128 bytes
    size_t tr = (size_t)std::min<int64_t>(tile_rows, ny), tc = (size_t)std::min<int64_t>(tile_cols, nx);
    size_t worst = (tr + 2) * up(tc + 2 + 32, 32) * sizeof(float);
    if (worst > kPackBytes)
        return nfail(LT_ERR_INVALID_ARG, "a packed tile needs " + std::to_string(worst) +
                                             " bytes; the static scratch holds " + std::to_string(kPackBytes) +
                                             " (64 MiB less 1 MiB of descriptors)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return nfail(LT_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return nfail(LT_ERR_UNSUPPORTED, "the stream is capturing: the descriptor upload reads a host buffer that "
                                         "lives only for the call, so this call is not recorded");
    unsigned char *scr = nullptr;
    lt_status st = scratch_ptr(&scr);
    if (st) return st;

    DView uv{(uint64_t)(uintptr_t)U, {ld_u, 1, 0}, {0, 0, 0}, {ny - 1, nx - 1, 0}};
    DView vv{(uint64_t)(uintptr_t)V, {ld_v, 1, 0}, {0, 0, 0}, {ny - 1, nx - 1, 0}};
    ExecParams ep{};
    ep.shape[0][0] = ep.shape[1][0] = ny;
    ep.shape[0][1] = ep.shape[1][1] = nx;
    ep.shape[0][2] = ep.shape[1][2] = 1;
    ep.nd[0] = ep.nd[1] = 2;

    const int64_t nty = (ny + tile_rows - 1) / tile_rows, ntx = (nx + tile_cols - 1) / tile_cols;
    const size_t per_tile_desc = sizeof(CopyPiece) + sizeof(ExecTask);
    std::vector<CopyPiece> packs;
    std::vector<ExecTask> tasks;
    int64_t t = 0, ntiles = nty * ntx;
    while (t < ntiles) {
        packs.clear();
        tasks.clear();
        size_t used = 0;
        // gather tiles while their packed regions and descriptors fit
        for (; t < ntiles; ++t) {
            int64_t ty = t / ntx, tx = t % ntx;
            int64_t r0 = ty * tile_rows, r1 = std::min(r0 + tile_rows, ny) - 1;
            int64_t c0 = tx * tile_cols, c1 = std::min(c0 + tile_cols, nx) - 1;
            int64_t rr0 = std::max<int64_t>(0, r0 - 1), rr1 = std::min(ny - 1, r1 + 1);
            int64_t rc0 = std::max<int64_t>(0, c0 - 1), rc1 = std::min(nx - 1, c1 + 1);
            int64_t org = rc0 / 32 * 32;
            int64_t ext = (int64_t)up((size_t)(rc1 + 1 - org), 32);
            size_t bytes = up((size_t)((rr1 - rr0 + 1) * ext) * sizeof(float), 1024);
            if (used + bytes > kPackBytes || (packs.size() + 1) * per_tile_desc + 512 > kDescBytes) break;
            uint64_t tbase = (uint64_t)(uintptr_t)(scr + kDescBytes + used);
            DView tv{tbase - (uint64_t)((rr0 * ext + org) * (int64_t)sizeof(float)), {ext, 1, 0}, {rr0, org, 0},
                     {rr1, rc1, 0}};
            CopyPiece cp{};
            cp.src = uv;
            cp.dst = tv;
            cp.nd = 2;
            cp.esize = 4;
            cp.lo[0] = rr0;
            cp.hi[0] = rr1;
            cp.lo[1] = rc0;
            cp.hi[1] = rc1;
            packs.push_back(cp);
            ExecTask et{};
            et.t_lo[0] = c0;
            et.t_hi[0] = c1;
            et.t_lo[1] = r0;
            et.t_hi[1] = r1;
            et.v[0] = tv;
            et.v[1] = vv;
            tasks.push_back(et);
            used += bytes;
        }
        uint64_t units = 0;
        for (auto &p : packs) {
            p.unit_begin = units;
            units += copy_piece_units(p);
        }
        ep.ntasks = (int32_t)tasks.size();
        uint32_t ctas = k::prepare_jacobi2d(tasks.data(), (int)tasks.size(), ep);
        size_t pbytes = packs.size() * sizeof(CopyPiece);
        size_t tbytes = tasks.size() * sizeof(ExecTask);
        std::vector<unsigned char> host(up(pbytes, 256) + tbytes);
        std::memcpy(host.data(), packs.data(), pbytes);
        std::memcpy(host.data() + up(pbytes, 256), tasks.data(), tbytes);
        // pageable source: the copy is staged before the call returns
        cudaError_t e = cudaMemcpyAsync(scr, host.data(), host.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = k::copy_pieces((const CopyPiece *)scr, (int)packs.size(), units, s);
        if (e == cudaSuccess && ctas)
            e = k::launch_jacobi2d((const ExecTask *)(scr + up(pbytes, 256)), ctas, ep, s);
        if (e != cudaSuccess) return nfail(LT_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    }
    return LT_OK;
}
