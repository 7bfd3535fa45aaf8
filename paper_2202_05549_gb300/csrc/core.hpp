// Internal types of the annotated-launch engine: boxes, annotations,
// distributions and launch plans.  Host-only C++17; no CUDA here.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "lightning.h"

namespace lt {

// Dense n-D box of element (or thread) indices, bounds inclusive.  Axis 0 is
// the slowest axis of an array.  Thread boxes use axis 0 = x, 1 = y, 2 = z.
struct Box {
    int nd = 0;
    int64_t lo[3] = {0, 0, 0};
    int64_t hi[3] = {-1, -1, -1};

    bool empty() const {
        if (nd == 0) return true;
        for (int d = 0; d < nd; ++d)
            if (lo[d] > hi[d]) return true;
        return false;
    }
    int64_t extent(int d) const { return hi[d] - lo[d] + 1; }
    int64_t volume() const {
        if (empty()) return 0;
        int64_t v = 1;
        for (int d = 0; d < nd; ++d) v *= extent(d);
        return v;
    }
    Box intersect(const Box &o) const {
        Box r;
        r.nd = nd;
        for (int d = 0; d < nd; ++d) {
            r.lo[d] = lo[d] > o.lo[d] ? lo[d] : o.lo[d];
            r.hi[d] = hi[d] < o.hi[d] ? hi[d] : o.hi[d];
        }
        return r;
    }
    bool contains(const Box &o) const {
        if (o.empty()) return true;
        for (int d = 0; d < nd; ++d)
            if (o.lo[d] < lo[d] || o.hi[d] > hi[d]) return false;
        return true;
    }
    bool operator==(const Box &o) const {
        if (nd != o.nd) return false;
        for (int d = 0; d < nd; ++d)
            if (lo[d] != o.lo[d] || hi[d] != o.hi[d]) return false;
        return true;
    }
};

// true iff `target` is covered by the union of `parts`
bool box_covered(const Box &target, const std::vector<Box> &parts);

// ---------------------------------------------------------------- annotations
enum VarKind { VAR_GLOBAL = 0, VAR_BLOCK = 1, VAR_LOCAL = 2 };
enum Mode { MODE_READ = 0, MODE_WRITE = 1, MODE_READWRITE = 2, MODE_REDUCE = 3 };
enum ReduceOp { RED_ADD = 0, RED_MUL = 1, RED_MIN = 2, RED_MAX = 3 };

struct Var {
    std::string name;
    int kind = VAR_GLOBAL;
    int dim = 0;  // 0 = x, 1 = y, 2 = z
};

struct Affine {
    std::vector<int64_t> coef;  // one per bound variable
    int64_t c = 0;
};

struct Index {
    bool slice = false;
    bool has_lo = true, has_hi = true;
    Affine lo, hi;  // equal for a plain index
};

struct Stmt {
    int mode = MODE_READ;
    int op = RED_ADD;
    std::string array;
    std::vector<Index> idx;
};

struct Annotation {
    std::vector<Var> vars;
    std::vector<Stmt> stmts;
    std::string text;
};

// Parse the grammar documented in lightning.h.  Returns false and sets *err.
bool parse_annotation(const std::string &text, Annotation *out, std::string *err);

// Range [lo, hi] of every bound variable over the threads of one superblock.
// tbox: thread box (x, y, z) inclusive; block: block dims (x, y, z).
void var_ranges(const Annotation &a, const Box &tbox, const int64_t block[3], std::vector<int64_t> *vlo,
                std::vector<int64_t> *vhi);

// Access region of statement s for the given variable ranges, clipped to the
// array domain `shape` (ndim = s.idx.size()).  Empty box if nothing lies in
// the domain.
Box eval_region(const Stmt &s, const std::vector<int64_t> &vlo, const std::vector<int64_t> &vhi,
                const int64_t *shape);

// ---------------------------------------------------------------- distributions
size_t dtype_size(int dtype);

struct ChunkGeom {
    Box box;                // elements held (owned tile + halo, clipped)
    Box owned;              // the tile of the distribution (no halo)
    int64_t s_origin[3];    // global index of storage element 0 per axis
    int64_t s_ext[3];       // storage extents (innermost padded to 128 B)
    int64_t stride[3];      // element strides per axis
    size_t bytes = 0;       // storage bytes
};

struct ArrayGeom {
    int dtype = LT_F32;
    int nd = 1;
    int64_t shape[3] = {1, 1, 1};
    lt_dist dist{};
    int64_t ntile[3] = {1, 1, 1};
    int64_t tile[3] = {1, 1, 1};
    std::vector<ChunkGeom> chunks;

    size_t esize() const { return dtype_size(dtype); }
    Box domain() const {
        Box b;
        b.nd = nd;
        for (int d = 0; d < nd; ++d) {
            b.lo[d] = 0;
            b.hi[d] = shape[d] - 1;
        }
        return b;
    }
};

// Build the chunk list; false + *err on invalid distribution.
bool make_geometry(int dtype, int nd, const int64_t shape[3], const lt_dist &dist, ArrayGeom *g, std::string *err);

// Chunks whose box intersects `region`, in chunk index order.
std::vector<int64_t> chunks_intersecting(const ArrayGeom &g, const Box &region);

// Storage layout for a temporary chunk covering `region` (same padding rules).
ChunkGeom temp_geometry(const ArrayGeom &g, const Box &region);

// ---------------------------------------------------------------- plans
enum ArgKind {
    ARG_VALUE = 0,    // value parameter
    ARG_NONE = 1,     // empty access region
    ARG_DIRECT = 2,   // one chunk encloses the region: use it in place
    ARG_PACK = 3,     // read region spans chunks: assemble a temporary
    ARG_TEMPW = 4,    // write region spans chunks: temporary, scattered after
    ARG_REDUCE = 5,   // per-superblock partials, reduced after all superblocks
};

struct Piece {
    int64_t chunk = -1;  // chunk of the array
    Box box;             // global element box
};

struct ArgPlan {
    int param = -1;       // parameter index
    int stmt = -1;        // annotation statement index
    int kind = ARG_NONE;
    int mode = MODE_READ;
    int op = RED_ADD;
    Box region;
    int64_t chunk = -1;          // ARG_DIRECT
    std::vector<Piece> pieces;   // PACK sources, TEMPW / REDUCE destinations
    std::vector<Piece> replicas; // DIRECT writes: other chunks to refresh (src = chunk)
};

struct SuperblockPlan {
    int64_t index = 0;
    Box threads;             // x, y, z thread box
    std::vector<ArgPlan> args;
};

struct KernelSig;  // built-in signature (runtime side)

struct LaunchPlan {
    std::vector<SuperblockPlan> sbs;
    int64_t nsb[3] = {1, 1, 1};
};

struct PlanArray {
    const ArrayGeom *geom = nullptr;  // nullptr for value parameters
};

// Plan a launch: split the grid into superblocks and classify every
// argument of every superblock.  `stmt_of_param[p]` gives the statement of
// array parameter p (-1 for values).
bool plan_launch(const Annotation &a, const std::vector<int> &stmt_of_param, const std::vector<PlanArray> &arrays,
                 const uint64_t grid[3], const uint64_t block[3], const int64_t superblock[3], LaunchPlan *out,
                 std::string *err);

std::string plan_to_json(const LaunchPlan &p);

// Record the calling thread's error message (returned by lt_last_error).
lt_status set_last_error(lt_status st, const std::string &msg);

}  // namespace lt
