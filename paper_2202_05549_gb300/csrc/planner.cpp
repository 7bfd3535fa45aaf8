// Annotation parser, access-region evaluation, distributions and the launch
// planner (Sec. 2.3 "Data Annotations", Sec. 2.2 distributions, Sec. 2.4
// "Execution Planner").  Host-only C++17.
#include <algorithm>
#include <cctype>
#include <cstdio>
#include <sstream>

#include "core.hpp"

namespace lt {

// ============================================================== coverage
static bool covered_rec(const Box &t, const std::vector<Box> &parts, int d) {
    if (parts.empty()) return false;
    if (d == t.nd) return true;
    std::vector<int64_t> b;
    b.reserve(parts.size() * 2 + 2);
    b.push_back(t.lo[d]);
    b.push_back(t.hi[d] + 1);
    for (const Box &p : parts) {
        b.push_back(p.lo[d]);
        b.push_back(p.hi[d] + 1);
    }
    std::sort(b.begin(), b.end());
    b.erase(std::unique(b.begin(), b.end()), b.end());
    std::vector<Box> sub;
    for (size_t k = 0; k + 1 < b.size(); ++k) {
        int64_t s0 = b[k], s1 = b[k + 1] - 1;
        if (s0 < t.lo[d] || s1 > t.hi[d]) continue;
        sub.clear();
        for (const Box &p : parts)
            if (p.lo[d] <= s0 && p.hi[d] >= s1) sub.push_back(p);
        Box ts = t;
        ts.lo[d] = s0;
        ts.hi[d] = s1;
        if (!covered_rec(ts, sub, d + 1)) return false;
    }
    return true;
}

bool box_covered(const Box &target, const std::vector<Box> &parts) {
    if (target.empty()) return true;
    std::vector<Box> clipped;
    int64_t vol = 0;
    for (const Box &p : parts) {
        Box q = target.intersect(p);
        if (!q.empty()) {
            clipped.push_back(q);
            vol += q.volume();
        }
    }
    if (vol < target.volume()) return false;
    return covered_rec(target, clipped, 0);
}

// ============================================================== parser
namespace {

struct Tok {
    enum K { END, IDENT, INT, SYM } k = END;
    std::string s;
    int64_t v = 0;
};

struct Lexer {
    const std::string &t;
    size_t p = 0;
    explicit Lexer(const std::string &text) : t(text) {}
    bool next(Tok *out, std::string *err) {
        while (p < t.size() && std::isspace((unsigned char)t[p])) ++p;
        Tok k;
        if (p >= t.size()) {
            *out = k;
            return true;
        }
        char c = t[p];
        if (std::isalpha((unsigned char)c) || c == '_') {
            size_t q = p;
            while (q < t.size() && (std::isalnum((unsigned char)t[q]) || t[q] == '_')) ++q;
            k.k = Tok::IDENT;
            k.s = t.substr(p, q - p);
            p = q;
        } else if (std::isdigit((unsigned char)c)) {
            size_t q = p;
            int64_t v = 0;
            while (q < t.size() && std::isdigit((unsigned char)t[q])) {
                if (v > (INT64_MAX - 9) / 10) {
                    *err = "integer literal too large";
                    return false;
                }
                v = v * 10 + (t[q] - '0');
                ++q;
            }
            k.k = Tok::INT;
            k.v = v;
            k.s = t.substr(p, q - p);
            p = q;
        } else if (c == '=' && p + 1 < t.size() && t[p + 1] == '>') {
            k.k = Tok::SYM;
            k.s = "=>";
            p += 2;
        } else if (std::string("[](),:+-*").find(c) != std::string::npos) {
            k.k = Tok::SYM;
            k.s = std::string(1, c);
            ++p;
        } else {
            *err = std::string("unexpected character '") + c + "'";
            return false;
        }
        *out = k;
        return true;
    }
};

struct Parser {
    std::vector<Tok> toks;
    size_t p = 0;
    Annotation *a = nullptr;
    std::string err;

    const Tok &peek() const { return toks[p]; }
    bool is_sym(const char *s) const { return peek().k == Tok::SYM && peek().s == s; }
    bool is_ident(const char *s) const { return peek().k == Tok::IDENT && peek().s == s; }
    bool expect_sym(const char *s) {
        if (!is_sym(s)) {
            err = std::string("expected '") + s + "' near token " + std::to_string(p) + " ('" + peek().s + "')";
            return false;
        }
        ++p;
        return true;
    }
    int var_index(const std::string &n) const {
        for (size_t i = 0; i < a->vars.size(); ++i)
            if (a->vars[i].name == n) return (int)i;
        return -1;
    }
    Affine zero() const {
        Affine f;
        f.coef.assign(a->vars.size(), 0);
        return f;
    }
    static bool is_const(const Affine &f) {
        for (int64_t c : f.coef)
            if (c) return false;
        return true;
    }
    // sum := ['-'] prod (('+'|'-') prod)*
    bool sum(Affine *out) {
        Affine acc = zero();
        int sign = 1;
        if (is_sym("-")) {
            sign = -1;
            ++p;
        } else if (is_sym("+")) {
            ++p;
        }
        for (;;) {
            Affine t;
            if (!prod(&t)) return false;
            for (size_t i = 0; i < acc.coef.size(); ++i) acc.coef[i] += sign * t.coef[i];
            acc.c += sign * t.c;
            if (is_sym("+")) {
                sign = 1;
                ++p;
            } else if (is_sym("-")) {
                sign = -1;
                ++p;
            } else {
                break;
            }
        }
        *out = acc;
        return true;
    }
    // prod := atom ('*' atom)*, at most one non-constant factor
    bool prod(Affine *out) {
        Affine f;
        if (!atom(&f)) return false;
        while (is_sym("*")) {
            ++p;
            Affine g;
            if (!atom(&g)) return false;
            if (!is_const(f) && !is_const(g)) {
                err = "index expression is not affine (product of variables)";
                return false;
            }
            if (is_const(f)) std::swap(f, g);
            // f may be non-constant, g constant
            for (auto &c : f.coef) c *= g.c;
            f.c *= g.c;
        }
        *out = f;
        return true;
    }
    bool atom(Affine *out) {
        Affine f = zero();
        const Tok &t = peek();
        if (t.k == Tok::INT) {
            f.c = t.v;
            ++p;
        } else if (t.k == Tok::IDENT) {
            int vi = var_index(t.s);
            if (vi < 0) {
                err = "unknown variable '" + t.s + "' in index expression";
                return false;
            }
            f.coef[vi] = 1;
            ++p;
        } else if (is_sym("(")) {
            ++p;
            if (!sum(&f)) return false;
            if (!expect_sym(")")) return false;
        } else if (is_sym("-")) {
            ++p;
            if (!atom(&f)) return false;
            for (auto &c : f.coef) c = -c;
            f.c = -f.c;
        } else {
            err = "expected an index expression near '" + t.s + "'";
            return false;
        }
        *out = f;
        return true;
    }
    bool index(Index *out) {
        Index ix;
        bool starts_colon = is_sym(":");
        if (starts_colon) {
            ix.slice = true;
            ix.has_lo = false;
            ix.lo = zero();
            ++p;
        } else {
            if (!sum(&ix.lo)) return false;
            if (is_sym(":")) {
                ix.slice = true;
                ++p;
            } else {
                ix.hi = ix.lo;
                *out = ix;
                return true;
            }
        }
        // after ':'
        if (is_sym(",") || is_sym("]")) {
            ix.has_hi = false;
            ix.hi = zero();
        } else {
            if (!sum(&ix.hi)) return false;
        }
        *out = ix;
        return true;
    }
    bool bindings() {
        for (;;) {
            int kind;
            if (is_ident("global"))
                kind = VAR_GLOBAL;
            else if (is_ident("block"))
                kind = VAR_BLOCK;
            else if (is_ident("local"))
                kind = VAR_LOCAL;
            else {
                err = "expected 'global', 'block' or 'local' near '" + peek().s + "'";
                return false;
            }
            ++p;
            std::vector<std::string> names;
            if (is_sym("[")) {
                ++p;
                for (;;) {
                    if (peek().k != Tok::IDENT) {
                        err = "expected a variable name in binding";
                        return false;
                    }
                    names.push_back(peek().s);
                    ++p;
                    if (is_sym(",")) {
                        ++p;
                        continue;
                    }
                    if (!expect_sym("]")) return false;
                    break;
                }
            } else if (peek().k == Tok::IDENT) {
                names.push_back(peek().s);
                ++p;
            } else {
                err = "expected a variable or '[' after binding kind";
                return false;
            }
            if (names.size() > 3) {
                err = "a binding has at most 3 variables";
                return false;
            }
            int n = (int)names.size();
            for (int i = 0; i < n; ++i) {
                const std::string &nm = names[i];
                if (nm == "read" || nm == "write" || nm == "readwrite" || nm == "reduce" || nm == "global" ||
                    nm == "block" || nm == "local") {
                    err = "reserved word used as variable: " + nm;
                    return false;
                }
                if (var_index(nm) >= 0) {
                    err = "variable bound twice: " + nm;
                    return false;
                }
                Var v;
                v.name = nm;
                v.kind = kind;
                v.dim = n - 1 - i;  // last variable is x
                a->vars.push_back(v);
            }
            if (is_sym(",")) {
                ++p;
                continue;
            }
            return expect_sym("=>");
        }
    }
    bool stmt(Stmt *out) {
        Stmt s;
        if (is_ident("read")) {
            s.mode = MODE_READ;
            ++p;
        } else if (is_ident("write")) {
            s.mode = MODE_WRITE;
            ++p;
        } else if (is_ident("readwrite")) {
            s.mode = MODE_READWRITE;
            ++p;
        } else if (is_ident("reduce")) {
            s.mode = MODE_REDUCE;
            ++p;
            if (!expect_sym("(")) return false;
            if (is_sym("+")) {
                s.op = RED_ADD;
                ++p;
            } else if (is_sym("*")) {
                s.op = RED_MUL;
                ++p;
            } else if (is_ident("min")) {
                s.op = RED_MIN;
                ++p;
            } else if (is_ident("max")) {
                s.op = RED_MAX;
                ++p;
            } else {
                err = "reduce operator must be +, *, min or max";
                return false;
            }
            if (!expect_sym(")")) return false;
        } else {
            err = "expected an access mode (read, write, readwrite, reduce) near '" + peek().s + "'";
            return false;
        }
        if (peek().k != Tok::IDENT) {
            err = "expected an array name after the access mode";
            return false;
        }
        s.array = peek().s;
        ++p;
        if (!expect_sym("[")) return false;
        for (;;) {
            Index ix;
            if (!index(&ix)) return false;
            s.idx.push_back(ix);
            if (is_sym(",")) {
                ++p;
                continue;
            }
            if (!expect_sym("]")) return false;
            break;
        }
        if (s.idx.size() > 3) {
            err = "arrays have at most 3 dimensions";
            return false;
        }
        *out = s;
        return true;
    }
};

}  // namespace

bool parse_annotation(const std::string &text, Annotation *out, std::string *err) {
    Annotation a;
    a.text = text;
    Parser ps;
    ps.a = &a;
    Lexer lx(text);
    for (;;) {
        Tok t;
        if (!lx.next(&t, err)) return false;
        ps.toks.push_back(t);
        if (t.k == Tok::END) break;
    }
    if (!ps.bindings()) {
        *err = ps.err;
        return false;
    }
    for (;;) {
        Stmt s;
        if (!ps.stmt(&s)) {
            *err = ps.err;
            return false;
        }
        for (const Stmt &o : a.stmts)
            if (o.array == s.array) {
                *err = "array '" + s.array + "' appears in two statements";
                return false;
            }
        a.stmts.push_back(s);
        if (ps.is_sym(",")) {
            ++ps.p;
            continue;
        }
        if (ps.peek().k != Tok::END) {
            *err = "unexpected trailing text near '" + ps.peek().s + "'";
            return false;
        }
        break;
    }
    *out = a;
    return true;
}

void var_ranges(const Annotation &a, const Box &tbox, const int64_t block[3], std::vector<int64_t> *vlo,
                std::vector<int64_t> *vhi) {
    vlo->assign(a.vars.size(), 0);
    vhi->assign(a.vars.size(), 0);
    for (size_t i = 0; i < a.vars.size(); ++i) {
        int d = a.vars[i].dim;
        int64_t t0 = tbox.lo[d], t1 = tbox.hi[d], B = block[d];
        switch (a.vars[i].kind) {
            case VAR_GLOBAL:
                (*vlo)[i] = t0;
                (*vhi)[i] = t1;
                break;
            case VAR_BLOCK:
                (*vlo)[i] = t0 / B;
                (*vhi)[i] = t1 / B;
                break;
            default:
                if (t1 - t0 + 1 >= B) {
                    (*vlo)[i] = 0;
                    (*vhi)[i] = B - 1;
                } else {
                    (*vlo)[i] = t0 % B;
                    (*vhi)[i] = t1 % B;
                    if ((*vhi)[i] < (*vlo)[i]) {
                        (*vlo)[i] = 0;
                        (*vhi)[i] = B - 1;
                    }
                }
        }
    }
}

static void affine_minmax(const Affine &f, const std::vector<int64_t> &vlo, const std::vector<int64_t> &vhi,
                          int64_t *mn, int64_t *mx) {
    int64_t a = f.c, b = f.c;
    for (size_t i = 0; i < f.coef.size(); ++i) {
        int64_t c = f.coef[i];
        if (c > 0) {
            a += c * vlo[i];
            b += c * vhi[i];
        } else if (c < 0) {
            a += c * vhi[i];
            b += c * vlo[i];
        }
    }
    *mn = a;
    *mx = b;
}

Box eval_region(const Stmt &s, const std::vector<int64_t> &vlo, const std::vector<int64_t> &vhi,
                const int64_t *shape) {
    Box r;
    r.nd = (int)s.idx.size();
    for (int d = 0; d < r.nd; ++d) {
        const Index &ix = s.idx[d];
        int64_t mn, mx, lo, hi;
        if (ix.has_lo) {
            affine_minmax(ix.lo, vlo, vhi, &mn, &mx);
            lo = mn;
        } else {
            lo = 0;
        }
        if (ix.has_hi) {
            affine_minmax(ix.hi, vlo, vhi, &mn, &mx);
            hi = mx;
        } else {
            hi = shape[d] - 1;
        }
        if (lo < 0) lo = 0;
        if (hi > shape[d] - 1) hi = shape[d] - 1;
        r.lo[d] = lo;
        r.hi[d] = hi;
    }
    return r;
}

// ============================================================== distributions
size_t dtype_size(int dtype) {
    switch (dtype) {
        case LT_F32: return 4;
        case LT_BF16: return 2;
        case LT_U8: return 1;
        case LT_U32: return 4;
        case LT_F64: return 8;
        default: return 0;
    }
}

static void storage_for(const Box &box, int nd, int order, size_t esize, ChunkGeom *c) {
    int inner = (order == LT_ORDER_COL) ? 0 : nd - 1;
    int64_t A = (int64_t)(128 / esize);
    for (int d = 0; d < 3; ++d) {
        c->s_origin[d] = 0;
        c->s_ext[d] = 1;
        c->stride[d] = 0;
    }
    for (int d = 0; d < nd; ++d) {
        if (d == inner) {
            int64_t o = (box.lo[d] / A) * A;
            int64_t e = box.hi[d] + 1 - o;
            e = (e + A - 1) / A * A;
            c->s_origin[d] = o;
            c->s_ext[d] = e;
        } else {
            c->s_origin[d] = box.lo[d];
            c->s_ext[d] = box.extent(d);
        }
    }
    if (order == LT_ORDER_COL) {
        c->stride[0] = 1;
        c->stride[1] = c->s_ext[0];
    } else {
        int64_t s = 1;
        for (int d = nd - 1; d >= 0; --d) {
            c->stride[d] = s;
            s *= c->s_ext[d];
        }
    }
    size_t n = 1;
    for (int d = 0; d < nd; ++d) n *= (size_t)c->s_ext[d];
    c->bytes = n * esize;
}

bool make_geometry(int dtype, int nd, const int64_t shape[3], const lt_dist &dist, ArrayGeom *g, std::string *err) {
    if (dtype_size(dtype) == 0) {
        *err = "unknown dtype";
        return false;
    }
    if (nd < 1 || nd > 3) {
        *err = "ndim must be 1, 2 or 3";
        return false;
    }
    for (int d = 0; d < nd; ++d)
        if (shape[d] < 1) {
            *err = "every extent must be >= 1";
            return false;
        }
    if (dist.order != LT_ORDER_ROW && !(dist.order == LT_ORDER_COL && nd == 2)) {
        *err = "column-major chunk order is only for 2-D arrays";
        return false;
    }
    g->dtype = dtype;
    g->nd = nd;
    g->dist = dist;
    for (int d = 0; d < 3; ++d) g->shape[d] = d < nd ? shape[d] : 1;
    for (int d = 0; d < nd; ++d) {
        if (dist.halo[d] < 0 || dist.chunk[d] < 0) {
            *err = "chunk extents and halo widths must be >= 0";
            return false;
        }
        int64_t t = shape[d];
        switch (dist.kind) {
            case LT_DIST_BLOCK: break;
            case LT_DIST_ROWS:
                if (d == 0 && dist.chunk[0] > 0) t = dist.chunk[0];
                break;
            case LT_DIST_COLS:
                if (nd < 2) {
                    *err = "column distribution needs a 2-D or 3-D array";
                    return false;
                }
                if (d == 1 && dist.chunk[1] > 0) t = dist.chunk[1];
                break;
            case LT_DIST_TILES:
                if (dist.chunk[d] > 0) t = dist.chunk[d];
                break;
            default:
                *err = "unknown distribution kind";
                return false;
        }
        if (t > shape[d]) t = shape[d];
        g->tile[d] = t;
        g->ntile[d] = (shape[d] + t - 1) / t;
    }
    for (int d = nd; d < 3; ++d) {
        g->tile[d] = 1;
        g->ntile[d] = 1;
    }
    int64_t n = g->ntile[0] * g->ntile[1] * g->ntile[2];
    if (n > (int64_t)1 << 24) {
        *err = "too many chunks";
        return false;
    }
    g->chunks.clear();
    g->chunks.reserve((size_t)n);
    size_t es = dtype_size(dtype);
    for (int64_t t0 = 0; t0 < g->ntile[0]; ++t0)
        for (int64_t t1 = 0; t1 < g->ntile[1]; ++t1)
            for (int64_t t2 = 0; t2 < g->ntile[2]; ++t2) {
                int64_t t[3] = {t0, t1, t2};
                ChunkGeom c;
                c.owned.nd = nd;
                c.box.nd = nd;
                for (int d = 0; d < nd; ++d) {
                    c.owned.lo[d] = t[d] * g->tile[d];
                    c.owned.hi[d] = std::min((t[d] + 1) * g->tile[d], shape[d]) - 1;
                    int64_t h = dist.halo[d];
                    c.box.lo[d] = std::max<int64_t>(0, c.owned.lo[d] - h);
                    c.box.hi[d] = std::min<int64_t>(shape[d] - 1, c.owned.hi[d] + h);
                }
                storage_for(c.box, nd, dist.order, es, &c);
                g->chunks.push_back(c);
            }
    return true;
}

std::vector<int64_t> chunks_intersecting(const ArrayGeom &g, const Box &region) {
    std::vector<int64_t> out;
    if (region.empty()) return out;
    int64_t t0[3] = {0, 0, 0}, t1[3] = {0, 0, 0};
    for (int d = 0; d < g.nd; ++d) {
        int64_t h = g.dist.halo[d];
        int64_t lo = region.lo[d] - h, hi = region.hi[d] + h;
        if (lo < 0) lo = 0;
        if (hi > g.shape[d] - 1) hi = g.shape[d] - 1;
        t0[d] = lo / g.tile[d];
        t1[d] = hi / g.tile[d];
    }
    for (int64_t a = t0[0]; a <= t1[0]; ++a)
        for (int64_t b = t0[1]; b <= t1[1]; ++b)
            for (int64_t c = t0[2]; c <= t1[2]; ++c) {
                int64_t idx = (a * g.ntile[1] + b) * g.ntile[2] + c;
                if (!g.chunks[(size_t)idx].box.intersect(region).empty()) out.push_back(idx);
            }
    return out;
}

ChunkGeom temp_geometry(const ArrayGeom &g, const Box &region) {
    ChunkGeom c;
    c.box = region;
    c.owned = region;
    storage_for(region, g.nd, g.dist.order, g.esize(), &c);
    return c;
}

// ============================================================== planner
bool plan_launch(const Annotation &a, const std::vector<int> &stmt_of_param, const std::vector<PlanArray> &arrays,
                 const uint64_t grid[3], const uint64_t block[3], const int64_t superblock[3], LaunchPlan *out,
                 std::string *err) {
    int64_t G[3], B[3], S[3];
    for (int d = 0; d < 3; ++d) {
        G[d] = (int64_t)(grid[d] ? grid[d] : 1);
        B[d] = (int64_t)(block[d] ? block[d] : 1);
        if (G[d] < 1 || B[d] < 1 || G[d] > ((int64_t)1 << 50)) {
            *err = "grid and block extents must be >= 1";
            return false;
        }
        int64_t s = superblock[d] > 0 ? superblock[d] : G[d];
        s = (s + B[d] - 1) / B[d] * B[d];
        S[d] = s;
        out->nsb[d] = (G[d] + s - 1) / s;
    }
    int64_t total = out->nsb[0] * out->nsb[1] * out->nsb[2];
    if (total > ((int64_t)1 << 22)) {
        *err = "too many superblocks (more than 4M)";
        return false;
    }
    out->sbs.clear();
    out->sbs.reserve((size_t)total);
    std::vector<int64_t> vlo, vhi;
    for (int64_t z = 0; z < out->nsb[2]; ++z)
        for (int64_t y = 0; y < out->nsb[1]; ++y)
            for (int64_t x = 0; x < out->nsb[0]; ++x) {
                SuperblockPlan sb;
                sb.index = (z * out->nsb[1] + y) * out->nsb[0] + x;
                sb.threads.nd = 3;
                int64_t k[3] = {x, y, z};
                for (int d = 0; d < 3; ++d) {
                    sb.threads.lo[d] = k[d] * S[d];
                    sb.threads.hi[d] = std::min((k[d] + 1) * S[d], G[d]) - 1;
                }
                var_ranges(a, sb.threads, B, &vlo, &vhi);
                for (size_t p = 0; p < stmt_of_param.size(); ++p) {
                    ArgPlan ap;
                    ap.param = (int)p;
                    int si = stmt_of_param[p];
                    if (si < 0) {
                        ap.kind = ARG_VALUE;
                        sb.args.push_back(ap);
                        continue;
                    }
                    const Stmt &st = a.stmts[(size_t)si];
                    const ArrayGeom &g = *arrays[p].geom;
                    ap.stmt = si;
                    ap.mode = st.mode;
                    ap.op = st.op;
                    ap.region = eval_region(st, vlo, vhi, g.shape);
                    if (ap.region.empty()) {
                        ap.kind = ARG_NONE;
                        sb.args.push_back(ap);
                        continue;
                    }
                    std::vector<int64_t> cand = chunks_intersecting(g, ap.region);
                    int64_t best = -1, best_vol = -1;
                    for (int64_t c : cand) {
                        const ChunkGeom &cg = g.chunks[(size_t)c];
                        if (!cg.box.contains(ap.region)) continue;
                        int64_t v = cg.owned.intersect(ap.region).volume();
                        if (v > best_vol) {
                            best_vol = v;
                            best = c;
                        }
                    }
                    if (st.mode == MODE_REDUCE) {
                        ap.kind = ARG_REDUCE;
                        for (int64_t c : cand)
                            ap.pieces.push_back({c, g.chunks[(size_t)c].box.intersect(ap.region)});
                    } else if (best >= 0) {
                        ap.kind = ARG_DIRECT;
                        ap.chunk = best;
                        if (st.mode != MODE_READ)
                            for (int64_t c : cand)
                                if (c != best)
                                    ap.replicas.push_back({c, g.chunks[(size_t)c].box.intersect(ap.region)});
                    } else if (st.mode == MODE_READ) {
                        ap.kind = ARG_PACK;
                        for (int64_t c : cand) {
                            Box b = g.chunks[(size_t)c].owned.intersect(ap.region);
                            if (!b.empty()) ap.pieces.push_back({c, b});
                        }
                    } else {
                        ap.kind = ARG_TEMPW;
                        for (int64_t c : cand)
                            ap.pieces.push_back({c, g.chunks[(size_t)c].box.intersect(ap.region)});
                        if (st.mode == MODE_READWRITE)
                            for (int64_t c : cand) {
                                Box b = g.chunks[(size_t)c].owned.intersect(ap.region);
                                if (!b.empty()) ap.replicas.push_back({c, b});  // pack sources
                            }
                    }
                    sb.args.push_back(ap);
                }
                out->sbs.push_back(std::move(sb));
            }
    return true;
}

static void box_json(std::ostringstream &o, const Box &b) {
    o << "{\"lo\":[";
    for (int d = 0; d < b.nd; ++d) o << (d ? "," : "") << b.lo[d];
    o << "],\"hi\":[";
    for (int d = 0; d < b.nd; ++d) o << (d ? "," : "") << b.hi[d];
    o << "]}";
}

static const char *kind_name(int k) {
    switch (k) {
        case ARG_VALUE: return "value";
        case ARG_NONE: return "none";
        case ARG_DIRECT: return "direct";
        case ARG_PACK: return "pack";
        case ARG_TEMPW: return "temp_write";
        default: return "reduce";
    }
}

static const char *mode_name(int m) {
    switch (m) {
        case MODE_READ: return "read";
        case MODE_WRITE: return "write";
        case MODE_READWRITE: return "readwrite";
        default: return "reduce";
    }
}

std::string plan_to_json(const LaunchPlan &p) {
    std::ostringstream o;
    o << "{\"nsb\":[" << p.nsb[0] << "," << p.nsb[1] << "," << p.nsb[2] << "],\"superblocks\":[";
    for (size_t s = 0; s < p.sbs.size(); ++s) {
        const SuperblockPlan &sb = p.sbs[s];
        o << (s ? "," : "") << "{\"index\":" << sb.index << ",\"threads\":";
        box_json(o, sb.threads);
        o << ",\"args\":[";
        for (size_t k = 0; k < sb.args.size(); ++k) {
            const ArgPlan &ap = sb.args[k];
            o << (k ? "," : "") << "{\"param\":" << ap.param << ",\"kind\":\"" << kind_name(ap.kind) << "\"";
            if (ap.kind != ARG_VALUE) {
                o << ",\"mode\":\"" << mode_name(ap.mode) << "\",\"region\":";
                box_json(o, ap.region);
                o << ",\"chunk\":" << ap.chunk << ",\"pieces\":[";
                for (size_t q = 0; q < ap.pieces.size(); ++q) {
                    o << (q ? "," : "") << "{\"chunk\":" << ap.pieces[q].chunk << ",\"box\":";
                    box_json(o, ap.pieces[q].box);
                    o << "}";
                }
                o << "],\"replicas\":[";
                for (size_t q = 0; q < ap.replicas.size(); ++q) {
                    o << (q ? "," : "") << "{\"chunk\":" << ap.replicas[q].chunk << ",\"box\":";
                    box_json(o, ap.replicas[q].box);
                    o << "}";
                }
                o << "]";
            }
            o << "}";
        }
        o << "]}";
    }
    o << "]}";
    return o.str();
}

}  // namespace lt
