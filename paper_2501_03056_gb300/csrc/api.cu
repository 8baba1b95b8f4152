// extern "C" entry points of the relaxation library (include/fppg.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>

#include "../../include/fppg.h"
#include "body.h"

using namespace fppg;

namespace fppg {
void set_global_error(const char *msg);
}

struct fppg_ctx {
    Body body;
    Group group;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t n = 0;
    bool has_particles = false;
    int fixed_features = 0;
    std::vector<int32_t> cls_host;
    int mobile_mask = (1 << FPPG_S) | (1 << FPPG_V) | (1 << FPPG_F);   // classes that move
    int cascade = 0;               // surface re-projection rule (fppg_set_projection_rule)
    // Boolean operations this body takes part in (fppg_boolean), in order:
    // the other operand, FPPG_UNION / FPPG_DIFFERENCE / FPPG_INTERSECTION,
    // whether this body is the first operand, and this body's
    // intersection-curve segments with the other one [curve_lo, curve_hi)
    struct BoolRel {
        fppg_ctx *other;
        int op;
        bool first;
        int curve_lo, curve_hi;
    };
    std::vector<BoolRel> rels;
    BoolRel *rel_with(const fppg_ctx *o) {
        for (BoolRel &r : rels)
            if (r.other == o) return &r;
        return nullptr;
    }
    int64_t n_ghost = 0;           // the last n_ghost particles are ghosts (fppg_set_ghost_count)
    int split_buf = -1;            // grid buffer of the last fppg_relax_forces, until its step
    // device staging of the host particle arrays of set / get, kept between
    // calls (both synchronise the stream before they return)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    ~fppg_ctx() {
        if (stage) cudaFree(stage);
    }
};

struct fppg_batch {
    Group group;
    std::vector<fppg_ctx *> ctxs;
    std::vector<int64_t> off;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

// errors of calls without a handle (creation, the static-scratch entry
// point) go to a fixed per-thread buffer, so reporting them never allocates
thread_local char g_global_err[256] = {0};

int fail(std::string &dst, int code, const std::string &msg) {
    dst = msg;
    return code;
}

int fail_global(int code, const char *msg) {
    fppg::set_global_error(msg);
    return code;
}

#define CUDA_OR(dst, x)                                                                 \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess)                                                          \
            return fail(dst, e_ == cudaErrorMemoryAllocation ? FPPG_ERR_OOM : FPPG_ERR_CUDA, \
                        std::string(#x) + ": " + cudaGetErrorString(e_));               \
    } while (0)

__global__ void k_pack(const float *__restrict__ xyz, const int32_t *__restrict__ cls, int64_t n, int body,
                       float4 *__restrict__ pos, int32_t *__restrict__ cons) {
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    pos[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2],
                         __uint_as_float(class_bit(cls[i]) | ((uint32_t)body << 8)));
    cons[i] = -1;
}

__global__ void k_unpack(const float4 *__restrict__ pos, int64_t n, float *__restrict__ xyz) {
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    xyz[3 * i] = p.x;
    xyz[3 * i + 1] = p.y;
    xyz[3 * i + 2] = p.z;
}

__global__ void k_set_body(float4 *__restrict__ pos, int64_t n, int body) {
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    float4 p = pos[i];
    p.w = __uint_as_float((__float_as_uint(p.w) & 0xffu) | ((uint32_t)body << 8));
    pos[i] = p;
}

inline unsigned nb(int64_t n) { return (unsigned)std::max<int64_t>((n + 255) / 256, 1); }

// f(begin, end) over [0, n) in chunks on up to 32 host threads (at least 2^20
// items each); a thread that cannot be started runs its chunk here
template <typename F>
void host_parallel(int64_t n, F &&f) {
    const int64_t per = (int64_t)1 << 20;
    const int64_t hw = std::max<int64_t>((int64_t)std::thread::hardware_concurrency(), 1);
    const int nt = (int)std::min<int64_t>(std::min<int64_t>((n + per - 1) / per, hw), 32);
    if (nt <= 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)nt);
    for (int t = 1; t < nt; t++) {
        const int64_t a = n * t / nt, b = n * (t + 1) / nt;
        try {
            th.emplace_back([&f, a, b] { f(a, b); });
        } catch (...) {
            f(a, b);
        }
    }
    f((int64_t)0, n / nt);
    for (std::thread &x : th) x.join();
}

MeshView view_of(const Body &b) {
    return MeshView{b.geo, b.vx, b.pn, b.hrng, b.compact, b.tlist, b.seg, b.lines, b.occ, b.drank, b.coff, b.cand};
}

// (re)build the single-body group of a context
// the staging buffer of ctx with at least `bytes` bytes
int stage_buf(fppg_ctx *ctx, size_t bytes, void **out) {
    if (bytes > ctx->stage_bytes) {
        if (ctx->stage) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        CUDA_OR(ctx->err, dev_malloc(&ctx->stage, bytes));
        ctx->stage_bytes = bytes;
    }
    *out = ctx->stage;
    return FPPG_OK;
}

int ctx_group(fppg_ctx *c) {
    Group &g = c->group;
    g.d.B = 1;
    g.d.total_cells = (int64_t)c->body.ng_n[0] * c->body.ng_n[1] * c->body.ng_n[2];
    g.hp.assign(1, make_params(c->body, 0u, 0, (int)c->n, c->fixed_features));
    g.hp[0].mobile = c->mobile_mask;
    g.hp[0].cascade = c->cascade;
    if (g.cell_order) g.hp[0].row_rank = g.d.row_rank;   // the body's table (fppg_set_cell_order)
    g.mesh = view_of(c->body);
    const int r = g.upload_params(c->stream, c->err);
    return r == 0 ? FPPG_OK : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
}

} // namespace

void fppg::set_global_error(const char *msg) { snprintf(g_global_err, sizeof(g_global_err), "%s", msg); }

namespace {
// allocations to go before one fails (fppg_debug_fail_allocation); -1: none
std::atomic<int64_t> g_fail_after{-1};
} // namespace

cudaError_t fppg::dev_malloc_raw(void **p, size_t bytes) {
    int64_t k = g_fail_after.load();
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1)) {
            if (k == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

extern "C" {

int fppg_create(const float *verts_host, int64_t nv, const int32_t *tris_host, int64_t nt, float dx, float h,
                fppg_ctx **out) {
    g_global_err[0] = 0;
    if (!out) return fail_global(FPPG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!verts_host || !tris_host || nv < 3 || nt < 1 || nv > (1 << 30) || nt > (1 << 29))
        return fail_global(FPPG_ERR_ARG, "empty or oversized mesh");
    if (!(dx > 0.f) || !(h > 0.f) || !std::isfinite(dx) || !std::isfinite(h))
        return fail_global(FPPG_ERR_ARG, "dx and h must be finite and positive");
    for (int64_t i = 0; i < 3 * nv; i++)
        if (!std::isfinite(verts_host[i])) return fail_global(FPPG_ERR_ARG, "non-finite vertex");
    for (int64_t i = 0; i < 3 * nt; i++)
        if (tris_host[i] < 0 || tris_host[i] >= nv)
            return fail_global(FPPG_ERR_ARG, "triangle index out of range");
    fppg_ctx *c = new (std::nothrow) fppg_ctx();
    if (!c) return fail_global(FPPG_ERR_OOM, "host allocation failed");
    c->body.verts_host.assign(verts_host, verts_host + 3 * nv);
    c->body.tris_host.assign(tris_host, tris_host + 3 * nt);
    int r = c->body.build_mesh(verts_host, nv, tris_host, nt, dx, h, c->stream, c->err);
    if (r == 0) r = ctx_group(c);
    if (r != 0) {
        set_global_error(c->err.c_str());
        delete c;
        return r == 1 ? FPPG_ERR_ARG : r;
    }
    *out = c;
    return FPPG_OK;
}

int fppg_destroy(fppg_ctx *ctx) {
    if (!ctx) return FPPG_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (const fppg_ctx::BoolRel &r : ctx->rels) {
        auto &o = r.other->rels;
        for (size_t q = 0; q < o.size(); q++)
            if (o[q].other == ctx) {
                o.erase(o.begin() + (long)q);
                break;
            }
    }
    delete ctx;
    return FPPG_OK;
}

const char *fppg_last_error(const fppg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_global_err; }

int fppg_set_stream(fppg_ctx *ctx, void *stream) {
    if (!ctx) return FPPG_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return FPPG_OK;
}

int fppg_set_fixed_features(fppg_ctx *ctx, int32_t fixed) {
    if (!ctx) return FPPG_ERR_ARG;
    ctx->fixed_features = fixed ? 1 : 0;
    return ctx_group(ctx);
}

int fppg_set_mobile_classes(fppg_ctx *ctx, int32_t mask) {
    if (!ctx) return FPPG_ERR_ARG;
    if (mask & ~((1 << FPPG_S) | (1 << FPPG_V) | (1 << FPPG_F)))
        return fail(ctx->err, FPPG_ERR_ARG, "only S, V and F can be mobile");
    ctx->mobile_mask = mask;
    return ctx_group(ctx);
}

int fppg_set_projection_rule(fppg_ctx *ctx, int32_t rule) {
    if (!ctx) return FPPG_ERR_ARG;
    if (rule != FPPG_PROJECT_CLOSEST && rule != FPPG_PROJECT_CASCADE)
        return fail(ctx->err, FPPG_ERR_ARG, "unknown projection rule");
    ctx->cascade = rule == FPPG_PROJECT_CASCADE ? 1 : 0;
    return ctx_group(ctx);
}

int fppg_set_cell_order(fppg_ctx *ctx, int32_t order) {
    if (!ctx) return FPPG_ERR_ARG;
    if (order != FPPG_ORDER_ROWS && order != FPPG_ORDER_MORTON_ROWS)
        return fail(ctx->err, FPPG_ERR_ARG, "unknown cell order");
    const int r = ctx->group.set_cell_order(order, ctx->stream, ctx->err);
    if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
    return ctx_group(ctx);
}

int fppg_extract_features(fppg_ctx *ctx, float dihedral_deg, int64_t *n_edges) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!std::isfinite(dihedral_deg)) return fail(ctx->err, FPPG_ERR_ARG, "dihedral_deg must be finite");
    int r = ctx->body.extract_features(dihedral_deg, ctx->stream, ctx->err);
    // the lines are rebuilt from the feature edges alone: intersection-curve
    // lines are gone (fppg_boolean_curve adds them again)
    for (fppg_ctx::BoolRel &rel : ctx->rels) rel.curve_lo = rel.curve_hi = 0;
    if (r) {
        // the group must not keep a view of feature segments that are gone
        const std::string msg = ctx->err;
        ctx_group(ctx);
        ctx->err = msg;
        return r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA;
    }
    if (n_edges) *n_edges = (int64_t)ctx->body.fe.size() / 2;
    return ctx_group(ctx);
}

int fppg_get_feature_edges(fppg_ctx *ctx, int32_t *edges_host, int64_t cap, int64_t *n) {
    if (!ctx) return FPPG_ERR_ARG;
    if (cap < 0) return fail(ctx->err, FPPG_ERR_ARG, "negative capacity");
    const int64_t m = (int64_t)ctx->body.fe.size() / 2;
    if (n) *n = m;
    if (edges_host) std::copy(ctx->body.fe.begin(), ctx->body.fe.begin() + 2 * std::min(cap, m), edges_host);
    return FPPG_OK;
}

int fppg_get_feature_lines(fppg_ctx *ctx, int64_t *line_nseg_host, int32_t *closed_host, int64_t cap_lines,
                           int32_t *seg_v_host, int64_t cap_seg, int64_t *n_lines, int64_t *n_seg) {
    if (!ctx) return FPPG_ERR_ARG;
    if (cap_lines < 0 || cap_seg < 0) return fail(ctx->err, FPPG_ERR_ARG, "negative capacity");
    const Body &b = ctx->body;
    if (n_lines) *n_lines = b.nlines;
    if (n_seg) *n_seg = b.nseg;
    for (int64_t l = 0; l < std::min<int64_t>(cap_lines, b.nlines); l++) {
        if (line_nseg_host) line_nseg_host[l] = b.line_nseg[l];
        if (closed_host) closed_host[l] = b.line_closed[l];
    }
    if (seg_v_host) std::copy(b.seg_v.begin(), b.seg_v.begin() + 2 * std::min<int64_t>(cap_seg, b.nseg), seg_v_host);
    return FPPG_OK;
}

int fppg_map_particles(fppg_ctx *ctx, const fppg_map_opts *opts, int64_t *n_out) {
    NvtxRange nvtx_("fppg_map_particles");
    if (!ctx || !opts) return FPPG_ERR_ARG;
    if (opts->band_cells < 0 || opts->band_cells > 64 || opts->inner_cells < 0 || opts->inner_cells > 64)
        return fail(ctx->err, FPPG_ERR_ARG, "band_cells or inner_cells outside 0..64");
    int64_t n = 0;
    std::vector<int32_t> cls;
    ctx->has_particles = false;     // until the new set is complete
    int r = map_particles(ctx->group, ctx->body, opts->surface, opts->volume, opts->features, opts->band_cells,
                          opts->band_cells > 0 ? opts->inner_cells : 0, ctx->stream, &n, cls, ctx->err);
    if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : (r == 6 ? FPPG_ERR_INTERNAL : FPPG_ERR_CUDA));
    ctx->n = n;
    ctx->cls_host.swap(cls);
    ctx->has_particles = true;
    if (n_out) *n_out = n;
    return ctx_group(ctx);
}

int fppg_set_particles(fppg_ctx *ctx, const float *xyz_host, const int32_t *cls_host, int64_t n) {
    if (!ctx) return FPPG_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 31) return fail(ctx->err, FPPG_ERR_ARG, "particle count out of range");
    if (n > 0 && (!xyz_host || !cls_host)) return fail(ctx->err, FPPG_ERR_ARG, "NULL particle buffer");
    // the upload into the staging buffer (scratch, not yet the state) runs
    // while the host checks the input
    float *dx = nullptr;
    int32_t *dc = nullptr;
    if (n > 0) {
        void *st = nullptr;
        int r = stage_buf(ctx, 16 * (size_t)n, &st);
        if (r) return r;
        dx = (float *)st;
        dc = (int32_t *)(dx + 3 * n);
        CUDA_OR(ctx->err, cudaMemcpyAsync(dx, xyz_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_OR(ctx->err, cudaMemcpyAsync(dc, cls_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    // branch-free scans (they vectorise), on several host threads: a class
    // outside 0..4, an exponent field of all ones (inf or NaN)
    std::atomic<uint32_t> bad_cls{0u}, bad_xyz{0u};
    host_parallel(n, [&](int64_t a, int64_t b) {
        uint32_t bc = 0u, bx = 0u;
        for (int64_t i = a; i < b; i++) bc |= (uint32_t)((uint32_t)cls_host[i] > 4u);
        for (int64_t i = 3 * a; i < 3 * b; i++) {
            uint32_t w;
            memcpy(&w, xyz_host + i, sizeof(w));
            bx |= (uint32_t)((w & 0x7f800000u) == 0x7f800000u);
        }
        if (bc) bad_cls.fetch_or(bc);
        if (bx) bad_xyz.fetch_or(bx);
    });
    if (bad_cls.load() || bad_xyz.load()) {
        cudaStreamSynchronize(ctx->stream);   // the staging copies end before the buffer is reused
        return fail(ctx->err, FPPG_ERR_ARG, bad_cls.load() ? "class outside 0..4" : "non-finite coordinate");
    }
    Group &g = ctx->group;
    ctx->has_particles = false;     // until the new set is complete
    ctx->split_buf = -1;
    ctx->n_ghost = 0;
    if (n != g.d.N || !g.d.pos) {
        int r = g.alloc_particles(n, ctx->err);
        if (r) return r;
    }
    ctx->n = n;
    if ((int64_t)ctx->cls_host.size() != n) ctx->cls_host.resize((size_t)n);
    int32_t *ch = ctx->cls_host.data();
    host_parallel(n, [&](int64_t a, int64_t b) { std::copy(cls_host + a, cls_host + b, ch + a); });
    if (n > 0) k_pack<<<nb(n), 256, 0, ctx->stream>>>(dx, dc, n, 0, g.d.pos, g.d.cons);
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    ctx->has_particles = true;
    return ctx_group(ctx);
}

int fppg_set_constraints(fppg_ctx *ctx, const int32_t *cons_host, int64_t n) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (n != ctx->n || (n > 0 && !cons_host)) return fail(ctx->err, FPPG_ERR_ARG, "constraint count mismatch");
    std::atomic<uint32_t> bad{0u};
    const int32_t *cl = ctx->cls_host.data();
    const int64_t nt = ctx->body.nt, ns = ctx->body.nseg;
    host_parallel(n, [&](int64_t a, int64_t b) {
        uint32_t e = 0u;
        for (int64_t i = a; i < b; i++) {
            const int64_t lim = cl[i] == FPPG_S ? nt : cl[i] == FPPG_F ? ns : 0;
            e |= (uint32_t)(cons_host[i] < -1 || cons_host[i] >= lim);
        }
        if (e) bad.fetch_or(e);
    });
    if (bad.load()) return fail(ctx->err, FPPG_ERR_ARG, "constraint id out of range for its class");
    if (n > 0)
        CUDA_OR(ctx->err, cudaMemcpyAsync(ctx->group.d.cons, cons_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                                          ctx->stream));
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    return FPPG_OK;
}

int fppg_boolean(fppg_ctx *a, fppg_ctx *b, int32_t op, int64_t *n_a, int64_t *n_b) {
    NvtxRange nvtx_("fppg_boolean");
    if (!a || !b || a == b) return fail_global(FPPG_ERR_ARG, "a Boolean operation needs two different bodies");
    if (op != FPPG_UNION && op != FPPG_DIFFERENCE && op != FPPG_INTERSECTION)
        return fail(a->err, FPPG_ERR_ARG, "unknown Boolean operation");
    if (!a->has_particles || !b->has_particles) return fail(a->err, FPPG_ERR_STATE, "no particles set");
    if (a->rel_with(b)) return fail(a->err, FPPG_ERR_STATE, "the two bodies are already in a Boolean operation");
    if ((int)a->rels.size() >= kMaxPartners || (int)b->rels.size() >= kMaxPartners)
        return fail(a->err, FPPG_ERR_STATE, "a body takes part in at most four Boolean operations");
    if (a->body.dx != b->body.dx || a->body.h != b->body.h || a->fixed_features != b->fixed_features)
        return fail(a->err, FPPG_ERR_ARG, "Boolean operands need the same dx, h and feature setting");
    if (!a->body.closed || !b->body.closed)
        return fail(a->err, FPPG_ERR_ARG, "Boolean operands need closed, consistently oriented meshes");
    cudaStream_t s = a->stream;
    CUDA_OR(a->err, cudaStreamSynchronize(b->stream));
    int32_t *in = nullptr;
    const int64_t na = a->n, nbp = b->n;
    CUDA_OR(a->err, dev_malloc(&in, sizeof(int32_t) * (size_t)std::max<int64_t>(na + nbp, 1)));
    ray_parity(b->group, a->group.d.pos, na, in, s);
    ray_parity(a->group, b->group.d.pos, nbp, in + na, s);
    std::vector<int32_t> inside((size_t)(na + nbp));
    if (na + nbp > 0)
        CUDA_OR(a->err, cudaMemcpyAsync(inside.data(), in, sizeof(int32_t) * (na + nbp), cudaMemcpyDeviceToHost, s));
    CUDA_OR(a->err, cudaStreamSynchronize(s));
    cudaFree(in);
    // keep rules (inside = ray parity against the other body; vol = volume
    // or innermost): union a keeps !inside, b keeps !inside || vol (the
    // overlap keeps one copy of its volume particles); difference a - b: a
    // keeps !inside, b keeps inside && !vol (the cavity wall); intersection:
    // a keeps inside, b keeps inside && !vol
    fppg_ctx *m[2] = {a, b};
    for (int q = 0; q < 2; q++) {
        fppg_ctx *c = m[q];
        const int64_t n = c->n, base = q == 0 ? 0 : na;
        std::vector<float> xyz(3 * (size_t)std::max<int64_t>(n, 1));
        std::vector<int32_t> cls((size_t)std::max<int64_t>(n, 1)), cons((size_t)std::max<int64_t>(n, 1));
        int r = fppg_get_particles(c, xyz.data(), cls.data(), cons.data(), n, nullptr);
        if (r) return r;
        std::vector<float> kx;
        std::vector<int32_t> kc, kk;
        for (int64_t i = 0; i < n; i++) {
            const bool vol = cls[i] == FPPG_V || cls[i] == FPPG_I, in = inside[base + i] != 0;
            const bool keep = op == FPPG_UNION ? (q == 0 ? !in : (!in || vol))
                                               : op == FPPG_DIFFERENCE ? (q == 0 ? !in : (in && !vol))
                                                                       : (q == 0 ? in : (in && !vol));
            if (!keep) continue;
            kx.insert(kx.end(), &xyz[3 * i], &xyz[3 * i] + 3);
            kc.push_back(cls[i]);
            kk.push_back(cons[i]);
        }
        r = fppg_set_particles(c, kx.data(), kc.data(), (int64_t)kc.size());
        if (!r) r = fppg_set_constraints(c, kk.data(), (int64_t)kk.size());
        if (r) return r;
    }
    a->rels.push_back(fppg_ctx::BoolRel{b, op, true, 0, 0});
    b->rels.push_back(fppg_ctx::BoolRel{a, op, false, 0, 0});
    if (n_a) *n_a = a->n;
    if (n_b) *n_b = b->n;
    return FPPG_OK;
}

int fppg_union(fppg_ctx *a, fppg_ctx *b, int64_t *n_a, int64_t *n_b) {
    return fppg_boolean(a, b, FPPG_UNION, n_a, n_b);
}

int fppg_boolean_curve(fppg_ctx *a, fppg_ctx *b, int64_t *n_added) {
    NvtxRange nvtx_("fppg_boolean_curve");
    if (!a || !b || a == b) return fail_global(FPPG_ERR_ARG, "the intersection curve needs two different bodies");
    fppg_ctx::BoolRel *rel = a->rel_with(b);
    if (!rel) return fail(a->err, FPPG_ERR_STATE, "the intersection curve follows fppg_boolean on the pair");
    if (!a->has_particles) return fail(a->err, FPPG_ERR_STATE, "no particles set");
    Body &bd = a->body;
    if (rel->curve_hi > rel->curve_lo || (b->rel_with(a)->curve_hi > b->rel_with(a)->curve_lo))
        return fail(a->err, FPPG_ERR_STATE, "the intersection curve is there already");
    const int nseg_before = bd.nseg;
    const size_t verts_before = bd.verts_host.size();
    const bool has_before = bd.has_features;
    const int64_t n = a->n;
    std::vector<float> xyz(3 * (size_t)n);
    std::vector<int32_t> cls((size_t)n), cons((size_t)n);
    int r = fppg_get_particles(a, xyz.data(), cls.data(), cons.data(), n, nullptr);
    if (r) return r;
    std::vector<float> fx;
    std::vector<int32_t> fc, fs;
    r = bd.add_curve(b->body, fx, fc, fs, a->stream, a->err);
    if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
    xyz.insert(xyz.end(), fx.begin(), fx.end());
    cls.insert(cls.end(), fc.begin(), fc.end());
    cons.insert(cons.end(), fs.begin(), fs.end());
    r = fppg_set_particles(a, xyz.data(), cls.data(), (int64_t)cls.size());
    if (!r) r = fppg_set_constraints(a, cons.data(), (int64_t)cons.size());
    if (r) {
        // no curve without its particles: the host lines go back to the
        // body's own (the device copy only holds more segments than used)
        const std::string msg = a->err;
        bd.drop_lines_after(nseg_before, verts_before, has_before);
        ctx_group(a);
        a->err = msg;
        return r;
    }
    rel->curve_lo = nseg_before;
    rel->curve_hi = bd.nseg;
    if (n_added) *n_added = (int64_t)fc.size();
    return FPPG_OK;
}

int fppg_get_curve_points(fppg_ctx *ctx, float *xyz_host, int64_t cap, int64_t *n) {
    if (!ctx) return FPPG_ERR_ARG;
    if (cap < 0) return fail(ctx->err, FPPG_ERR_ARG, "negative capacity");
    const Body &b = ctx->body;
    const int64_t m = (int64_t)b.verts_host.size() / 3 - b.nv;
    if (n) *n = m;
    if (xyz_host)
        std::copy(b.verts_host.begin() + 3 * (size_t)b.nv, b.verts_host.begin() + 3 * (size_t)(b.nv + std::min(cap, m)),
                  xyz_host);
    return FPPG_OK;
}

int fppg_get_particles(fppg_ctx *ctx, float *xyz_host, int32_t *cls_host, int32_t *cons_host, int64_t cap,
                       int64_t *n_out) {
    if (!ctx) return FPPG_ERR_ARG;
    if (n_out) *n_out = ctx->n;
    const int64_t m = std::min(cap, ctx->n);
    if (m <= 0) return FPPG_OK;
    if (xyz_host) {
        void *st = nullptr;
        int r = stage_buf(ctx, 12 * (size_t)ctx->n, &st);
        if (r) return r;
        float *dx = (float *)st;
        k_unpack<<<nb(ctx->n), 256, 0, ctx->stream>>>(ctx->group.d.pos, ctx->n, dx);
        CUDA_OR(ctx->err, cudaMemcpyAsync(xyz_host, dx, sizeof(float) * 3 * m, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    }
    if (cons_host)
        CUDA_OR(ctx->err, cudaMemcpyAsync(cons_host, ctx->group.d.cons, sizeof(int32_t) * m, cudaMemcpyDeviceToHost,
                                          ctx->stream));
    if (cls_host) std::copy(ctx->cls_host.begin(), ctx->cls_host.begin() + m, cls_host);
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    return FPPG_OK;
}

static int relax_impl(fppg_ctx *ctx, int32_t n_iter, bool energy_mode) {
    NvtxRange nvtx_("fppg_relax");
    if (!ctx) return FPPG_ERR_ARG;
    if (n_iter < 0) return fail(ctx->err, FPPG_ERR_ARG, "n_iter < 0");
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (!ctx->rels.empty())
        return fail(ctx->err, FPPG_ERR_STATE, "a Boolean operand relaxes in a batch together with its partners");
    for (int32_t it = 0; it < n_iter; it++) iterate(ctx->group, ctx->stream, energy_mode);
    CUDA_OR(ctx->err, cudaGetLastError());
    return FPPG_OK;
}

int fppg_relax(fppg_ctx *ctx, int32_t n_iter) { return relax_impl(ctx, n_iter, false); }

int fppg_set_ghost_count(fppg_ctx *ctx, int64_t n_ghost) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (n_ghost < 0 || n_ghost > ctx->n) return fail(ctx->err, FPPG_ERR_ARG, "ghost count outside 0..n");
    ctx->n_ghost = n_ghost;
    tag_ghosts(ctx->group, ctx->n - n_ghost, ctx->stream);
    CUDA_OR(ctx->err, cudaGetLastError());
    return FPPG_OK;
}

int fppg_relax_forces(fppg_ctx *ctx, float *amax_host) {
    if (!ctx || !amax_host) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (!ctx->rels.empty())
        return fail(ctx->err, FPPG_ERR_STATE, "a Boolean operand relaxes in a batch together with its partners");
    uint32_t a = 0u;
    if (ctx->n > 0) {
        Group &g = ctx->group;
        ctx->split_buf = build_grid(g, ctx->stream);
        forces(g, ctx->stream, nullptr);
        CUDA_OR(ctx->err, cudaMemcpyAsync(&a, g.d.amax, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    } else {
        ctx->split_buf = 0;
    }
    memcpy(amax_host, &a, sizeof(float));
    return FPPG_OK;
}

int fppg_relax_step(fppg_ctx *ctx, float amax) {
    if (!ctx) return FPPG_ERR_ARG;
    if (ctx->split_buf < 0) return fail(ctx->err, FPPG_ERR_STATE, "fppg_relax_step needs a fppg_relax_forces first");
    if (!(amax >= 0.f) || !std::isfinite(amax)) return fail(ctx->err, FPPG_ERR_ARG, "amax must be finite, >= 0");
    const int buf = ctx->split_buf;
    ctx->split_buf = -1;
    if (ctx->n == 0) return FPPG_OK;
    Group &g = ctx->group;
    uint32_t a;
    memcpy(&a, &amax, sizeof(a));
    CUDA_OR(ctx->err, cudaMemcpyAsync(g.d.amax, &a, sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    step_and_project(g, ctx->stream, buf);
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    return FPPG_OK;
}

int fppg_relax_energy(fppg_ctx *ctx, int32_t n_iter) { return relax_impl(ctx, n_iter, true); }

int fppg_stats(fppg_ctx *ctx, fppg_stats_t *out) {
    if (!ctx || !out) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    int r = stats(ctx->group, ctx->stream, out->mean_rho, out->std_rho, &out->min_pair_over_dx,
                  &out->max_disp_over_dx, out->count, ctx->err);
    return r == 0 ? FPPG_OK : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
}

int fppg_debug_grid(fppg_ctx *ctx, uint32_t *key_host, uint32_t *perm_host, uint32_t *cells_host,
                    uint32_t *start_host, uint32_t *end_host, int64_t cap_cells, int64_t *n_cells) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    Group &g = ctx->group;
    const int64_t n = ctx->n;
    if (n == 0) {
        if (n_cells) *n_cells = 0;
        return FPPG_OK;
    }
    int buf = build_grid(g, ctx->stream);
    std::vector<uint32_t> ks(n), perm(n);
    CUDA_OR(ctx->err, cudaMemcpyAsync(ks.data(), g.d.key[buf], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR(ctx->err, cudaMemcpyAsync(perm.data(), g.d.id[buf], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    // the dense start table: cell c holds the slots [fstart[8c], fstart[8c + 8])
    std::vector<uint32_t> table((size_t)kSlabs * (size_t)g.d.total_cells + 1);
    CUDA_OR(ctx->err, cudaMemcpyAsync(table.data(), g.d.fstart, sizeof(uint32_t) * table.size(),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    if (key_host)
        for (int64_t k = 0; k < n; k++) key_host[perm[k]] = ks[k];
    if (perm_host) std::copy(perm.begin(), perm.end(), perm_host);
    int64_t m = 0;
    for (int64_t c = 0; c < g.d.total_cells; c++) {
        const uint32_t cs = table[(size_t)kSlabs * c], ce = table[(size_t)kSlabs * (c + 1)];
        if (ce <= cs) continue;
        if (m < cap_cells) {
            if (cells_host) cells_host[m] = (uint32_t)c;
            if (start_host) start_host[m] = cs;
            if (end_host) end_host[m] = ce;
        }
        m++;
    }
    if (n_cells) *n_cells = m;
    return FPPG_OK;
}

int fppg_debug_forces(fppg_ctx *ctx, float *acc_host, int32_t *count_host, float *amax_host) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    Group &g = ctx->group;
    const int64_t n = ctx->n;
    if (n == 0) return FPPG_OK;
    float *dacc = nullptr;
    int32_t *dcnt_s = nullptr, *dcnt = nullptr;
    CUDA_OR(ctx->err, dev_malloc(&dacc, sizeof(float) * 3 * n));
    CUDA_OR(ctx->err, dev_malloc(&dcnt_s, sizeof(int32_t) * n));
    CUDA_OR(ctx->err, dev_malloc(&dcnt, sizeof(int32_t) * n));
    int buf = build_grid(g, ctx->stream);
    forces(g, ctx->stream, dcnt_s);
    unpermute(g, buf, ctx->stream, dacc, dcnt_s, dcnt);
    uint32_t am = 0;
    if (acc_host) CUDA_OR(ctx->err, cudaMemcpyAsync(acc_host, dacc, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (count_host)
        CUDA_OR(ctx->err, cudaMemcpyAsync(count_host, dcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR(ctx->err, cudaMemcpyAsync(&am, g.d.amax, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    if (amax_host) memcpy(amax_host, &am, 4);
    cudaFree(dacc);
    cudaFree(dcnt_s);
    cudaFree(dcnt);
    return FPPG_OK;
}

int fppg_debug_search(fppg_ctx *ctx, int64_t *queued, int32_t *closed) {
    if (!ctx) return FPPG_ERR_ARG;
    uint32_t q[2] = {0u, 0u};
    if (ctx->group.d.work_count) {
        CUDA_OR(ctx->err, cudaMemcpyAsync(q, ctx->group.d.work_count, sizeof(q), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
    }
    if (queued) *queued = (int64_t)q[0] + q[1];
    if (closed) *closed = ctx->body.closed ? 1 : 0;
    return FPPG_OK;
}

int fppg_debug_cell_lists(fppg_ctx *ctx, int64_t *cells, int64_t *entries, int64_t *overflow) {
    if (!ctx) return FPPG_ERR_ARG;
    const Body &b = ctx->body;
    int64_t ov = 0;
    if (overflow && b.n_dil > 0) {
        std::vector<uint32_t> off((size_t)b.n_dil);
        CUDA_OR(ctx->err, cudaMemcpy(off.data(), b.coff, sizeof(uint32_t) * off.size(), cudaMemcpyDeviceToHost));
        for (uint32_t o : off) ov += o >> 31;
    }
    if (cells) *cells = b.n_dil;
    if (entries) *entries = b.n_cand;
    if (overflow) *overflow = ov;
    return FPPG_OK;
}

int fppg_work_counts(fppg_ctx *ctx, int64_t *candidates, int64_t *pairs, int64_t *tested) {
    if (!ctx) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    Group &g = ctx->group;
    const int64_t n = ctx->n;
    int64_t c = 0, p = 0, t = 0;
    if (n > 0) {
        int32_t *dcnt = nullptr, *dcand = nullptr, *dtest = nullptr;
        CUDA_OR(ctx->err, dev_malloc(&dcnt, sizeof(int32_t) * n));
        CUDA_OR(ctx->err, dev_malloc(&dcand, sizeof(int32_t) * n));
        CUDA_OR(ctx->err, dev_malloc(&dtest, sizeof(int32_t) * n));
        build_grid(g, ctx->stream);
        forces(g, ctx->stream, dcnt, dcand, dtest);
        std::vector<int32_t> hc(n), hp(n), ht(n);
        CUDA_OR(ctx->err, cudaMemcpyAsync(hc.data(), dcand, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaMemcpyAsync(hp.data(), dcnt, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaMemcpyAsync(ht.data(), dtest, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_OR(ctx->err, cudaStreamSynchronize(ctx->stream));
        cudaFree(dcnt);
        cudaFree(dcand);
        cudaFree(dtest);
        for (int64_t k = 0; k < n; k++) {
            c += hc[k];
            t += ht[k];
            if (hc[k] > 0) p += hp[k];
        }
    }
    if (candidates) *candidates = c;
    if (pairs) *pairs = p;
    if (tested) *tested = t;
    return FPPG_OK;
}

int fppg_project_points(fppg_ctx *ctx, const float *y_host, const int32_t *cls_host, const int32_t *cons_host,
                        int64_t n, float *x_host, int32_t *cons_out_host, int32_t *ok_host) {
    if (!ctx) return FPPG_ERR_ARG;
    if (n < 0 || (n > 0 && (!y_host || !cls_host || !x_host || !cons_out_host || !ok_host)))
        return fail(ctx->err, FPPG_ERR_ARG, "bad projection buffers");
    if (n == 0) return FPPG_OK;
    for (int64_t i = 0; i < n; i++)
        if (cls_host[i] < 0 || cls_host[i] > 4) return fail(ctx->err, FPPG_ERR_ARG, "class outside 0..4");
    float *dy = nullptr, *dxo = nullptr;
    int32_t *dcls = nullptr, *dcin = nullptr, *dcout = nullptr, *dok = nullptr;
    CUDA_OR(ctx->err, dev_malloc(&dy, sizeof(float) * 3 * n));
    CUDA_OR(ctx->err, dev_malloc(&dxo, sizeof(float) * 3 * n));
    CUDA_OR(ctx->err, dev_malloc(&dcls, sizeof(int32_t) * n));
    CUDA_OR(ctx->err, dev_malloc(&dcout, sizeof(int32_t) * n));
    CUDA_OR(ctx->err, dev_malloc(&dok, sizeof(int32_t) * n));
    if (cons_host) CUDA_OR(ctx->err, dev_malloc(&dcin, sizeof(int32_t) * n));
    cudaStream_t s = ctx->stream;
    CUDA_OR(ctx->err, cudaMemcpyAsync(dy, y_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
    CUDA_OR(ctx->err, cudaMemcpyAsync(dcls, cls_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    if (cons_host) CUDA_OR(ctx->err, cudaMemcpyAsync(dcin, cons_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    project_points(ctx->group, dy, dcls, dcin, n, dxo, dcout, dok, s);
    CUDA_OR(ctx->err, cudaMemcpyAsync(x_host, dxo, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    CUDA_OR(ctx->err, cudaMemcpyAsync(cons_out_host, dcout, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    CUDA_OR(ctx->err, cudaMemcpyAsync(ok_host, dok, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    CUDA_OR(ctx->err, cudaStreamSynchronize(s));
    void *p[] = {dy, dxo, dcls, dcin, dcout, dok};
    for (void *q : p)
        if (q) cudaFree(q);
    return FPPG_OK;
}

int fppg_energy(fppg_ctx *ctx, const float *y_dev, const float *verts_dev, double *E_host, float *gy_dev,
                float *gV_dev) {
    if (!ctx || !y_dev || !E_host) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (ctx->n == 0) {
        *E_host = 0.0;
        return FPPG_OK;
    }
    int r = energy(ctx->group, ctx->body, y_dev, verts_dev, E_host, gy_dev, gV_dev, ctx->stream, ctx->err);
    return r == 0 ? FPPG_OK : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
}

int fppg_copy_positions_dev(fppg_ctx *ctx, float *xyz_dev) {
    if (!ctx || !xyz_dev) return FPPG_ERR_ARG;
    if (!ctx->has_particles) return fail(ctx->err, FPPG_ERR_STATE, "no particles set");
    if (ctx->n) k_unpack<<<nb(ctx->n), 256, 0, ctx->stream>>>(ctx->group.d.pos, ctx->n, xyz_dev);
    CUDA_OR(ctx->err, cudaGetLastError());
    return FPPG_OK;
}

// ---- batches ------------------------------------------------------------------
int fppg_batch_create(fppg_ctx *const *ctxs, int32_t n, fppg_batch **out) {
    if (!out) return FPPG_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n <= 0 || n > (1 << 20)) return fail_global(FPPG_ERR_ARG, "bad body list");
    for (int32_t i = 0; i < n; i++)
        if (!ctxs[i] || !ctxs[i]->has_particles)
            return fail_global(FPPG_ERR_STATE, "every body needs particles before batching");
    fppg_batch *b = new (std::nothrow) fppg_batch();
    if (!b) return fail_global(FPPG_ERR_OOM, "host allocation failed");
    b->ctxs.assign(ctxs, ctxs + n);
    b->stream = ctxs[0]->stream;
    Group &g = b->group;
    g.owns_mesh = true;
    DevGroup &d = g.d;
    d.B = n;
    // Bodies joined by Boolean operations form one assembly: one neighbour
    // grid over all their boxes (set up at the assembly's first body) and
    // one time step; root[i] = the assembly's first body
    auto index_of = [&](const fppg_ctx *c) {
        for (int32_t q = 0; q < n; q++)
            if (ctxs[q] == c) return q;
        return -1;
    };
    std::vector<int> root(n);
    for (int32_t i = 0; i < n; i++) root[i] = i;
    auto find = [&](int i) {
        while (root[i] != i) i = root[i] = root[root[i]];
        return i;
    };
    for (int32_t i = 0; i < n; i++)
        for (const fppg_ctx::BoolRel &r : ctxs[i]->rels) {
            const int j = index_of(r.other);
            if (j < 0) {
                delete b;
                return fail_global(FPPG_ERR_STATE, "a Boolean operand needs every partner in the same batch");
            }
            const int x = find(i), y = find(j);
            if (x != y) root[std::max(x, y)] = std::min(x, y);
        }
    std::vector<int> members(n, 0);
    for (int32_t i = 0; i < n; i++) members[find(i)]++;
    int64_t N = 0, cells = 0, nt = 0, nv = 0, hs = 0, nc = 0, np = 0, ns = 0, nl = 0, ow = 0;
    int64_t dw = 0, dl = 0, dc = 0;   // candidate-list ranks, starts and lists
    for (int32_t i = 0; i < n; i++) {
        const fppg_ctx *c = ctxs[i];
        const Body &bd = c->body;
        AsmParams A = make_params(bd, (uint32_t)cells, (int)N, (int)(N + c->n), c->fixed_features);
        A.amax_slot = i;
        A.mobile = c->mobile_mask;
        A.cascade = c->cascade;
        const int r0 = find(i);
        int64_t grid_cells = (int64_t)bd.ng_n[0] * bd.ng_n[1] * bd.ng_n[2];
        if (r0 < i) {
            const AsmParams &Q = g.hp[r0];
            for (int k = 0; k < 3; k++) {
                A.ng_o[k] = Q.ng_o[k];
                A.ng_n[k] = Q.ng_n[k];
            }
            A.ng_inv = Q.ng_inv;
            A.key_base = Q.key_base;
            grid_cells = 0;
        } else if (members[i] > 1) {
            float lo[3], hi[3];
            for (int k = 0; k < 3; k++) {
                lo[k] = bd.bbmin[k];
                hi[k] = bd.bbmax[k];
            }
            for (int32_t q = i + 1; q < n; q++)
                if (find(q) == i)
                    for (int k = 0; k < 3; k++) {
                        lo[k] = std::min(lo[k], ctxs[q]->body.bbmin[k]);
                        hi[k] = std::max(hi[k], ctxs[q]->body.bbmax[k]);
                    }
            if (!grid_setup(lo, hi, bd.ng_cell, 1.0, 1, A.ng_o, &A.ng_inv, A.ng_n)) {
                delete b;
                return fail_global(FPPG_ERR_ARG,
                                   "the shared grid of a Boolean assembly needs more than 2^20 cells per axis");
            }
            grid_cells = (int64_t)A.ng_n[0] * A.ng_n[1] * A.ng_n[2];
        }
        if (members[r0] > 1) {
            A.amax_slot = r0;
            A.slab_r2 = slab_reach2(A.R2, A.ng_inv);
        }
        // partner rules (1 stay outside, 2 stay inside): surface and feature
        // particles, then volume particles
        for (const fppg_ctx::BoolRel &r : c->rels) {
            const int q = A.npart++;
            const bool first = r.first;
            A.partner[q] = index_of(r.other);
            A.partner_surf[q] = r.op == FPPG_UNION ? 1 : r.op == FPPG_DIFFERENCE ? (first ? 1 : 2) : 2;
            A.partner_vol[q] = r.op == FPPG_UNION ? 0 : r.op == FPPG_DIFFERENCE ? (first ? 1 : 0) : (first ? 2 : 0);
            A.curve_lo[q] = r.curve_lo;
            A.curve_hi[q] = r.curve_hi;
            if (A.partner_vol[q] != 0) A.vol_rules = 1;
        }
        A.tri_off = (int)nt;
        A.vert_off = (int)nv;
        A.hash_off = (uint32_t)hs;
        A.compact_off = (uint32_t)nc;
        A.tlist_off = (uint32_t)np;
        A.seg_off = (int)ns;
        A.line_off = (int)nl;
        A.occ_off = (uint32_t)ow;
        A.dil_off = (uint32_t)(ow + bd.occ_words);
        A.drank_off = (uint32_t)dw;
        A.coff_off = (uint32_t)dl;
        A.cand_off = (uint32_t)dc;
        g.hp.push_back(A);
        b->off.push_back(N);
        N += c->n;
        cells += grid_cells;
        nt += bd.nt;
        nv += bd.nv;
        hs += bd.hash_size;
        nc += bd.ncompact;
        np += bd.npairs;
        ns += bd.nseg;
        nl += bd.nlines;
        ow += 2 * bd.occ_words;
        dw += bd.occ_words;
        dl += bd.n_dil + 1;
        dc += bd.n_cand;
    }
    b->off.push_back(N);
    if (cells >= ((int64_t)1 << 29) || N > ((int64_t)1 << 31) || ow >= 0xffffffffLL || dl >= 0xffffffffLL ||
        dc >= 0x7fffffffLL) {
        delete b;
        return fail_global(FPPG_ERR_ARG, "batch too large for 32-bit keys");
    }
    d.total_cells = cells;
    std::string &err = b->err;
    int r = g.alloc_particles(N, err);
    auto A = [&](void **p, size_t bytes) { return dev_malloc(p, std::max<size_t>(bytes, 16)); };
    if (!r && (A((void **)&d.geo, sizeof(float4) * 5 * nt) || A((void **)&d.vx, sizeof(float4) * 3 * nt) ||
               A((void **)&d.pn, sizeof(float4) * 6 * nt) || A((void **)&d.hrng, sizeof(uint2) * hs) ||
               A((void **)&d.compact, sizeof(uint4) * nc) || A((void **)&d.tlist, sizeof(int32_t) * np) ||
               A((void **)&d.seg, sizeof(float4) * 3 * ns) || A((void **)&d.lines, sizeof(int2) * nl) ||
               A((void **)&d.occ, sizeof(uint32_t) * ow) || A((void **)&d.drank, sizeof(uint32_t) * dw) ||
               A((void **)&d.coff, sizeof(uint32_t) * dl) || A((void **)&d.cand, sizeof(int32_t) * dc)))
        r = FPPG_ERR_OOM;
    cudaStream_t s = b->stream;
    for (int32_t i = 0; i < n && !r; i++) {
        const Body &bd = ctxs[i]->body;
        const AsmParams &P = g.hp[i];
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
        };
        cp(d.geo + 5 * (size_t)P.tri_off, bd.geo, sizeof(float4) * 5 * bd.nt);
        cp(d.vx + 3 * (size_t)P.tri_off, bd.vx, sizeof(float4) * 3 * bd.nt);
        cp(d.pn + 6 * (size_t)P.tri_off, bd.pn, sizeof(float4) * 6 * bd.nt);
        cp(d.hrng + P.hash_off, bd.hrng, sizeof(uint2) * bd.hash_size);
        cp(d.compact + P.compact_off, bd.compact, sizeof(uint4) * bd.ncompact);
        cp(d.tlist + P.tlist_off, bd.tlist, sizeof(int32_t) * bd.npairs);
        if (bd.nseg) cp(d.seg + 3 * (size_t)P.seg_off, bd.seg, sizeof(float4) * 3 * bd.nseg);
        if (bd.nlines) cp(d.lines + P.line_off, bd.lines, sizeof(int2) * bd.nlines);
        cp(d.occ + P.occ_off, bd.occ, sizeof(uint32_t) * 2 * bd.occ_words);
        cp(d.drank + P.drank_off, bd.drank, sizeof(uint32_t) * bd.occ_words);
        cp(d.coff + P.coff_off, bd.coff, sizeof(uint32_t) * (bd.n_dil + 1));
        if (bd.n_cand) cp(d.cand + P.cand_off, bd.cand, sizeof(int32_t) * bd.n_cand);
        const int64_t cn = ctxs[i]->n;
        cp(d.pos + b->off[i], ctxs[i]->group.d.pos, sizeof(float4) * cn);
        cp(d.cons + b->off[i], ctxs[i]->group.d.cons, sizeof(int32_t) * cn);
        if (cn) k_set_body<<<nb(cn), 256, 0, s>>>(d.pos + b->off[i], cn, i);
    }
    g.mesh = MeshView{d.geo, d.vx, d.pn, d.hrng, d.compact, d.tlist, d.seg, d.lines, d.occ, d.drank, d.coff, d.cand};
    if (!r) r = g.upload_params(s, err);
    if (!r && cudaStreamSynchronize(s) != cudaSuccess) r = FPPG_ERR_CUDA;
    if (r) {
        set_global_error(err.empty() ? "batch allocation failed" : err.c_str());
        delete b;
        return r;
    }
    *out = b;
    return FPPG_OK;
}

int fppg_batch_destroy(fppg_batch *b) {
    if (!b) return FPPG_ERR_ARG;
    cudaStreamSynchronize(b->stream);
    delete b;
    return FPPG_OK;
}

int fppg_batch_set_stream(fppg_batch *b, void *stream) {
    if (!b) return FPPG_ERR_ARG;
    b->stream = (cudaStream_t)stream;
    return FPPG_OK;
}

int fppg_batch_set_graph_iters(fppg_batch *b, int32_t graph_iters) {
    if (!b || graph_iters <= 0 || graph_iters > 100000) return FPPG_ERR_ARG;
    if (b->group.graph && b->group.graph_iters != graph_iters) {
        cudaGraphExecDestroy(b->group.graph);
        b->group.graph = nullptr;
    }
    b->group.graph_iters = graph_iters;
    return FPPG_OK;
}

int fppg_batch_time_force(fppg_batch *b, int32_t enable) {
    if (!b) return FPPG_ERR_ARG;
    if (b->group.time_force != (enable != 0) && b->group.graph) {
        cudaGraphExecDestroy(b->group.graph);
        b->group.graph = nullptr;
    }
    b->group.time_force = enable != 0;
    return FPPG_OK;
}

static int build_graph(fppg_batch *b) {
    Group &g = b->group;
    if (g.graph_iters <= 0) g.graph_iters = 50;
    if (!g.graph_stream) CUDA_OR(b->err, cudaStreamCreateWithFlags(&g.graph_stream, cudaStreamNonBlocking));
    if (g.time_force) {
        while ((int)g.ev.size() < kPhaseEvents * g.graph_iters) {
            cudaEvent_t e;
            CUDA_OR(b->err, cudaEventCreate(&e));
            g.ev.push_back(e);
        }
    }
    g.ev_used = 0;
    cudaGraph_t graph;
    CUDA_OR(b->err, cudaStreamBeginCapture(g.graph_stream, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < g.graph_iters; it++) iterate(g, g.graph_stream, false);
    CUDA_OR(b->err, cudaStreamEndCapture(g.graph_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&g.graph, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_OR(b->err, e);
    return FPPG_OK;
}

int fppg_batch_relax(fppg_batch *b, int32_t n_iter, int32_t use_graph) {
    NvtxRange nvtx_("fppg_batch_relax");
    if (!b) return FPPG_ERR_ARG;
    if (n_iter < 0) return fail(b->err, FPPG_ERR_ARG, "n_iter < 0");
    Group &g = b->group;
    int32_t done = 0;
    if (use_graph) {
        if (!g.graph) {
            int r = build_graph(b);
            if (r) return r;
        }
        for (; done + g.graph_iters <= n_iter; done += g.graph_iters)
            CUDA_OR(b->err, cudaGraphLaunch(g.graph, b->stream));
    }
    const bool t = g.time_force;
    g.time_force = false;   // eager iterations are not timed
    for (; done < n_iter; done++) iterate(g, b->stream, false);
    g.time_force = t;
    CUDA_OR(b->err, cudaGetLastError());
    return FPPG_OK;
}

int fppg_batch_phase_ms(fppg_batch *b, double *ms4) {
    if (!b || !ms4) return FPPG_ERR_ARG;
    Group &g = b->group;
    if (!g.time_force || !g.graph || (int)g.ev.size() < kPhaseEvents * g.graph_iters)
        return fail(b->err, FPPG_ERR_STATE, "phase timing not active");
    CUDA_OR(b->err, cudaStreamSynchronize(b->stream));
    double tot[kPhaseEvents - 1] = {};
    for (int i = 0; i < g.graph_iters; i++)
        for (int k = 0; k + 1 < kPhaseEvents; k++) {
            float t = 0.f;
            CUDA_OR(b->err, cudaEventElapsedTime(&t, g.ev[kPhaseEvents * i + k], g.ev[kPhaseEvents * i + k + 1]));
            tot[k] += t;
        }
    for (int k = 0; k + 1 < kPhaseEvents; k++) ms4[k] = tot[k] / g.graph_iters;
    return FPPG_OK;
}

int fppg_batch_force_ms(fppg_batch *b, double *ms) {
    if (!b || !ms) return FPPG_ERR_ARG;
    double ph[kPhaseEvents - 1];
    const int r = fppg_batch_phase_ms(b, ph);
    if (r == FPPG_OK) *ms = ph[1];
    return r;
}

int fppg_batch_store(fppg_batch *b) {
    if (!b) return FPPG_ERR_ARG;
    cudaStream_t s = b->stream;
    DevGroup &d = b->group.d;
    for (size_t i = 0; i < b->ctxs.size(); i++) {
        fppg_ctx *c = b->ctxs[i];
        const int64_t cn = c->n;
        if (!cn) continue;
        CUDA_OR(b->err, cudaMemcpyAsync(c->group.d.pos, d.pos + b->off[i], sizeof(float4) * cn,
                                        cudaMemcpyDeviceToDevice, s));
        CUDA_OR(b->err, cudaMemcpyAsync(c->group.d.cons, d.cons + b->off[i], sizeof(int32_t) * cn,
                                        cudaMemcpyDeviceToDevice, s));
        k_set_body<<<nb(cn), 256, 0, s>>>(c->group.d.pos, cn, 0);
    }
    CUDA_OR(b->err, cudaStreamSynchronize(s));
    return FPPG_OK;
}

int fppg_batch_load(fppg_batch *b) {
    if (!b) return FPPG_ERR_ARG;
    cudaStream_t s = b->stream;
    DevGroup &d = b->group.d;
    for (size_t i = 0; i < b->ctxs.size(); i++) {
        fppg_ctx *c = b->ctxs[i];
        const int64_t cn = c->n;
        if (cn != b->off[i + 1] - b->off[i]) return fail(b->err, FPPG_ERR_STATE, "a body changed its particle count");
        if (!cn) continue;
        CUDA_OR(b->err, cudaMemcpyAsync(d.pos + b->off[i], c->group.d.pos, sizeof(float4) * cn,
                                        cudaMemcpyDeviceToDevice, s));
        CUDA_OR(b->err, cudaMemcpyAsync(d.cons + b->off[i], c->group.d.cons, sizeof(int32_t) * cn,
                                        cudaMemcpyDeviceToDevice, s));
        k_set_body<<<nb(cn), 256, 0, s>>>(d.pos + b->off[i], cn, (int)i);
    }
    CUDA_OR(b->err, cudaGetLastError());
    return FPPG_OK;
}

namespace {
struct TuneKey {
    int n_bucket, v_share;
    std::string gpu;
    bool operator<(const TuneKey &o) const {
        return std::tie(n_bucket, v_share, gpu) < std::tie(o.n_bucket, o.v_share, o.gpu);
    }
};
struct TuneVal {
    int variant, block, search_ctas, incremental, cell_order;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;
} // namespace

// switch the ordering of the keys; entering the incremental form forgets
// the previous order (its arrays may be stale after full sorts)
static void set_ordering(Group &g, bool incremental, cudaStream_t s) {
    if (incremental && !g.d.incremental) g.invalidate_order(s);
    g.d.incremental = incremental;
}

int fppg_batch_autotune(fppg_batch *b, int32_t iters, int32_t *variant, int32_t *block, int32_t *search_ctas,
                        int32_t *incremental, int32_t *cell_order, double *ms_per_iter) {
    NvtxRange nvtx_("fppg_batch_autotune");
    if (!b || iters <= 0 || iters > 10000) return FPPG_ERR_ARG;
    Group &g = b->group;
    DevGroup &d = g.d;
    cudaStream_t s = b->stream;
    int dev = 0, sms = 152;
    cudaDeviceProp prop;
    CUDA_OR(b->err, cudaGetDevice(&dev));
    CUDA_OR(b->err, cudaGetDeviceProperties(&prop, dev));
    sms = prop.multiProcessorCount;
    int64_t nv = 0;
    for (const fppg_ctx *c : b->ctxs)
        for (int32_t cl : c->cls_host) nv += cl == FPPG_V;
    int nb = 0;
    while ((int64_t)1 << (nb + 1) <= std::max<int64_t>(d.N, 1)) nb++;
    const TuneKey key{nb, d.N ? (int)(10 * nv / d.N) : 0, prop.name};
    TuneVal best{g.force_variant, g.force_block, g.search_thread ? 0 : g.search_blocks / std::max(sms, 1),
                 d.incremental ? 1 : 0, g.cell_order};
    double best_ms = 0.0;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        float4 *pos0 = nullptr;
        int32_t *cons0 = nullptr;
        CUDA_OR(b->err, dev_malloc(&pos0, sizeof(float4) * std::max<int64_t>(d.N, 1)));
        if (dev_malloc(&cons0, sizeof(int32_t) * std::max<int64_t>(d.N, 1)) != cudaSuccess) {
            cudaFree(pos0);
            return fail(b->err, FPPG_ERR_OOM, "autotune: out of device memory");
        }
        CUDA_OR(b->err, cudaMemcpyAsync(pos0, d.pos, sizeof(float4) * d.N, cudaMemcpyDeviceToDevice, s));
        CUDA_OR(b->err, cudaMemcpyAsync(cons0, d.cons, sizeof(int32_t) * d.N, cudaMemcpyDeviceToDevice, s));
        cudaEvent_t e0, e1;
        CUDA_OR(b->err, cudaEventCreate(&e0));
        CUDA_OR(b->err, cudaEventCreate(&e1));
        const bool tf = g.time_force;
        g.time_force = false;
        best_ms = 1e30;
        // one trial: the state restored, one untimed iteration, `iters` timed
        auto trial = [&](int v, int tb, int sc, int inc, int co, float *ms) -> int {
            g.force_variant = v;
            g.force_block = tb;
            g.search_thread = sc == 0;
            g.search_blocks = (sc == 0 ? 16 : sc) * sms;
            set_ordering(g, inc != 0, s);
            if (co != g.cell_order) {
                const int r = g.set_cell_order(co, s, b->err);
                if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
            }
            CUDA_OR(b->err, cudaMemcpyAsync(d.pos, pos0, sizeof(float4) * d.N, cudaMemcpyDeviceToDevice, s));
            CUDA_OR(b->err, cudaMemcpyAsync(d.cons, cons0, sizeof(int32_t) * d.N, cudaMemcpyDeviceToDevice, s));
            iterate(g, s, false);
            CUDA_OR(b->err, cudaEventRecord(e0, s));
            for (int it = 0; it < iters; it++) iterate(g, s, false);
            CUDA_OR(b->err, cudaEventRecord(e1, s));
            CUDA_OR(b->err, cudaEventSynchronize(e1));
            CUDA_OR(b->err, cudaEventElapsedTime(ms, e0, e1));
            return FPPG_OK;
        };
        const int inc0 = best.incremental, co0 = best.cell_order;
        auto consider = [&](int v, int tb, int sc, int inc, int co) -> int {
            float ms = 0.f;
            const int r = trial(v, tb, sc, inc, co, &ms);
            if (r) return r;
            if (ms / iters < best_ms) {
                best_ms = ms / iters;
                best = TuneVal{v, tb, sc, inc, co};
            }
            return FPPG_OK;
        };
        // the force kernel (variant, block) with the warp search on 4 CTAs
        // per SM, then the search grid with the fastest force kernel
        for (int v = 0; v < 2; v++)
            for (int tb : {128, 256})
                if (const int r = consider(v, tb, 4, inc0, co0)) return r;
        {
            const int v = best.variant, tb = best.block;
            for (int sc : {0, 8, 16})   // 0: one thread per queued particle
                if (const int r = consider(v, tb, sc, inc0, co0)) return r;
        }
        // the other ordering of the keys, then the other order of the grid
        // rows, with the fastest kernels
        if (const int r = consider(best.variant, best.block, best.search_ctas, 1 - inc0, co0)) return r;
        if (const int r = consider(best.variant, best.block, best.search_ctas, best.incremental, 1 - co0))
            if (r != FPPG_ERR_ARG) return r;   // a grid too large for the Morton table keeps row-major rows
        g.time_force = tf;
        CUDA_OR(b->err, cudaMemcpyAsync(d.pos, pos0, sizeof(float4) * d.N, cudaMemcpyDeviceToDevice, s));
        CUDA_OR(b->err, cudaMemcpyAsync(d.cons, cons0, sizeof(int32_t) * d.N, cudaMemcpyDeviceToDevice, s));
        CUDA_OR(b->err, cudaStreamSynchronize(s));
        cudaFree(pos0);
        cudaFree(cons0);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    g.force_variant = best.variant;
    g.force_block = best.block;
    g.search_thread = best.search_ctas == 0;
    g.search_blocks = (best.search_ctas == 0 ? 16 : best.search_ctas) * sms;
    set_ordering(g, best.incremental != 0, s);
    if (best.cell_order != g.cell_order) {
        const int r = g.set_cell_order(best.cell_order, s, b->err);
        if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
    }
    if (g.graph) {
        cudaGraphExecDestroy(g.graph);
        g.graph = nullptr;
    }
    if (variant) *variant = best.variant;
    if (block) *block = best.block;
    if (search_ctas) *search_ctas = best.search_ctas;
    if (incremental) *incremental = best.incremental;
    if (cell_order) *cell_order = best.cell_order;
    if (ms_per_iter) *ms_per_iter = cached ? 0.0 : best_ms;
    return FPPG_OK;
}

int fppg_batch_set_mobile_classes(fppg_batch *b, int32_t mask) {
    if (!b) return FPPG_ERR_ARG;
    if (mask & ~((1 << FPPG_S) | (1 << FPPG_V) | (1 << FPPG_F)))
        return fail(b->err, FPPG_ERR_ARG, "only S, V and F can be mobile");
    for (AsmParams &A : b->group.hp) A.mobile = mask;
    // the kernels read the parameters from device memory: a captured
    // graph sees the new mask without being captured again
    return b->group.upload_params(b->stream, b->err) ? FPPG_ERR_CUDA : FPPG_OK;
}

int fppg_batch_configure(fppg_batch *b, int32_t variant, int32_t block, int32_t search_ctas) {
    if (!b || variant < 0 || variant > 1 || (block != 128 && block != 256) || search_ctas < 0 || search_ctas > 64)
        return FPPG_ERR_ARG;
    Group &g = b->group;
    int dev = 0;
    cudaDeviceProp prop;
    CUDA_OR(b->err, cudaGetDevice(&dev));
    CUDA_OR(b->err, cudaGetDeviceProperties(&prop, dev));
    g.force_variant = variant;
    g.force_block = block;
    g.search_thread = search_ctas == 0;
    g.search_blocks = (search_ctas == 0 ? 16 : search_ctas) * prop.multiProcessorCount;
    if (g.graph) {
        cudaGraphExecDestroy(g.graph);
        g.graph = nullptr;
    }
    return FPPG_OK;
}

int fppg_debug_fail_allocation(int64_t k) {
    if (k < -1) return fail_global(FPPG_ERR_ARG, "k must be -1 (off) or a count of allocations");
    g_fail_after.store(k);
    return FPPG_OK;
}

int fppg_check_status(uint32_t *word, int32_t *checked) {
    if (!word) return FPPG_ERR_ARG;
#ifdef FPPG_CHECKED
    if (checked) *checked = 1;
#else
    if (checked) *checked = 0;
#endif
    *word = check_word_take();
    return *word == 0xffffffffu ? FPPG_ERR_CUDA : FPPG_OK;
}

int fppg_grid_lattice(const fppg_ctx *ctx, float *origin_host, float *d_host) {
    if (!ctx || !origin_host || !d_host) return fail_global(FPPG_ERR_ARG, "fppg_grid_lattice: NULL argument");
    for (int a = 0; a < 3; a++) origin_host[a] = ctx->body.tg_o[a];
    *d_host = ctx->body.dx;
    return FPPG_OK;
}

int fppg_device_sm_count(int32_t *sms) {
    if (!sms) return fail_global(FPPG_ERR_ARG, "sms is NULL");
    int dev = 0, v = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_global(FPPG_ERR_CUDA, cudaGetErrorString(e));
    *sms = v;
    return FPPG_OK;
}

int fppg_set_incremental(fppg_ctx *ctx, int32_t incremental) {
    if (!ctx || incremental < 0 || incremental > 1) return FPPG_ERR_ARG;
    set_ordering(ctx->group, incremental != 0, ctx->stream);
    CUDA_OR(ctx->err, cudaGetLastError());
    return FPPG_OK;
}

int fppg_batch_set_incremental(fppg_batch *b, int32_t incremental) {
    if (!b || incremental < 0 || incremental > 1) return FPPG_ERR_ARG;
    Group &g = b->group;
    set_ordering(g, incremental != 0, b->stream);
    if (g.graph) {
        cudaGraphExecDestroy(g.graph);
        g.graph = nullptr;
    }
    CUDA_OR(b->err, cudaGetLastError());
    return FPPG_OK;
}

int fppg_batch_set_cell_order(fppg_batch *b, int32_t order) {
    if (!b || (order != FPPG_ORDER_ROWS && order != FPPG_ORDER_MORTON_ROWS)) return FPPG_ERR_ARG;
    const int r = b->group.set_cell_order(order, b->stream, b->err);
    if (r) return r == 1 ? FPPG_ERR_ARG : (r == 3 ? FPPG_ERR_OOM : FPPG_ERR_CUDA);
    return FPPG_OK;
}

int32_t fppg_batch_kernels_per_iter(const fppg_batch *b) {
    // keys, 3 per radix pass, gather, the start scan, force, step, search
    return b ? grid_kernels(b->group.d) + 3 : -1;
}

int64_t fppg_batch_size(const fppg_batch *b) { return b ? b->group.d.N : -1; }

const char *fppg_batch_last_error(const fppg_batch *b) { return b ? b->err.c_str() : g_global_err; }

} // extern "C"
