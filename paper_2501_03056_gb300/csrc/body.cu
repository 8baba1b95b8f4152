// Host side of a body (feature lines) and of a group (allocation, params).
#include <algorithm>
#include <cmath>

#include "body.h"

namespace fppg {


// Feature lines from the sorted feature-edge list (Sec. 3.2.2): walks that
// start at singular vertices (feature degree 1 or > 2) in ascending vertex
// order, each incident uncoloured edge in ascending edge order, continuing
// through degree-2 vertices; then closed loops from the lowest uncoloured
// edge.  Edges are coloured as they are walked.
void Body::build_lines() {
    verts_host.resize(3 * (size_t)nv);   // intersection-curve lines are rebuilt by their own call
    const int64_t m = (int64_t)fe.size() / 2;
    std::vector<int32_t> deg(nv, 0);
    for (int64_t e = 0; e < m; e++) {
        deg[fe[2 * e]]++;
        deg[fe[2 * e + 1]]++;
    }
    std::vector<int64_t> first(nv + 1, 0);
    for (int v = 0; v < nv; v++) first[v + 1] = first[v] + deg[v];
    std::vector<int64_t> incident(2 * m), fill(first.begin(), first.end() - 1);
    for (int64_t e = 0; e < m; e++) {
        incident[fill[fe[2 * e]]++] = e;
        incident[fill[fe[2 * e + 1]]++] = e;
    }
    sing.clear();
    for (int v = 0; v < nv; v++)
        if (deg[v] == 1 || deg[v] > 2) sing.push_back(v);
    std::vector<char> used(m, 0);
    line_first.clear();
    line_nseg.clear();
    line_closed.clear();
    seg_v.clear();
    auto other = [&](int64_t e, int32_t v) { return fe[2 * e] == v ? fe[2 * e + 1] : fe[2 * e]; };
    auto next_edge = [&](int32_t v, int64_t from) {
        return incident[first[v]] == from ? incident[first[v] + 1] : incident[first[v]];
    };
    for (int32_t s : sing) {
        for (int64_t q = first[s]; q < first[s + 1]; q++) {
            int64_t e = incident[q];
            if (used[e]) continue;
            const int64_t start = (int64_t)seg_v.size() / 2;
            int32_t cur = s;
            while (true) {
                used[e] = 1;
                const int32_t nxt = other(e, cur);
                seg_v.push_back(cur);
                seg_v.push_back(nxt);
                if (deg[nxt] != 2) break;
                const int64_t e2 = next_edge(nxt, e);
                if (used[e2]) break;
                e = e2;
                cur = nxt;
            }
            line_first.push_back(start);
            line_nseg.push_back((int64_t)seg_v.size() / 2 - start);
            line_closed.push_back(0);
        }
    }
    for (int64_t e0 = 0; e0 < m; e0++) {
        if (used[e0]) continue;
        const int64_t start = (int64_t)seg_v.size() / 2;
        const int32_t v0 = fe[2 * e0];
        int32_t cur = v0;
        int64_t e = e0;
        int closed = 0;
        while (true) {
            used[e] = 1;
            const int32_t nxt = other(e, cur);
            seg_v.push_back(cur);
            seg_v.push_back(nxt);
            if (nxt == v0) {
                closed = 1;
                break;
            }
            const int64_t e2 = next_edge(nxt, e);
            if (used[e2]) break;
            e = e2;
            cur = nxt;
        }
        line_first.push_back(start);
        line_nseg.push_back((int64_t)seg_v.size() / 2 - start);
        line_closed.push_back(closed);
    }
    nseg = (int)(seg_v.size() / 2);
    nseg_own = nseg;
    nlines = (int)line_first.size();
    has_features = true;
}

void Body::drop_features() {
    has_features = false;
    fe.clear();
    sing.clear();
    line_first.clear();
    line_nseg.clear();
    line_closed.clear();
    seg_v.clear();
    nseg = nlines = nseg_own = 0;
    verts_host.resize(3 * (size_t)nv);   // curve points go with the lines
}

int Body::upload_lines(cudaStream_t s, std::string &err, bool keep_on_failure) {
    std::vector<float4> hs(3 * (size_t)std::max(nseg, 1));
    std::vector<int2> hl((size_t)std::max(nlines, 1));
    for (int l = 0; l < nlines; l++) {
        hl[l] = make_int2((int)line_first[l], (int)line_nseg[l]);
        for (int64_t q = line_first[l]; q < line_first[l] + line_nseg[l]; q++) {
            const float *a = &verts_host[3 * (size_t)seg_v[2 * q]];
            const float *b = &verts_host[3 * (size_t)seg_v[2 * q + 1]];
            double e[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
            double len = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            float lb;
            int li = l;
            memcpy(&lb, &li, 4);
            hs[3 * q] = make_float4(a[0], a[1], a[2], lb);
            hs[3 * q + 1] = make_float4(b[0], b[1], b[2], 0.f);
            hs[3 * q + 2] = len > 0 ? make_float4((float)(e[0] / len), (float)(e[1] / len), (float)(e[2] / len),
                                                  (float)len)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float4 *nseg_d = nullptr;
    int2 *nlines_d = nullptr;
    if (dev_malloc(&nseg_d, sizeof(float4) * hs.size()) != cudaSuccess ||
        dev_malloc(&nlines_d, sizeof(int2) * hl.size()) != cudaSuccess) {
        if (nseg_d) cudaFree(nseg_d);
        if (nlines_d) cudaFree(nlines_d);
        err = "feature lines: out of device memory";
        if (keep_on_failure) return 3;   // the caller restores the host lines the old buffers hold
        // no half-built feature set: the body is left without features
        if (seg) cudaFree(seg);
        if (lines) cudaFree(lines);
        seg = nullptr;
        lines = nullptr;
        drop_features();
        return 3;
    }
    if (seg) cudaFree(seg);
    if (lines) cudaFree(lines);
    seg = nseg_d;
    lines = nlines_d;
    cudaMemcpyAsync(seg, hs.data(), sizeof(float4) * hs.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(lines, hl.data(), sizeof(int2) * hl.size(), cudaMemcpyHostToDevice, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        err = std::string("feature lines: ") + cudaGetErrorString(e);
        return 4;
    }
    return 0;
}

static double host_alpha3(double h) { return 21.0 / (16.0 * M_PI * h * h * h); }

static double host_W(double r, double h) {
    double q = r / h;
    if (q > 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return host_alpha3(h) * t * t * t * t * (2.0 * q + 1.0);
}

// ideal kernel sum of a perfect lattice of spacing dx in dim dimensions
static double lattice_w0(double dx, double h, int dim) {
    int m = (int)std::ceil(2.0 * h / dx) + 1;
    double s = 0.0;
    for (int i = -m; i <= m; i++)
        for (int j = (dim >= 2 ? -m : 0); j <= (dim >= 2 ? m : 0); j++)
            for (int k = (dim >= 3 ? -m : 0); k <= (dim >= 3 ? m : 0); k++)
                s += host_W(dx * std::sqrt((double)(i * i + j * j + k * k)), h);
    return s;
}

AsmParams make_params(const Body &b, uint32_t key_base, int p_begin, int p_end, int fixed_features) {
    AsmParams A;
    memset(&A, 0, sizeof(A));
    for (int k = 0; k < 3; k++) {
        A.ng_o[k] = b.ng_o[k];
        A.ng_n[k] = b.ng_n[k];
        A.tg_o[k] = b.tg_o[k];
        A.tg_n[k] = b.tg_n[k];
    }
    A.ng_inv = b.ng_inv;
    A.slab_r2 = slab_reach2(b.R2, b.ng_inv);
    A.tg_inv = b.tg_inv;
    A.key_base = key_base;
    A.hash_mask = (uint32_t)(b.hash_size - 1);
    A.occ_off = 0;
    A.dil_off = (uint32_t)b.occ_words;
    A.nt = b.nt;
    A.nv = b.nv;
    A.nseg = b.nseg;
    A.nlines = b.nlines;
    A.fixed_features = fixed_features;
    const double h = (double)b.h;
    A.h = b.h;
    A.R2 = b.R2;
    A.half_inv_h = (float)(1.0 / (2.0 * h));
    A.alpha = (float)host_alpha3(h);
    A.w_zero = A.alpha;
    A.force_scale = (float)(5.0 * host_alpha3(h) / (h * h));
    A.step_h = (float)(h / 16.0);
    A.dx = b.dx;
    A.edge_tol = b.edge_tol;
    A.closed = b.closed ? 1 : 0;
    A.mobile = (1 << kClsS) | (1 << kClsV) | (1 << kClsF);
    A.cascade = 0;
    A.npart = 0;
    A.vol_rules = 0;
    A.amax_slot = 0;
    A.w0[0] = (float)lattice_w0((double)b.dx, h, 2);
    A.w0[1] = (float)lattice_w0((double)b.dx, h, 3);
    A.w0[2] = (float)lattice_w0((double)b.dx, h, 1);
    A.p_begin = p_begin;
    A.p_end = p_end;
    return A;
}

// the bits of v moved to the even bit positions
static uint64_t spread_even(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

void morton_row_ranks(int ny, int nz, std::vector<uint32_t> &rank) {
    const int64_t m = (int64_t)ny * nz;
    std::vector<std::pair<uint64_t, uint32_t>> code((size_t)m);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++) {
            const uint32_t r = (uint32_t)y + (uint32_t)ny * (uint32_t)z;
            code[r] = {spread_even((uint32_t)y) | (spread_even((uint32_t)z) << 1), r};
        }
    std::sort(code.begin(), code.end());
    rank.resize((size_t)m);
    for (int64_t q = 0; q < m; q++) rank[code[(size_t)q].second] = (uint32_t)q;
}

#define CKA(x)                                                                  \
    do {                                                                        \
        cudaError_t e_ = (x);                                                   \
        if (e_ != cudaSuccess) {                                                \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);              \
            return e_ == cudaErrorMemoryAllocation ? 3 : 4;                     \
        }                                                                       \
    } while (0)

// Every particle and grid array of the group freed and cleared (N = 0), so
// that the next allocation starts from scratch.
void Group::release_particles() {
    DevGroup &g = d;
    void *ptrs[] = {g.pos,    g.cons,   g.cons_s,   g.key[0], g.key[1],  g.id[0],   g.id[1],  g.pos_s,
                    g.pos_p,  g.cert,   g.acc_s,    g.hist,   g.coef_s,  g.work,    g.fstart, g.bstart,
                    g.amax,   g.maxdisp, g.work_count, g.totals};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    free_order_state();
    g.pos = g.pos_s = g.pos_p = g.cert = g.acc_s = nullptr;
    g.cons = g.cons_s = nullptr;
    g.key[0] = g.key[1] = g.id[0] = g.id[1] = nullptr;
    g.hist = g.fstart = g.bstart = g.amax = g.maxdisp = g.work_count = g.totals = nullptr;
    g.coef_s = nullptr;
    g.work = nullptr;
    g.N = 0;
}

int Group::alloc_particles(int64_t N, std::string &err) {
    const int r = alloc_particles_once(N, err);
    if (r) release_particles();   // no half-allocated group: the next call starts over
    return r;
}

void Group::free_order_state() {
    DevGroup &g = d;
    void *ptrs[] = {g.key_id, g.chg_bits, g.keep_bits, g.tile_cnt, g.tile_pos, g.ck[0], g.ck[1], g.cv[0],
                    g.cv[1],  g.uk,       g.uv,        g.split,    g.counts,   g.scan_tmp_n};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    g.key_id = g.chg_bits = g.keep_bits = g.tile_cnt = g.tile_pos = nullptr;
    g.uk = g.uv = g.split = g.counts = g.scan_tmp_n = nullptr;
    g.ck[0] = g.ck[1] = g.cv[0] = g.cv[1] = nullptr;
}

__global__ void k_iota_u32(uint32_t *__restrict__ a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (uint32_t)i;
}

// The arrays of the incremental ordering: the previous order starts as the
// identity over ids with no key recorded, so the first grid build sorts
// every particle.  Allocated with the particles.
int Group::alloc_order_state(std::string &err) {
    DevGroup &g = d;
    free_order_state();
    const size_t n1 = (size_t)std::max<int64_t>(g.N, 1);
    const int64_t nblk = (std::max<int64_t>(g.N, 1) + 2047) / 2048;
    CKA(dev_malloc(&g.key_id, sizeof(uint32_t) * n1));
    // tiles of 2048 (those of the compactions), 32 flags a word
    const int64_t ntile = (std::max<int64_t>(g.N, 1) + 2047) / 2048;
    const size_t nword = (size_t)(ntile * 64);
    CKA(dev_malloc(&g.chg_bits, sizeof(uint32_t) * nword));
    CKA(dev_malloc(&g.keep_bits, sizeof(uint32_t) * nword));
    CKA(dev_malloc(&g.tile_cnt, sizeof(uint32_t) * (size_t)(2 * ntile)));
    CKA(dev_malloc(&g.tile_pos, sizeof(uint32_t) * (size_t)(2 * ntile)));
    for (int k = 0; k < 2; k++) {
        CKA(dev_malloc(&g.ck[k], sizeof(uint32_t) * n1));
        CKA(dev_malloc(&g.cv[k], sizeof(uint32_t) * n1));
    }
    CKA(dev_malloc(&g.uk, sizeof(uint32_t) * n1));
    CKA(dev_malloc(&g.uv, sizeof(uint32_t) * n1));
    CKA(dev_malloc(&g.split, sizeof(uint32_t) * (size_t)(nblk + 2)));
    CKA(dev_malloc(&g.counts, 2 * sizeof(uint32_t)));
    CKA(dev_malloc(&g.scan_tmp_n, sizeof(uint32_t) * (size_t)scan_tmp_elems(2 * ntile)));
    CKA(cudaMemset(g.key_id, 0xff, sizeof(uint32_t) * n1));
    k_iota_u32<<<(unsigned)((n1 + 255) / 256), 256>>>(g.id[0], (int64_t)n1);
    CKA(cudaGetLastError());
    CKA(cudaDeviceSynchronize());
    return 0;
}

void Group::invalidate_order(cudaStream_t s) {
    if (d.key_id && d.N > 0) cudaMemsetAsync(d.key_id, 0xff, sizeof(uint32_t) * (size_t)d.N, s);
}

int Group::alloc_particles_once(int64_t N, std::string &err) {
    DevGroup &g = d;
    void *old[] = {g.pos,   g.cons,  g.cons_s, g.key[0], g.key[1], g.id[0], g.id[1],
                   g.pos_s, g.pos_p, g.cert,   g.acc_s,  g.hist,   g.coef_s, g.work};
    for (void *p : old)
        if (p) cudaFree(p);
    g.pos = g.pos_s = g.pos_p = g.cert = g.acc_s = nullptr;
    g.cons = g.cons_s = nullptr;
    g.key[0] = g.key[1] = g.id[0] = g.id[1] = nullptr;
    g.hist = nullptr;
    g.coef_s = nullptr;
    g.work = nullptr;
    g.N = N;
    const size_t n1 = (size_t)std::max<int64_t>(N, 1);
    g.n_tiles = (int)std::max<int64_t>(radix_tiles(N), 1);
    g.key_bits = fine_key_bits(g.total_cells);
    int digit_bits = 8;
    g.passes = radix_pass_plan(g.key_bits, &digit_bits);
    CKA(dev_malloc(&g.pos, sizeof(float4) * n1));
    CKA(dev_malloc(&g.cons, sizeof(int32_t) * n1));
    CKA(dev_malloc(&g.cons_s, sizeof(int32_t) * n1));
    for (int k = 0; k < 2; k++) {
        CKA(dev_malloc(&g.key[k], sizeof(uint32_t) * n1));
        CKA(dev_malloc(&g.id[k], sizeof(uint32_t) * n1));
    }
    CKA(dev_malloc(&g.pos_s, sizeof(float4) * n1));
    CKA(dev_malloc(&g.pos_p, sizeof(float4) * (n1 + 1)));
    CKA(dev_malloc(&g.cert, sizeof(float4) * n1));
    CKA(cudaMemset(g.cert, 0, sizeof(float4) * n1));
    CKA(dev_malloc(&g.acc_s, sizeof(float4) * n1));
    CKA(dev_malloc(&g.coef_s, sizeof(float) * (n1 + 1)));
    CKA(dev_malloc(&g.work, (sizeof(int4) + sizeof(uint2)) * n1));   // queue entries, then their ranges
    if (!g.work_count) {
        CKA(dev_malloc(&g.work_count, 2 * sizeof(uint32_t)));
        CKA(cudaMemset(g.work_count, 0, 2 * sizeof(uint32_t)));
    }
    CKA(dev_malloc(&g.hist, sizeof(uint32_t) * kMaxDigits * (size_t)g.n_tiles));
    if (!g.totals) CKA(dev_malloc(&g.totals, sizeof(uint32_t) * kMaxDigits));
    if (!g.fstart) {
        // dense start table of every fine key (+1), the counts it is scanned
        // from (zero between iterations) and the scan's block sums
        const size_t f1 = (size_t)kSlabs * (size_t)std::max<int64_t>(g.total_cells, 1) + 1;
        CKA(dev_malloc(&g.fstart, sizeof(uint32_t) * f1));
        CKA(dev_malloc(&g.bstart, sizeof(uint32_t) * (size_t)(start_blocks((int64_t)f1) + 1)));
    }
    // the incremental ordering for large groups (the autotuner may switch)
    {
        const int r = alloc_order_state(err);
        if (r) return r;
        g.incremental = N >= kIncrementalMinN;
    }
    if (!g.amax) {
        CKA(dev_malloc(&g.amax, sizeof(uint32_t) * (size_t)std::max(g.B, 1)));
        CKA(dev_malloc(&g.maxdisp, sizeof(uint32_t) * (size_t)std::max(g.B, 1)));
        CKA(cudaMemset(g.amax, 0, sizeof(uint32_t) * (size_t)std::max(g.B, 1)));
        CKA(cudaMemset(g.maxdisp, 0, sizeof(uint32_t) * (size_t)std::max(g.B, 1)));
    }
    return 0;
}

int Group::upload_params(cudaStream_t s, std::string &err) {
    if (!d.params) CKA(dev_malloc(&d.params, sizeof(AsmParams) * (size_t)std::max<int>(d.B, 1)));
    CKA(cudaMemcpyAsync(d.params, hp.data(), sizeof(AsmParams) * hp.size(), cudaMemcpyHostToDevice, s));
    CKA(cudaStreamSynchronize(s));
    return 0;
}

int Group::set_cell_order(int order, cudaStream_t s, std::string &err) {
    if (order && !d.row_rank) {
        // one table per grid: a body shares the grid (and the table) of the
        // first body with its key base (the members of a Boolean assembly)
        std::vector<uint32_t> all, t;
        row_off.assign(hp.size(), 0);
        for (size_t i = 0; i < hp.size(); i++) {
            size_t owner = i;
            for (size_t j = 0; j < i; j++)
                if (hp[j].key_base == hp[i].key_base) {
                    owner = j;
                    break;
                }
            if (owner != i) {
                row_off[i] = row_off[owner];
                continue;
            }
            const int64_t rows = (int64_t)hp[i].ng_n[1] * hp[i].ng_n[2];
            if (rows > ((int64_t)1 << 26) || (int64_t)all.size() + rows > ((int64_t)1 << 28)) {
                err = "the Morton row order supports grids of at most 2^26 rows";
                return 1;
            }
            row_off[i] = (int64_t)all.size();
            morton_row_ranks(hp[i].ng_n[1], hp[i].ng_n[2], t);
            all.insert(all.end(), t.begin(), t.end());
        }
        CKA(dev_malloc(&d.row_rank, sizeof(uint32_t) * std::max<size_t>(all.size(), 1)));
        CKA(cudaMemcpyAsync(d.row_rank, all.data(), sizeof(uint32_t) * all.size(), cudaMemcpyHostToDevice, s));
    }
    cell_order = order;
    d.morton_rows = order != 0;
    for (size_t i = 0; i < hp.size(); i++) hp[i].row_rank = order ? d.row_rank + row_off[i] : nullptr;
    invalidate_order(s);
    return upload_params(s, err);
}

void Group::free_all() {
    escr.release();
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    if (graph_stream) cudaStreamDestroy(graph_stream);
    graph_stream = nullptr;
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    DevGroup &g = d;
    void *ptrs[] = {g.params, g.row_rank, g.pos, g.cons, g.cons_s, g.key[0], g.key[1], g.id[0], g.id[1], g.pos_s, g.pos_p, g.cert,
                    g.acc_s, g.fstart, g.bstart, g.amax, g.maxdisp, g.hist, g.totals, g.coef_s, g.work,
                    g.work_count};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (owns_mesh) {
        void *m[] = {g.geo, g.vx, g.pn, g.hrng, g.compact, g.tlist, g.seg, g.lines, g.occ, g.drank, g.coff, g.cand};
        for (void *p : m)
            if (p) cudaFree(p);
    }
    d = DevGroup();
}

} // namespace fppg
