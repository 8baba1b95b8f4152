// Internal declarations of the FPPG relaxation library (GB300, sm_103a).
//
// Data layout in HBM (one "group" = one or more bodies relaxed together):
//   particles   pos   float4[N]  x, y, z, w = bits((1 << class) | body << 8)
//               cons  int32[N]   triangle (S) / feature segment (F) / -1
//               key, id  u32[N] x 2 (radix ping-pong), pos_s / acc_s float4[N]
//               in key order, pos_p float4[N + 1] pos_s as slot pairs;
//               cert  float4[N]  {x, y, z, r}: a ball of radius r around x
//               that is free of surface and inside the body (r = 0: none)
//               key = 8 (key_base + cell) + x-slab of the cell
//   grid        fstart u32[F + 1], F = 8 x total cells: the first key slot
//               whose fine key is >= f, dense over every fine key of every
//               body's neighbour grid (rebuilt every iteration from the
//               sorted keys), so the slots of fine keys [a, b] are
//               [fstart[a], fstart[b + 1])
//               bstart u32[F / 256 + 2]: the first slot of every block of
//               256 fine keys, the step that builds fstart
//   triangles   geo   float4[5 nt]  v0, n, m0, m1 (w = c1), m2 (w = c2)
//               vx    float4[3 nt]  v0, v1, v2 (w = vertex id bits)
//               pn    float4[6 nt]  edge pseudonormals 0..2, vertex ones 0..2
//   hash        hrng  uint2[sum hash sizes]   {begin, length} in compact
//               compact uint4[occupied cells] {cell key, list begin, length, 0}
//               tlist int32[pairs]            triangle ids grouped by cell
//               occ   u32 bitmaps   occupied triangle cells, then the same
//                                   dilated by one cell (any of the 27)
//   features    seg   float4[3 nseg]  a (w = line bits), b, unit tangent
//               lines int2[nlines]    {first segment, count}
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

namespace fppg {

constexpr int kClsS = 0, kClsV = 1, kClsF = 2, kClsI = 3, kClsP = 4;

// Which source classes act on each target class (bit c = class c acts):
// S <- S, F, P;  V <- all;  F <- F, P;  I, P never move.
__host__ __device__ constexpr uint32_t acts_on_bits(int c) {
    return c == kClsS ? ((1u << kClsS) | (1u << kClsF) | (1u << kClsP))
                      : c == kClsV ? 0x1Fu : c == kClsF ? ((1u << kClsF) | (1u << kClsP)) : 0u;
}

// Eq. 10 primes, exactly as printed.
constexpr uint32_t kHashP1 = 738560931u, kHashP2 = 19349663u, kHashP3 = 83492791u;

constexpr int kMaxPartners = 4;   // Boolean operations one body takes part in

struct AsmParams {
    // neighbour grid (cell 2h (1 + 2^-8))
    float ng_o[3];
    float ng_inv;
    int ng_n[3];
    uint32_t key_base;     // in cells; fine keys start at 8 key_base
    float slab_r2;         // (2h / cell)^2 (1 + 2^-12): reach in cell units, squared
    // triangle grid (cell dx)
    float tg_o[3];
    float tg_inv;
    int tg_n[3];
    uint32_t hash_off;     // offset of this body's hash table
    uint32_t hash_mask;
    uint32_t compact_off;  // offset of its C_compact entries
    uint32_t tlist_off;    // offset of its triangle list
    uint32_t occ_off;      // word offset of its triangle-cell occupancy bitmap
    uint32_t dil_off;      // word offset of the dilated bitmap (any of 27 cells)
    uint32_t drank_off;    // offset of its dilated-bit ranks (one per bitmap word)
    uint32_t coff_off;     // offset of its candidate-list starts (dilated cells + 1)
    uint32_t cand_off;     // offset of its candidate lists
    int tri_off;           // offset of its triangles (ids are local)
    int nt;
    int vert_off;
    int nv;
    int seg_off;           // offset of its feature segments (ids are local)
    int nseg;
    int line_off;
    int nlines;
    int fixed_features;
    // kernel and step
    float h;
    float R2;          // (2h)^2 rounded to FP32
    float half_inv_h;  // 1 / (2h)
    float force_scale; // 5 alpha_3 / h^2: -dW/dr / r = force_scale (1 - q/2)^3
    float step_h;      // h / 16
    float dx;
    float w0[3];       // ideal kernel sums of S, V, F
    float w_zero;      // W(0) = alpha_3
    float alpha;       // alpha_3
    float edge_tol;    // a foot this close outside a triangle edge still counts as inside
    int closed;        // closed, consistently oriented mesh: inside certificates apply
    int mobile;        // bit c: class c may move (S, V, F; I and P never do)
    int cascade;       // surface re-projection: 0 closest over 27 cells, 1 the cascade of Sec. 3.3.3
    // Boolean operations this body takes part in (Sec. 3.2.3), one entry per
    // partner: its body index in the group, the rule for surface / feature
    // particles (0 none, 1 stay outside the partner, 2 stay inside), the
    // rule for volume particles, and this body's intersection-curve
    // segments with that partner [curve_lo, curve_hi) (on both surfaces:
    // exempt from that partner's rule)
    int npart;
    int partner[kMaxPartners];
    int partner_surf[kMaxPartners];
    int partner_vol[kMaxPartners];
    int curve_lo[kMaxPartners], curve_hi[kMaxPartners];
    int vol_rules;     // some partner has a volume rule
    int amax_slot;     // body whose amax / time step this body shares (itself, or its assembly's first body)
    // order of the neighbour grid's rows (y, z): null for row-major
    // (y + ny z), else the rank of each row y + ny z in the Morton order of
    // Eq. 9 restricted to (y, z); x stays the fastest axis inside a row
    const uint32_t *row_rank;
    int p_begin, p_end;
};

// Read-only mesh arrays of a group (all bodies concatenated).
struct MeshView {
    const float4 *geo;
    const float4 *vx;
    const float4 *pn;
    const uint2 *hrng;
    const uint4 *compact;
    const int32_t *tlist;
    const float4 *seg;
    const int2 *lines;
    const uint32_t *occ;
    const uint32_t *drank;   // candidate lists of the dilated cells (Body)
    const uint32_t *coff;
    const int32_t *cand;
};

// Device arrays of one group.
struct DevGroup {
    int B = 0;           // bodies
    int64_t N = 0;       // particles
    int64_t total_cells = 0;
    int key_bits = 0;
    int passes = 0;      // radix passes (8-bit digits)
    int n_tiles = 0;
    int nt = 0, nv = 0, nseg = 0, nlines = 0;
    AsmParams *params = nullptr;
    uint32_t *row_rank = nullptr;  // Morton ranks of the grid rows of every grid of the group (null: row-major)
    bool morton_rows = false;      // the parameters point at row_rank (the order in force)
    // particles
    float4 *pos = nullptr;
    int32_t *cons = nullptr;
    int32_t *cons_s = nullptr;   // cons in key order, gathered with the positions (null: not gathered)
    uint32_t *key[2] = {nullptr, nullptr};
    uint32_t *id[2] = {nullptr, nullptr};
    float4 *pos_s = nullptr;
    float4 *pos_p = nullptr;   // pos_s as slot pairs: [m] {x, x', y, y'}, [(N + 1) / 2 + m] {z, z', w, w'}
    float4 *cert = nullptr;    // id order: inside certificate {centre, radius} of a volume particle
    float4 *acc_s = nullptr;
    uint32_t *fstart = nullptr;   // F + 1 entries (F = kSlabs * total_cells)
    uint32_t *bstart = nullptr;   // start_blocks(F + 1) + 1 entries
    // incremental ordering (the previous iteration's order repaired, see
    // order_incremental); null unless incremental is set
    bool incremental = false;
    uint32_t *key_id = nullptr;    // by id: fine key at the last grid build (~0: none)
    uint32_t *chg_bits = nullptr;  // by id: key changed, one bit each (bit i & 31 of word i >> 5)
    uint32_t *keep_bits = nullptr; // by previous slot: key kept, one bit each
    uint32_t *tile_cnt = nullptr;  // set bits of every tile of 2048: the changed tiles, then the kept ones
    uint32_t *tile_pos = nullptr;  // their exclusive scan
    uint32_t *ck[2] = {nullptr, nullptr}, *cv[2] = {nullptr, nullptr};   // changed (key, id), radix ping-pong
    uint32_t *uk = nullptr, *uv = nullptr;   // kept (key, id) in previous order
    uint32_t *split = nullptr;     // merge tile splits
    uint32_t *counts = nullptr;    // [0] changed, [1] kept
    uint32_t *scan_tmp_n = nullptr; // scan_tmp_elems(2 x tiles) entries
    uint32_t *amax = nullptr;
    uint32_t *maxdisp = nullptr;
    int4 *work = nullptr;          // search queue {key slot, trial point}, N entries, then N uint2
                                   // candidate-list ranges (queue_ranges)
    uint32_t *work_count = nullptr; // [0] entries from the front (S, F), [1] from the back (V)
    uint32_t *hist = nullptr;  // kMaxDigits * n_tiles
    uint32_t *totals = nullptr; // kMaxDigits
    // mesh
    float4 *geo = nullptr, *vx = nullptr, *pn = nullptr;
    uint2 *hrng = nullptr;
    uint4 *compact = nullptr;
    int32_t *tlist = nullptr;
    float4 *seg = nullptr;
    int2 *lines = nullptr;
    uint32_t *occ = nullptr;
    uint32_t *drank = nullptr, *coff = nullptr;
    int32_t *cand = nullptr;
    // energy scratch
    float *coef_s = nullptr;
};

// the candidate-list range of each search-queue entry, stored after the
// queue's N int4 entries in the same allocation
inline uint2 *queue_ranges(const DevGroup &d) { return reinterpret_cast<uint2 *>(d.work + d.N); }

// ---- small device helpers ------------------------------------------------
// the class is stored one-hot in the low byte of w, so "does class c act on
// me" is (acts_on_bits(me) & bits(w)) != 0
__device__ inline int cls_of(float w) { return __ffs(__float_as_uint(w) & 0xffu) - 1; }

__host__ __device__ constexpr uint32_t class_bit(int c) { return 1u << c; }

// the approximate square-root instruction: relative error of a few 2^-23,
// exactly 0 at 0
__device__ inline float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ inline int body_of(float w) { return (int)(__float_as_uint(w) >> 8); }

// cell coordinate: clamp((x - o) * inv, 0, n - 1), FP32 without contraction
__device__ inline int cell_coord(float x, float o, float inv, int n) {
    float t = __fsub_rn(x, o);
    t = __fmul_rn(t, inv);
    t = fmaxf(t, 0.0f);
    t = fminf(t, (float)(n - 1));
    return (int)t;
}

// ---- neighbour grid rows --------------------------------------------------
// Keys are refined by 8 slabs along x inside each cell: key = 8 (key_base +
// cell) + slab, the slab being the fine coordinate clamp(floor(8 t), 0,
// 8 n - 1) with t = (x - o) * inv.  Since 8 t is exact, fine >> 3 is
// cell_coord(x).  A grid row (fixed y, z) is then one contiguous key range
// ordered by x in steps of 1/8 cell, so a particle walks, per row, only the
// slabs that can hold a point within 2h of it.
constexpr int kSlabBits = 3;
constexpr int kSlabs = 1 << kSlabBits;

__device__ inline int fine_coord(float x, float o, float inv, int n) {
    float t = __fsub_rn(x, o);
    t = __fmul_rn(t, inv);
    t = __fmul_rn(t, (float)kSlabs);
    t = fmaxf(t, 0.0f);
    t = fminf(t, (float)(kSlabs * n - 1));
    return (int)t;
}

// bits of the largest fine key of a grid of `cells` cells
inline int fine_key_bits(int64_t cells) {
    const uint64_t m = (uint64_t)(cells > 0 ? cells : 1) * kSlabs - 1;
    int b = 0;
    while (b < 64 && (m >> b) != 0) b++;
    return b;
}

// (2h / cell)^2 with a relative margin of 2^-12, so that the row reach
// below never cuts off a pair that the FP32 test r^2 < (2h)^2 accepts
inline float slab_reach2(float R2, float inv) {
    return (float)((double)R2 * (double)inv * (double)inv * (1.0 + 1.0 / 4096.0));
}

// A particle's place in the grid: unclamped cell coordinates t, clamped
// cells c and the slack (cell units) that covers the FP32 rounding of t and
// of the reach arithmetic (relative errors of a few 2^-24 of |t|).
// Bounds-checked build (compiled with -DFPPG_CHECKED): the hot-path kernels
// check the indices they compute before using them; a failed check ORs its
// code into the device word read by fppg_check_status and the access is
// skipped, so a bad index never reaches memory.  In the normal build every
// check is the constant true and compiles away.
enum CheckCode : uint32_t {
    kChkGather = 1u,     // a sorted id or fine key outside the particle / key count
    kChkRange = 2u,      // a row's slot range outside [0, N]
    kChkQueue = 4u,      // a search-queue slot outside [0, N)
    kChkEntry = 8u,      // a queued key slot outside [0, N)
    kChkTri = 16u,       // a candidate triangle outside the body's triangles
    kChkMerge = 32u,     // a merge tile's split outside its lists
    kChkCompact = 64u,   // a compaction position outside [0, N)
};
#ifdef FPPG_CHECKED
__device__ bool fppg_check_failed(uint32_t code);
#define FPPG_CHECK(cond, code) ((cond) || fppg_check_failed(code))
#else
#define FPPG_CHECK(cond, code) true
#endif

// index of grid row (y, z) in key order: row-major, or its Morton rank
__device__ inline uint32_t grid_row(const AsmParams &A, int y, int z) {
    const uint32_t r = (uint32_t)y + (uint32_t)A.ng_n[1] * (uint32_t)z;
    return A.row_rank ? A.row_rank[r] : r;
}

// the same with the order fixed at compile time (the force pass)
template <bool MORTON>
__device__ inline uint32_t grid_row_of(const AsmParams &A, int y, int z) {
    const uint32_t r = (uint32_t)y + (uint32_t)A.ng_n[1] * (uint32_t)z;
    return MORTON ? A.row_rank[r] : r;
}

// the fine keys in blocks of 256 for building the start table (relax.cu)
constexpr int kStartBlock = 256;
constexpr int64_t start_blocks(int64_t f1) { return (f1 + kStartBlock - 1) / kStartBlock; }

struct GridPoint {
    float t[3];
    int c[3];
    float slack;
};

__device__ inline GridPoint grid_point(const AsmParams &A, float x, float y, float z) {
    GridPoint g;
    const float v[3] = {x, y, z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        g.t[k] = __fmul_rn(__fsub_rn(v[k], A.ng_o[k]), A.ng_inv);
        g.c[k] = (int)fminf(fmaxf(g.t[k], 0.0f), (float)(A.ng_n[k] - 1));
    }
    g.slack = 0x1p-12f + (fabsf(g.t[0]) + fabsf(g.t[1]) + fabsf(g.t[2]) + 4.0f) * 0x1p-19f;
    return g;
}

// Lower bound (cell units) of the distance from the particle to any point
// keyed into grid row offset d (-1, 0, +1) along a y or z axis: a point of
// row c + 1 has t >= c + 1, one of row c - 1 has t < c.
__device__ inline float row_gap(float t, int c, int d, float slack) {
    if (d == 0) return 0.0f;
    const float g = d < 0 ? t - (float)c : (float)(c + 1) - t;
    return fmaxf(g - slack, 0.0f);
}

// Slot range [s, e) of the particles of grid row `row` (index of its x = 0
// cell) whose fine x lies within reach of the particle, given the row's
// y / z gaps: the fine keys from the slab of t - w to the slab of t + w,
// cut to the cells x0..x1 of the 3 x 3 x 3 stencil, read from the dense
// start table (two loads).  Empty (s >= e) when no point of the row can be
// within 2h.  w carries the slack of the FP32 reach arithmetic, and the
// approximate root is within a few 2^-23 of the exact one, far inside the
// 2^-12 relative margin of slab_r2.
__device__ inline void row_slots(const AsmParams &A, const uint32_t *__restrict__ fstart, const GridPoint &g,
                                 float gy, float gz, uint32_t row, uint32_t &s, uint32_t &e) {
    s = 0xffffffffu;
    e = 0u;
    const float w2 = A.slab_r2 - gy * gy - gz * gz;
    if (!(w2 > 0.0f)) return;
    const float w = sqrt_approx(w2) + g.slack;
    // fine coordinates of t -/+ w under the key's own clamp to [0, 8 n - 1]
    // (monotone, so every point within reach has its fine x in [flo, fhi]),
    // cut to the stencil cells x0..x1; the particle's own slab is inside
    const int x0 = max(g.c[0] - 1, 0), x1 = min(g.c[0] + 1, A.ng_n[0] - 1);
    const float flo = fmaxf(fminf(floorf((g.t[0] - w) * (float)kSlabs), (float)(kSlabs * A.ng_n[0] - 1)),
                            (float)(kSlabs * x0));
    const float fhi = fminf(fmaxf(floorf((g.t[0] + w) * (float)kSlabs), 0.0f), (float)(kSlabs * x1 + kSlabs - 1));
    if (!(flo <= fhi)) return;   // only for non-finite coordinates
    const uint32_t f0 = kSlabs * row;
    const uint32_t a = fstart[f0 + (uint32_t)(int)flo], b = fstart[f0 + (uint32_t)(int)fhi + 1u];
    if (a < b) {       // empty stays (~0, 0): neutral under a warp min / max
        s = a;
        e = b;
    }
}

// slots [s, e) of the whole cells x0..x1 of grid row `row`
__device__ inline void cells_slots(const uint32_t *__restrict__ fstart, uint32_t row, int x0, int x1, uint32_t &s,
                                   uint32_t &e) {
    s = fstart[kSlabs * (row + (uint32_t)x0)];
    e = fstart[kSlabs * (row + (uint32_t)x1 + 1u)];
}

// ---- triangle grid -------------------------------------------------------
// C_compact entry of triangle cell (x, y, z) through the Eq. 10 hash:
// [beg, beg + len) in the triangle list; false for a cell without triangles
__device__ inline bool tri_cell(const MeshView &M, const AsmParams &A, int x, int y, int z, uint32_t &beg,
                                uint32_t &len) {
    const uint32_t h = (kHashP1 * (uint32_t)x + kHashP2 * (uint32_t)y + kHashP3 * (uint32_t)z) & A.hash_mask;
    const uint2 r = M.hrng[A.hash_off + h];
    const uint32_t key = (uint32_t)x + (uint32_t)A.tg_n[0] * ((uint32_t)y + (uint32_t)A.tg_n[1] * (uint32_t)z);
    for (uint32_t e = r.x; e < r.x + r.y; e++) {
        const uint4 c = M.compact[A.compact_off + e];
        if (c.x == key) {
            beg = A.tlist_off + c.y;
            len = c.z;
            return true;
        }
    }
    return false;
}

__device__ inline bool test_bit(const uint32_t *m, uint32_t off, uint32_t c) {
    return (m[off + (c >> 5)] >> (c & 31u)) & 1u;
}

__device__ inline uint32_t tri_key(const AsmParams &A, int x, int y, int z) {
    return (uint32_t)x + (uint32_t)A.tg_n[0] * ((uint32_t)y + (uint32_t)A.tg_n[1] * (uint32_t)z);
}

// FP32 squared distance (dx dx + dy dy) + dz dz without contraction
__device__ inline float dist2_rn(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ inline bool is_mobile(int cls, const AsmParams &A) {
    return (cls == kClsS || cls == kClsV || (cls == kClsF && !A.fixed_features)) && ((A.mobile >> cls) & 1);
}

// Ghost particles (bit 7 of w, above the one-hot class bits): copies of
// another domain's particles near a shared face (spatial decomposition over
// several GPUs).  A ghost acts on its neighbours by its class, but it never
// moves, has no force of its own and is left out of amax and the statistics.
constexpr uint32_t kGhostBit = 0x80u;
__device__ inline bool is_ghost(float w) { return (__float_as_uint(w) & kGhostBit) != 0u; }

// ---- host side -------------------------------------------------------------
// Every device allocation of the library goes through dev_malloc, so that a
// test can make one chosen allocation fail as if the device were out of
// memory (fppg_debug_fail_allocation) and check the error path.
cudaError_t dev_malloc_raw(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

struct Status {
    int code = 0;
    std::string msg;
};

// radix sort of (key, value) pairs, stable, 8-bit digits, LSD
// Returns the index (0 or 1) of the buffer that holds the result.
int radix_sort_u32(uint32_t *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int bits, uint32_t *hist,
                   uint32_t *totals, cudaStream_t s);
int radix_sort_u64(uint64_t *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int bits, uint32_t *hist,
                   uint32_t *totals, cudaStream_t s);
// the same with the count read from device memory (*n_dev <= n_max; the
// launches and the histogram are sized for n_max; values given)
int radix_sort_u32_dev(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max, const uint32_t *n_dev, int bits,
                       uint32_t *hist, uint32_t *totals, cudaStream_t s);
int64_t radix_tiles(int64_t n);
// radix passes for keys of `bits` bits and their digit width (*digit_bits);
// the histogram holds kMaxDigits rows of radix_tiles(n)
int radix_pass_plan(int bits, int *digit_bits);
constexpr int kMaxDigits = 256;
// exclusive scan of n uint32 values into out (may alias in); returns the total
// through *total_dev (device pointer, nullable)
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *tmp,
                        int64_t tmp_elems, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);
// the same scan of counts that are cleared (set to 0) as they are read, so
// the count array starts the next accumulation at zero
void exclusive_scan_u32_clear(uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, int64_t tmp_elems,
                              cudaStream_t s);
// kernel launches of exclusive_scan_u32 (no total) / _clear on n elements
int scan_launches(int64_t n);
int scan_clear_launches(int64_t n);

} // namespace fppg
