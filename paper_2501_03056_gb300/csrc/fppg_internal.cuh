// Internal declarations of the FPPG relaxation library (GB300, sm_103a).
//
// Data layout in HBM (one "group" = one or more bodies relaxed together):
//   particles   pos   float4[N]  x, y, z, w = bits((1 << class) | body << 8)
//               cons  int32[N]   triangle (S) / feature segment (F) / -1
//               key, id  u32[N] x 2 (radix ping-pong), pos_s / acc_s float4[N]
//               in key order
//   grid        cells uint4[total cells] {start, end, epoch, 0}: dense over
//               every body's neighbour grid, validated by epoch (never cleared)
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

struct AsmParams {
    // neighbour grid (cell 2h (1 + 2^-8))
    float ng_o[3];
    float ng_inv;
    int ng_n[3];
    uint32_t key_base;
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
    // particles
    float4 *pos = nullptr;
    int32_t *cons = nullptr;
    uint32_t *key[2] = {nullptr, nullptr};
    uint32_t *id[2] = {nullptr, nullptr};
    float4 *pos_s = nullptr;
    float4 *acc_s = nullptr;
    uint4 *cells = nullptr;
    uint32_t *epoch = nullptr;
    uint32_t *amax = nullptr;
    uint32_t *maxdisp = nullptr;
    int4 *work = nullptr;          // search queue {key slot, trial point}
    uint32_t *work_count = nullptr;
    uint32_t *hist = nullptr;  // 256 * n_tiles
    uint32_t *totals = nullptr; // 256
    // mesh
    float4 *geo = nullptr, *vx = nullptr, *pn = nullptr;
    uint2 *hrng = nullptr;
    uint4 *compact = nullptr;
    int32_t *tlist = nullptr;
    float4 *seg = nullptr;
    int2 *lines = nullptr;
    uint32_t *occ = nullptr;
    // energy scratch
    float *rho_s = nullptr;
};

// ---- small device helpers ------------------------------------------------
// the class is stored one-hot in the low byte of w, so "does class c act on
// me" is (acts_on_bits(me) & bits(w)) != 0
__device__ inline int cls_of(float w) { return __ffs(__float_as_uint(w) & 0xffu) - 1; }

__host__ __device__ constexpr uint32_t class_bit(int c) { return 1u << c; }

__device__ inline int body_of(float w) { return (int)(__float_as_uint(w) >> 8); }

// cell coordinate: clamp((x - o) * inv, 0, n - 1), FP32 without contraction
__device__ inline int cell_coord(float x, float o, float inv, int n) {
    float t = __fsub_rn(x, o);
    t = __fmul_rn(t, inv);
    t = fmaxf(t, 0.0f);
    t = fminf(t, (float)(n - 1));
    return (int)t;
}

// FP32 squared distance (dx dx + dy dy) + dz dz without contraction
__device__ inline float dist2_rn(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ inline bool is_mobile(int cls, const AsmParams &A) {
    return cls == kClsS || cls == kClsV || (cls == kClsF && !A.fixed_features);
}

// ---- host side -------------------------------------------------------------
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
int64_t radix_tiles(int64_t n);
// exclusive scan of n uint32 values into out (may alias in); returns the total
// through *total_dev (device pointer, nullable)
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *tmp,
                        int64_t tmp_elems, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);

} // namespace fppg
