// Set-up of a body's device geometry (Sec. 3.1, Sec. 3.2.2).
//
// Compiled with -fmad=false: every FP64 expression here is evaluated
// operation by operation in the order written, so the unit normals and the
// dihedral test decide exactly like any other IEEE implementation of the
// same formulas.
//   k_tri_prep      unit normals, in-plane edge normals, vertex copies,
//                   edge keys v1 * nv + v2 (v1 < v2) and corner keys
//   k_edge_runs     per edge (sorted keys): edge pseudonormal = normalised
//                   sum of the unit normals of its faces
//   k_vertex_runs   per vertex: angle-weighted pseudonormal
//   k_bin_*         triangle-box overlap by separating axes (Sec. 3.1.2)
//                   on cells inflated by 1e-6 dx, emitted as (cell, tri)
//   compact + hash  C_compact and the Eq. 10 hash with H_begin/H_length
//   k_feature_flags dihedral rule on the sorted edge list
#include <algorithm>
#include <cmath>
#include <cstring>

#include "body.h"

namespace fppg {

namespace {

struct d3 {
    double x, y, z;
};
__device__ inline d3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ inline d3 sub(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline d3 cross(d3 a, d3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ inline d3 vload(const float *v, int i) { return {(double)v[3 * i], (double)v[3 * i + 1], (double)v[3 * i + 2]}; }
__device__ inline float4 f4(d3 a, float w) { return make_float4((float)a.x, (float)a.y, (float)a.z, w); }

__global__ void k_tri_prep(const float *__restrict__ verts, const int32_t *__restrict__ tris, int nt, int nv,
                           float4 *__restrict__ geo, float4 *__restrict__ vx, double *__restrict__ nu,
                           uint64_t *__restrict__ ekey, uint32_t *__restrict__ ckey) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int id[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    d3 v[3] = {vload(verts, id[0]), vload(verts, id[1]), vload(verts, id[2])};
    d3 e1 = sub(v[1], v[0]), e2 = sub(v[2], v[0]);
    d3 n = cross(e1, e2);
    double len = sqrt(dot(n, n));
    d3 u = len > 0.0 ? mk(n.x / len, n.y / len, n.z / len) : mk(0.0, 0.0, 0.0);
    nu[3 * t] = u.x;
    nu[3 * t + 1] = u.y;
    nu[3 * t + 2] = u.z;
    geo[5 * t + 0] = f4(v[0], 0.0f);
    geo[5 * t + 1] = f4(u, 0.0f);
    for (int k = 0; k < 3; k++) {
        d3 e = sub(v[(k + 1) % 3], v[k]);
        d3 m = cross(u, e);
        double ml = sqrt(dot(m, m));
        m = ml > 0.0 ? mk(m.x / ml, m.y / ml, m.z / ml) : mk(0.0, 0.0, 0.0);
        double ck = dot(sub(v[k], v[0]), m);
        // a degenerate triangle is never projectable: its first edge test
        // can never pass
        float w = (float)ck;
        if (len <= 0.0 && k == 1) w = INFINITY;
        geo[5 * t + 2 + k] = f4(m, k == 0 ? 0.0f : w);
        vx[3 * t + k] = f4(v[k], __int_as_float(id[k]));
        int a = id[k], b = id[(k + 1) % 3];
        uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
        ekey[3 * t + k] = lo * (uint64_t)nv + hi;
        ckey[3 * t + k] = (uint32_t)id[k];
    }
}

__global__ void k_edge_runs(const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, int64_t m,
                            const double *__restrict__ nu, float4 *__restrict__ pn) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || (i > 0 && key[i] == key[i - 1])) return;
    d3 s = mk(0.0, 0.0, 0.0);
    int64_t j = i;
    for (; j < m && key[j] == key[i]; j++) {
        uint32_t t = val[j] / 3;
        s = mk(s.x + nu[3 * t], s.y + nu[3 * t + 1], s.z + nu[3 * t + 2]);
    }
    double len = sqrt(dot(s, s));
    d3 e = len > 0.0 ? mk(s.x / len, s.y / len, s.z / len) : mk(0.0, 0.0, 0.0);
    for (int64_t q = i; q < j; q++) {
        uint32_t t = val[q] / 3, k = val[q] % 3;
        pn[6 * t + k] = f4(e, 0.0f);
    }
}

__global__ void k_vertex_runs(const uint32_t *__restrict__ key, const uint32_t *__restrict__ val, int64_t m,
                              const float *__restrict__ verts, const int32_t *__restrict__ tris,
                              const double *__restrict__ nu, float4 *__restrict__ vpn) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || (i > 0 && key[i] == key[i - 1])) return;
    d3 s = mk(0.0, 0.0, 0.0);
    for (int64_t j = i; j < m && key[j] == key[i]; j++) {
        uint32_t t = val[j] / 3, k = val[j] % 3;
        d3 p = vload(verts, tris[3 * t + k]);
        d3 u = sub(vload(verts, tris[3 * t + (k + 1) % 3]), p);
        d3 w = sub(vload(verts, tris[3 * t + (k + 2) % 3]), p);
        double lu = sqrt(dot(u, u)), lw = sqrt(dot(w, w));
        double c = (lu > 0.0 && lw > 0.0) ? dot(u, w) / (lu * lw) : 1.0;
        c = fmin(1.0, fmax(-1.0, c));
        double ang = acos(c);
        s = mk(s.x + ang * nu[3 * t], s.y + ang * nu[3 * t + 1], s.z + ang * nu[3 * t + 2]);
    }
    double len = sqrt(dot(s, s));
    d3 e = len > 0.0 ? mk(s.x / len, s.y / len, s.z / len) : mk(0.0, 0.0, 0.0);
    vpn[key[i]] = f4(e, 0.0f);
}

__global__ void k_fill_vertex_pn(const int32_t *__restrict__ tris, int nt, const float4 *__restrict__ vpn,
                                 float4 *__restrict__ pn) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    for (int k = 0; k < 3; k++) pn[6 * t + 3 + k] = vpn[tris[3 * t + k]];
}

// ---- triangle-box overlap (separating axes) ---------------------------------
__device__ inline bool axis_separates(d3 ax, d3 v0, d3 v1, d3 v2, double hs) {
    double p0 = dot(ax, v0), p1 = dot(ax, v1), p2 = dot(ax, v2);
    double mn = fmin(p0, fmin(p1, p2)), mx = fmax(p0, fmax(p1, p2));
    double r = hs * (fabs(ax.x) + fabs(ax.y) + fabs(ax.z));
    return mn > r || mx < -r;
}

__device__ bool tri_box_overlap(d3 ctr, double hs, d3 a, d3 b, d3 c) {
    d3 v0 = sub(a, ctr), v1 = sub(b, ctr), v2 = sub(c, ctr);
    d3 f[3] = {sub(v1, v0), sub(v2, v1), sub(v0, v2)};
    double vk[3][3] = {{v0.x, v1.x, v2.x}, {v0.y, v1.y, v2.y}, {v0.z, v1.z, v2.z}};
    for (int k = 0; k < 3; k++) {
        double mn = fmin(vk[k][0], fmin(vk[k][1], vk[k][2])), mx = fmax(vk[k][0], fmax(vk[k][1], vk[k][2]));
        if (mn > hs || mx < -hs) return false;
    }
    d3 n = cross(f[0], f[1]);
    if (fabs(dot(n, v0)) > hs * (fabs(n.x) + fabs(n.y) + fabs(n.z))) return false;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            d3 e = mk(i == 0 ? 1.0 : 0.0, i == 1 ? 1.0 : 0.0, i == 2 ? 1.0 : 0.0);
            if (axis_separates(cross(e, f[j]), v0, v1, v2, hs)) return false;
        }
    return true;
}

struct TriGrid {
    float o[3];
    int n[3];
    double cell;
};

// Binning of the triangles into the cells of the triangle grid, one thread
// per (triangle, candidate cell) so that a large triangle's work is spread
// over many threads.  The candidates of triangle t are the cells of its
// bounding box widened by 1e-5 of a cell (the tested box is inflated by
// 1e-6 of a cell, so no cell outside can pass the overlap test), in the
// order z, y, x (x fastest); the accepted pairs come out in that order for
// every triangle in turn.

// per triangle: its candidate box and the number of candidate cells
// (total64: the 64-bit sum of the counts, so that the host can refuse a
// mesh whose candidates would not fit 32-bit offsets)
__global__ void k_bin_boxes(const float *__restrict__ verts, const int32_t *__restrict__ tris, int nt, TriGrid g,
                            int4 *__restrict__ box_lo, int4 *__restrict__ box_n, uint32_t *__restrict__ ncand,
                            unsigned long long *__restrict__ total64) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    if (t < nt) {
        d3 a = vload(verts, tris[3 * t]), b = vload(verts, tris[3 * t + 1]), c = vload(verts, tris[3 * t + 2]);
        double av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z}, cv[3] = {c.x, c.y, c.z};
        int lo[3], cnt[3];
        m = 1;
        for (int k = 0; k < 3; k++) {
            double mn = fmin(av[k], fmin(bv[k], cv[k])), mx = fmax(av[k], fmax(bv[k], cv[k]));
            double lf = floor((mn - (double)g.o[k]) / g.cell - 1e-5), hf = floor((mx - (double)g.o[k]) / g.cell + 1e-5);
            lf = fmax(lf, 0.0);
            hf = fmin(hf, (double)(g.n[k] - 1));
            lo[k] = (int)lf;
            cnt[k] = hf >= lf ? (int)(hf - lf) + 1 : 0;
            m *= (unsigned long long)cnt[k];
        }
        box_lo[t] = make_int4(lo[0], lo[1], lo[2], 0);
        box_n[t] = make_int4(cnt[0], cnt[1], cnt[2], 0);
        ncand[t] = m > 0xffffffffull ? 0xffffffffu : (uint32_t)m;
    }
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(total64, m);
}

// per candidate q: its triangle (the last t with coff[t] <= q) and cell;
// flag[q] = the triangle-box overlap test, key[q] the cell key
__global__ void k_bin_test(const float *__restrict__ verts, const int32_t *__restrict__ tris, int nt, TriGrid g,
                           const int4 *__restrict__ box_lo, const int4 *__restrict__ box_n,
                           const uint32_t *__restrict__ coff, int64_t nc, uint32_t *__restrict__ flag,
                           uint32_t *__restrict__ key, uint32_t *__restrict__ tri) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    int lo_t = 0, hi_t = nt - 1;                 // coff is ascending: upper bound of q, minus one
    while (lo_t < hi_t) {
        const int mid = (lo_t + hi_t + 1) >> 1;
        if ((int64_t)coff[mid] <= q) lo_t = mid;
        else hi_t = mid - 1;
    }
    const int t = lo_t;
    const int4 l = box_lo[t], n = box_n[t];
    const uint32_t r = (uint32_t)(q - (int64_t)coff[t]);
    const int x = l.x + (int)(r % (uint32_t)n.x);
    const int y = l.y + (int)((r / (uint32_t)n.x) % (uint32_t)n.y);
    const int z = l.z + (int)(r / ((uint32_t)n.x * (uint32_t)n.y));
    d3 a = vload(verts, tris[3 * t]), b = vload(verts, tris[3 * t + 1]), c = vload(verts, tris[3 * t + 2]);
    const double hs = 0.5 * g.cell + 1e-6 * g.cell;
    const d3 ctr = mk((double)g.o[0] + (x + 0.5) * g.cell, (double)g.o[1] + (y + 0.5) * g.cell,
                      (double)g.o[2] + (z + 0.5) * g.cell);
    flag[q] = tri_box_overlap(ctr, hs, a, b, c) ? 1u : 0u;
    key[q] = (uint32_t)x + (uint32_t)g.n[0] * ((uint32_t)y + (uint32_t)g.n[1] * (uint32_t)z);
    tri[q] = (uint32_t)t;
}

// the accepted candidates, compacted in candidate order
__global__ void k_bin_emit(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                           const uint32_t *__restrict__ key, const uint32_t *__restrict__ tri, int64_t nc,
                           uint32_t *__restrict__ pkey, uint32_t *__restrict__ ptri) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc || !flag[q]) return;
    pkey[pos[q]] = key[q];
    ptri[pos[q]] = tri[q];
}

__global__ void k_run_flags(const uint32_t *__restrict__ key, int64_t m, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// occupied cell -> compact entry {cell key, tlist begin, length, hash}
__global__ void k_compact(const uint32_t *__restrict__ key, int64_t m, const uint32_t *__restrict__ flag,
                          const uint32_t *__restrict__ pos, TriGrid g, uint32_t hmask, uint4 *__restrict__ compact,
                          uint32_t *__restrict__ hkey) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !flag[i]) return;
    int64_t j = i;
    while (j < m && key[j] == key[i]) j++;
    uint32_t c = key[i];
    uint32_t x = c % (uint32_t)g.n[0], yz = c / (uint32_t)g.n[0];
    uint32_t y = yz % (uint32_t)g.n[1], z = yz / (uint32_t)g.n[1];
    uint32_t h = (kHashP1 * x + kHashP2 * y + kHashP3 * z) & hmask;   // Eq. 10
    compact[pos[i]] = make_uint4(c, (uint32_t)i, (uint32_t)(j - i), h);
    hkey[pos[i]] = h;
}

__global__ void k_gather_compact(const uint4 *__restrict__ in, const uint32_t *__restrict__ perm, int64_t m,
                                 uint4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        uint4 e = in[perm[i]];
        e.w = 0;
        out[i] = e;
    }
}

__global__ void k_hash_ranges(const uint32_t *__restrict__ hsorted, int64_t m, uint2 *__restrict__ hrng) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || (i > 0 && hsorted[i] == hsorted[i - 1])) return;
    int64_t j = i;
    while (j < m && hsorted[j] == hsorted[i]) j++;
    hrng[hsorted[i]] = make_uint2((uint32_t)i, (uint32_t)(j - i));
}

// occupied cell c: its bit in the occupancy map and the bits of its 27
// neighbours in the dilated map
__global__ void k_mark_occupancy(const uint4 *__restrict__ compact, int64_t m, TriGrid g, int64_t words,
                                 uint32_t *__restrict__ occ) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t c = compact[i].x;
    atomicOr(occ + (c >> 5), 1u << (c & 31u));
    int x = (int)(c % (uint32_t)g.n[0]), yz = (int)(c / (uint32_t)g.n[0]);
    int y = yz % g.n[1], z = yz / g.n[1];
    for (int zz = max(z - 1, 0); zz <= min(z + 1, g.n[2] - 1); zz++)
        for (int yy = max(y - 1, 0); yy <= min(y + 1, g.n[1] - 1); yy++)
            for (int xx = max(x - 1, 0); xx <= min(x + 1, g.n[0] - 1); xx++) {
                uint32_t d = (uint32_t)xx + (uint32_t)g.n[0] * ((uint32_t)yy + (uint32_t)g.n[1] * (uint32_t)zz);
                atomicOr(occ + words + (d >> 5), 1u << (d & 31u));
            }
}

// A closed, consistently oriented surface: every edge has exactly two faces
// that traverse it in opposite directions, and no face is degenerate.  Any
// violation sets *open.
__global__ void k_closed_check(const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, int64_t m,
                               const int32_t *__restrict__ tris, const double *__restrict__ nu,
                               uint32_t *__restrict__ open) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t t = val[i] / 3;
    if (nu[3 * t] == 0.0 && nu[3 * t + 1] == 0.0 && nu[3 * t + 2] == 0.0) atomicOr(open, 1u);
    if (i > 0 && key[i] == key[i - 1]) return;
    int64_t j = i;
    while (j < m && key[j] == key[i]) j++;
    if (j - i != 2) {
        atomicOr(open, 1u);
        return;
    }
    const uint32_t t1 = val[i] / 3, k1 = val[i] % 3, t2 = val[i + 1] / 3, k2 = val[i + 1] % 3;
    const int32_t a1 = tris[3 * t1 + k1], b1 = tris[3 * t1 + (k1 + 1) % 3];
    const int32_t a2 = tris[3 * t2 + k2], b2 = tris[3 * t2 + (k2 + 1) % 3];
    if (!(a1 == b2 && b1 == a2)) atomicOr(open, 1u);
}

// ---- candidate lists of the dilated cells ------------------------------------
// For every cell of the dilated occupancy map (a cell with a triangle among
// its 27 neighbours) the distinct triangles binned into those 27 cells, so
// that the search reads one list instead of probing 27 cells through the
// hash.  The set is the one the 27-cell probe gathers, without repeats.

__global__ void k_word_popc(const uint32_t *__restrict__ words, int64_t n, uint32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = __popc(words[i]);
}

// cell key of every set bit, in key order: dcell[rank] = key
__global__ void k_bit_cells(const uint32_t *__restrict__ words, int64_t n, const uint32_t *__restrict__ rank,
                            uint32_t *__restrict__ dcell) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n) return;
    uint32_t bits = words[w], r = rank[w];
    while (bits) {
        const int j = __ffs(bits) - 1;
        dcell[r++] = (uint32_t)(32 * w + j);
        bits &= bits - 1u;
    }
}

constexpr int kListBuf = 512;   // gathered ids per warp (with repeats); more: the cell keeps the probe

// one warp per dilated cell: gather the 27 cells' triangle ids, keep the
// first occurrence of each; WRITE = 0 counts (cnt[r], 0 and ovf[r] = 1 on
// overflow), WRITE = 1 writes the list at off[r]
template <bool WRITE>
__global__ void __launch_bounds__(256) k_cell_lists(AsmParams A, MeshView M, const uint32_t *__restrict__ dcell,
                                                    int64_t D, uint32_t *__restrict__ cnt, uint8_t *__restrict__ ovf,
                                                    const uint32_t *__restrict__ off, int32_t *__restrict__ list) {
    __shared__ int32_t sbuf[8][kListBuf];
    int32_t *buf = sbuf[threadIdx.x / 32];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t r = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; r < D; r += warps) {
        const uint32_t c = dcell[r];
        const int x = (int)(c % (uint32_t)A.tg_n[0]), yz = (int)(c / (uint32_t)A.tg_n[0]);
        const int y = yz % A.tg_n[1], z = yz / A.tg_n[1];
        uint32_t beg = 0, len = 0;
        if (lane < 27) {
            const int xx = x + lane % 3 - 1, yy = y + (lane / 3) % 3 - 1, zz = z + lane / 9 - 1;
            if (xx >= 0 && yy >= 0 && zz >= 0 && xx < A.tg_n[0] && yy < A.tg_n[1] && zz < A.tg_n[2] &&
                test_bit(M.occ, A.occ_off, tri_key(A, xx, yy, zz)))
                tri_cell(M, A, xx, yy, zz, beg, len);
        }
        uint32_t o = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, o, d);
            if (lane >= d) o += t;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, o, 31);
        o -= len;
        if (total > (uint32_t)kListBuf) {
            if (!WRITE && lane == 0) {
                cnt[r] = 0;
                ovf[r] = 1;
            }
            __syncwarp();
            continue;
        }
        for (uint32_t q = 0; q < len; q++) buf[o + q] = M.tlist[beg + q];
        __syncwarp();
        uint32_t written = 0;
        for (uint32_t q0 = 0; q0 < total; q0 += 32) {
            const uint32_t q = q0 + lane;
            bool first = false;
            int32_t id = 0;
            if (q < total) {
                id = buf[q];
                first = true;
                for (uint32_t p = 0; p < q; p++)
                    if (buf[p] == id) {
                        first = false;
                        break;
                    }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, first);
            if (WRITE && first) list[off[r] + written + __popc(m & ((1u << lane) - 1u))] = id;
            written += __popc(m);
        }
        if (!WRITE && lane == 0) {
            cnt[r] = written;
            ovf[r] = 0;
        }
        __syncwarp();
    }
}

__global__ void k_flag_overflow(uint32_t *__restrict__ off, const uint8_t *__restrict__ ovf, int64_t D) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < D && ovf[r]) off[r] |= 0x80000000u;
}

__global__ void k_feature_flags(const uint64_t *__restrict__ key, const uint32_t *__restrict__ val, int64_t m,
                                const double *__restrict__ nu, double cthr, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint32_t f = 0;
    if (i == 0 || key[i] != key[i - 1]) {
        int64_t j = i;
        while (j < m && key[j] == key[i]) j++;
        if (j - i != 2) {
            f = 1; // boundary or non-manifold edge
        } else {
            uint32_t t1 = val[i] / 3, t2 = val[i + 1] / 3;
            double d = nu[3 * t1] * nu[3 * t2] + nu[3 * t1 + 1] * nu[3 * t2 + 1] + nu[3 * t1 + 2] * nu[3 * t2 + 2];
            f = d < cthr ? 1u : 0u;
        }
    }
    flag[i] = f;
}

__global__ void k_feature_emit(const uint64_t *__restrict__ key, int64_t m, const uint32_t *__restrict__ flag,
                               const uint32_t *__restrict__ pos, int nv, int32_t *__restrict__ fe) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !flag[i]) return;
    uint64_t k = key[i];
    fe[2 * pos[i]] = (int32_t)(k / (uint64_t)nv);
    fe[2 * pos[i] + 1] = (int32_t)(k % (uint64_t)nv);
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b) != 0) b++;
    return b;
}

} // namespace

// Grid rule shared with every other implementation of the method:
// origin = bbmin - shift * cell (FP64, rounded to FP32), inv = 1 / cell
// (FP64, rounded), n = ceil((bbmax - origin) / cell) + margin.  The triangle
// grid uses shift 2.5 with margin 2 (a face on the bounding box passes
// through cell centres), the neighbour grid shift 1 with margin 1.
// The count of every axis is checked in FP64 before it becomes an int:
// false (n left at 0) when it is not finite or above kGridAxisMax, so that a
// cell far below the box extent is an argument error, not a wrapped count.
bool grid_setup(const float *bbmin, const float *bbmax, float cell, double shift, int margin, float *o, float *inv,
                int *n) {
    bool ok = std::isfinite(cell) && cell > 0.f;
    for (int a = 0; a < 3; a++) {
        o[a] = (float)((double)bbmin[a] - shift * (double)cell);
        const double c = std::ceil(((double)bbmax[a] - (double)o[a]) / (double)cell) + margin;
        if (!(c >= 1.0 && c <= (double)kGridAxisMax)) ok = false;
        n[a] = ok ? (int)c : 0;
    }
    if (!ok) n[0] = n[1] = n[2] = 0;
    *inv = (float)(1.0 / (double)cell);
    return ok;
}

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                     \
            return e_ == cudaErrorMemoryAllocation ? 3 : 4;                            \
        }                                                                              \
    } while (0)

template <typename T>
static cudaError_t dalloc(T **p, int64_t n) {
    return dev_malloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
}

void Body::free_mesh() {
    void *ptrs[] = {d_verts, d_tris, geo, vx, pn, hrng, compact, tlist, nu, ekey, eval, seg, lines, occ,
                    drank, coff, cand};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    drank = coff = nullptr;
    cand = nullptr;
    n_dil = n_cand = 0;
    d_verts = nullptr;
    d_tris = nullptr;
    geo = vx = pn = nullptr;
    hrng = nullptr;
    compact = nullptr;
    tlist = nullptr;
    nu = nullptr;
    ekey = nullptr;
    eval = nullptr;
    seg = nullptr;
    lines = nullptr;
    occ = nullptr;
}

int Body::build_mesh(const float *verts_host, int64_t nv_, const int32_t *tris_host, int64_t nt_, float dx_,
                     float h_, cudaStream_t s, std::string &err) {
    nv = (int)nv_;
    nt = (int)nt_;
    dx = dx_;
    h = h_;
    float bbmin[3] = {INFINITY, INFINITY, INFINITY}, bbmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv_; i++)
        for (int k = 0; k < 3; k++) {
            bbmin[k] = std::min(bbmin[k], verts_host[3 * i + k]);
            bbmax[k] = std::max(bbmax[k], verts_host[3 * i + k]);
        }
    {
        double ext = 0.0;
        for (int k = 0; k < 3; k++) ext = std::max(ext, (double)bbmax[k] - (double)bbmin[k]);
        edge_tol = (float)std::ldexp(ext, -20);
    }
    for (int k = 0; k < 3; k++) {
        this->bbmin[k] = bbmin[k];
        this->bbmax[k] = bbmax[k];
    }
    const bool tg_ok = grid_setup(bbmin, bbmax, dx, 2.5, 2, tg_o, &tg_inv, tg_n);
    float R = 2.0f * h;
    R2 = (float)((double)R * (double)R);
    ng_cell = (float)((double)R * (1.0 + 1.0 / 256.0));
    const bool ng_ok = grid_setup(bbmin, bbmax, ng_cell, 1.0, 1, ng_o, &ng_inv, ng_n);
    if (!tg_ok || !ng_ok || (double)tg_n[0] * tg_n[1] * tg_n[2] >= 4294967295.0 ||
        (double)ng_n[0] * ng_n[1] * ng_n[2] >= 536870912.0) {
        // neighbour keys carry 3 slab bits below the cell index
        err = "grid too large for 32-bit cell keys (dx too small for the mesh extent)";
        return 1;
    }
    CK(dalloc(&d_verts, 3 * (int64_t)nv));
    CK(dalloc(&d_tris, 3 * (int64_t)nt));
    CK(cudaMemcpyAsync(d_verts, verts_host, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_tris, tris_host, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, s));
    CK(dalloc(&geo, 5 * (int64_t)nt));
    CK(dalloc(&vx, 3 * (int64_t)nt));
    CK(dalloc(&pn, 6 * (int64_t)nt));
    CK(dalloc(&nu, 3 * (int64_t)nt));
    const int64_t m = 3 * (int64_t)nt;
    uint64_t *ek[2] = {nullptr, nullptr};
    uint32_t *ev[2] = {nullptr, nullptr}, *ck[2] = {nullptr, nullptr}, *cv[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr, *tot = nullptr;
    float4 *vpn = nullptr;
    CK(dalloc(&ek[0], m));
    CK(dalloc(&ek[1], m));
    CK(dalloc(&ev[0], m));
    CK(dalloc(&ev[1], m));
    CK(dalloc(&ck[0], m));
    CK(dalloc(&ck[1], m));
    CK(dalloc(&cv[0], m));
    CK(dalloc(&cv[1], m));
    CK(dalloc(&vpn, nv));
    int64_t tiles = radix_tiles(m);
    CK(dalloc(&hist, kMaxDigits * std::max<int64_t>(tiles, 1)));
    CK(dalloc(&tot, kMaxDigits));
    k_tri_prep<<<blocks(nt), 256, 0, s>>>(d_verts, d_tris, nt, nv, geo, vx, nu, ek[0], ck[0]);
    int eb = radix_sort_u64(ek, ev, true, m, bits_for((uint64_t)nv * (uint64_t)nv), hist, tot, s);
    k_edge_runs<<<blocks(m), 256, 0, s>>>(ek[eb], ev[eb], m, nu, pn);
    uint32_t *open = nullptr;
    CK(dalloc(&open, 1));
    CK(cudaMemsetAsync(open, 0, sizeof(uint32_t), s));
    k_closed_check<<<blocks(m), 256, 0, s>>>(ek[eb], ev[eb], m, d_tris, nu, open);
    int cb = radix_sort_u32(ck, cv, true, m, bits_for((uint64_t)nv), hist, tot, s);
    k_vertex_runs<<<blocks(m), 256, 0, s>>>(ck[cb], cv[cb], m, d_verts, d_tris, nu, vpn);
    k_fill_vertex_pn<<<blocks(nt), 256, 0, s>>>(d_tris, nt, vpn, pn);
    // keep the sorted edge list for feature extraction
    ekey = ek[eb];
    eval = ev[eb];
    cudaFree(ek[eb ^ 1]);
    cudaFree(ev[eb ^ 1]);
    cudaFree(ck[0]);
    cudaFree(ck[1]);
    cudaFree(cv[0]);
    cudaFree(cv[1]);

    // ---- triangle binning, C_compact and the hash -------------------------
    TriGrid g;
    for (int k = 0; k < 3; k++) {
        g.o[k] = tg_o[k];
        g.n[k] = tg_n[k];
    }
    g.cell = (double)dx;
    uint32_t *cnt = nullptr, *off = nullptr, *total = nullptr, *scratch = nullptr;
    int4 *blo = nullptr, *bn = nullptr;
    int64_t sc = scan_tmp_elems(std::max<int64_t>(nt, 1) + 1);
    CK(dalloc(&cnt, (int64_t)nt + 1));
    CK(dalloc(&off, (int64_t)nt + 1));
    CK(dalloc(&blo, nt));
    CK(dalloc(&bn, nt));
    CK(dalloc(&total, 4));
    CK(dalloc(&scratch, sc));
    CK(cudaMemsetAsync(total, 0, 16, s));
    unsigned long long *total64 = reinterpret_cast<unsigned long long *>(total + 2);
    k_bin_boxes<<<blocks(nt, 128), 128, 0, s>>>(d_verts, d_tris, nt, g, blo, bn, cnt, total64);
    exclusive_scan_u32(cnt, off, nt, total, scratch, sc, s);
    uint32_t ncand_h = 0, open_h = 1;
    unsigned long long ncand64 = 0;
    CK(cudaMemcpyAsync(&ncand_h, total, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&ncand64, total64, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&open_h, open, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    closed = nt > 0 && open_h == 0;
    cudaFree(open);
    if (ncand64 >= (1ull << 31) || ncand64 != (unsigned long long)ncand_h) {
        err = "triangle binning: the triangles span more than 2^31 candidate cells (dx too small for them)";
        cudaFree(cnt);
        cudaFree(off);
        cudaFree(blo);
        cudaFree(bn);
        cudaFree(total);
        cudaFree(scratch);
        return 1;
    }
    const int64_t nc = ncand_h;
    uint32_t *cflag = nullptr, *cpos = nullptr, *ckey = nullptr, *ctri = nullptr;
    CK(dalloc(&cflag, nc));
    CK(dalloc(&cpos, nc));
    CK(dalloc(&ckey, nc));
    CK(dalloc(&ctri, nc));
    const int64_t sc_c = scan_tmp_elems(std::max<int64_t>(nc, 1));
    if (sc_c > sc) {
        cudaFree(scratch);
        CK(dalloc(&scratch, sc_c));
        sc = sc_c;
    }
    if (nc > 0) {
        k_bin_test<<<blocks(nc, 128), 128, 0, s>>>(d_verts, d_tris, nt, g, blo, bn, off, nc, cflag, ckey, ctri);
        exclusive_scan_u32(cflag, cpos, nc, total + 1, scratch, sc, s);
    } else {
        CK(cudaMemsetAsync(total + 1, 0, 4, s));
    }
    uint32_t npairs_h = 0;
    CK(cudaMemcpyAsync(&npairs_h, total + 1, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    npairs = npairs_h;
    uint32_t *pk[2] = {nullptr, nullptr}, *pt[2] = {nullptr, nullptr}, *flag = nullptr, *pos = nullptr;
    CK(dalloc(&pk[0], npairs));
    CK(dalloc(&pk[1], npairs));
    CK(dalloc(&pt[0], npairs));
    CK(dalloc(&pt[1], npairs));
    CK(dalloc(&flag, npairs));
    CK(dalloc(&pos, npairs));
    if (nc > 0) k_bin_emit<<<blocks(nc, 256), 256, 0, s>>>(cflag, cpos, ckey, ctri, nc, pk[0], pt[0]);
    cudaFree(cflag);
    cudaFree(cpos);
    cudaFree(ckey);
    cudaFree(ctri);
    cudaFree(blo);
    cudaFree(bn);
    int64_t pt_tiles = radix_tiles(npairs);
    cudaFree(hist);
    CK(dalloc(&hist, kMaxDigits * std::max<int64_t>(std::max(pt_tiles, tiles), 1)));
    int pb = radix_sort_u32(pk, pt, false, npairs, bits_for((uint64_t)tg_n[0] * tg_n[1] * tg_n[2]), hist, tot, s);
    CK(dalloc(&tlist, npairs));
    CK(cudaMemcpyAsync(tlist, pt[pb], sizeof(uint32_t) * npairs, cudaMemcpyDeviceToDevice, s));
    k_run_flags<<<blocks(npairs), 256, 0, s>>>(pk[pb], npairs, flag);
    int64_t sc2 = scan_tmp_elems(std::max<int64_t>(npairs, 1));
    if (sc2 > sc) {
        cudaFree(scratch);
        CK(dalloc(&scratch, sc2));
        sc = sc2;
    }
    exclusive_scan_u32(flag, pos, npairs, total, scratch, sc, s);
    uint32_t nocc = 0;
    CK(cudaMemcpyAsync(&nocc, total, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ncompact = nocc;
    hash_size = 1;
    while (hash_size < 2 * std::max<int64_t>(ncompact, 1)) hash_size <<= 1;
    uint4 *cmp_unsorted = nullptr;
    uint32_t *hk[2] = {nullptr, nullptr}, *hv[2] = {nullptr, nullptr};
    CK(dalloc(&cmp_unsorted, ncompact));
    CK(dalloc(&compact, ncompact));
    CK(dalloc(&hk[0], ncompact));
    CK(dalloc(&hk[1], ncompact));
    CK(dalloc(&hv[0], ncompact));
    CK(dalloc(&hv[1], ncompact));
    CK(dalloc(&hrng, hash_size));
    CK(cudaMemsetAsync(hrng, 0, sizeof(uint2) * hash_size, s));
    k_compact<<<blocks(npairs), 256, 0, s>>>(pk[pb], npairs, flag, pos, g, (uint32_t)(hash_size - 1), cmp_unsorted,
                                              hk[0]);
    int hb = radix_sort_u32(hk, hv, true, ncompact, bits_for((uint64_t)hash_size - 1), hist, tot, s);
    k_gather_compact<<<blocks(ncompact), 256, 0, s>>>(cmp_unsorted, hv[hb], ncompact, compact);
    k_hash_ranges<<<blocks(ncompact), 256, 0, s>>>(hk[hb], ncompact, hrng);
    occ_words = ((int64_t)tg_n[0] * tg_n[1] * tg_n[2] + 31) / 32;
    CK(dalloc(&occ, 2 * occ_words));
    CK(cudaMemsetAsync(occ, 0, sizeof(uint32_t) * 2 * occ_words, s));
    k_mark_occupancy<<<blocks(ncompact), 256, 0, s>>>(compact, ncompact, g, occ_words, occ);

    // ---- candidate lists of the dilated cells -----------------------------
    uint32_t *wpop = nullptr, *dcell = nullptr, *lcnt = nullptr, *ltot = nullptr, *lscr = nullptr;
    uint8_t *lovf = nullptr;
    CK(dalloc(&drank, occ_words));
    CK(dalloc(&wpop, occ_words));
    CK(dalloc(&ltot, 1));
    int64_t lsc = scan_tmp_elems(occ_words);
    CK(dalloc(&lscr, lsc));
    k_word_popc<<<blocks(occ_words), 256, 0, s>>>(occ + occ_words, occ_words, wpop);
    exclusive_scan_u32(wpop, drank, occ_words, ltot, lscr, lsc, s);
    uint32_t nd = 0;
    CK(cudaMemcpyAsync(&nd, ltot, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    n_dil = nd;
    CK(dalloc(&dcell, n_dil));
    CK(dalloc(&lcnt, n_dil));
    CK(dalloc(&lovf, n_dil));
    CK(dalloc(&coff, n_dil + 1));
    k_bit_cells<<<blocks(occ_words), 256, 0, s>>>(occ + occ_words, occ_words, drank, dcell);
    {
        AsmParams A;
        memset(&A, 0, sizeof(A));
        for (int k = 0; k < 3; k++) A.tg_n[k] = tg_n[k];
        A.hash_mask = (uint32_t)(hash_size - 1);
        const MeshView M{geo, vx, pn, hrng, compact, tlist, nullptr, nullptr, occ, nullptr, nullptr, nullptr};
        const unsigned lb = (unsigned)std::min<int64_t>(std::max<int64_t>((n_dil + 7) / 8, 1), 65535);
        k_cell_lists<false><<<lb, 256, 0, s>>>(A, M, dcell, n_dil, lcnt, lovf, nullptr, nullptr);
        cudaFree(lscr);
        lsc = scan_tmp_elems(std::max<int64_t>(n_dil, 1));
        CK(dalloc(&lscr, lsc));
        exclusive_scan_u32(lcnt, coff, n_dil, coff + n_dil, lscr, lsc, s);
        uint32_t nc_ = 0;
        CK(cudaMemcpyAsync(&nc_, coff + n_dil, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        n_cand = nc_;
        CK(dalloc(&cand, n_cand));
        k_cell_lists<true><<<lb, 256, 0, s>>>(A, M, dcell, n_dil, lcnt, lovf, coff, cand);
        k_flag_overflow<<<blocks(std::max<int64_t>(n_dil, 1)), 256, 0, s>>>(coff, lovf, n_dil);
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    {
        void *lt[] = {wpop, dcell, lcnt, ltot, lscr, lovf};
        for (void *p : lt) cudaFree(p);
    }
    void *tmp[] = {cnt, off, total, scratch, pk[0], pk[1], pt[0], pt[1], flag, pos, cmp_unsorted,
                   hk[0], hk[1], hv[0], hv[1], hist, tot, vpn};
    for (void *p : tmp) cudaFree(p);
    return 0;
}

// Feature edges on the device (sorted (v1, v2)), lines by a colouring walk on
// the host (a few thousand edges at most), segments back to the device.
int Body::extract_features(float deg, cudaStream_t s, std::string &err) {
    const int64_t m = 3 * (int64_t)nt;
    double cthr = std::cos((double)deg * M_PI / 180.0);
    uint32_t *flag = nullptr, *pos = nullptr, *total = nullptr, *scratch = nullptr;
    int32_t *dfe = nullptr;
    auto release = [&]() {
        void *p[] = {flag, pos, total, scratch, dfe};
        for (void *q : p)
            if (q) cudaFree(q);
    };
    // the old features stay as they are until the new edge list is on the host
#define CKF(x)                                                                         \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            release();                                                                 \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                     \
            return e_ == cudaErrorMemoryAllocation ? 3 : 4;                            \
        }                                                                              \
    } while (0)
    int64_t sc = scan_tmp_elems(m);
    CKF(dalloc(&flag, m));
    CKF(dalloc(&pos, m));
    CKF(dalloc(&total, 1));
    CKF(dalloc(&scratch, sc));
    k_feature_flags<<<blocks(m), 256, 0, s>>>(ekey, eval, m, nu, cthr, flag);
    exclusive_scan_u32(flag, pos, m, total, scratch, sc, s);
    uint32_t nfe = 0;
    CKF(cudaMemcpyAsync(&nfe, total, 4, cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
    CKF(dalloc(&dfe, 2 * (int64_t)nfe));
    k_feature_emit<<<blocks(m), 256, 0, s>>>(ekey, m, flag, pos, nv, dfe);
    std::vector<int32_t> fe_new(2 * (size_t)nfe, 0);
    if (nfe) CKF(cudaMemcpyAsync(fe_new.data(), dfe, sizeof(int32_t) * 2 * nfe, cudaMemcpyDeviceToHost, s));
    CKF(cudaStreamSynchronize(s));
#undef CKF
    release();
    fe.swap(fe_new);
    build_lines();
    return upload_lines(s, err);
}

} // namespace fppg
