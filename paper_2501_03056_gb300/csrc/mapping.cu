// Initial particles of a body (Sec. 3.2), on the device.
//
// Compiled with -fmad=false: the ray-parity arithmetic is evaluated exactly
// in the written order, so inside / outside is decided as by any other IEEE
// implementation of the same formulas.
//   k_column_parity  one warp per (x, y) column of the triangle grid: the
//                    +z ray of Fig. 6 from every cell centre (displaced by
//                    (1.234567e-6, 2.345678e-6) dx in x, y so it never meets
//                    an edge or vertex exactly) against the triangles binned
//                    into the column, each triangle counted once
//   k_dilate_axis    Chebyshev distance <= band to a cell with triangles,
//                    by three one-axis dilations of the occupancy bitmap
//   k_map_cells      per cell in key order: a cell with triangles maps its
//                    centre to the nearest triangle of the cell whose foot
//                    is inside (else it is discarded, Fig. 9b); an empty
//                    cell inside the body gives a volume particle
#include <cfloat>
#include <cmath>

#include "body.h"

namespace fppg {
namespace {

constexpr int kColBuf = 256;   // crossing candidates per column and warp

__device__ inline bool bit_of(const uint32_t *m, uint64_t c) { return (m[c >> 5] >> (c & 31u)) & 1u; }

__device__ inline double centre(const float *o, int a, int i, double dx) {
    return (double)(float)((double)o[a] + ((double)i + 0.5) * dx);
}

struct MapGrid {
    float o[3];
    int n[3];
    double dx;
    uint32_t hash_mask;
    float edge_tol;
};

__device__ inline bool cell_tris(const uint2 *hrng, const uint4 *compact, const MapGrid &g, int x, int y, int z,
                                 uint32_t &beg, uint32_t &len) {
    const uint32_t h = (kHashP1 * (uint32_t)x + kHashP2 * (uint32_t)y + kHashP3 * (uint32_t)z) & g.hash_mask;
    const uint2 r = hrng[h];
    const uint32_t key = (uint32_t)x + (uint32_t)g.n[0] * ((uint32_t)y + (uint32_t)g.n[1] * (uint32_t)z);
    for (uint32_t e = r.x; e < r.x + r.y; e++) {
        const uint4 c = compact[e];
        if (c.x == key) {
            beg = c.y;
            len = c.z;
            return true;
        }
    }
    return false;
}

__global__ void __launch_bounds__(256) k_column_parity(const float *__restrict__ V, const int32_t *__restrict__ T,
                                                       const uint32_t *__restrict__ occ, const uint2 *__restrict__ hrng,
                                                       const uint4 *__restrict__ compact,
                                                       const int32_t *__restrict__ tlist, MapGrid g,
                                                       uint8_t *__restrict__ inside, uint32_t *__restrict__ error) {
    __shared__ int32_t s_tri[8][kColBuf];
    __shared__ double s_z[8][kColBuf];
    __shared__ int s_cnt[8];
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int64_t col = (int64_t)blockIdx.x * 8 + w;
    if (col >= (int64_t)g.n[0] * g.n[1]) return;                 // whole warp
    const int x = (int)(col % g.n[0]), y = (int)(col / g.n[0]);
    const double qx = centre(g.o, 0, x, g.dx) + 1.234567e-6 * g.dx;
    const double qy = centre(g.o, 1, y, g.dx) + 2.345678e-6 * g.dx;
    if (lane == 0) s_cnt[w] = 0;
    __syncwarp();
    bool overflow = false;
    for (int z0 = 0; z0 < g.n[2]; z0 += 32) {
        const int z = z0 + lane;
        uint32_t beg = 0, len = 0;
        if (z < g.n[2]) {
            const uint64_t key = (uint64_t)x + (uint64_t)g.n[0] * ((uint64_t)y + (uint64_t)g.n[1] * (uint64_t)z);
            if (bit_of(occ, key)) cell_tris(hrng, compact, g, x, y, z, beg, len);
        }
        for (uint32_t e = beg; e < beg + len; e++) {
            const int t = tlist[e];
            const float *a = V + 3 * T[3 * t], *b = V + 3 * T[3 * t + 1], *c = V + 3 * T[3 * t + 2];
            const double ax = a[0], ay = a[1], bx = b[0], by = b[1], cx = c[0], cy = c[1];
            const double d = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay);
            if (d == 0.0) continue;
            const double l1 = ((bx - qx) * (cy - qy) - (cx - qx) * (by - qy)) / d;
            const double l2 = ((cx - qx) * (ay - qy) - (ax - qx) * (cy - qy)) / d;
            const double l3 = 1.0 - l1 - l2;
            if (l1 < 0 || l2 < 0 || l3 < 0) continue;
            const double zc = l1 * (double)a[2] + l2 * (double)b[2] + l3 * (double)c[2];
            const int slot = atomicAdd(&s_cnt[w], 1);
            if (slot < kColBuf) {
                s_tri[w][slot] = t;
                s_z[w][slot] = zc;
            } else {
                overflow = true;
            }
        }
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, overflow)) {
        if (lane == 0) atomicOr(error, 1u);
        return;
    }
    const int m = s_cnt[w];
    // a triangle binned into several cells of the column is counted once:
    // an entry counts only if no earlier entry holds the same triangle
    for (int z0 = 0; z0 < g.n[2]; z0 += 32) {
        const int z = z0 + lane;
        if (z >= g.n[2]) continue;
        const double qz = centre(g.o, 2, z, g.dx);
        int cross = 0;
        for (int e = 0; e < m; e++) {
            if (!(s_z[w][e] > qz)) continue;
            bool first = true;
            for (int f = 0; f < e && first; f++) first = s_tri[w][f] != s_tri[w][e];
            cross += first;
        }
        inside[(uint64_t)x + (uint64_t)g.n[0] * ((uint64_t)y + (uint64_t)g.n[1] * (uint64_t)z)] = (uint8_t)(cross & 1);
    }
}

// one-axis dilation by `band` cells of bitmap src into dst (bytes)
__global__ void k_dilate_axis(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, MapGrid g, int axis,
                              int band) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t total = (int64_t)g.n[0] * g.n[1] * g.n[2];
    if (c >= total) return;
    int idx[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((int64_t)g.n[0] * g.n[1]))};
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? g.n[0] : (int64_t)g.n[0] * g.n[1]);
    uint8_t v = 0;
    for (int d = -band; d <= band && !v; d++) {
        const int q = idx[axis] + d;
        if (q < 0 || q >= g.n[axis]) continue;
        v = src[c + (int64_t)d * stride];
    }
    dst[c] = v;
}

__global__ void k_occ_bytes(const uint32_t *__restrict__ occ, int64_t total, uint8_t *__restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (c < total) out[c] = bit_of(occ, (uint64_t)c) ? 1 : 0;
}

// nearest triangle of cell (x, y, z) whose foot of the centre is inside
// (the FP32 rule of the constraint step); -1 when none
__device__ int map_surface_cell(const float4 *__restrict__ geo, const uint2 *__restrict__ hrng,
                                const uint4 *__restrict__ compact, const int32_t *__restrict__ tlist, const MapGrid &g,
                                int x, int y, int z, float3 p, float &dist) {
    uint32_t beg = 0, len = 0;
    if (!cell_tris(hrng, compact, g, x, y, z, beg, len)) return -1;
    float best = FLT_MAX, bd = 0.f;
    int bt = -1;
    for (uint32_t e = beg; e < beg + len; e++) {
        const int t = tlist[e];
        const float4 *q = geo + 5 * (size_t)t;
        const float ux = __fsub_rn(p.x, q[0].x), uy = __fsub_rn(p.y, q[0].y), uz = __fsub_rn(p.z, q[0].z);
        auto dotu = [&](float4 m) { return ux * m.x + uy * m.y + uz * m.z; };
        if (dotu(q[2]) < -g.edge_tol) continue;
        if (dotu(q[3]) - q[3].w < -g.edge_tol) continue;
        if (dotu(q[4]) - q[4].w < -g.edge_tol) continue;
        const float d = dotu(q[1]);
        const float ad = fabsf(d);
        if (ad < best || (ad == best && t < bt)) {
            best = ad;
            bd = d;
            bt = t;
        }
    }
    dist = bd;
    return bt;
}

// pass 0: flags (surface kept / volume); pass 1: emit at the scanned slots
template <bool EMIT>
__global__ void k_map_cells(const float4 *__restrict__ geo, const uint2 *__restrict__ hrng,
                            const uint4 *__restrict__ compact, const int32_t *__restrict__ tlist,
                            const uint32_t *__restrict__ occ, const uint8_t *__restrict__ inside,
                            const uint8_t *__restrict__ band, const uint8_t *__restrict__ inner, MapGrid g,
                            int surface, int volume,
                            uint32_t *__restrict__ sflag, uint32_t *__restrict__ vflag,
                            const uint32_t *__restrict__ soff, const uint32_t *__restrict__ voff, int64_t base_s,
                            int64_t base_v, float4 *__restrict__ pos, int32_t *__restrict__ cons,
                            int32_t *__restrict__ cls) {
    const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t total = (int64_t)g.n[0] * g.n[1] * g.n[2];
    if (c >= total) return;
    const int x = (int)(c % g.n[0]), y = (int)((c / g.n[0]) % g.n[1]), z = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    const float3 p = make_float3((float)centre(g.o, 0, x, g.dx), (float)centre(g.o, 1, y, g.dx),
                                 (float)centre(g.o, 2, z, g.dx));
    uint32_t fs = 0, fv = 0;
    if (bit_of(occ, (uint64_t)c)) {
        if (surface) {
            float d;
            const int t = map_surface_cell(geo, hrng, compact, tlist, g, x, y, z, p, d);
            if (t >= 0) {
                fs = 1;
                if (EMIT) {
                    const float4 n = geo[5 * (size_t)t + 1];
                    const int64_t o = base_s + soff[c];
                    pos[o] = make_float4(p.x - d * n.x, p.y - d * n.y, p.z - d * n.z, __uint_as_float(class_bit(kClsS)));
                    cons[o] = t;
                    cls[o] = kClsS;
                }
            }
        }
    } else if (volume && inside[c] && (inner == nullptr || inner[c])) {
        fv = 1;
        if (EMIT) {
            const int cl = (band == nullptr || band[c]) ? kClsV : kClsI;
            const int64_t o = base_v + voff[c];
            pos[o] = make_float4(p.x, p.y, p.z, __uint_as_float(class_bit(cl)));
            cons[o] = -1;
            cls[o] = cl;
        }
    }
    if (!EMIT) {
        sflag[c] = fs;
        vflag[c] = fv;
    }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>((n + t - 1) / t, 1); }

} // namespace

// Feature particles of Sec. 3.2.2 on the host from the walked lines: n =
// ceil(L / dx) pieces of length L / n; open lines add their singular end
// points once (class P); loops carry n points.  seg gets the segment each
// feature particle was placed on (-1 for singular points), so its first
// step already projects onto its own line.
void Body::feature_particles(std::vector<float> &xyz, std::vector<int32_t> &cls, std::vector<int32_t> &seg, int l0,
                             int l1) const {
    std::vector<char> done(verts_host.size() / 3, 0);
    if (l1 < 0) l1 = nlines;
    auto seglen = [&](int64_t q) {
        const float *a = &verts_host[3 * (size_t)seg_v[2 * q]], *b = &verts_host[3 * (size_t)seg_v[2 * q + 1]];
        const double e0 = (double)b[0] - a[0], e1 = (double)b[1] - a[1], e2 = (double)b[2] - a[2];
        return std::sqrt(e0 * e0 + e1 * e1 + e2 * e2);
    };
    auto emit = [&](double x, double y, double z, int c, int64_t q) {
        xyz.push_back((float)x);
        xyz.push_back((float)y);
        xyz.push_back((float)z);
        cls.push_back(c);
        seg.push_back((int32_t)q);
    };
    for (int l = l0; l < l1; l++) {
        const int64_t f = line_first[l], ns = line_nseg[l];
        double L = 0.0;
        for (int64_t q = f; q < f + ns; q++) L += seglen(q);
        int64_t np = (int64_t)std::ceil(L / (double)dx);
        if (np < 1) np = 1;
        const double sp = L / (double)np;
        const bool closed = line_closed[l] != 0;
        if (!closed) {
            for (int32_t v : {seg_v[2 * f], seg_v[2 * (f + ns - 1) + 1]})
                if (!done[v]) {
                    done[v] = 1;
                    emit(verts_host[3 * (size_t)v], verts_host[3 * (size_t)v + 1], verts_host[3 * (size_t)v + 2], kClsP,
                         -1);
                }
        }
        int64_t q = f;
        double cum = 0.0;
        for (int64_t k = closed ? 0 : 1; k <= np - 1; k++) {
            const double target = sp * (double)k;
            while (q < f + ns - 1 && cum + seglen(q) <= target) {
                cum += seglen(q);
                q++;
            }
            const double len = seglen(q), t = len > 0 ? (target - cum) / len : 0.0;
            const float *a = &verts_host[3 * (size_t)seg_v[2 * q]], *b = &verts_host[3 * (size_t)seg_v[2 * q + 1]];
            emit(a[0] + t * ((double)b[0] - a[0]), a[1] + t * ((double)b[1] - a[1]), a[2] + t * ((double)b[2] - a[2]),
                 kClsF, q);
        }
    }
}

#define CKM(x)                                                                       \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                   \
            return e_ == cudaErrorMemoryAllocation ? 3 : 4;                          \
        }                                                                            \
    } while (0)

int map_particles(Group &g, Body &b, int surface, int volume, int features, int band_cells, int inner_cells,
                  cudaStream_t s, int64_t *n_out, std::vector<int32_t> &cls_host, std::string &err) {
    MapGrid mg;
    for (int k = 0; k < 3; k++) {
        mg.o[k] = b.tg_o[k];
        mg.n[k] = b.tg_n[k];
    }
    mg.dx = (double)b.dx;
    mg.hash_mask = (uint32_t)(b.hash_size - 1);
    mg.edge_tol = b.edge_tol;
    const int64_t cells = (int64_t)mg.n[0] * mg.n[1] * mg.n[2];
    if (cells >= 0xffffffffLL) {
        err = "map_particles: triangle grid too large";
        return 1;
    }
    std::vector<float> fxyz;
    std::vector<int32_t> fcls, fseg;
    if (features && b.has_features) b.feature_particles(fxyz, fcls, fseg);
    const int64_t nf = (int64_t)fcls.size();

    uint8_t *inside = nullptr, *band = nullptr, *tmp = nullptr, *inner = nullptr;
    uint32_t *sflag = nullptr, *vflag = nullptr, *soff = nullptr, *voff = nullptr, *tot = nullptr, *scr = nullptr,
             *error = nullptr;
    auto cleanup = [&]() {
        void *p[] = {inside, band, tmp, inner, sflag, vflag, soff, voff, tot, scr, error};
        for (void *q : p)
            if (q) cudaFree(q);
    };
    const int64_t sc = scan_tmp_elems(cells);
    if (dev_malloc(&inside, cells) || dev_malloc(&sflag, 4 * cells) || dev_malloc(&vflag, 4 * cells) ||
        dev_malloc(&soff, 4 * cells) || dev_malloc(&voff, 4 * cells) || dev_malloc(&tot, 8) ||
        dev_malloc(&scr, 4 * sc) || dev_malloc(&error, 4)) {
        cleanup();
        err = "map_particles: out of device memory";
        return 3;
    }
    cudaMemsetAsync(error, 0, 4, s);
    cudaMemsetAsync(inside, 0, cells, s);
    if (volume)
        k_column_parity<<<nblk((int64_t)mg.n[0] * mg.n[1], 8), 256, 0, s>>>(b.d_verts, b.d_tris, b.occ, b.hrng,
                                                                             b.compact, b.tlist, mg, inside, error);
    if (volume && band_cells > 0) {
        if (dev_malloc(&band, cells) || dev_malloc(&tmp, cells)) {
            cleanup();
            err = "map_particles: out of device memory";
            return 3;
        }
        k_occ_bytes<<<nblk(cells), 256, 0, s>>>(b.occ, cells, band);
        for (int axis = 0; axis < 3; axis++) {
            k_dilate_axis<<<nblk(cells), 256, 0, s>>>(band, tmp, mg, axis, band_cells);
            std::swap(band, tmp);
        }
        if (inner_cells > 0) {
            if (dev_malloc(&inner, cells)) {
                cleanup();
                err = "map_particles: out of device memory";
                return 3;
            }
            k_occ_bytes<<<nblk(cells), 256, 0, s>>>(b.occ, cells, inner);
            for (int axis = 0; axis < 3; axis++) {
                k_dilate_axis<<<nblk(cells), 256, 0, s>>>(inner, tmp, mg, axis, band_cells + inner_cells);
                std::swap(inner, tmp);
            }
        }
    }
    k_map_cells<false><<<nblk(cells), 256, 0, s>>>(b.geo, b.hrng, b.compact, b.tlist, b.occ, inside, band, inner, mg,
                                                   surface,
                                                   volume, sflag, vflag, nullptr, nullptr, 0, 0, nullptr, nullptr,
                                                   nullptr);
    exclusive_scan_u32(sflag, soff, cells, tot, scr, sc, s);
    exclusive_scan_u32(vflag, voff, cells, tot + 1, scr, sc, s);
    uint32_t counts[2] = {0, 0}, errh = 0;
    CKM(cudaMemcpyAsync(counts, tot, 8, cudaMemcpyDeviceToHost, s));
    CKM(cudaMemcpyAsync(&errh, error, 4, cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    if (errh) {
        cleanup();
        err = "map_particles: a grid column crosses more than 256 triangle entries";
        return 6;
    }
    const int64_t ns = counts[0], nvol = counts[1], N = nf + ns + nvol;
    int r = g.alloc_particles(N, err);
    if (r) {
        cleanup();
        return r;
    }
    int32_t *dcls = nullptr;
    if (dev_malloc(&dcls, 4 * std::max<int64_t>(N, 1))) {
        cleanup();
        err = "map_particles: out of device memory";
        return 3;
    }
    if (nf) {
        std::vector<float4> p4(nf);
        const std::vector<int32_t> &c4 = fseg;   // constraints: the segment of each feature particle
        for (int64_t i = 0; i < nf; i++) {
            uint32_t bits = class_bit(fcls[i]);
            float w;
            memcpy(&w, &bits, 4);
            p4[i] = make_float4(fxyz[3 * i], fxyz[3 * i + 1], fxyz[3 * i + 2], w);
        }
        CKM(cudaMemcpyAsync(g.d.pos, p4.data(), sizeof(float4) * nf, cudaMemcpyHostToDevice, s));
        CKM(cudaMemcpyAsync(g.d.cons, c4.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
        CKM(cudaMemcpyAsync(dcls, fcls.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
        CKM(cudaStreamSynchronize(s));
    }
    k_map_cells<true><<<nblk(cells), 256, 0, s>>>(b.geo, b.hrng, b.compact, b.tlist, b.occ, inside, band, inner, mg,
                                                  surface,
                                                  volume, nullptr, nullptr, soff, voff, nf, nf + ns, g.d.pos,
                                                  g.d.cons, dcls);
    cls_host.assign(N, 0);
    if (N) CKM(cudaMemcpyAsync(cls_host.data(), dcls, 4 * N, cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    cudaFree(dcls);
    cleanup();
    *n_out = N;
    return 0;
}

} // namespace fppg
