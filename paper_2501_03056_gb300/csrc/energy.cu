// Uniformity energy E = sum over mobile i of (rho_i - W0_{c_i})^2 and its
// hand-written backward, with rho_i = W(0) + sum over masked neighbours of
// W(r_ij) (the kernel sum that Eq. 15's pressure force equalises).
//
//   k_rho        rho in key order (masked, FP32), kept as the coefficient
//                2 (rho_k - W0_k) of mobile particles, and E (FP64 atomics)
//   k_grad       dE/dx_k = sum_j dW/dr(r_kj) e_kj * coef, coef =
//                2 (rho_k - W0_k) [j acts on k, k mobile] +
//                2 (rho_j - W0_j) [k acts on j, j mobile]
//   k_vjp        through x = y - ((y - v_a) . n) n (frozen triangle): dE/dy
//                and, per particle, its three vertex contributions
//   k_vertex_sum dE/dverts: the contributions sorted by vertex (stable radix
//                sort, so each vertex keeps them in key order) and summed in
//                that order -- no atomics, the same bits on every run
// E is summed by a fixed two-level tree (k_sum_fixed), also run to run exact.
// energy_accel() turns -dE/dx into the acceleration of the limited step, so
// the same step / projection kernel runs an energy-descent relaxation.
#include <cfloat>
#include <type_traits>

#include "body.h"

namespace fppg {

namespace {

constexpr int TPB = 256;
inline unsigned nblocks(int64_t n) { return (unsigned)std::max<int64_t>((n + TPB - 1) / TPB, 1); }

__device__ inline float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ inline float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ inline float w0_of(const AsmParams &A, int c) { return c == kClsS ? A.w0[0] : c == kClsV ? A.w0[1] : A.w0[2]; }

// the classes that feel a particle of class c (its own mask is acts_on_bits)
__device__ constexpr uint32_t felt_by_bits(int c) {
    uint32_t m = 0u;
    for (int t = 0; t <= kClsP; t++)
        if (acts_on_bits(t) & class_bit(c)) m |= class_bit(t);
    return m;
}

// The pair sums walk the same candidates as the force pass: per grid row of
// the 3 x 3 rows around p, the slots that the reach cut keeps (a superset of
// the particles within 2h), read two at a time from the slot-pair copy
// ({x0, x1, y0, y1}, {z0, z1, w0, w1}) into packed FP32x2 operands.  The
// first and last pair of a range may hold a slot outside it (EDGE), masked
// out.  Weights use max(1 - r / 2h, 0), so a slot beyond 2h adds exactly 0
// and one within rounding of 2h a term below 1e-18 of the largest.
template <typename F>
__device__ inline void for_row_ranges(const float4 &p, bool on, const AsmParams &A, const uint32_t *fstart, F &&f) {
    const int ny = A.ng_n[1], nz = A.ng_n[2];
    const GridPoint g = grid_point(A, p.x, p.y, p.z);
    const int cy = g.c[1], cz = g.c[2];
    for (int dz = -1; dz <= 1; dz++) {
        const int z = cz + dz;
        const float gz = row_gap(g.t[2], cz, dz, g.slack);
        for (int dy = -1; dy <= 1; dy++) {
            const int y = cy + dy;
            uint32_t s = 0xffffffffu, e = 0u;
            if (on && z >= 0 && z < nz && y >= 0 && y < ny) {
                const uint32_t row = A.key_base + (uint32_t)A.ng_n[0] * grid_row(A, y, z);
                row_slots(A, fstart, g, row_gap(g.t[1], cy, dy, g.slack), gz, row, s, e);
            }
            f(s, e);
        }
    }
}

// the slot pairs [s >> 1, (e + 1) >> 1) of range [s, e): f(edge, m) with
// edge true for the first and the last
template <typename F>
__device__ inline void for_pairs(uint32_t s, uint32_t e, F &&f) {
    if (s >= e) return;
    uint32_t m = s >> 1;
    const uint32_t m1 = (e + 1) >> 1;
    f(std::true_type{}, m);
    if (m + 1 >= m1) return;
    for (m = m + 1; m + 1 < m1; m++) f(std::false_type{}, m);
    f(std::true_type{}, m1 - 1);
}

struct PairGeo {
    float2 dx, dy, dz, t;   // q - p per axis; max(1 - r / 2h, 0)
    float2 r;
    uint32_t w0, w1;        // class bits of the two slots
};

// pos_p: the {x, y} halves of the slot pairs, pos_b: the {z, w} halves
__device__ inline PairGeo pair_geo(const float4 *__restrict__ pos_p, const float4 *__restrict__ pos_b, uint32_t m,
                                   float2 npx, float2 npy, float2 npz, float hih) {
    const float4 A = pos_p[m], B = pos_b[m];
    PairGeo o;
    o.dx = __fadd2_rn(make_float2(A.x, A.y), npx);
    o.dy = __fadd2_rn(make_float2(A.z, A.w), npy);
    o.dz = __fadd2_rn(make_float2(B.x, B.y), npz);
    const float2 r2 = __fadd2_rn(__fadd2_rn(__fmul2_rn(o.dx, o.dx), __fmul2_rn(o.dy, o.dy)), __fmul2_rn(o.dz, o.dz));
    o.r = make_float2(sqrt_approx(r2.x), sqrt_approx(r2.y));
    const float2 t = __ffma2_rn(o.r, make_float2(-hih, -hih), make_float2(1.f, 1.f));
    o.t = make_float2(fmaxf(t.x, 0.f), fmaxf(t.y, 0.f));
    o.w0 = __float_as_uint(B.z);
    o.w1 = __float_as_uint(B.w);
    return o;
}

// sum over the masked slots of (1 - q/2)^4 (1 + 2q), q = r / h, the particle
// itself included (r = 0 gives exactly 1); ALL: every class acts on the lane
template <bool ALL>
__device__ inline void rho_range(const float4 *__restrict__ pos_p, const float4 *__restrict__ pos_b, uint32_t s,
                                 uint32_t e, float2 npx, float2 npy, float2 npz, uint32_t mbits, float hih,
                                 float2 &acc) {
    for_pairs(s, e, [&](auto edge, uint32_t m) {
        constexpr bool EDGE = decltype(edge)::value;
        const PairGeo g = pair_geo(pos_p, pos_b, m, npx, npy, npz, hih);
        const float2 t2 = __fmul2_rn(g.t, g.t);
        const float2 poly = __ffma2_rn(g.r, make_float2(4.f * hih, 4.f * hih), make_float2(1.f, 1.f));
        float2 w = __fmul2_rn(__fmul2_rn(t2, t2), poly);
        bool k0 = !EDGE || 2 * m >= s, k1 = !EDGE || 2 * m + 1 < e;
        if (!ALL) {
            k0 = k0 && (mbits & g.w0) != 0u;
            k1 = k1 && (mbits & g.w1) != 0u;
        }
        if (EDGE || !ALL) {
            w.x = k0 ? w.x : 0.f;
            w.y = k1 ? w.y : 0.f;
        }
        acc = __fadd2_rn(acc, w);
    });
}

// k_rho: coef_s[k] = 2 (rho_k - W0_k) for mobile k in key order, else 0 (and
// 0 in the padding slot N, read by the slot pairs of an odd count); E[k]
// (nullable) gets (rho_k - W0_k)^2 in FP64 (0 for fixed particles)
__global__ void __launch_bounds__(TPB) k_rho(const float4 *__restrict__ pos_s, const float4 *__restrict__ pos_p,
                                             int64_t N, const AsmParams *__restrict__ P,
                                             const uint32_t *__restrict__ fstart, float *__restrict__ coef_s,
                                             double *__restrict__ E) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool active = k < N;
    const float4 p = active ? pos_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int cls = active ? cls_of(p.w) : kClsI;
    const AsmParams &A = P[active ? body_of(p.w) : 0];
    const bool mob = active && is_mobile(cls, A) && !is_ghost(p.w);
    const uint32_t mbits = mob ? acts_on_bits(cls) : 0u;
    const float hih = A.half_inv_h;
    const float2 npx = make_float2(-p.x, -p.x), npy = make_float2(-p.y, -p.y), npz = make_float2(-p.z, -p.z);
    const bool all_cls = __all_sync(0xffffffffu, mbits == 0u || mbits == 0x1Fu);
    const float4 *pos_b = pos_p + (N + 1) / 2;
    float2 acc = make_float2(0.f, 0.f);
    for_row_ranges(p, mob, A, fstart, [&](uint32_t s, uint32_t e) {
        if (all_cls) rho_range<true>(pos_p, pos_b, s, e, npx, npy, npz, mbits, hih, acc);
        else rho_range<false>(pos_p, pos_b, s, e, npx, npy, npz, mbits, hih, acc);
    });
    double e = 0.0;
    if (mob) {
        const float rho = A.alpha * (acc.x + acc.y);
        const float d = rho - w0_of(A, cls);
        coef_s[k] = 2.f * d;
        const double dd = (double)rho - (double)w0_of(A, cls);
        e = dd * dd;
    } else if (k <= N) {
        coef_s[k] = 0.f;
    }
    if (E && active) E[k] = e;
}

// Deterministic sum of x[0..n): a fixed grid of kSumBlocks blocks strides
// over x in a fixed order, each block reduces by a fixed shared-memory
// tree into part[block], and one block then reduces part[] the same way
// (out = part when it is the second stage).  No atomics: the bits do not
// depend on scheduling.
constexpr int kSumBlocks = 256;

__global__ void __launch_bounds__(TPB) k_sum_fixed(const double *__restrict__ x, int64_t n,
                                                   double *__restrict__ out) {
    __shared__ double sh[TPB];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) a += x[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = TPB / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// sum over the slots of (1 - q/2)^3 c_kj (q - p), c_kj = ek [j acts on k] +
// coef_j [k acts on j]; ALLV: the lane is a volume particle (every class acts
// on it, only volume particles feel it)
template <bool ALLV>
__device__ inline void grad_range(const float4 *__restrict__ pos_p, const float4 *__restrict__ pos_b,
                                  const float2 *__restrict__ coef2, uint32_t s,
                                  uint32_t e, float2 npx, float2 npy, float2 npz, uint32_t bk, uint32_t fk, float ek,
                                  float hih, float2 &gx, float2 &gy, float2 &gz) {
    for_pairs(s, e, [&](auto edge, uint32_t m) {
        constexpr bool EDGE = decltype(edge)::value;
        const PairGeo g = pair_geo(pos_p, pos_b, m, npx, npy, npz, hih);
        const float2 c = coef2[m];
        float2 cf;
        if (ALLV) {
            cf.x = ek + ((g.w0 & class_bit(kClsV)) ? c.x : 0.f);
            cf.y = ek + ((g.w1 & class_bit(kClsV)) ? c.y : 0.f);
        } else {
            cf.x = ((bk & g.w0) ? ek : 0.f) + ((fk & g.w0) ? c.x : 0.f);
            cf.y = ((bk & g.w1) ? ek : 0.f) + ((fk & g.w1) ? c.y : 0.f);
        }
        if (EDGE) {
            cf.x = 2 * m >= s ? cf.x : 0.f;
            cf.y = 2 * m + 1 < e ? cf.y : 0.f;
        }
        const float2 w = __fmul2_rn(__fmul2_rn(__fmul2_rn(g.t, g.t), g.t), cf);
        gx = __ffma2_rn(w, g.dx, gx);
        gy = __ffma2_rn(w, g.dy, gy);
        gz = __ffma2_rn(w, g.dz, gz);
    });
}

// out_s[k] = sign * dE/dx_k in key order; amax (nullable) gets the largest
// |out| per body over mobile particles (and out is 0 for the others)
__global__ void __launch_bounds__(TPB) k_grad(const float4 *__restrict__ pos_s, const float4 *__restrict__ pos_p,
                                              int64_t N, const AsmParams *__restrict__ P,
                                              const uint32_t *__restrict__ fstart, const float *__restrict__ coef_s,
                                              float sign, float4 *__restrict__ out_s, uint32_t *__restrict__ amax) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool active = k < N;
    const float4 p = active ? pos_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ck = active ? cls_of(p.w) : kClsI;
    const AsmParams &A = P[active ? body_of(p.w) : 0];
    const bool mk = active && is_mobile(ck, A) && !is_ghost(p.w);
    const float ek = mk ? coef_s[k] : 0.f;
    const uint32_t bk = mk ? acts_on_bits(ck) : 0u, fk = felt_by_bits(ck);
    const float hih = A.half_inv_h;
    const float2 npx = make_float2(-p.x, -p.x), npy = make_float2(-p.y, -p.y), npz = make_float2(-p.z, -p.z);
    const float2 *coef2 = reinterpret_cast<const float2 *>(coef_s);
    const float4 *pos_b = pos_p + (N + 1) / 2;
    const bool allv = __all_sync(0xffffffffu, !active || ck == kClsV);
    float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
    for_row_ranges(p, active, A, fstart, [&](uint32_t s, uint32_t e) {
        if (allv) grad_range<true>(pos_p, pos_b, coef2, s, e, npx, npy, npz, bk, fk, ek, hih, gx, gy, gz);
        else grad_range<false>(pos_p, pos_b, coef2, s, e, npx, npy, npz, bk, fk, ek, hih, gx, gy, gz);
    });
    const float sc = sign * A.force_scale;
    float fx = (gx.x + gx.y) * sc, fy = (gy.x + gy.y) * sc, fz = (gz.x + gz.y) * sc;
    float mag = 0.f;
    if (amax && !mk) fx = fy = fz = 0.f;
    if (active) {
        mag = sqrtf(fx * fx + fy * fy + fz * fz);
        out_s[k] = make_float4(fx, fy, fz, mag);
    }
    if (amax) {
        const int slot = A.amax_slot;
        uint32_t peers = __match_any_sync(0xffffffffu, slot);
        uint32_t m = __reduce_max_sync(peers, __float_as_uint(mag));
        if ((uint32_t)(__ffs(peers) - 1) == (threadIdx.x & 31u)) atomicMax(amax + slot, m);
    }
}

// x = y - ((y - a) . n) n for S particles with a triangle; w bits kept
__global__ void k_project_frozen(const float *__restrict__ y, const float4 *__restrict__ pos,
                                 const int32_t *__restrict__ cons, int64_t N, const float *__restrict__ V,
                                 const int32_t *__restrict__ T, float4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= N) return;
    const float4 p = pos[i];
    float3 yy = make_float3(y[3 * i], y[3 * i + 1], y[3 * i + 2]);
    const int t = cons[i];
    if (cls_of(p.w) == kClsS && t >= 0) {
        const float3 a = make_float3(V[3 * T[3 * t]], V[3 * T[3 * t] + 1], V[3 * T[3 * t] + 2]);
        const float3 b = make_float3(V[3 * T[3 * t + 1]], V[3 * T[3 * t + 1] + 1], V[3 * T[3 * t + 1] + 2]);
        const float3 c = make_float3(V[3 * T[3 * t + 2]], V[3 * T[3 * t + 2] + 1], V[3 * T[3 * t + 2] + 2]);
        const float3 m = cross(sub(b, a), sub(c, a));
        const float il = rsqrtf(dot(m, m));
        const float3 n = make_float3(m.x * il, m.y * il, m.z * il);
        const float s = dot(sub(yy, a), n);
        yy = make_float3(yy.x - s * n.x, yy.y - s * n.y, yy.z - s * n.z);
    }
    out[i] = make_float4(yy.x, yy.y, yy.z, p.w);
}

// vkey[3k + c] / vcon[3k + c]: vertex and contribution of corner c of the
// frozen triangle of the particle in key slot k (vertex nv = none)
__global__ void k_vjp(const float4 *__restrict__ gx_s, const uint32_t *__restrict__ id_s, int64_t N,
                      const float *__restrict__ y, const float4 *__restrict__ pos, const int32_t *__restrict__ cons,
                      const float *__restrict__ V, const int32_t *__restrict__ T, int nv, float *__restrict__ gy,
                      uint32_t *__restrict__ vkey, float4 *__restrict__ vcon) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    const uint32_t i = id_s[k];
    const float3 g = f3(gx_s[k]);
    const int t = cons[i];
    if (vkey)
        for (int c = 0; c < 3; c++) vkey[3 * k + c] = (uint32_t)nv;
    if (!(cls_of(pos[i].w) == kClsS && t >= 0)) {
        if (gy) {
            gy[3 * (size_t)i] = g.x;
            gy[3 * (size_t)i + 1] = g.y;
            gy[3 * (size_t)i + 2] = g.z;
        }
        return;
    }
    const int ia = T[3 * t], ib = T[3 * t + 1], ic = T[3 * t + 2];
    const float3 a = make_float3(V[3 * ia], V[3 * ia + 1], V[3 * ia + 2]);
    const float3 e1 = sub(make_float3(V[3 * ib], V[3 * ib + 1], V[3 * ib + 2]), a);
    const float3 e2 = sub(make_float3(V[3 * ic], V[3 * ic + 1], V[3 * ic + 2]), a);
    const float3 m = cross(e1, e2);
    const float ml = sqrtf(dot(m, m));
    const float3 n = make_float3(m.x / ml, m.y / ml, m.z / ml);
    const float3 ya = sub(make_float3(y[3 * (size_t)i], y[3 * (size_t)i + 1], y[3 * (size_t)i + 2]), a);
    const float s = dot(ya, n), gn = dot(g, n);
    if (gy) {
        gy[3 * (size_t)i] = g.x - gn * n.x;
        gy[3 * (size_t)i + 1] = g.y - gn * n.y;
        gy[3 * (size_t)i + 2] = g.z - gn * n.z;
    }
    if (!vkey) return;
    // dE along dn with u = -(gn (y - a) + s g), dn = (I - n n^T) dm / |m|
    const float3 u = make_float3(-(gn * ya.x + s * g.x), -(gn * ya.y + s * g.y), -(gn * ya.z + s * g.z));
    const float un = dot(u, n);
    const float3 ut = make_float3((u.x - un * n.x) / ml, (u.y - un * n.y) / ml, (u.z - un * n.z) / ml);
    const float3 gb = cross(e2, ut), gc = cross(ut, e1);
    vkey[3 * k] = (uint32_t)ia;
    vcon[3 * k] = make_float4(-gb.x - gc.x + gn * n.x, -gb.y - gc.y + gn * n.y, -gb.z - gc.z + gn * n.z, 0.f);
    vkey[3 * k + 1] = (uint32_t)ib;
    vcon[3 * k + 1] = make_float4(gb.x, gb.y, gb.z, 0.f);
    vkey[3 * k + 2] = (uint32_t)ic;
    vcon[3 * k + 2] = make_float4(gc.x, gc.y, gc.z, 0.f);
}

// gV[v] = the contributions of vertex v summed in FP64 in sorted order (the
// stable sort keeps key-slot order within a vertex): the thread at the
// start of each run of equal vertices walks its run
__global__ void k_vertex_sum(const uint32_t *__restrict__ vkey_s, const uint32_t *__restrict__ idx_s, int64_t M,
                             const float4 *__restrict__ vcon, int nv, float *__restrict__ gV) {
    const int64_t j = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (j >= M) return;
    const uint32_t v = vkey_s[j];
    if (v >= (uint32_t)nv || (j > 0 && vkey_s[j - 1] == v)) return;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t q = j; q < M && vkey_s[q] == v; q++) {
        const float4 c = vcon[idx_s[q]];
        sx += (double)c.x;
        sy += (double)c.y;
        sz += (double)c.z;
    }
    gV[3 * (size_t)v] = (float)sx;
    gV[3 * (size_t)v + 1] = (float)sy;
    gV[3 * (size_t)v + 2] = (float)sz;
}

} // namespace

void energy_accel(Group &g, cudaStream_t s) {
    DevGroup &d = g.d;
    k_rho<<<nblocks(d.N + 1), TPB, 0, s>>>(d.pos_s, d.pos_p, d.N, d.params, d.fstart, d.coef_s,
                                            nullptr);
    k_grad<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.pos_p, d.N, d.params, d.fstart, d.coef_s, -1.f,
                                        d.acc_s, d.amax);
}

// The scratch of energy(): kept in the group between calls (allocated on the
// first call, grown when the particle count grows), so a repeated energy and
// backward costs no allocation and no implicit device synchronisation.
static int energy_scratch(Group &g, int64_t N, std::string &err) {
    EnergyScratch &e = g.escr;
    if (e.n >= N && e.xs) return 0;
    e.release();
    const int64_t M = 3 * N;
    const size_t n1 = (size_t)std::max<int64_t>(N, 1), m1 = (size_t)std::max<int64_t>(M, 1);
    if (dev_malloc(&e.xs, sizeof(float4) * n1) != cudaSuccess ||
        dev_malloc(&e.e_s, sizeof(double) * n1) != cudaSuccess ||
        dev_malloc(&e.part, sizeof(double) * (kSumBlocks + 1)) != cudaSuccess ||
        dev_malloc(&e.vcon, sizeof(float4) * m1) != cudaSuccess ||
        dev_malloc(&e.vk[0], 4 * m1) != cudaSuccess || dev_malloc(&e.vk[1], 4 * m1) != cudaSuccess ||
        dev_malloc(&e.vi[0], 4 * m1) != cudaSuccess || dev_malloc(&e.vi[1], 4 * m1) != cudaSuccess ||
        dev_malloc(&e.hist, 4 * (size_t)kMaxDigits * std::max<int64_t>(radix_tiles(M), 1)) != cudaSuccess ||
        dev_malloc(&e.tot, 4 * (size_t)kMaxDigits) != cudaSuccess) {
        e.release();
        err = "energy: out of device memory";
        return 3;
    }
    e.n = N;
    return 0;
}

int energy(Group &g, const Body &b, const float *y_dev, const float *verts_dev, double *E, float *gy, float *gV,
           cudaStream_t s, std::string &err) {
    DevGroup &d = g.d;
    const int64_t N = d.N, M = 3 * N;          // M: vertex contributions (three per particle)
    if (const int r = energy_scratch(g, N, err)) return r;
    EnergyScratch &es = g.escr;
    const float *V = verts_dev ? verts_dev : b.d_verts;
    float4 *saved = d.pos;
    k_project_frozen<<<nblocks(N), TPB, 0, s>>>(y_dev, d.pos, d.cons, N, V, b.d_tris, es.xs);
    d.pos = es.xs;
    int buf = build_grid(g, s);
    d.pos = saved;
    k_rho<<<nblocks(N + 1), TPB, 0, s>>>(d.pos_s, d.pos_p, N, d.params, d.fstart, d.coef_s, es.e_s);
    k_sum_fixed<<<kSumBlocks, TPB, 0, s>>>(es.e_s, N, es.part);
    k_sum_fixed<<<1, TPB, 0, s>>>(es.part, kSumBlocks, es.part + kSumBlocks);
    if (gy || gV) {
        k_grad<<<nblocks(N), TPB, 0, s>>>(d.pos_s, d.pos_p, N, d.params, d.fstart, d.coef_s, 1.f, d.acc_s, nullptr);
        k_vjp<<<nblocks(N), TPB, 0, s>>>(d.acc_s, d.id[buf], N, y_dev, d.pos, d.cons, V, b.d_tris, b.nv, gy,
                                          gV ? es.vk[0] : nullptr, es.vcon);
        if (gV) {
            cudaMemsetAsync(gV, 0, sizeof(float) * 3 * (size_t)b.nv, s);
            int bits = 1;
            while (bits < 32 && ((uint64_t)b.nv >> bits) != 0) bits++;
            const int vb = radix_sort_u32(es.vk, es.vi, true, M, bits, es.hist, es.tot, s);
            k_vertex_sum<<<nblocks(M), TPB, 0, s>>>(es.vk[vb], es.vi[vb], M, es.vcon, b.nv, gV);
        }
    }
    cudaMemcpyAsync(E, es.part + kSumBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("energy: ") + cudaGetErrorString(e);
        return 4;
    }
    return 0;
}

} // namespace fppg
