// Uniformity energy E = sum over mobile i of (rho_i - W0_{c_i})^2 and its
// hand-written backward, with rho_i = W(0) + sum over masked neighbours of
// W(r_ij) (the kernel sum that Eq. 15's pressure force equalises).
//
//   k_rho        rho in key order (masked, FP32) and E (FP64 atomics)
//   k_grad       dE/dx_k = sum_j dW/dr(r_kj) e_kj * coef, coef =
//                2 (rho_k - W0_k) [j acts on k, k mobile] +
//                2 (rho_j - W0_j) [k acts on j, j mobile]
//   k_vjp        through x = y - ((y - v_a) . n) n (frozen triangle): dE/dy
//                and the vertex gradients (atomics into gV)
// energy_accel() turns -dE/dx into the acceleration of the limited step, so
// the same step / projection kernel runs an energy-descent relaxation.
#include <cfloat>

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

// every slot j of the 3 x 3 grid rows around p that the reach cut keeps (a
// superset of the particles within 2h of p), row by row, slots ascending
template <typename F>
__device__ inline void for_rows(const float4 &p, const AsmParams &A, const uint4 *cells, const uint2 *slab,
                                uint32_t ep, F &&f) {
    const int ny = A.ng_n[1], nz = A.ng_n[2];
    const GridPoint g = grid_point(A, p.x, p.y, p.z);
    const int cy = g.c[1], cz = g.c[2];
    for (int z = max(cz - 1, 0); z <= min(cz + 1, nz - 1); z++) {
        const float gz = row_gap(g.t[2], cz, z - cz, g.slack);
        for (int y = max(cy - 1, 0); y <= min(cy + 1, ny - 1); y++) {
            const uint32_t row = A.key_base + (uint32_t)A.ng_n[0] * ((uint32_t)y + (uint32_t)ny * (uint32_t)z);
            uint32_t s, e;
            row_slots(A, cells, slab, ep, g, row_gap(g.t[1], cy, y - cy, g.slack), gz, row, s, e);
            for (uint32_t j = s; j < e; j++) f(j);
        }
    }
}

__global__ void __launch_bounds__(TPB) k_rho(const float4 *__restrict__ pos_s, int64_t N,
                                             const AsmParams *__restrict__ P, const uint4 *__restrict__ cells,
                                             const uint2 *__restrict__ slab, const uint32_t *__restrict__ epoch,
                                             float *__restrict__ rho_s,
                                             double *__restrict__ E) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    double e = 0.0;
    if (k < N) {
        const float4 p = pos_s[k];
        const int cls = cls_of(p.w);
        const AsmParams &A = P[body_of(p.w)];
        const uint32_t mbits = acts_on_bits(cls);
        float rho = 0.f;
        for_rows(p, A, cells, slab, *epoch, [&](uint32_t j) {
            const float4 q = pos_s[j];
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            const float r2 = dist2_rn(dx, dy, dz);
            if (r2 < A.R2 && (int64_t)j != k && (mbits & __float_as_uint(q.w)) != 0u) {
                const float qh = sqrtf(r2) * A.half_inv_h;
                const float t = 1.f - qh;
                rho += t * t * t * t * (4.f * qh + 1.f);
            }
        });
        rho = A.alpha * (rho + 1.f);
        rho_s[k] = rho;
        if (is_mobile(cls, A)) {
            const double d = (double)rho - (double)w0_of(A, cls);
            e = d * d;
        }
    }
    if (E) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(E, e);
    }
}

// out_s[k] = sign * dE/dx_k in key order; amax (nullable) gets the largest
// |out| per body over mobile particles
__global__ void __launch_bounds__(TPB) k_grad(const float4 *__restrict__ pos_s, int64_t N,
                                              const AsmParams *__restrict__ P, const uint4 *__restrict__ cells,
                                              const uint2 *__restrict__ slab, const uint32_t *__restrict__ epoch,
                                              const float *__restrict__ rho_s,
                                              float sign, float4 *__restrict__ out_s, uint32_t *__restrict__ amax) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool active = k < N;
    const float4 p = active ? pos_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int ck = cls_of(p.w);
    const int b = active ? body_of(p.w) : 0;
    const AsmParams &A = P[b];
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (active) {
        const bool mk = is_mobile(ck, A);
        const float ek = mk ? 2.f * (rho_s[k] - w0_of(A, ck)) : 0.f;
        const uint32_t bk = acts_on_bits(ck);
        for_rows(p, A, cells, slab, *epoch, [&](uint32_t j) {
            const float4 q = pos_s[j];
            const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
            const float r2 = dist2_rn(dx, dy, dz);
            if (!(r2 < A.R2) || (int64_t)j == k) return;
            const int cj = cls_of(q.w);
            float coef = 0.f;
            if (mk && (bk & class_bit(cj)) != 0u) coef += ek;
            if (is_mobile(cj, A) && (acts_on_bits(cj) & class_bit(ck)) != 0u) coef += 2.f * (rho_s[j] - w0_of(A, cj));
            if (coef == 0.f) return;
            const float t = 1.f - sqrtf(r2) * A.half_inv_h;
            const float w = -A.force_scale * t * t * t * coef;   // dW/dr / r * coef
            gx += w * dx;
            gy += w * dy;
            gz += w * dz;
        });
    }
    gx *= sign;
    gy *= sign;
    gz *= sign;
    float mag = 0.f;
    if (amax && active && !is_mobile(ck, A)) gx = gy = gz = 0.f;
    if (active) {
        mag = sqrtf(gx * gx + gy * gy + gz * gz);
        out_s[k] = make_float4(gx, gy, gz, mag);
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

__global__ void k_vjp(const float4 *__restrict__ gx_s, const uint32_t *__restrict__ id_s, int64_t N,
                      const float *__restrict__ y, const float4 *__restrict__ pos, const int32_t *__restrict__ cons,
                      const float *__restrict__ V, const int32_t *__restrict__ T, float *__restrict__ gy,
                      float *__restrict__ gV) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    const uint32_t i = id_s[k];
    const float3 g = f3(gx_s[k]);
    const int t = cons[i];
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
    if (!gV) return;
    // dE along dn with u = -(gn (y - a) + s g), dn = (I - n n^T) dm / |m|
    const float3 u = make_float3(-(gn * ya.x + s * g.x), -(gn * ya.y + s * g.y), -(gn * ya.z + s * g.z));
    const float un = dot(u, n);
    const float3 ut = make_float3((u.x - un * n.x) / ml, (u.y - un * n.y) / ml, (u.z - un * n.z) / ml);
    const float3 gb = cross(e2, ut), gc = cross(ut, e1);
    atomicAdd(gV + 3 * ib, gb.x);
    atomicAdd(gV + 3 * ib + 1, gb.y);
    atomicAdd(gV + 3 * ib + 2, gb.z);
    atomicAdd(gV + 3 * ic, gc.x);
    atomicAdd(gV + 3 * ic + 1, gc.y);
    atomicAdd(gV + 3 * ic + 2, gc.z);
    atomicAdd(gV + 3 * ia, -gb.x - gc.x + gn * n.x);
    atomicAdd(gV + 3 * ia + 1, -gb.y - gc.y + gn * n.y);
    atomicAdd(gV + 3 * ia + 2, -gb.z - gc.z + gn * n.z);
}

} // namespace

void energy_accel(Group &g, cudaStream_t s) {
    DevGroup &d = g.d;
    k_rho<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.cells, d.slab, d.epoch, d.rho_s, nullptr);
    k_grad<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.cells, d.slab, d.epoch, d.rho_s, -1.f, d.acc_s,
                                        d.amax);
}

int energy(Group &g, const Body &b, const float *y_dev, const float *verts_dev, double *E, float *gy, float *gV,
           cudaStream_t s, std::string &err) {
    DevGroup &d = g.d;
    float4 *xs = nullptr;
    double *dE = nullptr;
    if (cudaMalloc(&xs, sizeof(float4) * (size_t)std::max<int64_t>(d.N, 1)) != cudaSuccess ||
        cudaMalloc(&dE, sizeof(double)) != cudaSuccess) {
        cudaFree(xs);
        err = "energy: out of device memory";
        return 3;
    }
    const float *V = verts_dev ? verts_dev : b.d_verts;
    cudaMemsetAsync(dE, 0, sizeof(double), s);
    float4 *saved = d.pos;
    k_project_frozen<<<nblocks(d.N), TPB, 0, s>>>(y_dev, d.pos, d.cons, d.N, V, b.d_tris, xs);
    d.pos = xs;
    int buf = build_grid(g, s);
    d.pos = saved;
    k_rho<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.cells, d.slab, d.epoch, d.rho_s, dE);
    if (gy || gV) {
        if (gV) cudaMemsetAsync(gV, 0, sizeof(float) * 3 * (size_t)b.nv, s);
        k_grad<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.cells, d.slab, d.epoch, d.rho_s, 1.f, d.acc_s,
                                             nullptr);
        k_vjp<<<nblocks(d.N), TPB, 0, s>>>(d.acc_s, d.id[buf], d.N, y_dev, d.pos, d.cons, V, b.d_tris, gy, gV);
    }
    cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(xs);
    cudaFree(dE);
    if (e != cudaSuccess) {
        err = std::string("energy: ") + cudaGetErrorString(e);
        return 4;
    }
    return 0;
}

} // namespace fppg
