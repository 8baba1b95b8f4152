// Boolean union of two bodies (Sec. 3.2.3, Fig. 10): the inside test that
// decides which particles of one body lie inside the other.
//
// Ray parity of Fig. 6 for arbitrary points, in FP64 without contraction
// (compiled with -fmad=false): the +z ray from the point (displaced by
// (1.234567e-6, 2.345678e-6) dx in x, y) crosses a triangle
// when the point lies in the triangle's xy projection (barycentric
// coordinates all >= 0) and the crossing height is above the point; odd
// crossings = inside.  Instead of every triangle, the ray's column of
// triangle cells is walked upwards: a triangle crossed at height z is binned
// in the cell whose FP64 box holds (x, y, z) (boxes inflated by 1e-6 dx), so
// counting a crossing only in that cell visits every crossing exactly once.
#include "body.h"

namespace fppg {

namespace {

__global__ void k_ray_parity(const float4 *__restrict__ pos, int64_t n, const AsmParams *__restrict__ P,
                             MeshView M, int32_t *__restrict__ inside) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const AsmParams &A = P[0];
    const float4 pf = pos[i];
    const double cell = (double)A.dx;
    // the ray starts displaced by (1.234567e-6, 2.345678e-6) dx in x, y (as
    // in the generation), so that it meets no edge or vertex exactly
    const double q[3] = {(double)pf.x + 1.234567e-6 * cell, (double)pf.y + 2.345678e-6 * cell, (double)pf.z};
    int c[3];
    for (int k = 0; k < 3; k++) c[k] = (int)floor((q[k] - (double)A.tg_o[k]) / cell);
    int cross = 0;
    if (c[0] >= 0 && c[0] < A.tg_n[0] && c[1] >= 0 && c[1] < A.tg_n[1] && c[2] < A.tg_n[2]) {
        // one cell lower as well: a crossing just above the point may round into it
        for (int z = max(c[2] - 1, 0); z < A.tg_n[2]; z++) {
            if (!test_bit(M.occ, A.occ_off, tri_key(A, c[0], c[1], z))) continue;
            uint32_t beg, len;
            if (!tri_cell(M, A, c[0], c[1], z, beg, len)) continue;
            const double zlo = (double)A.tg_o[2] + z * cell, zhi = (double)A.tg_o[2] + (z + 1) * cell;
            for (uint32_t e = beg; e < beg + len; e++) {
                const size_t g = (size_t)(A.tri_off + M.tlist[e]);
                const float4 va = M.vx[3 * g], vb = M.vx[3 * g + 1], vc = M.vx[3 * g + 2];
                const double a0 = va.x, a1 = va.y, a2 = va.z, b0 = vb.x, b1 = vb.y, b2 = vb.z;
                const double c0 = vc.x, c1 = vc.y, c2 = vc.z;
                const double d = (b0 - a0) * (c1 - a1) - (c0 - a0) * (b1 - a1);
                if (d == 0.0) continue;
                const double l1 = ((b0 - q[0]) * (c1 - q[1]) - (c0 - q[0]) * (b1 - q[1])) / d;
                const double l2 = ((c0 - q[0]) * (a1 - q[1]) - (a0 - q[0]) * (c1 - q[1])) / d;
                const double l3 = 1.0 - l1 - l2;
                if (l1 < 0 || l2 < 0 || l3 < 0) continue;
                const double h = l1 * a2 + l2 * b2 + l3 * c2;
                if (h > q[2] && h >= zlo && h < zhi) cross++;
            }
        }
    }
    inside[i] = cross & 1;
}

} // namespace

// inside[i] (device, n entries) = ray parity of point i of `pos` against
// body 0 of group `other`
void ray_parity(const Group &other, const float4 *pos, int64_t n, int32_t *inside, cudaStream_t s) {
    if (n <= 0) return;
    k_ray_parity<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(pos, n, other.d.params, other.mesh, inside);
}

} // namespace fppg
