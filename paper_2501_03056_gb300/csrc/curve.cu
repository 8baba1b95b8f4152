// Intersection curve of two bodies (Sec. 3.2.3): where the surfaces of the
// two operands of a Boolean operation cross, the result has a crease.  It is
// read as a feature line (Sec. 3.2.2): a polyline with feature particles
// placed along it, which then relax along the line like the body's own.
//
// Set-up arithmetic in FP64 on the host, evaluated in the written order
// (compiled with -ffp-contract=off): the side of a vertex with respect to a
// plane is a sign decision, and both segments that share a crossing point
// must compute it from the same numbers.
//
// Per triangle pair (a of body A, b of body B) whose boxes overlap: a's
// vertices against b's plane (unnormalised normal, b's vertex 0 as origin;
// zero counts as the positive side) give the two edges of a that cross it,
// and b's vertices against a's plane the two edges of b.  The crossing point
// of an edge (u < v) is u + (v - u) du / (du - dv), named by the key (mesh of
// the edge, u, v, the other triangle).  Along the line of the two planes
// (direction na x nb) the pair's segment is the overlap of a's two points and
// b's two points, kept when it has positive length.
//
// Chaining, in a fixed order: segments sorted by (a, b); two ends with the
// same key join (a key met by other than two ends joins nothing); ends still
// free join the first free end of another segment, in (segment, end) order,
// within 2^-30 of A's largest extent (a point where the curve meets an edge
// of each mesh at once carries two keys).  Open chains first, each walked
// from the free end of the first segment that has one; then loops, each
// from its first unvisited segment, leaving by the end of larger key.
#include <algorithm>
#include <cmath>

#include "body.h"

namespace fppg {

namespace {

struct CurveKey {
    int32_t side;    // 0: an edge of A crossing a triangle of B; 1: the reverse
    int32_t u, v;    // the edge, u < v
    int64_t other;   // the triangle it crosses
};

int key_cmp(const CurveKey &x, const CurveKey &y) {
    if (x.side != y.side) return x.side < y.side ? -1 : 1;
    if (x.u != y.u) return x.u < y.u ? -1 : 1;
    if (x.v != y.v) return x.v < y.v ? -1 : 1;
    if (x.other != y.other) return x.other < y.other ? -1 : 1;
    return 0;
}

struct CurveSeg {
    int64_t a, b;
    CurveKey key[2];
    double p[2][3];
};

struct MeshD {
    std::vector<double> V;            // vertex coordinates (FP32 values)
    const std::vector<int32_t> *T;
    int64_t nt;
    const double *vert(int64_t t, int i) const { return &V[3 * (size_t)(*T)[3 * t + i]]; }
};

inline double dotd(const double *x, const double *y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; }

inline void diffd(const double *x, const double *y, double *o) {
    for (int k = 0; k < 3; k++) o[k] = x[k] - y[k];
}

inline void crossd(const double *x, const double *y, double *o) {
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
}

void normal_of(const MeshD &m, int64_t t, double *n) {
    double e1[3], e2[3];
    diffd(m.vert(t, 1), m.vert(t, 0), e1);
    diffd(m.vert(t, 2), m.vert(t, 0), e2);
    crossd(e1, e2, n);
}

// the two edges of triangle t that cross plane (n, o), in edge order (0-1,
// 1-2, 2-0), each as (smaller, larger) vertex id; false when all three
// vertices lie on one side
bool crossing_pair(const MeshD &m, int64_t t, const double *n, const double *o, int32_t lo[2], int32_t hi[2]) {
    bool side[3];
    for (int i = 0; i < 3; i++) {
        double w[3];
        diffd(m.vert(t, i), o, w);
        side[i] = dotd(n, w) >= 0.0;
    }
    int found = 0;
    for (int i = 0; i < 3; i++) {
        const int j = i == 2 ? 0 : i + 1;
        if (side[i] == side[j]) continue;
        const int32_t x = (*m.T)[3 * t + i], y = (*m.T)[3 * t + j];
        lo[found] = std::min(x, y);
        hi[found] = std::max(x, y);
        found++;
    }
    return found == 2;
}

void crossing_point(const MeshD &m, int32_t u, int32_t v, const double *n, const double *o, double *p) {
    const double *pu = &m.V[3 * (size_t)u], *pv = &m.V[3 * (size_t)v];
    double wu[3], wv[3], e[3];
    diffd(pu, o, wu);
    diffd(pv, o, wv);
    const double du = dotd(n, wu), dv = dotd(n, wv);
    diffd(pv, pu, e);
    const double t = du / (du - dv);
    for (int k = 0; k < 3; k++) p[k] = pu[k] + e[k] * t;
}

bool pair_segment(const MeshD &A, int64_t a, const MeshD &B, int64_t b, CurveSeg &out) {
    double na[3], nb[3];
    normal_of(A, a, na);
    normal_of(B, b, nb);
    const double *oa = A.vert(a, 0), *ob = B.vert(b, 0);
    int32_t au[2], av[2], bu[2], bv[2];
    if (!crossing_pair(A, a, nb, ob, au, av)) return false;
    if (!crossing_pair(B, b, na, oa, bu, bv)) return false;
    double dir[3];
    crossd(na, nb, dir);
    double q[4][3], t[4];
    CurveKey k[4];
    for (int i = 0; i < 2; i++) {
        crossing_point(A, au[i], av[i], nb, ob, q[i]);
        crossing_point(B, bu[i], bv[i], na, oa, q[2 + i]);
        k[i] = CurveKey{0, au[i], av[i], b};
        k[2 + i] = CurveKey{1, bu[i], bv[i], a};
    }
    for (int i = 0; i < 4; i++) t[i] = dotd(dir, q[i]);
    // each triangle's interval along dir, then their overlap
    const int a_lo = t[0] <= t[1] ? 0 : 1, a_hi = 1 - a_lo;
    const int b_lo = t[2] <= t[3] ? 2 : 3, b_hi = 5 - b_lo;
    const int s = t[a_lo] >= t[b_lo] ? a_lo : b_lo;
    const int e = t[a_hi] <= t[b_hi] ? a_hi : b_hi;
    if (!(t[s] < t[e])) return false;
    out.a = a;
    out.b = b;
    out.key[0] = k[s];
    out.key[1] = k[e];
    for (int c = 0; c < 3; c++) {
        out.p[0][c] = q[s][c];
        out.p[1][c] = q[e][c];
    }
    return true;
}

void box_of(const MeshD &m, int64_t t, double *lo, double *hi) {
    for (int c = 0; c < 3; c++) {
        lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) {
            const double x = m.vert(t, i)[c];
            lo[c] = std::min(lo[c], x);
            hi[c] = std::max(hi[c], x);
        }
}

// Every triangle pair whose closed boxes overlap, found through a uniform
// grid over A's triangles (a pair of overlapping boxes shares a point, and
// that point's cell lies in both boxes' cell ranges), with its segment.
std::vector<CurveSeg> crossing_segments(const MeshD &A, const MeshD &B) {
    std::vector<double> alo(3 * (size_t)A.nt), ahi(3 * (size_t)A.nt);
    double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY}, mean = 0.0;
    for (int64_t a = 0; a < A.nt; a++) {
        box_of(A, a, &alo[3 * a], &ahi[3 * a]);
        double w = 0.0;
        for (int c = 0; c < 3; c++) {
            glo[c] = std::min(glo[c], alo[3 * a + c]);
            ghi[c] = std::max(ghi[c], ahi[3 * a + c]);
            w = std::max(w, ahi[3 * a + c] - alo[3 * a + c]);
        }
        mean += w;
    }
    // cells about twice a triangle's size, at most ~4 per triangle
    double cell = 2.0 * mean / (double)std::max<int64_t>(A.nt, 1);
    const double ext = std::max({ghi[0] - glo[0], ghi[1] - glo[1], ghi[2] - glo[2]});
    if (!(cell > 0.0)) cell = ext > 0.0 ? ext : 1.0;
    double nd[3];
    for (;;) {
        double tot = 1.0;
        for (int c = 0; c < 3; c++) {
            nd[c] = std::floor((ghi[c] - glo[c]) / cell) + 1.0;
            tot *= nd[c];
        }
        if (tot <= 4.0 * (double)std::max<int64_t>(A.nt, 1) + 64.0) break;
        cell *= 1.25;
    }
    const int64_t n[3] = {(int64_t)nd[0], (int64_t)nd[1], (int64_t)nd[2]};
    // clamped in FP64 before the conversion: a box of B far outside A's
    // grid maps to its boundary cells
    auto cell_of = [&](double x, int c) {
        return (int64_t)std::min(std::max(std::floor((x - glo[c]) / cell), 0.0), nd[c] - 1.0);
    };
    auto cell_range = [&](const double *lo, const double *hi, int64_t *c0, int64_t *c1) {
        for (int c = 0; c < 3; c++) {
            c0[c] = cell_of(lo[c], c);
            c1[c] = cell_of(hi[c], c);
        }
    };
    const int64_t ncell = n[0] * n[1] * n[2];
    std::vector<int64_t> start((size_t)ncell + 1, 0);
    std::vector<int64_t> c0(3 * (size_t)A.nt), c1(3 * (size_t)A.nt);
    auto for_cells = [&](const int64_t *l, const int64_t *h, auto &&f) {
        for (int64_t z = l[2]; z <= h[2]; z++)
            for (int64_t y = l[1]; y <= h[1]; y++)
                for (int64_t x = l[0]; x <= h[0]; x++) f((z * n[1] + y) * n[0] + x);
    };
    for (int64_t a = 0; a < A.nt; a++) {
        cell_range(&alo[3 * a], &ahi[3 * a], &c0[3 * a], &c1[3 * a]);
        for_cells(&c0[3 * a], &c1[3 * a], [&](int64_t id) { start[id + 1]++; });
    }
    for (int64_t i = 0; i < ncell; i++) start[i + 1] += start[i];
    std::vector<int64_t> members((size_t)start[ncell]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t a = 0; a < A.nt; a++)
        for_cells(&c0[3 * a], &c1[3 * a], [&](int64_t id) { members[(size_t)fill[id]++] = a; });
    std::vector<CurveSeg> segs;
    std::vector<int64_t> seen((size_t)A.nt, -1);
    for (int64_t b = 0; b < B.nt; b++) {
        double lo[3], hi[3];
        box_of(B, b, lo, hi);
        int64_t l[3], h[3];
        cell_range(lo, hi, l, h);
        for_cells(l, h, [&](int64_t id) {
            for (int64_t e = start[id]; e < start[id + 1]; e++) {
                const int64_t a = members[(size_t)e];
                if (seen[a] == b) continue;
                seen[a] = b;
                bool apart = false;
                for (int c = 0; c < 3; c++)
                    if (alo[3 * a + c] > hi[c] || ahi[3 * a + c] < lo[c]) apart = true;
                if (apart) continue;
                CurveSeg g;
                if (pair_segment(A, a, B, b, g)) segs.push_back(g);
            }
        });
    }
    std::sort(segs.begin(), segs.end(),
              [](const CurveSeg &x, const CurveSeg &y) { return x.a != y.a ? x.a < y.a : x.b < y.b; });
    return segs;
}

}  // namespace

// Appends the feature lines of the curve where this body's surface crosses
// `other`'s and returns their feature particles (positions, class, segment).
// The curve points join verts_host after the mesh vertices (rounded to FP32)
// and the lines follow the body's own.  On failure (out of device memory for
// the new segments) the body is left as it was.
int Body::add_curve(const Body &other, std::vector<float> &xyz, std::vector<int32_t> &cls,
                    std::vector<int32_t> &fseg, cudaStream_t s, std::string &err) {
    MeshD A{std::vector<double>(verts_host.begin(), verts_host.begin() + 3 * (size_t)nv), &tris_host, nt};
    MeshD B{std::vector<double>(other.verts_host.begin(), other.verts_host.begin() + 3 * (size_t)other.nv),
            &other.tris_host, other.nt};
    const std::vector<CurveSeg> S = crossing_segments(A, B);
    const int64_t ns = (int64_t)S.size();
    // join[2 q + e]: the end that end e of segment q continues into, or -1
    std::vector<int64_t> join(2 * (size_t)ns, -1);
    {
        std::vector<int64_t> ends(2 * (size_t)ns);
        for (int64_t i = 0; i < 2 * ns; i++) ends[i] = i;
        std::sort(ends.begin(), ends.end(), [&](int64_t x, int64_t y) {
            const int c = key_cmp(S[x / 2].key[x % 2], S[y / 2].key[y % 2]);
            return c != 0 ? c < 0 : x < y;
        });
        for (int64_t i = 0; i < 2 * ns;) {
            int64_t j = i + 1;
            while (j < 2 * ns && key_cmp(S[ends[j] / 2].key[ends[j] % 2], S[ends[i] / 2].key[ends[i] % 2]) == 0) j++;
            if (j - i == 2) {
                join[ends[i]] = ends[i + 1];
                join[ends[i + 1]] = ends[i];
            }
            i = j;
        }
    }
    double ext = 0.0;
    for (int c = 0; c < 3; c++) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t v = 0; v < nv; v++) {
            lo = std::min(lo, A.V[3 * v + c]);
            hi = std::max(hi, A.V[3 * v + c]);
        }
        ext = std::max(ext, hi - lo);
    }
    const double tol = std::ldexp(ext, -30);
    for (int64_t i = 0; i < 2 * ns; i++) {
        if (join[i] >= 0) continue;
        for (int64_t j = i + 1; j < 2 * ns; j++) {
            if (join[j] >= 0 || j / 2 == i / 2) continue;
            double w[3];
            diffd(S[i / 2].p[i % 2], S[j / 2].p[j % 2], w);
            if (std::sqrt(dotd(w, w)) <= tol) {
                join[i] = j;
                join[j] = i;
                break;
            }
        }
    }
    // walks: open chains, then loops
    std::vector<char> visited((size_t)ns, 0);
    std::vector<double> P;
    std::vector<int64_t> first, count;
    std::vector<int32_t> closed_l;
    for (int pass = 0; pass < 2; pass++)
        for (int64_t q0 = 0; q0 < ns; q0++) {
            if (visited[q0]) continue;
            int enter;
            if (pass == 0) {
                if (join[2 * q0] >= 0 && join[2 * q0 + 1] >= 0) continue;
                enter = join[2 * q0] < 0 ? 0 : 1;
            } else {
                enter = key_cmp(S[q0].key[0], S[q0].key[1]) < 0 ? 0 : 1;
            }
            const int64_t f = (int64_t)P.size() / 3;
            P.insert(P.end(), S[q0].p[enter], S[q0].p[enter] + 3);
            int64_t q = q0;
            int is_loop = 0;
            for (;;) {
                visited[q] = 1;
                const int leave = 1 - enter;
                const int64_t nx = join[2 * q + leave];
                if (nx >= 0 && nx / 2 == q0) {
                    is_loop = 1;
                    break;
                }
                P.insert(P.end(), S[q].p[leave], S[q].p[leave] + 3);
                if (nx < 0 || visited[nx / 2]) break;
                q = nx / 2;
                enter = (int)(nx % 2);
            }
            first.push_back(f);
            count.push_back((int64_t)P.size() / 3 - f);
            closed_l.push_back(is_loop);
        }
    const int64_t npts = (int64_t)P.size() / 3;
    if ((int64_t)verts_host.size() / 3 + npts > ((int64_t)1 << 31) - 1 ||
        (int64_t)nseg + npts > ((int64_t)1 << 31) - 1) {
        err = "intersection curve: too many points";
        return 1;
    }
    // the new state, kept only if the segments reach the device
    const size_t old_verts = verts_host.size(), old_segv = seg_v.size(), old_lines = line_first.size();
    const int old_nseg = nseg, old_nlines = nlines;
    const bool old_has = has_features;
    const int64_t v0 = (int64_t)verts_host.size() / 3;
    for (int64_t i = 0; i < 3 * npts; i++) verts_host.push_back((float)P[(size_t)i]);
    const int l_first = nlines;
    for (size_t l = 0; l < first.size(); l++) {
        const int64_t m = count[l], nsl = closed_l[l] ? m : m - 1;
        line_first.push_back(nseg);
        line_nseg.push_back(nsl);
        line_closed.push_back(closed_l[l]);
        for (int64_t q = 0; q < nsl; q++) {
            seg_v.push_back((int32_t)(v0 + first[l] + q));
            seg_v.push_back((int32_t)(v0 + first[l] + (q + 1) % m));
        }
        nseg += (int)nsl;
        nlines++;
    }
    has_features = true;
    const int r = upload_lines(s, err, true);
    if (r) {
        verts_host.resize(old_verts);
        seg_v.resize(old_segv);
        line_first.resize(old_lines);
        line_nseg.resize(old_lines);
        line_closed.resize(old_lines);
        nseg = old_nseg;
        nlines = old_nlines;
        has_features = old_has;
        return r;
    }
    feature_particles(xyz, cls, fseg, l_first, nlines);
    return 0;
}

void Body::drop_lines_after(int nseg_keep, size_t verts_keep, bool has_features_keep) {
    int keep = 0;
    while (keep < nlines && line_first[keep] < nseg_keep) keep++;
    line_first.resize(keep);
    line_nseg.resize(keep);
    line_closed.resize(keep);
    seg_v.resize(2 * (size_t)nseg_keep);
    nseg = nseg_keep;
    nlines = keep;
    verts_host.resize(verts_keep);
    has_features = has_features_keep;
}

} // namespace fppg
