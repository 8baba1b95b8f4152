/*
 * FP64 CPU oracle for the FPPG relaxation hot path (arXiv 2501.03056).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Every step follows the paper in its own order and notation:
 *   Sec. 3.1.1  uniform background grid, cell = particle spacing dx
 *   Sec. 3.1.2  triangle-box overlap (separating axes) marks surface cells,
 *               ray parity (Fig. 6) classifies points as inside / outside
 *   Sec. 3.1.3  cell keys (row-major here; Eq. 9 Morton as an alternative),
 *               cell lists sorted by key, C_compact begin/length
 *   Sec. 3.2.1  projection onto the nearest triangle whose foot is inside
 *               (cross-product test of Fig. 8)
 *   Sec. 3.2.2  edge-face map, dihedral feature rule, singular points,
 *               feature lines by colouring walk, even spacing L/ceil(L/dx)
 *   Sec. 3.3.1  pairwise pressure force, Eq. 15, Wendland C2 kernel Eq. 16/17
 *   Sec. 3.3.2  velocity reset and Euler update, Eqs. 22-23, tangential
 *               displacement, Eqs. 24-25
 *   Sec. 3.3.3  surface re-projection over the 27 neighbouring cells, revert
 *               when no triangle is projectable; Algorithm 1
 *   Sec. 3.3.4  volume particles feel volume, surface and innermost ones
 *
 * Readings where the paper is silent or garbled (all shared with the CUDA
 * side by documentation only):
 *   - alpha_3 = 21 / (16 pi h^3): the printed 21/(6 pi h^3) does not
 *     integrate to one over the support 2h; q = r / h.
 *   - the time step follows the acceleration criterion dt = 0.25 sqrt(h/amax)
 *     of the cited feature-aware SPH work; with v reset to 0 the move is
 *     a dt^2, so the fastest particle moves exactly h/16.
 *   - Eqs. 24-25 are read as removing the normal component of the
 *     displacement (the printed form projects the position itself).
 *   - force constants m = 1, p0 / rho_t^2 terms folded into K = 1; the step
 *     is invariant to K because dt normalises by amax.
 *   - interaction mask: S <- {S, F, P}; V <- {S, V, F, I, P}; F <- {F, P};
 *     I and P (singular feature points) never move.
 *   - one Jacobi update per iteration over all mobile classes with a single
 *     amax per body.
 *   - volume particles are kept inside by the sign of the angle-weighted
 *     pseudonormal of the closest triangle feature (Baerentzen and Aanaes
 *     2005); a volume particle with no triangle within the 27 cells is
 *     accepted.
 *   - decisions that turn floating point into an integer (cell keys, the
 *     neighbour test r^2 < (2h)^2, which triangle / segment is chosen, inside
 *     or outside) are taken in FP32 like the kernels; every continuous
 *     quantity (forces, displacements, feet, energies) is FP64.
 *
 * Parity status per function is listed in the tests that pin it; the
 * end-state quality versus the paper's own figures is unpinned (the paper
 * publishes no particle data).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_S 0
#define OR_V 1
#define OR_F 2
#define OR_I 3
#define OR_P 4

#define OR_MAX_PARTNERS 4   /* Boolean operations one body takes part in */

typedef struct {
    uint32_t key;
    uint32_t id;
} or_kv;

typedef struct {
    /* mesh (Sec. 3.1) */
    int64_t nv, nt;
    int64_t nv_all;     /* nv plus the points of intersection-curve lines (V, Vf hold them all) */
    int64_t nseg_own;   /* segments of the body's own feature lines; curve segments follow */
    /* intersection-curve lines: segments [curve_lo[q], curve_hi[q]) lie on
     * the curve with body curve_with[q] */
    int32_t ncurves;
    int64_t curve_lo[OR_MAX_PARTNERS], curve_hi[OR_MAX_PARTNERS];
    const void *curve_with[OR_MAX_PARTNERS];
    double *V;      /* [nv*3] vertices (FP64 copy of the FP32 input)        */
    float *Vf;      /* [nv*3] vertices as given                             */
    int32_t *T;     /* [nt*3]                                              */
    double *Nrm;    /* [nt*3] cross(b - a, c - a), not normalised          */
    double *Nu;     /* [nt*3] unit normals                                  */
    float *Nuf;     /* [nt*3] unit normals rounded to FP32                  */
    float *EPf;     /* [nt*9] edge pseudonormals, edge k = (v_k, v_k+1)     */
    float *VPf;     /* [nv*3] angle-weighted vertex pseudonormals           */
    float dx, h;
    float edge_tol;  /* a foot this close outside an edge still counts as inside */
    /* triangle grid, cell = dx (Sec. 3.1.1) */
    float tg_o[3];
    float tg_inv;
    int32_t tg_n[3];
    int64_t npairs;
    int64_t *pair_key; /* sorted (cell key, triangle) pairs = C_compact   */
    int32_t *pair_tri;
    /* neighbour grid, cell = 2h (1 + 2^-8) */
    int32_t cell_order;   /* 0: rows y + ny z in order; 1: rows in Morton order (row_rank) */
    uint32_t *row_rank;   /* [ny * nz] place of row y + ny z in the Morton order of (y, z) */
    float ng_o[3];
    float ng_inv;
    float ng_cell;
    int32_t ng_n[3];
    float R2;
    /* features (Sec. 3.2.2) */
    double feat_deg;
    int64_t nfe;
    int32_t *fe;        /* [nfe*2] feature edges (v1 < v2), sorted           */
    int64_t nsing;
    int32_t *sing;      /* singular vertices, ascending                      */
    int64_t nlines;
    int64_t *line_first;  /* first segment of each line                     */
    int64_t *line_nseg;
    int32_t *line_closed;
    int64_t nseg;
    int32_t *seg_v;       /* [nseg*2] vertex ids of each segment            */
    int32_t *seg_line;
    /* particles */
    int64_t n;
    double *X;
    int32_t *cls;
    int32_t *cons;
    int fixed_features;
    int64_t n_ghost;   /* the last n_ghost particles are ghosts: they act, never move */
    double *split_acc; /* forces of oracle_relax_forces, kept for oracle_relax_step */
    int mobile_mask;   /* bit c: class c may move (S, V, F; I and P never do) */
    int cascade;       /* surface re-projection: 0 closest over 27 cells, 1 the cascade of Sec. 3.3.3 */
    double last_maxdisp;
    double last_amax;
    int64_t last_reverts;
} or_ctx;

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void subf(const float *a, const float *b, float *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static float dotf(const float *a, const float *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void crossf(const float *a, const float *b, float *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Wendland C2 kernel, Eqs. 16-17 (3-D, support 2h)                          */
/* ------------------------------------------------------------------------ */
double oracle_alpha3(double h) { return 21.0 / (16.0 * M_PI * h * h * h); }

double oracle_W(double r, double h)
{
    double q = r / h;
    if (q > 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return oracle_alpha3(h) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr = alpha/h * d/dq[(1 - q/2)^4 (2q + 1)] = -5 alpha q (1 - q/2)^3 / h */
double oracle_dW(double r, double h)
{
    double q = r / h;
    if (q > 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * oracle_alpha3(h) * q * t * t * t / h;
}

/* Lattice sum of W over a cubic (dim 3), square (dim 2) or linear (dim 1)
 * lattice of spacing dx, origin included: the ideal kernel sum W0 of a
 * perfectly uniform distribution of the class. */
double oracle_lattice_sum(double dx, double h, int dim)
{
    int m = (int)ceil(2.0 * h / dx) + 1;
    double s = 0.0;
    for (int i = -m; i <= m; i++)
        for (int j = (dim >= 2 ? -m : 0); j <= (dim >= 2 ? m : 0); j++)
            for (int k = (dim >= 3 ? -m : 0); k <= (dim >= 3 ? m : 0); k++) {
                double r = dx * sqrt((double)(i * i + j * j + k * k));
                s += oracle_W(r, h);
            }
    return s;
}

/* ------------------------------------------------------------------------ */
/* grids: FP32 cell coordinate rule (Sec. 3.1.1 / 3.1.3)                     */
/* ------------------------------------------------------------------------ */
/* origin = bbmin - shift * cell (FP64, rounded to FP32); inv = 1 / cell in
 * FP64 rounded to FP32; n = ceil((bbmax - origin) / cell) + margin.  The
 * triangle grid uses shift 2.5 (half a cell more than its margin of 2), so a
 * face lying on the bounding box passes through cell centres, not between
 * two layers of cells; the neighbour grid uses shift = margin = 1. */
static void grid_setup(const float *bbmin, const float *bbmax, float cell, double shift, int margin,
                       float *o, float *inv, int32_t *n)
{
    for (int a = 0; a < 3; a++) {
        o[a] = (float)((double)bbmin[a] - shift * (double)cell);
        n[a] = (int32_t)ceil(((double)bbmax[a] - (double)o[a]) / (double)cell) + margin;
    }
    *inv = (float)(1.0 / (double)cell);
}

/* cell coordinate of a point along one axis: clamp((x - o) * inv, 0, n - 1),
 * evaluated in FP32 without contraction, truncated to an integer. */
static int32_t cell_coord(float x, float o, float inv, int32_t n)
{
    float t = x - o;
    t = t * inv;
    t = fmaxf(t, 0.0f);
    t = fminf(t, (float)(n - 1));
    return (int32_t)t;
}

/* Eq. 9: interleave the bits of (x, y, z) into a Morton code (x lowest). */
uint64_t oracle_morton3(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t code = 0;
    for (int b = 0; b < 21; b++) {
        code |= (uint64_t)((x >> b) & 1u) << (3 * b);
        code |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        code |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return code;
}

/* ------------------------------------------------------------------------ */
/* mesh preprocessing                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t v1, v2, tri, k;
} or_edge;

static int edge_cmp(const void *pa, const void *pb)
{
    const or_edge *a = pa, *b = pb;
    if (a->v1 != b->v1) return a->v1 < b->v1 ? -1 : 1;
    if (a->v2 != b->v2) return a->v2 < b->v2 ? -1 : 1;
    if (a->tri != b->tri) return a->tri < b->tri ? -1 : 1;
    return a->k < b->k ? -1 : (a->k > b->k);
}

/* Edge-face map of Sec. 3.2.2: every triangle edge as (v1 < v2, face). */
static or_edge *edge_face_map(const or_ctx *c)
{
    or_edge *E = malloc(sizeof(or_edge) * 3 * (size_t)c->nt);
    for (int64_t t = 0; t < c->nt; t++)
        for (int k = 0; k < 3; k++) {
            int32_t a = c->T[3 * t + k], b = c->T[3 * t + (k + 1) % 3];
            or_edge *e = &E[3 * t + k];
            e->v1 = a < b ? a : b;
            e->v2 = a < b ? b : a;
            e->tri = (int32_t)t;
            e->k = k;
        }
    qsort(E, 3 * (size_t)c->nt, sizeof(or_edge), edge_cmp);
    return E;
}

static void mesh_prepare(or_ctx *c)
{
    int64_t nt = c->nt, nv = c->nv;
    c->Nrm = malloc(sizeof(double) * 3 * nt);
    c->Nu = malloc(sizeof(double) * 3 * nt);
    c->Nuf = malloc(sizeof(float) * 3 * nt);
    c->EPf = malloc(sizeof(float) * 9 * nt);
    c->VPf = malloc(sizeof(float) * 3 * nv);
    for (int64_t t = 0; t < nt; t++) {
        const double *a = c->V + 3 * c->T[3 * t], *b = c->V + 3 * c->T[3 * t + 1], *cc = c->V + 3 * c->T[3 * t + 2];
        double e1[3], e2[3], n[3];
        sub3(b, a, e1);
        sub3(cc, a, e2);
        cross3(e1, e2, n);
        double len = sqrt(dot3(n, n));
        for (int k = 0; k < 3; k++) {
            c->Nrm[3 * t + k] = n[k];
            c->Nu[3 * t + k] = len > 0 ? n[k] / len : 0.0;
            c->Nuf[3 * t + k] = (float)c->Nu[3 * t + k];
        }
    }
    /* edge pseudonormal: normalised sum of the unit normals of all faces on
     * the edge (two for a closed manifold) */
    or_edge *E = edge_face_map(c);
    int64_t m = 3 * nt;
    for (int64_t s = 0; s < m;) {
        int64_t e = s;
        while (e < m && E[e].v1 == E[s].v1 && E[e].v2 == E[s].v2) e++;
        double sum[3] = {0, 0, 0};
        for (int64_t q = s; q < e; q++)
            for (int k = 0; k < 3; k++) sum[k] += c->Nu[3 * E[q].tri + k];
        double len = sqrt(dot3(sum, sum));
        for (int64_t q = s; q < e; q++)
            for (int k = 0; k < 3; k++)
                c->EPf[9 * E[q].tri + 3 * E[q].k + k] = (float)(len > 0 ? sum[k] / len : 0.0);
        s = e;
    }
    free(E);
    /* vertex pseudonormal: sum of incident unit normals weighted by the
     * triangle's angle at the vertex */
    double *acc = calloc(3 * (size_t)nv, sizeof(double));
    for (int64_t t = 0; t < nt; t++)
        for (int k = 0; k < 3; k++) {
            int32_t vi = c->T[3 * t + k];
            const double *p = c->V + 3 * vi;
            const double *q1 = c->V + 3 * c->T[3 * t + (k + 1) % 3];
            const double *q2 = c->V + 3 * c->T[3 * t + (k + 2) % 3];
            double u[3], w[3];
            sub3(q1, p, u);
            sub3(q2, p, w);
            double lu = sqrt(dot3(u, u)), lw = sqrt(dot3(w, w));
            double cosang = (lu > 0 && lw > 0) ? dot3(u, w) / (lu * lw) : 1.0;
            if (cosang > 1.0) cosang = 1.0;
            if (cosang < -1.0) cosang = -1.0;
            double ang = acos(cosang);
            for (int j = 0; j < 3; j++) acc[3 * vi + j] += ang * c->Nu[3 * t + j];
        }
    for (int64_t v = 0; v < nv; v++) {
        double len = sqrt(dot3(acc + 3 * v, acc + 3 * v));
        for (int j = 0; j < 3; j++) c->VPf[3 * v + j] = (float)(len > 0 ? acc[3 * v + j] / len : 0.0);
    }
    free(acc);
}

/* ------------------------------------------------------------------------ */
/* triangle-box overlap by separating axes (Sec. 3.1.2)                       */
/* ------------------------------------------------------------------------ */
/* Box given by its centre and half size; the box is inflated by 1e-6 dx so
 * that a triangle lying exactly on a cell face counts in both cells. */
static int axis_separates(const double *ax, const double *v0, const double *v1, const double *v2, double hs)
{
    double p0 = dot3(ax, v0), p1 = dot3(ax, v1), p2 = dot3(ax, v2);
    double mn = fmin(p0, fmin(p1, p2)), mx = fmax(p0, fmax(p1, p2));
    double r = hs * (fabs(ax[0]) + fabs(ax[1]) + fabs(ax[2]));
    return mn > r || mx < -r;
}

static int tri_box_overlap(const double *ctr, double hs, const double *a, const double *b, const double *c)
{
    double v0[3], v1[3], v2[3], f[3][3];
    sub3(a, ctr, v0);
    sub3(b, ctr, v1);
    sub3(c, ctr, v2);
    sub3(v1, v0, f[0]);
    sub3(v2, v1, f[1]);
    sub3(v0, v2, f[2]);
    /* box face normals */
    for (int k = 0; k < 3; k++) {
        double mn = fmin(v0[k], fmin(v1[k], v2[k])), mx = fmax(v0[k], fmax(v1[k], v2[k]));
        if (mn > hs || mx < -hs) return 0;
    }
    /* triangle normal */
    double n[3];
    cross3(f[0], f[1], n);
    if (fabs(dot3(n, v0)) > hs * (fabs(n[0]) + fabs(n[1]) + fabs(n[2]))) return 0;
    /* nine edge cross products */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double e[3] = {0, 0, 0}, ax[3];
            e[i] = 1.0;
            cross3(e, f[j], ax);
            if (axis_separates(ax, v0, v1, v2, hs)) return 0;
        }
    return 1;
}

typedef struct {
    int64_t key;
    int32_t tri;
} or_pair;

static int pair_cmp(const void *pa, const void *pb)
{
    const or_pair *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->tri < b->tri ? -1 : (a->tri > b->tri);
}

static void bin_triangles(or_ctx *c)
{
    double cell = (double)c->dx, hs = 0.5 * cell + 1e-6 * cell;
    int64_t cap = 1024, np = 0;
    or_pair *P = malloc(sizeof(or_pair) * cap);
    for (int64_t t = 0; t < c->nt; t++) {
        const double *a = c->V + 3 * c->T[3 * t], *b = c->V + 3 * c->T[3 * t + 1], *cc = c->V + 3 * c->T[3 * t + 2];
        int32_t lo[3], hi[3];
        for (int k = 0; k < 3; k++) {
            double mn = fmin(a[k], fmin(b[k], cc[k])), mx = fmax(a[k], fmax(b[k], cc[k]));
            lo[k] = (int32_t)floor((mn - (double)c->tg_o[k]) / cell) - 1;
            hi[k] = (int32_t)floor((mx - (double)c->tg_o[k]) / cell) + 1;
            if (lo[k] < 0) lo[k] = 0;
            if (hi[k] > c->tg_n[k] - 1) hi[k] = c->tg_n[k] - 1;
        }
        for (int32_t z = lo[2]; z <= hi[2]; z++)
            for (int32_t y = lo[1]; y <= hi[1]; y++)
                for (int32_t x = lo[0]; x <= hi[0]; x++) {
                    double ctr[3] = {(double)c->tg_o[0] + (x + 0.5) * cell, (double)c->tg_o[1] + (y + 0.5) * cell,
                                     (double)c->tg_o[2] + (z + 0.5) * cell};
                    if (!tri_box_overlap(ctr, hs, a, b, cc)) continue;
                    if (np == cap) {
                        cap *= 2;
                        P = realloc(P, sizeof(or_pair) * cap);
                    }
                    P[np].key = (int64_t)x + (int64_t)c->tg_n[0] * ((int64_t)y + (int64_t)c->tg_n[1] * z);
                    P[np].tri = (int32_t)t;
                    np++;
                }
    }
    qsort(P, (size_t)np, sizeof(or_pair), pair_cmp);
    c->npairs = np;
    c->pair_key = malloc(sizeof(int64_t) * (np ? np : 1));
    c->pair_tri = malloc(sizeof(int32_t) * (np ? np : 1));
    for (int64_t i = 0; i < np; i++) {
        c->pair_key[i] = P[i].key;
        c->pair_tri[i] = P[i].tri;
    }
    free(P);
}

static int64_t lower_bound_i64(const int64_t *a, int64_t n, int64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* context                                                                  */
/* ------------------------------------------------------------------------ */
or_ctx *oracle_create(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, float dx, float h)
{
    if (nv <= 0 || nt <= 0 || !(dx > 0) || !(h > 0)) return NULL;
    for (int64_t i = 0; i < 3 * nt; i++)
        if (tris[i] < 0 || tris[i] >= nv) return NULL;
    or_ctx *c = calloc(1, sizeof(or_ctx));
    c->nv = nv;
    c->nv_all = nv;
    c->nt = nt;
    c->dx = dx;
    c->h = h;
    c->V = malloc(sizeof(double) * 3 * nv);
    c->Vf = malloc(sizeof(float) * 3 * nv);
    c->T = malloc(sizeof(int32_t) * 3 * nt);
    memcpy(c->Vf, verts, sizeof(float) * 3 * nv);
    memcpy(c->T, tris, sizeof(int32_t) * 3 * nt);
    float bbmin[3] = {INFINITY, INFINITY, INFINITY}, bbmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; i++)
        for (int k = 0; k < 3; k++) {
            c->V[3 * i + k] = (double)verts[3 * i + k];
            bbmin[k] = fminf(bbmin[k], verts[3 * i + k]);
            bbmax[k] = fmaxf(bbmax[k], verts[3 * i + k]);
        }
    mesh_prepare(c);
    {
        double ext = 0.0;
        for (int k = 0; k < 3; k++) ext = fmax(ext, (double)bbmax[k] - (double)bbmin[k]);
        c->edge_tol = (float)ldexp(ext, -20);
    }
    grid_setup(bbmin, bbmax, dx, 2.5, 2, c->tg_o, &c->tg_inv, c->tg_n);
    bin_triangles(c);
    float R = 2.0f * h;
    c->R2 = (float)((double)R * (double)R);
    c->ng_cell = (float)((double)R * (1.0 + 1.0 / 256.0));
    grid_setup(bbmin, bbmax, c->ng_cell, 1.0, 1, c->ng_o, &c->ng_inv, c->ng_n);
    c->feat_deg = -1.0;
    c->mobile_mask = (1 << OR_S) | (1 << OR_V) | (1 << OR_F);
    return c;
}

static void free_features(or_ctx *c)
{
    free(c->fe);
    free(c->sing);
    free(c->line_first);
    free(c->line_nseg);
    free(c->line_closed);
    free(c->seg_v);
    free(c->seg_line);
    c->fe = c->sing = c->line_closed = c->seg_v = c->seg_line = NULL;
    c->line_first = c->line_nseg = NULL;
    c->nfe = c->nsing = c->nlines = c->nseg = 0;
    c->nseg_own = 0;
    c->ncurves = 0;
    c->nv_all = c->nv;   /* the points of intersection-curve lines go with them */
}

void oracle_destroy(or_ctx *c)
{
    if (!c) return;
    free(c->row_rank);
    free(c->split_acc);
    free(c->V);
    free(c->Vf);
    free(c->T);
    free(c->Nrm);
    free(c->Nu);
    free(c->Nuf);
    free(c->EPf);
    free(c->VPf);
    free(c->pair_key);
    free(c->pair_tri);
    free_features(c);
    free(c->X);
    free(c->cls);
    free(c->cons);
    free(c);
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_fixed_features(or_ctx *c, int fixed) { c->fixed_features = fixed; }

/* Which classes move (bit c for class c; only S, V and F count): the
 * paper relaxes surface particles (Algorithm 1) and then the intermediate
 * volume particles "similarly" (Sec. 3.3.4); mask {S, F} then {V} runs
 * that schedule, the default {S, V, F} moves all at once. */
void oracle_set_mobile_classes(or_ctx *c, int mask) { c->mobile_mask = mask & ((1 << OR_S) | (1 << OR_V) | (1 << OR_F)); }

/* Surface re-projection rule: 0 = the closest projectable triangle over the
 * 27 cells (default), 1 = the cascade of Sec. 3.3.3 (see choose_surface). */
void oracle_set_cascade(or_ctx *c, int on) { c->cascade = on ? 1 : 0; }

void oracle_tri_grid(const or_ctx *c, float *o, float *inv, int32_t *n)
{
    for (int k = 0; k < 3; k++) {
        o[k] = c->tg_o[k];
        n[k] = c->tg_n[k];
    }
    *inv = c->tg_inv;
}

void oracle_nbr_grid(const or_ctx *c, float *o, float *inv, float *cell, int32_t *n, float *R2)
{
    for (int k = 0; k < 3; k++) {
        o[k] = c->ng_o[k];
        n[k] = c->ng_n[k];
    }
    *inv = c->ng_inv;
    *cell = c->ng_cell;
    *R2 = c->R2;
}

/* C_compact content: sorted (cell key, triangle) pairs.  Returns the count;
 * copies at most cap pairs. */
int64_t oracle_tri_bins(const or_ctx *c, int64_t *keys, int32_t *tris, int64_t cap)
{
    for (int64_t i = 0; i < c->npairs && i < cap; i++) {
        keys[i] = c->pair_key[i];
        tris[i] = c->pair_tri[i];
    }
    return c->npairs;
}

void oracle_pseudonormals(const or_ctx *c, float *face, float *edge, float *vert)
{
    if (face) memcpy(face, c->Nuf, sizeof(float) * 3 * c->nt);
    if (edge) memcpy(edge, c->EPf, sizeof(float) * 9 * c->nt);
    if (vert) memcpy(vert, c->VPf, sizeof(float) * 3 * c->nv);
}

/* ------------------------------------------------------------------------ */
/* features (Sec. 3.2.2)                                                     */
/* ------------------------------------------------------------------------ */
static int32_t other_end(const int32_t *fe, int64_t e, int32_t v) { return fe[2 * e] == v ? fe[2 * e + 1] : fe[2 * e]; }

int64_t oracle_extract_features(or_ctx *c, double dihedral_deg)
{
    free_features(c);
    c->feat_deg = dihedral_deg;
    double cthr = cos(dihedral_deg * M_PI / 180.0);
    or_edge *E = edge_face_map(c);
    int64_t m = 3 * c->nt, nfe = 0;
    int32_t *fe = malloc(sizeof(int32_t) * 2 * (m ? m : 1));
    for (int64_t s = 0; s < m;) {
        int64_t e = s;
        while (e < m && E[e].v1 == E[s].v1 && E[e].v2 == E[s].v2) e++;
        int feature;
        if (e - s != 2) {
            feature = 1; /* boundary or non-manifold edge */
        } else {
            /* angle between the two face normals above the threshold */
            double d = dot3(c->Nu + 3 * E[s].tri, c->Nu + 3 * E[s + 1].tri);
            feature = d < cthr;
        }
        if (feature) {
            fe[2 * nfe] = E[s].v1;
            fe[2 * nfe + 1] = E[s].v2;
            nfe++;
        }
        s = e;
    }
    free(E);
    c->nfe = nfe;
    c->fe = fe;
    /* vertex degrees and incidence lists (edges in ascending id) */
    int32_t *deg = calloc((size_t)c->nv, sizeof(int32_t));
    for (int64_t e = 0; e < nfe; e++) {
        deg[fe[2 * e]]++;
        deg[fe[2 * e + 1]]++;
    }
    int64_t *start = malloc(sizeof(int64_t) * (c->nv + 1));
    start[0] = 0;
    for (int64_t v = 0; v < c->nv; v++) start[v + 1] = start[v] + deg[v];
    int64_t *fill = malloc(sizeof(int64_t) * (c->nv ? c->nv : 1));
    for (int64_t v = 0; v < c->nv; v++) fill[v] = start[v];
    int64_t *inc = malloc(sizeof(int64_t) * (2 * nfe + 1));
    for (int64_t e = 0; e < nfe; e++) {
        inc[fill[fe[2 * e]]++] = e;
        inc[fill[fe[2 * e + 1]]++] = e;
    }
    /* singular points: feature degree 1 or above 2 */
    c->sing = malloc(sizeof(int32_t) * (c->nv ? c->nv : 1));
    c->nsing = 0;
    for (int64_t v = 0; v < c->nv; v++)
        if (deg[v] == 1 || deg[v] > 2) c->sing[c->nsing++] = (int32_t)v;
    /* feature lines: walks from singular points, then loops; colouring */
    char *col = calloc((size_t)nfe + 1, 1);
    int64_t lcap = 16, scap = 64;
    c->line_first = malloc(sizeof(int64_t) * lcap);
    c->line_nseg = malloc(sizeof(int64_t) * lcap);
    c->line_closed = malloc(sizeof(int32_t) * lcap);
    c->seg_v = malloc(sizeof(int32_t) * 2 * scap);
    c->seg_line = malloc(sizeof(int32_t) * scap);
#define PUSH_SEG(a, b)                                                  \
    do {                                                                \
        if (c->nseg == scap) {                                          \
            scap *= 2;                                                  \
            c->seg_v = realloc(c->seg_v, sizeof(int32_t) * 2 * scap);   \
            c->seg_line = realloc(c->seg_line, sizeof(int32_t) * scap); \
        }                                                               \
        c->seg_v[2 * c->nseg] = (a);                                    \
        c->seg_v[2 * c->nseg + 1] = (b);                                \
        c->seg_line[c->nseg] = (int32_t)c->nlines;                      \
        c->nseg++;                                                      \
    } while (0)
#define PUSH_LINE(first, closed)                                                  \
    do {                                                                          \
        if (c->nlines == lcap) {                                                  \
            lcap *= 2;                                                            \
            c->line_first = realloc(c->line_first, sizeof(int64_t) * lcap);       \
            c->line_nseg = realloc(c->line_nseg, sizeof(int64_t) * lcap);         \
            c->line_closed = realloc(c->line_closed, sizeof(int32_t) * lcap);     \
        }                                                                         \
        c->line_first[c->nlines] = (first);                                       \
        c->line_nseg[c->nlines] = c->nseg - (first);                              \
        c->line_closed[c->nlines] = (closed);                                     \
        c->nlines++;                                                              \
    } while (0)
    for (int64_t si = 0; si < c->nsing; si++) {
        int32_t s = c->sing[si];
        for (int64_t q = start[s]; q < start[s + 1]; q++) {
            int64_t e = inc[q];
            if (col[e]) continue;
            int64_t first = c->nseg;
            int32_t cur = s;
            for (;;) {
                col[e] = 1;
                int32_t nxt = other_end(fe, e, cur);
                PUSH_SEG(cur, nxt);
                if (deg[nxt] != 2) break;
                int64_t e2 = inc[start[nxt]] == e ? inc[start[nxt] + 1] : inc[start[nxt]];
                if (col[e2]) break;
                e = e2;
                cur = nxt;
            }
            PUSH_LINE(first, 0);
        }
    }
    for (int64_t e0 = 0; e0 < nfe; e0++) {
        if (col[e0]) continue;
        int64_t first = c->nseg, e = e0;
        int32_t v0 = fe[2 * e0], cur = v0;
        int closed = 0;
        for (;;) {
            col[e] = 1;
            int32_t nxt = other_end(fe, e, cur);
            PUSH_SEG(cur, nxt);
            if (nxt == v0) {
                closed = 1;
                break;
            }
            int64_t e2 = inc[start[nxt]] == e ? inc[start[nxt] + 1] : inc[start[nxt]];
            if (col[e2]) break;
            e = e2;
            cur = nxt;
        }
        PUSH_LINE(first, closed);
    }
#undef PUSH_SEG
#undef PUSH_LINE
    c->nseg_own = c->nseg;
    c->ncurves = 0;
    free(col);
    free(inc);
    free(fill);
    free(start);
    free(deg);
    return nfe;
}

int64_t oracle_feature_edges(const or_ctx *c, int32_t *out, int64_t cap)
{
    for (int64_t i = 0; i < c->nfe && i < cap; i++) {
        out[2 * i] = c->fe[2 * i];
        out[2 * i + 1] = c->fe[2 * i + 1];
    }
    return c->nfe;
}

int64_t oracle_singular_points(const or_ctx *c, int32_t *out, int64_t cap)
{
    for (int64_t i = 0; i < c->nsing && i < cap; i++) out[i] = c->sing[i];
    return c->nsing;
}

/* Lines as (first segment, segment count, closed) triples; segments as
 * vertex pairs.  Returns the number of lines. */
int64_t oracle_feature_lines(const or_ctx *c, int64_t *first, int64_t *nseg, int32_t *closed, int32_t *seg_v,
                             int64_t *nseg_total)
{
    for (int64_t l = 0; l < c->nlines; l++) {
        if (first) first[l] = c->line_first[l];
        if (nseg) nseg[l] = c->line_nseg[l];
        if (closed) closed[l] = c->line_closed[l];
    }
    if (seg_v) memcpy(seg_v, c->seg_v, sizeof(int32_t) * 2 * c->nseg);
    if (nseg_total) *nseg_total = c->nseg;
    return c->nlines;
}

static double seg_len(const or_ctx *c, int64_t s)
{
    double d[3];
    sub3(c->V + 3 * c->seg_v[2 * s + 1], c->V + 3 * c->seg_v[2 * s], d);
    return sqrt(dot3(d, d));
}

/* Feature particles: along each line n = ceil(L / dx) equal pieces of
 * length L / n (slightly below dx); open lines carry both end points, which
 * are singular points (class P, emitted once each); loops carry n points.
 * Writes up to cap points; returns the total count.  seg (nullable) gets,
 * per point, the segment of its own line it was placed on (Sec. 3.2.2
 * places every feature particle on a known line), -1 for singular points. */
static int64_t feature_particles_on_segments(const or_ctx *c, double dx, double *xyz, int32_t *cls, int32_t *seg,
                                             int64_t cap);

int64_t oracle_feature_particles(const or_ctx *c, double dx, double *xyz, int32_t *cls, int64_t cap)
{
    return feature_particles_on_segments(c, dx, xyz, cls, NULL, cap);
}

static int64_t feature_particles_of_lines(const or_ctx *c, double dx, int64_t l0, int64_t l1, double *xyz,
                                          int32_t *cls, int32_t *seg, int64_t cap);

static int64_t feature_particles_on_segments(const or_ctx *c, double dx, double *xyz, int32_t *cls, int32_t *seg,
                                             int64_t cap)
{
    return feature_particles_of_lines(c, dx, 0, c->nlines, xyz, cls, seg, cap);
}

/* the same for the lines l0 .. l1 - 1 */
static int64_t feature_particles_of_lines(const or_ctx *c, double dx, int64_t l0, int64_t l1, double *xyz,
                                          int32_t *cls, int32_t *seg, int64_t cap)
{
    int64_t cnt = 0;
    char *done = calloc((size_t)(c->nv_all ? c->nv_all : 1), 1);
#define EMIT(px, py, pz, cl, sg)         \
    do {                                 \
        if (cnt < cap) {                 \
            xyz[3 * cnt] = (px);         \
            xyz[3 * cnt + 1] = (py);     \
            xyz[3 * cnt + 2] = (pz);     \
            cls[cnt] = (cl);             \
            if (seg) seg[cnt] = (sg);    \
        }                                \
        cnt++;                           \
    } while (0)
    for (int64_t l = l0; l < l1; l++) {
        int64_t f = c->line_first[l], ns = c->line_nseg[l];
        double L = 0.0;
        for (int64_t s = f; s < f + ns; s++) L += seg_len(c, s);
        int64_t npc = (int64_t)ceil(L / dx);
        if (npc < 1) npc = 1;
        double sp = L / (double)npc;
        int closed = c->line_closed[l];
        if (!closed) {
            int32_t va = c->seg_v[2 * f], vb = c->seg_v[2 * (f + ns - 1) + 1];
            if (!done[va]) {
                done[va] = 1;
                EMIT(c->V[3 * va], c->V[3 * va + 1], c->V[3 * va + 2], OR_P, -1);
            }
            if (!done[vb]) {
                done[vb] = 1;
                EMIT(c->V[3 * vb], c->V[3 * vb + 1], c->V[3 * vb + 2], OR_P, -1);
            }
        }
        int64_t k0 = closed ? 0 : 1, k1 = closed ? npc - 1 : npc - 1;
        int64_t s = f;
        double cum = 0.0;
        for (int64_t k = k0; k <= k1; k++) {
            double target = sp * (double)k;
            while (s < f + ns - 1 && cum + seg_len(c, s) <= target) {
                cum += seg_len(c, s);
                s++;
            }
            double len = seg_len(c, s), t = len > 0 ? (target - cum) / len : 0.0;
            const double *a = c->V + 3 * c->seg_v[2 * s], *b = c->V + 3 * c->seg_v[2 * s + 1];
            EMIT(a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]), a[2] + t * (b[2] - a[2]), OR_F, (int32_t)s);
        }
    }
#undef EMIT
    free(done);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* particles                                                                */
/* ------------------------------------------------------------------------ */
int oracle_set_particles(or_ctx *c, const float *xyz, const int32_t *cls, int64_t n)
{
    for (int64_t i = 0; i < n; i++)
        if (cls[i] < 0 || cls[i] > 4) return -1;
    free(c->X);
    free(c->cls);
    free(c->cons);
    c->n = n;
    c->X = malloc(sizeof(double) * 3 * (n ? n : 1));
    c->cls = malloc(sizeof(int32_t) * (n ? n : 1));
    c->cons = malloc(sizeof(int32_t) * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++) c->X[3 * i + k] = (double)xyz[3 * i + k];
        c->cls[i] = cls[i];
        c->cons[i] = -1;
    }
    c->last_maxdisp = 0.0;
    c->n_ghost = 0;
    free(c->split_acc);
    c->split_acc = NULL;
    return 0;
}

/* Overwrite positions (FP64) and constraint ids, e.g. to start the oracle
 * from a given state. */
void oracle_set_state(or_ctx *c, const double *xyz, const int32_t *cons)
{
    if (xyz) memcpy(c->X, xyz, sizeof(double) * 3 * c->n);
    if (cons) memcpy(c->cons, cons, sizeof(int32_t) * c->n);
}

void oracle_get_particles(const or_ctx *c, double *xyz, int32_t *cls, int32_t *cons)
{
    if (xyz) memcpy(xyz, c->X, sizeof(double) * 3 * c->n);
    if (cls) memcpy(cls, c->cls, sizeof(int32_t) * c->n);
    if (cons) memcpy(cons, c->cons, sizeof(int32_t) * c->n);
}

static int is_mobile(const or_ctx *c, int32_t cl)
{
    int m = 0;
    if (cl == OR_S || cl == OR_V) m = 1;
    if (cl == OR_F) m = !c->fixed_features;
    return m && ((c->mobile_mask >> cl) & 1);
}

/* does a particle of class cj act on one of class ci (interaction rules of
 * Sec. 3.3.3 and Sec. 3.3.4) */
/* particle i moves: a mobile class and not a ghost (a copy of a particle that
 * another domain of a spatial decomposition owns) */
static int moves(const or_ctx *c, int64_t i) { return i < c->n - c->n_ghost && is_mobile(c, c->cls[i]); }

static int acts_on(int32_t ci, int32_t cj)
{
    switch (ci) {
    case OR_S: return cj == OR_S || cj == OR_F || cj == OR_P;
    case OR_V: return 1;
    case OR_F: return cj == OR_F || cj == OR_P;
    default: return 0;
    }
}

/* ------------------------------------------------------------------------ */
/* neighbour grid: keys, stable sort, cell ranges (Sec. 3.1.3)               */
/* ------------------------------------------------------------------------ */
static void cell_of(const or_ctx *c, const double *x, int32_t *ci)
{
    for (int k = 0; k < 3; k++) ci[k] = cell_coord((float)x[k], c->ng_o[k], c->ng_inv, c->ng_n[k]);
}

/* Sort key of a particle: its cell refined by one of 8 slabs along x.  The
 * paper sorts particles by cell (Sec. 3.1.3) and leaves their order inside
 * a cell open; this order takes, inside each cell, the fine x coordinate
 * clamp(floor(8 t), 0, 8 n - 1), t = (x - o) * inv in FP32, whose top bits
 * are the cell's x (8 t is exact).  key = 8 * cell index + slab, so every
 * cell owns the 8 consecutive keys [8 cell, 8 cell + 8). */
#define OR_SLABS 8

static int32_t fine_coord(float x, float o, float inv, int32_t n)
{
    float t = x - o;
    t = t * inv;
    t = t * (float)OR_SLABS;
    t = fmaxf(t, 0.0f);
    t = fminf(t, (float)(OR_SLABS * n - 1));
    return (int32_t)t;
}

/* Cell index of the key: x + nx * row, where row = y + ny z (row-major) or
 * its place in the Morton order of Eq. 9 over (y, z) (cell_order 1); x is
 * the fastest axis inside a row either way. */
static uint32_t cell_index(const or_ctx *c, const int32_t *ci)
{
    uint32_t row = (uint32_t)ci[1] + (uint32_t)c->ng_n[1] * (uint32_t)ci[2];
    if (c->cell_order) row = c->row_rank[row];
    return (uint32_t)ci[0] + (uint32_t)c->ng_n[0] * row;
}

/* Morton code of Eq. 9 over (y, z): bit b of y at position 2b, bit b of z
 * at position 2b + 1 */
static uint64_t morton_yz(uint32_t y, uint32_t z)
{
    uint64_t m = 0;
    for (int b = 0; b < 32; b++) {
        m |= (uint64_t)((y >> b) & 1u) << (2 * b);
        m |= (uint64_t)((z >> b) & 1u) << (2 * b + 1);
    }
    return m;
}

typedef struct {
    uint64_t code;
    uint32_t row;
} or_rowcode;

static int rowcode_cmp(const void *pa, const void *pb)
{
    const or_rowcode *a = pa, *b = pb;
    return a->code < b->code ? -1 : (a->code > b->code);
}

/* the rank table of the grid's rows (NULL for more than 2^26 rows) */
static uint32_t *morton_rank_table(const int32_t *ng_n)
{
    const int64_t m = (int64_t)ng_n[1] * ng_n[2];
    if (m > ((int64_t)1 << 26)) return NULL;
    or_rowcode *rc = malloc(sizeof(or_rowcode) * (size_t)(m ? m : 1));
    for (int32_t z = 0; z < ng_n[2]; z++)
        for (int32_t y = 0; y < ng_n[1]; y++) {
            const uint32_t r = (uint32_t)y + (uint32_t)ng_n[1] * (uint32_t)z;
            rc[r].code = morton_yz((uint32_t)y, (uint32_t)z);
            rc[r].row = r;
        }
    qsort(rc, (size_t)m, sizeof(or_rowcode), rowcode_cmp);
    uint32_t *rank = malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    for (int64_t q = 0; q < m; q++) rank[rc[q].row] = (uint32_t)q;
    free(rc);
    return rank;
}

/* 0 on success, -1 for an unknown order or a grid of more than 2^26 rows */
int oracle_set_cell_order(or_ctx *c, int32_t order)
{
    if (order != 0 && order != 1) return -1;
    if (order == 1 && !c->row_rank) {
        c->row_rank = morton_rank_table(c->ng_n);
        if (!c->row_rank) return -1;
    }
    c->cell_order = order;
    return 0;
}

static uint32_t key_of(const or_ctx *c, const double *x)
{
    int32_t ci[3];
    cell_of(c, x, ci);
    int32_t fx = fine_coord((float)x[0], c->ng_o[0], c->ng_inv, c->ng_n[0]);
    return OR_SLABS * cell_index(c, ci) + (uint32_t)(fx % OR_SLABS);
}

static int kv_cmp(const void *pa, const void *pb)
{
    const or_kv *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

/* sorted (key, id) list for positions X; ties by id = a stable sort of the
 * id-ordered keys */
static or_kv *build_cells(const or_ctx *c, const double *X, int64_t n)
{
    or_kv *L = malloc(sizeof(or_kv) * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        L[i].key = key_of(c, X + 3 * i);
        L[i].id = (uint32_t)i;
    }
    qsort(L, (size_t)n, sizeof(or_kv), kv_cmp);
    return L;
}

static int64_t lower_bound_kv(const or_kv *L, int64_t n, uint32_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (L[mid].key < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Keys of the current state in id order and the permutation that sorts them
 * stably (perm[k] = id of the k-th particle in key order). */
void oracle_keys(const or_ctx *c, uint32_t *key, uint32_t *perm)
{
    or_kv *L = build_cells(c, c->X, c->n);
    for (int64_t k = 0; k < c->n; k++) {
        key[L[k].id] = L[k].key;
        perm[k] = L[k].id;
    }
    free(L);
}

/* Occupied cells (cell index = key / 8) with their [start, end) ranges in
 * sorted order (C_compact begin / length). Returns the count. */
int64_t oracle_cell_ranges(const or_ctx *c, uint32_t *cell, uint32_t *start, uint32_t *end, int64_t cap)
{
    or_kv *L = build_cells(c, c->X, c->n);
    int64_t m = 0;
    for (int64_t k = 0; k < c->n;) {
        int64_t e = k;
        while (e < c->n && L[e].key / OR_SLABS == L[k].key / OR_SLABS) e++;
        if (m < cap) {
            cell[m] = L[k].key / OR_SLABS;
            start[m] = (uint32_t)k;
            end[m] = (uint32_t)e;
        }
        m++;
        k = e;
    }
    free(L);
    return m;
}

/* FP32 neighbour test: r^2 = (dx dx + dy dy) + dz dz < (2h)^2 */
static int within(const or_ctx *c, const double *xi, const double *xj)
{
    float dx = (float)xi[0] - (float)xj[0];
    float dy = (float)xi[1] - (float)xj[1];
    float dz = (float)xi[2] - (float)xj[2];
    float r2 = dx * dx + dy * dy;
    r2 = r2 + dz * dz;
    return r2 < c->R2;
}

typedef void (*pair_fn)(void *user, int64_t i, int64_t j);

/* visit the neighbours j of particle i (27 cells, FP32 test, class mask
 * unless unmasked) in stencil order */
static void for_neighbours(const or_ctx *c, const double *X, const int32_t *cls, const or_kv *L, int64_t n,
                           int64_t i, int masked, pair_fn fn, void *user)
{
    int32_t ci[3];
    cell_of(c, X + 3 * i, ci);
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int32_t cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= c->ng_n[0] || cc[1] >= c->ng_n[1] ||
                    cc[2] >= c->ng_n[2])
                    continue;
                uint32_t key = OR_SLABS * cell_index(c, cc);
                for (int64_t k = lower_bound_kv(L, n, key); k < n && L[k].key < key + OR_SLABS; k++) {
                    int64_t j = L[k].id;
                    if (j == i) continue;
                    if (masked && !acts_on(cls[i], cls[j])) continue;
                    if (!within(c, X + 3 * i, X + 3 * j)) continue;
                    fn(user, i, j);
                }
            }
}

/* ------------------------------------------------------------------------ */
/* pressure force, Eq. 15 with K = 1                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_ctx *c;
    const double *X;
    double a[3];
    int64_t cnt;
} force_acc;

static void force_pair(void *user, int64_t i, int64_t j)
{
    force_acc *fa = user;
    double d[3];
    sub3(fa->X + 3 * i, fa->X + 3 * j, d);
    double r = sqrt(dot3(d, d));
    fa->cnt++;
    if (r > 0.0) {
        double w = oracle_dW(r, (double)fa->c->h);
        for (int k = 0; k < 3; k++) fa->a[k] -= w * d[k] / r;   /* -dW/dr e_ij */
    }
}

/* acc [n*3] and the masked neighbour count of every particle; fixed
 * particles get zero acceleration but still report their count.  Returns
 * amax over mobile particles. */
static double compute_forces(const or_ctx *c, const double *X, double *acc, int32_t *count)
{
    or_kv *L = build_cells(c, X, c->n);
    double amax = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(max : amax)
    for (int64_t i = 0; i < c->n; i++) {
        force_acc fa = {c, X, {0, 0, 0}, 0};
        for_neighbours(c, X, c->cls, L, c->n, i, 1, force_pair, &fa);
        int mob = moves(c, i);
        for (int k = 0; k < 3; k++) acc[3 * i + k] = mob ? fa.a[k] : 0.0;
        if (count) count[i] = (int32_t)fa.cnt;
        if (mob) {
            double m = sqrt(dot3(fa.a, fa.a));
            if (m > amax) amax = m;
        }
    }
    free(L);
    return amax;
}

double oracle_forces(const or_ctx *c, double *acc, int32_t *count)
{
    return compute_forces(c, c->X, acc, count);
}

/* brute-force O(N^2) masked neighbour counts (validator) */
void oracle_brute_neighbours(const or_ctx *c, int32_t *count)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < c->n; i++) {
        int32_t m = 0;
        for (int64_t j = 0; j < c->n; j++) {
            if (j == i || !acts_on(c->cls[i], c->cls[j])) continue;
            if (within(c, c->X + 3 * i, c->X + 3 * j)) m++;
        }
        count[i] = m;
    }
}

/* ------------------------------------------------------------------------ */
/* projection (Sec. 3.2.1, 3.3.3, 3.3.4)                                     */
/* ------------------------------------------------------------------------ */
static void tri_cell_of(const or_ctx *c, const float *yf, int32_t *ci)
{
    for (int k = 0; k < 3; k++) ci[k] = cell_coord(yf[k], c->tg_o[k], c->tg_inv, c->tg_n[k]);
}

/* component along n of the cross product of edge (p -> q) and (p -> f):
 * non-negative when f is on the inner side of the edge (Fig. 8) */
static float edge_side(const float *p, const float *q, const float *f, const float *n)
{
    float e[3], w[3], cr[3];
    subf(q, p, e);
    subf(f, p, w);
    crossf(e, w, cr);
    return dotf(cr, n);
}

/* the cross-product test with a tolerance: f counts as inside the edge when
 * it lies at most tol outside it (signed distance = edge_side / |q - p|), so
 * that a foot on an edge shared by two triangles belongs to both */
static int edge_inside(const float *p, const float *q, const float *f, const float *n, float tol)
{
    float e[3];
    subf(q, p, e);
    return edge_side(p, q, f, n) >= -tol * sqrtf(dotf(e, e));
}

/* FP32 decision for one triangle: is the orthogonal foot of y inside, and
 * at what distance. */
static int is_degenerate(const or_ctx *c, int64_t t)
{
    const double *n = c->Nu + 3 * t;
    return n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0;
}

static int surface_candidate(const or_ctx *c, int64_t t, const float *y, float *dist)
{
    if (is_degenerate(c, t)) return 0; /* a zero-area triangle has no foot */
    const float *a = c->Vf + 3 * c->T[3 * t], *b = c->Vf + 3 * c->T[3 * t + 1], *cc = c->Vf + 3 * c->T[3 * t + 2];
    const float *n = c->Nuf + 3 * t;
    float ya[3], f[3];
    subf(y, a, ya);
    float d = dotf(ya, n);
    for (int k = 0; k < 3; k++) f[k] = y[k] - d * n[k];
    if (!edge_inside(a, b, f, n, c->edge_tol)) return 0;
    if (!edge_inside(b, cc, f, n, c->edge_tol)) return 0;
    if (!edge_inside(cc, a, f, n, c->edge_tol)) return 0;
    *dist = fabsf(d);
    return 1;
}

/* foot of y on the plane of triangle t, FP64 */
static void plane_foot(const or_ctx *c, int64_t t, const double *y, double *x)
{
    const double *a = c->V + 3 * c->T[3 * t], *n = c->Nu + 3 * t;
    double ya[3];
    sub3(y, a, ya);
    double s = dot3(ya, n);
    for (int k = 0; k < 3; k++) x[k] = y[k] - s * n[k];
}

/* Closest projectable triangle among those binned into the 3x3x3 cells
 * around y: smallest |plane distance|, ties to the lower triangle index.
 * Returns the triangle or -1 when none is projectable. */
static int64_t choose_surface_triangle(const or_ctx *c, const double *y)
{
    float yf[3] = {(float)y[0], (float)y[1], (float)y[2]};
    int32_t ci[3];
    tri_cell_of(c, yf, ci);
    float best = INFINITY;
    int64_t bt = -1;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int32_t cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= c->tg_n[0] || cc[1] >= c->tg_n[1] ||
                    cc[2] >= c->tg_n[2])
                    continue;
                int64_t key = (int64_t)cc[0] + (int64_t)c->tg_n[0] * ((int64_t)cc[1] + (int64_t)c->tg_n[1] * cc[2]);
                for (int64_t p = lower_bound_i64(c->pair_key, c->npairs, key); p < c->npairs && c->pair_key[p] == key;
                     p++) {
                    int64_t t = c->pair_tri[p];
                    float d;
                    if (!surface_candidate(c, t, yf, &d)) continue;
                    if (d < best || (d == best && t < bt)) {
                        best = d;
                        bt = t;
                    }
                }
            }
    return bt;
}

/* The re-projection cascade of Sec. 3.3.3: a particle that is still on its
 * triangle (foot inside it) stays there; otherwise the closest projectable
 * triangle of the cell that holds the trial point, as in the mapping of
 * Sec. 3.2.1; otherwise the closest projectable one over the 27 cells
 * around it; otherwise none (the particle reverts). */
static int64_t choose_surface_cascade(const or_ctx *c, const double *y, int32_t cons_in)
{
    float yf[3] = {(float)y[0], (float)y[1], (float)y[2]}, d;
    if (cons_in >= 0 && cons_in < c->nt && surface_candidate(c, cons_in, yf, &d)) return cons_in;
    int32_t ci[3];
    tri_cell_of(c, yf, ci);
    int64_t key = (int64_t)ci[0] + (int64_t)c->tg_n[0] * ((int64_t)ci[1] + (int64_t)c->tg_n[1] * ci[2]);
    float best = INFINITY;
    int64_t bt = -1;
    for (int64_t p = lower_bound_i64(c->pair_key, c->npairs, key); p < c->npairs && c->pair_key[p] == key; p++) {
        int64_t t = c->pair_tri[p];
        if (!surface_candidate(c, t, yf, &d)) continue;
        if (d < best || (d == best && t < bt)) {
            best = d;
            bt = t;
        }
    }
    return bt >= 0 ? bt : choose_surface_triangle(c, y);
}

/* FP32 closest point on triangle t to y; region 0 = face, 1 + k = edge k,
 * 4 + k = vertex k.  Returns the squared distance. */
static float closest_on_triangle(const or_ctx *c, int64_t t, const float *y, float *cp, int *region)
{
    const float *v[3] = {c->Vf + 3 * c->T[3 * t], c->Vf + 3 * c->T[3 * t + 1], c->Vf + 3 * c->T[3 * t + 2]};
    const float *n = c->Nuf + 3 * t;
    float ya[3], f[3];
    subf(y, v[0], ya);
    float d = dotf(ya, n);
    for (int k = 0; k < 3; k++) f[k] = y[k] - d * n[k];
    if (edge_side(v[0], v[1], f, n) >= 0.0f && edge_side(v[1], v[2], f, n) >= 0.0f &&
        edge_side(v[2], v[0], f, n) >= 0.0f) {
        memcpy(cp, f, sizeof(float) * 3);
        *region = 0;
        float w[3];
        subf(y, f, w);
        return dotf(w, w);
    }
    float best = INFINITY;
    for (int k = 0; k < 3; k++) {
        const float *p = v[k], *q = v[(k + 1) % 3];
        float e[3], w[3];
        subf(q, p, e);
        subf(y, p, w);
        float ee = dotf(e, e);
        float s = ee > 0.0f ? dotf(w, e) / ee : 0.0f;
        if (s < 0.0f) s = 0.0f;
        if (s > 1.0f) s = 1.0f;
        float pt[3] = {p[0] + s * e[0], p[1] + s * e[1], p[2] + s * e[2]}, u[3];
        subf(y, pt, u);
        float dd = dotf(u, u);
        if (dd < best) {
            best = dd;
            memcpy(cp, pt, sizeof(float) * 3);
            *region = s <= 0.0f ? 4 + k : (s >= 1.0f ? 4 + (k + 1) % 3 : 1 + k);
        }
    }
    return best;
}

/* Inside test of a volume particle: closest triangle among the 27 cells
 * (smallest distance, ties to the lower index) and the sign of (y - c) . psi
 * with psi the pseudonormal of the closest feature.  Returns 1 inside (or no
 * triangle near), 0 outside. */
static int closest_sign_inside(const or_ctx *c, const float *yf);

static int volume_inside_f(const or_ctx *c, const float *yf)
{
    int r = closest_sign_inside(c, yf);
    return r < 0 ? 1 : r;
}

/* The closest-feature sign test alone: 1 inside, 0 outside, -1 when no
 * triangle lies in the 27 cells around yf. */
static int closest_sign_inside(const or_ctx *c, const float *yf)
{
    int32_t ci[3];
    tri_cell_of(c, yf, ci);
    float best = INFINITY, bcp[3] = {0, 0, 0};
    int64_t bt = -1;
    int breg = 0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int32_t cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                if (cc[0] < 0 || cc[1] < 0 || cc[2] < 0 || cc[0] >= c->tg_n[0] || cc[1] >= c->tg_n[1] ||
                    cc[2] >= c->tg_n[2])
                    continue;
                int64_t key = (int64_t)cc[0] + (int64_t)c->tg_n[0] * ((int64_t)cc[1] + (int64_t)c->tg_n[1] * cc[2]);
                for (int64_t p = lower_bound_i64(c->pair_key, c->npairs, key); p < c->npairs && c->pair_key[p] == key;
                     p++) {
                    int64_t t = c->pair_tri[p];
                    if (is_degenerate(c, t)) continue;
                    float cp[3];
                    int reg;
                    float dd = closest_on_triangle(c, t, yf, cp, &reg);
                    if (dd < best || (dd == best && t < bt)) {
                        best = dd;
                        bt = t;
                        breg = reg;
                        memcpy(bcp, cp, sizeof(bcp));
                    }
                }
            }
    if (bt < 0) return -1;
    const float *psi;
    if (breg == 0) psi = c->Nuf + 3 * bt;
    else if (breg <= 3) psi = c->EPf + 9 * bt + 3 * (breg - 1);
    else psi = c->VPf + 3 * c->T[3 * bt + (breg - 4)];
    float w[3];
    subf(yf, bcp, w);
    return dotf(w, psi) <= 0.0f;
}

/* closest point on the own feature line (all lines when cons < 0): FP32
 * choice of the segment (smallest squared distance, ties to the lower
 * segment), FP64 point.  Returns the segment or -1. */
static int64_t project_feature(const or_ctx *c, const double *y, int32_t cons, double *x)
{
    if (c->nseg == 0) return -1;
    int64_t s0 = 0, s1 = c->nseg;
    if (cons >= 0 && cons < c->nseg) {
        int32_t l = c->seg_line[cons];
        s0 = c->line_first[l];
        s1 = s0 + c->line_nseg[l];
    }
    float yf[3] = {(float)y[0], (float)y[1], (float)y[2]};
    float best = INFINITY;
    int64_t bs = -1;
    for (int64_t s = s0; s < s1; s++) {
        const float *a = c->Vf + 3 * c->seg_v[2 * s], *b = c->Vf + 3 * c->seg_v[2 * s + 1];
        float e[3], w[3];
        subf(b, a, e);
        subf(yf, a, w);
        float ee = dotf(e, e);
        float t = ee > 0.0f ? dotf(w, e) / ee : 0.0f;
        if (t < 0.0f) t = 0.0f;
        if (t > 1.0f) t = 1.0f;
        float q[3] = {a[0] + t * e[0], a[1] + t * e[1], a[2] + t * e[2]}, u[3];
        subf(yf, q, u);
        float dd = dotf(u, u);
        if (dd < best) {
            best = dd;
            bs = s;
        }
    }
    const double *a = c->V + 3 * c->seg_v[2 * bs], *b = c->V + 3 * c->seg_v[2 * bs + 1];
    double e[3], w[3];
    sub3(b, a, e);
    sub3(y, a, w);
    double ee = dot3(e, e);
    double t = ee > 0.0 ? dot3(w, e) / ee : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    for (int k = 0; k < 3; k++) x[k] = a[k] + t * e[k];
    return bs;
}

/* Project one trial point according to its class.  Writes the new position
 * and constraint; returns 1 on success, 0 when the particle must revert. */
static int project_point(const or_ctx *c, int32_t cl, const double *y, int32_t cons_in, double *x, int32_t *cons_out)
{
    *cons_out = cons_in;
    if (cl == OR_S) {
        int64_t t = c->cascade ? choose_surface_cascade(c, y, cons_in) : choose_surface_triangle(c, y);
        if (t < 0) return 0;
        plane_foot(c, t, y, x);
        *cons_out = (int32_t)t;
        return 1;
    }
    if (cl == OR_V) {
        float yf[3] = {(float)y[0], (float)y[1], (float)y[2]};
        if (!volume_inside_f(c, yf)) return 0;
        memcpy(x, y, sizeof(double) * 3);
        return 1;
    }
    if (cl == OR_F) {
        int64_t s = project_feature(c, y, cons_in, x);
        if (s < 0) return 0;
        *cons_out = (int32_t)s;
        return 1;
    }
    memcpy(x, y, sizeof(double) * 3);
    return 1;
}

/* Projection of given FP32 points (the standalone form of the constraint
 * step).  ok[i] = 0 marks "not projectable" (x[i] then equals y[i]). */
void oracle_project_points(const or_ctx *c, const float *y, const int32_t *cls, const int32_t *cons_in, int64_t n,
                           double *x, int32_t *cons_out, int32_t *ok)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        double yd[3] = {(double)y[3 * i], (double)y[3 * i + 1], (double)y[3 * i + 2]};
        int r = project_point(c, cls[i], yd, cons_in ? cons_in[i] : -1, x + 3 * i, cons_out + i);
        if (!r) memcpy(x + 3 * i, yd, sizeof(yd));
        ok[i] = r;
    }
}

/* Brute force over all triangles: the closest projectable triangle (same
 * FP32 decision, no grid).  Validates the binned search. */
void oracle_brute_surface(const or_ctx *c, const float *y, int64_t n, int32_t *tri, float *dist)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        float best = INFINITY;
        int64_t bt = -1;
        for (int64_t t = 0; t < c->nt; t++) {
            float d;
            if (!surface_candidate(c, t, y + 3 * i, &d)) continue;
            if (d < best || (d == best && t < bt)) {
                best = d;
                bt = t;
            }
        }
        tri[i] = (int32_t)bt;
        dist[i] = best;
    }
}

/* Pseudonormal inside test on given points (1 inside or far, 0 outside). */
void oracle_volume_inside(const or_ctx *c, const float *y, int64_t n, int32_t *inside)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) inside[i] = volume_inside_f(c, y + 3 * i);
}

/* Ray parity of Fig. 6: count crossings of the +z ray from p with the
 * triangles (FP64, half-open edge rule).  1 = inside. */
void oracle_ray_parity(const or_ctx *c, const double *p, int64_t n, int32_t *inside)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        const double *q = p + 3 * i;
        int64_t cross = 0;
        for (int64_t t = 0; t < c->nt; t++) {
            const double *a = c->V + 3 * c->T[3 * t], *b = c->V + 3 * c->T[3 * t + 1], *cc = c->V + 3 * c->T[3 * t + 2];
            /* 2-D point-in-triangle in the xy plane, barycentric with a
             * consistent tie rule, then the crossing height */
            double d = (b[0] - a[0]) * (cc[1] - a[1]) - (cc[0] - a[0]) * (b[1] - a[1]);
            if (d == 0.0) continue;
            double l1 = ((b[0] - q[0]) * (cc[1] - q[1]) - (cc[0] - q[0]) * (b[1] - q[1])) / d;
            double l2 = ((cc[0] - q[0]) * (a[1] - q[1]) - (a[0] - q[0]) * (cc[1] - q[1])) / d;
            double l3 = 1.0 - l1 - l2;
            if (l1 < 0 || l2 < 0 || l3 < 0) continue;
            double z = l1 * a[2] + l2 * b[2] + l3 * cc[2];
            if (z > q[2]) cross++;
        }
        inside[i] = (int32_t)(cross & 1);
    }
}

/* ------------------------------------------------------------------------ */
/* one relaxation iteration (Algorithm 1, Eqs. 22-25, Sec. 3.3.3-3.3.4)      */
/* ------------------------------------------------------------------------ */
/* Apply the step to every mobile particle from accelerations acc and the
 * body's amax: dt = 0.25 sqrt(h / amax); v_{n+1} = 0 + a dt (velocity
 * reset); dr = v_{n+1} dt (Eq. 23); tangential part only for surface
 * (triangle normal) and feature (segment direction) particles; then the
 * projection of the trial point, or revert. */
static void apply_step_partners(or_ctx *c, const double *acc, double amax, const or_ctx *const *partner,
                                const int *surf_rule, const int *vol_rule, int npart);

static void apply_step(or_ctx *c, const double *acc, double amax)
{
    apply_step_partners(c, acc, amax, NULL, NULL, NULL, 0);
}

/* With Boolean partners (see oracle_boolean_relax_many), a projected
 * position must also respect every partner: rule 1 = stay outside it, rule
 * 2 = stay inside it, 0 = no rule; surf_rule for surface and feature
 * particles, vol_rule for volume particles.  The partner test is the
 * closest-feature sign of the partner's triangles within the 27 cells; with
 * none near, a particle is where it started (it moves less than a cell per
 * iteration) and the rule holds.  A feature particle on the intersection
 * curve with a partner lies on both surfaces: that partner's rule does not
 * apply to it (the others' do). */
static int partner_ok(const or_ctx *partner, int rule, const double *x)
{
    if (!partner || rule == 0) return 1;
    float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
    int t = closest_sign_inside(partner, xf);
    return rule == 1 ? t != 1 : t != 0;
}

static int on_curve_with(const or_ctx *c, int64_t seg, const void *partner)
{
    for (int32_t q = 0; q < c->ncurves; q++)
        if (c->curve_with[q] == partner && seg >= c->curve_lo[q] && seg < c->curve_hi[q]) return 1;
    return 0;
}

static void apply_step_partners(or_ctx *c, const double *acc, double amax, const or_ctx *const *partner,
                                const int *surf_rule, const int *vol_rule, int npart)
{
    double dt = amax > 0.0 ? 0.25 * sqrt((double)c->h / amax) : 0.0;
    double *Xn = malloc(sizeof(double) * 3 * (c->n ? c->n : 1));
    int32_t *Cn = malloc(sizeof(int32_t) * (c->n ? c->n : 1));
    double maxdisp = 0.0;
    int64_t reverts = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(max : maxdisp) reduction(+ : reverts)
    for (int64_t i = 0; i < c->n; i++) {
        const double *x = c->X + 3 * i;
        int32_t cl = c->cls[i];
        Cn[i] = c->cons[i];
        memcpy(Xn + 3 * i, x, sizeof(double) * 3);
        if (!moves(c, i)) continue;
        double v[3], dr[3], y[3];
        for (int k = 0; k < 3; k++) {
            v[k] = acc[3 * i + k] * dt;   /* Eq. 22 with v_n = 0 */
            dr[k] = v[k] * dt;            /* Eq. 23 */
        }
        int32_t cs = c->cons[i];
        if (cl == OR_S && cs >= 0) {      /* Eqs. 24-25: drop the normal part */
            const double *n = c->Nrm + 3 * cs;
            double s = dot3(dr, n) / dot3(n, n);
            for (int k = 0; k < 3; k++) dr[k] -= s * n[k];
        } else if (cl == OR_F && cs >= 0) { /* along the segment only */
            double tau[3];
            sub3(c->V + 3 * c->seg_v[2 * cs + 1], c->V + 3 * c->seg_v[2 * cs], tau);
            double s = dot3(dr, tau) / dot3(tau, tau);
            for (int k = 0; k < 3; k++) dr[k] = s * tau[k];
        }
        for (int k = 0; k < 3; k++) y[k] = x[k] + dr[k];
        double xn[3];
        int32_t cn;
        int ok = project_point(c, cl, y, cs, xn, &cn);
        for (int q = 0; q < npart && ok; q++) {
            if (cl == OR_S || (cl == OR_F && !on_curve_with(c, cn, partner[q])))
                ok = partner_ok(partner[q], surf_rule[q], xn);
            else if (cl == OR_V)
                ok = partner_ok(partner[q], vol_rule[q], xn);
        }
        if (ok) {
            memcpy(Xn + 3 * i, xn, sizeof(xn));
            Cn[i] = cn;
        } else {
            reverts++;
        }
        double d[3];
        sub3(Xn + 3 * i, x, d);
        double m = sqrt(dot3(d, d));
        if (m > maxdisp) maxdisp = m;
    }
    memcpy(c->X, Xn, sizeof(double) * 3 * c->n);
    memcpy(c->cons, Cn, sizeof(int32_t) * c->n);
    free(Xn);
    free(Cn);
    c->last_maxdisp = maxdisp;
    c->last_reverts = reverts;
}

int oracle_relax(or_ctx *c, int32_t n_iter)
{
    double *acc = malloc(sizeof(double) * 3 * (c->n ? c->n : 1));
    for (int32_t it = 0; it < n_iter; it++) {
        double amax = compute_forces(c, c->X, acc, NULL);
        c->last_amax = amax;
        apply_step(c, acc, amax);
    }
    free(acc);
    return 0;
}

/* One iteration in two halves for a spatial decomposition (the domains
 * share one time step, so the largest force is reduced over them between
 * the halves): forces of every particle (ghosts act, do not move), returning
 * this domain's amax; then the step of Eqs. 22-25 with the given amax and
 * the projections. */
void oracle_set_ghost_count(or_ctx *c, int64_t n_ghost)
{
    c->n_ghost = n_ghost < 0 ? 0 : (n_ghost > c->n ? c->n : n_ghost);
}

double oracle_relax_forces(or_ctx *c)
{
    free(c->split_acc);
    c->split_acc = malloc(sizeof(double) * 3 * (c->n ? c->n : 1));
    double amax = compute_forces(c, c->X, c->split_acc, NULL);
    c->last_amax = amax;
    return amax;
}

int oracle_relax_step(or_ctx *c, double amax)
{
    if (!c->split_acc) return -1;
    apply_step(c, c->split_acc, amax);
    free(c->split_acc);
    c->split_acc = NULL;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* intersection curve of two bodies: feature lines of a Boolean pair         */
/* ------------------------------------------------------------------------ */
/* Where the surfaces of two bodies cross, the result of a Boolean operation
 * (Sec. 3.2.3) has a crease; the paper does not say whether it carries
 * feature particles.  Reading: it does, like a feature line (Sec. 3.2.2):
 * the curve is the union of the segments where a triangle of A crosses a
 * triangle of B, chained into polylines, and feature particles are placed
 * along them as along feature lines; they belong to A (the first operand).
 *
 * One triangle pair (a, b): the signed distances of a's vertices to b's
 * plane (unnormalised normal, vertex 0 of b as origin; zero counts as
 * positive) pick the two edges of a that cross b's plane, and the same for
 * b against a's plane.  The crossing point of an edge (u < v, global vertex
 * ids) with the other triangle's plane is u + (v - u) du / (du - dv); it is
 * named by the key (mesh of the edge, u, v, other triangle), so the two
 * segments that meet there compute it from the same numbers.  Along the
 * line of the two planes (direction na x nb) the pair's segment is the
 * overlap of a's two points and b's two points; it is empty unless the
 * overlap has positive length.  The ends of the overlap are the segment's
 * ends, with their keys. */
typedef struct {
    int32_t side;      /* 0: an edge of A (other triangle of B), 1: an edge of B */
    int32_t u, v;      /* edge, u < v */
    int64_t other;     /* the triangle it crosses */
} or_ckey;

typedef struct {
    int64_t a, b;      /* the triangle pair */
    or_ckey k[2];
    double p[2][3];
} or_cseg;

static int ckey_cmp(const or_ckey *x, const or_ckey *y)
{
    if (x->side != y->side) return x->side < y->side ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    if (x->other != y->other) return x->other < y->other ? -1 : 1;
    return 0;
}

/* crossing point of edge (u, v) of mesh (V, T) with the plane (n, o) */
static void edge_plane_point(const double *V, int32_t u, int32_t v, const double *n, const double *o, double *p)
{
    double wu[3], wv[3], e[3];
    sub3(V + 3 * u, o, wu);
    sub3(V + 3 * v, o, wv);
    double du = dot3(n, wu), dv = dot3(n, wv);
    sub3(V + 3 * v, V + 3 * u, e);
    double t = du / (du - dv);
    for (int k = 0; k < 3; k++) p[k] = V[3 * u + k] + e[k] * t;
}

/* the two edges of triangle t (mesh V, T) whose end points lie on opposite
 * sides of plane (n, o); returns 0 when all three lie on one side */
static int crossing_edges(const double *V, const int32_t *T, int64_t t, const double *n, const double *o,
                          int32_t eu[2], int32_t ev[2])
{
    int pos[3];
    for (int i = 0; i < 3; i++) {
        double w[3];
        sub3(V + 3 * T[3 * t + i], o, w);
        pos[i] = dot3(n, w) >= 0.0;
    }
    if (pos[0] == pos[1] && pos[1] == pos[2]) return 0;
    int m = 0;
    for (int i = 0; i < 3; i++) {
        int j = (i + 1) % 3;
        if (pos[i] != pos[j]) {
            int32_t x = T[3 * t + i], y = T[3 * t + j];
            eu[m] = x < y ? x : y;
            ev[m] = x < y ? y : x;
            m++;
        }
    }
    return m == 2;
}

static int tri_pair_segment(const or_ctx *A, int64_t a, const or_ctx *B, int64_t b, or_cseg *out)
{
    double na[3], nb[3], e1[3], e2[3];
    const double *a0 = A->V + 3 * A->T[3 * a], *b0 = B->V + 3 * B->T[3 * b];
    sub3(A->V + 3 * A->T[3 * a + 1], a0, e1);
    sub3(A->V + 3 * A->T[3 * a + 2], a0, e2);
    cross3(e1, e2, na);
    sub3(B->V + 3 * B->T[3 * b + 1], b0, e1);
    sub3(B->V + 3 * B->T[3 * b + 2], b0, e2);
    cross3(e1, e2, nb);
    int32_t au[2], av[2], bu[2], bv[2];
    if (!crossing_edges(A->V, A->T, a, nb, b0, au, av)) return 0;
    if (!crossing_edges(B->V, B->T, b, na, a0, bu, bv)) return 0;
    double dir[3], pts[4][3], t[4];
    cross3(na, nb, dir);
    or_ckey keys[4];
    for (int i = 0; i < 2; i++) {
        edge_plane_point(A->V, au[i], av[i], nb, b0, pts[i]);
        keys[i] = (or_ckey){0, au[i], av[i], b};
        edge_plane_point(B->V, bu[i], bv[i], na, a0, pts[2 + i]);
        keys[2 + i] = (or_ckey){1, bu[i], bv[i], a};
    }
    for (int i = 0; i < 4; i++) t[i] = dot3(dir, pts[i]);
    int alo = t[0] <= t[1] ? 0 : 1, ahi = 1 - alo, blo = t[2] <= t[3] ? 2 : 3, bhi = 5 - blo;
    int lo = t[alo] >= t[blo] ? alo : blo;   /* the later start */
    int hi = t[ahi] <= t[bhi] ? ahi : bhi;   /* the earlier end */
    if (!(t[lo] < t[hi])) return 0;
    out->a = a;
    out->b = b;
    out->k[0] = keys[lo];
    out->k[1] = keys[hi];
    memcpy(out->p[0], pts[lo], sizeof(double) * 3);
    memcpy(out->p[1], pts[hi], sizeof(double) * 3);
    return 1;
}

typedef struct {
    or_ckey k;
    int64_t seg;
    int end;
} or_cend;

static int cend_cmp(const void *x, const void *y)
{
    const or_cend *p = x, *q = y;
    int c = ckey_cmp(&p->k, &q->k);
    if (c) return c;
    if (p->seg != q->seg) return p->seg < q->seg ? -1 : 1;
    return p->end - q->end;
}

static void aabb_of(const or_ctx *c, int64_t t, double *lo, double *hi)
{
    for (int k = 0; k < 3; k++) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
    }
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) {
            double x = c->V[3 * c->T[3 * t + i] + k];
            if (x < lo[k]) lo[k] = x;
            if (x > hi[k]) hi[k] = x;
        }
}

/* Chaining, in a fixed order: segments sorted by their triangle pair (a, b);
 * ends matched by key (a key met by other than two ends stops a chain), then
 * the ends left free matched by position (see below).
 * Open chains first: from each segment with a free end, in that order, a
 * walk from the free end; then loops: from the first unvisited segment, a
 * walk that leaves it by its end of larger key.  A walk appends the point of
 * every key it passes (a loop its first point once).  The polylines become
 * feature lines of A with their points appended to A's vertex arrays
 * (rounded to FP32), and feature particles are placed along them as along
 * A's own lines (Sec. 3.2.2: n = ceil(L / dx) pieces, open lines with their
 * end points as singular points).  Returns the particles added. */
int64_t oracle_boolean_curve(or_ctx *A, const or_ctx *B)
{
    const int64_t seg_before = A->nseg;
    /* the triangle pairs whose boxes overlap (brute force) */
    double *alo = malloc(sizeof(double) * 3 * A->nt), *ahi = malloc(sizeof(double) * 3 * A->nt);
    for (int64_t a = 0; a < A->nt; a++) aabb_of(A, a, alo + 3 * a, ahi + 3 * a);
    int64_t cap = 64, ns = 0;
    or_cseg *S = malloc(sizeof(or_cseg) * cap);
    for (int64_t b = 0; b < B->nt; b++) {
        double lo[3], hi[3];
        aabb_of(B, b, lo, hi);
        for (int64_t a = 0; a < A->nt; a++) {
            int apart = 0;
            for (int k = 0; k < 3; k++)
                if (alo[3 * a + k] > hi[k] || ahi[3 * a + k] < lo[k]) apart = 1;
            if (apart) continue;
            or_cseg g;
            if (!tri_pair_segment(A, a, B, b, &g)) continue;
            if (ns == cap) {
                cap *= 2;
                S = realloc(S, sizeof(or_cseg) * cap);
            }
            S[ns++] = g;
        }
    }
    free(alo);
    free(ahi);
    /* sort by (a, b): the loop above runs b outer, a inner */
    for (int64_t i = 1; i < ns; i++) {
        or_cseg x = S[i];
        int64_t j = i - 1;
        while (j >= 0 && (S[j].a > x.a || (S[j].a == x.a && S[j].b > x.b))) {
            S[j + 1] = S[j];
            j--;
        }
        S[j + 1] = x;
    }
    /* ends sorted by key: partner[2 s + e] = the other end with the same key */
    or_cend *E = malloc(sizeof(or_cend) * (2 * ns + 1));
    for (int64_t i = 0; i < ns; i++)
        for (int e = 0; e < 2; e++) E[2 * i + e] = (or_cend){S[i].k[e], i, e};
    qsort(E, (size_t)(2 * ns), sizeof(or_cend), cend_cmp);
    int64_t *partner = malloc(sizeof(int64_t) * (2 * ns + 1));
    for (int64_t i = 0; i < 2 * ns; i++) partner[i] = -1;
    for (int64_t i = 0; i < 2 * ns;) {
        int64_t j = i;
        while (j < 2 * ns && ckey_cmp(&E[j].k, &E[i].k) == 0) j++;
        if (j - i == 2) {
            partner[2 * E[i].seg + E[i].end] = 2 * E[i + 1].seg + E[i + 1].end;
            partner[2 * E[i + 1].seg + E[i + 1].end] = 2 * E[i].seg + E[i].end;
        }
        i = j;
    }
    free(E);
    /* a point where the curve meets an edge of each mesh at once has two keys
     * (degenerate, e.g. mirror-symmetric meshes): ends still free are joined
     * to the first free end (in segment order) within 2^-30 of the largest
     * extent of A */
    {
        double ext = 0.0;
        for (int k = 0; k < 3; k++) {
            double lo = INFINITY, hi = -INFINITY;
            for (int64_t v = 0; v < A->nv; v++) {
                if (A->V[3 * v + k] < lo) lo = A->V[3 * v + k];
                if (A->V[3 * v + k] > hi) hi = A->V[3 * v + k];
            }
            if (hi - lo > ext) ext = hi - lo;
        }
        const double tol = ldexp(ext, -30);
        for (int64_t i = 0; i < 2 * ns; i++) {
            if (partner[i] >= 0) continue;
            for (int64_t j = i + 1; j < 2 * ns; j++) {
                if (partner[j] >= 0 || j / 2 == i / 2) continue;
                double w[3];
                sub3(S[i / 2].p[i % 2], S[j / 2].p[j % 2], w);
                if (sqrt(dot3(w, w)) <= tol) {
                    partner[i] = j;
                    partner[j] = i;
                    break;
                }
            }
        }
    }
    /* walks */
    char *vis = calloc((size_t)(ns ? ns : 1), 1);
    int64_t pcap = 64, np = 0;
    double *P = malloc(sizeof(double) * 3 * pcap);
    int64_t lcap = 8, nl = 0, *lstart = malloc(sizeof(int64_t) * lcap), *lcount = malloc(sizeof(int64_t) * lcap);
    int32_t *lclosed = malloc(sizeof(int32_t) * lcap);
#define PUSH_PT(q)                                              \
    do {                                                        \
        if (np == pcap) {                                       \
            pcap *= 2;                                          \
            P = realloc(P, sizeof(double) * 3 * pcap);          \
        }                                                       \
        memcpy(P + 3 * np, (q), sizeof(double) * 3);           \
        np++;                                                   \
    } while (0)
    for (int pass = 0; pass < 2; pass++)
        for (int64_t s0 = 0; s0 < ns; s0++) {
            if (vis[s0]) continue;
            int e_in;
            if (pass == 0) {
                if (partner[2 * s0] >= 0 && partner[2 * s0 + 1] >= 0) continue;
                e_in = partner[2 * s0] < 0 ? 0 : 1;           /* the free end */
            } else {
                e_in = ckey_cmp(&S[s0].k[0], &S[s0].k[1]) < 0 ? 0 : 1;   /* leave by the larger key */
            }
            if (nl == lcap) {
                lcap *= 2;
                lstart = realloc(lstart, sizeof(int64_t) * lcap);
                lcount = realloc(lcount, sizeof(int64_t) * lcap);
                lclosed = realloc(lclosed, sizeof(int32_t) * lcap);
            }
            int64_t first = np, seg = s0;
            int closed = 0;
            PUSH_PT(S[s0].p[e_in]);
            for (;;) {
                vis[seg] = 1;
                int e_out = 1 - e_in;
                int64_t nx = partner[2 * seg + e_out];
                if (nx >= 0 && nx / 2 == s0) {
                    closed = 1;
                    break;
                }
                PUSH_PT(S[seg].p[e_out]);
                if (nx < 0 || vis[nx / 2]) break;
                seg = nx / 2;
                e_in = (int)(nx % 2);
            }
            lstart[nl] = first;
            lcount[nl] = np - first;
            lclosed[nl] = closed;
            nl++;
        }
#undef PUSH_PT
    free(vis);
    free(partner);
    free(S);
    /* the points join A's vertex arrays, rounded to FP32; each polyline a line */
    int64_t v0 = A->nv_all;
    A->nv_all += np;
    A->V = realloc(A->V, sizeof(double) * 3 * (A->nv_all ? A->nv_all : 1));
    A->Vf = realloc(A->Vf, sizeof(float) * 3 * (A->nv_all ? A->nv_all : 1));
    for (int64_t i = 0; i < np; i++)
        for (int k = 0; k < 3; k++) {
            A->Vf[3 * (v0 + i) + k] = (float)P[3 * i + k];
            A->V[3 * (v0 + i) + k] = (double)A->Vf[3 * (v0 + i) + k];
        }
    free(P);
    int64_t l_first = A->nlines, nseg_new = 0;
    for (int64_t l = 0; l < nl; l++) nseg_new += lclosed[l] ? lcount[l] : lcount[l] - 1;
    A->seg_v = realloc(A->seg_v, sizeof(int32_t) * 2 * (A->nseg + nseg_new + 1));
    A->seg_line = realloc(A->seg_line, sizeof(int32_t) * (A->nseg + nseg_new + 1));
    A->line_first = realloc(A->line_first, sizeof(int64_t) * (A->nlines + nl + 1));
    A->line_nseg = realloc(A->line_nseg, sizeof(int64_t) * (A->nlines + nl + 1));
    A->line_closed = realloc(A->line_closed, sizeof(int32_t) * (A->nlines + nl + 1));
    for (int64_t l = 0; l < nl; l++) {
        int64_t m = lcount[l], nseg_l = lclosed[l] ? m : m - 1, first = A->nseg;
        for (int64_t q = 0; q < nseg_l; q++) {
            A->seg_v[2 * A->nseg] = (int32_t)(v0 + lstart[l] + q);
            A->seg_v[2 * A->nseg + 1] = (int32_t)(v0 + lstart[l] + (q + 1) % m);
            A->seg_line[A->nseg] = (int32_t)A->nlines;
            A->nseg++;
        }
        A->line_first[A->nlines] = first;
        A->line_nseg[A->nlines] = nseg_l;
        A->line_closed[A->nlines] = lclosed[l];
        A->nlines++;
    }
    free(lstart);
    free(lcount);
    free(lclosed);
    if (A->ncurves < OR_MAX_PARTNERS) {
        A->curve_lo[A->ncurves] = seg_before;
        A->curve_hi[A->ncurves] = A->nseg;
        A->curve_with[A->ncurves] = B;
        A->ncurves++;
    }
    /* feature particles along the new lines, appended to A's particles */
    int64_t nf = feature_particles_of_lines(A, (double)A->dx, l_first, A->nlines, NULL, NULL, NULL, 0);
    double *fx = malloc(sizeof(double) * 3 * (nf ? nf : 1));
    int32_t *fc = malloc(sizeof(int32_t) * (nf ? nf : 1)), *fs = malloc(sizeof(int32_t) * (nf ? nf : 1));
    feature_particles_of_lines(A, (double)A->dx, l_first, A->nlines, fx, fc, fs, nf);
    A->X = realloc(A->X, sizeof(double) * 3 * (A->n + nf + 1));
    A->cls = realloc(A->cls, sizeof(int32_t) * (A->n + nf + 1));
    A->cons = realloc(A->cons, sizeof(int32_t) * (A->n + nf + 1));
    for (int64_t i = 0; i < nf; i++) {
        for (int k = 0; k < 3; k++) A->X[3 * (A->n + i) + k] = (double)(float)fx[3 * i + k];
        A->cls[A->n + i] = fc[i];
        A->cons[A->n + i] = fs[i];
    }
    A->n += nf;
    free(fx);
    free(fc);
    free(fs);
    return nf;
}

/* vertex coordinates of every intersection-curve point of A (the points
 * after its mesh vertices), FP32 */
int64_t oracle_curve_points(const or_ctx *c, float *out, int64_t cap)
{
    int64_t m = c->nv_all - c->nv;
    if (out) memcpy(out, c->Vf + 3 * c->nv, sizeof(float) * 3 * (size_t)(m < cap ? m : cap));
    return m;
}

/* ------------------------------------------------------------------------ */
/* Boolean operations on two bodies (Sec. 3.2.3, Fig. 10)                    */
/* ------------------------------------------------------------------------ */
/* The paper combines two bodies through their cell sets (interval union,
 * difference and intersection of C_compact).  Reading, on particles, with
 * "inside" = ray parity of Fig. 6 against the other mesh and "volume" =
 * volume or innermost class:
 *   op 0, union A + B:        A keeps what is outside B; B keeps what is
 *                             outside A and its volume particles (the
 *                             overlap keeps one copy of them).
 *   op 1, difference A - B:   A keeps what is outside B; B keeps its
 *                             surface, feature and singular particles
 *                             inside A (the wall of the cavity).
 *   op 2, intersection A * B: A keeps what is inside B; B keeps its
 *                             surface, feature and singular particles
 *                             inside A.
 * first = 1 for A, 0 for B.  keep[i] = 1 for the particles of self that
 * stay. */
void oracle_boolean_keep(const or_ctx *self, const or_ctx *other, int op, int first, int32_t *keep)
{
    /* the ray starts at the particle displaced by (1.234567e-6, 2.345678e-6) dx
     * in x, y (as in the generation), so that it meets no edge or vertex of
     * the other mesh exactly (a ray through an edge would cross both faces) */
    int32_t *inside = malloc(sizeof(int32_t) * (self->n ? self->n : 1));
    double *q = malloc(sizeof(double) * 3 * (self->n ? self->n : 1));
    for (int64_t i = 0; i < self->n; i++) {
        q[3 * i] = self->X[3 * i] + 1.234567e-6 * (double)other->dx;
        q[3 * i + 1] = self->X[3 * i + 1] + 2.345678e-6 * (double)other->dx;
        q[3 * i + 2] = self->X[3 * i + 2];
    }
    oracle_ray_parity(other, q, self->n, inside);
    free(q);
    for (int64_t i = 0; i < self->n; i++) {
        int vol = self->cls[i] == OR_V || self->cls[i] == OR_I;
        int in = inside[i];
        if (op == 0) keep[i] = first ? !in : (!in || vol);
        else if (op == 1) keep[i] = first ? !in : (in && !vol);
        else keep[i] = first ? in : (in && !vol);
    }
    free(inside);
}

/* partner rules of each operation for the first (A) and second (B) body:
 * surface / feature particles, then volume particles (1 outside, 2 inside) */
static void boolean_rules(int op, int first, int *surf, int *vol)
{
    if (op == 0) {
        *surf = 1;
        *vol = 0;
    } else if (op == 1) {
        *surf = first ? 1 : 2;
        *vol = first ? 1 : 0;
    } else {
        *surf = 2;
        *vol = first ? 2 : 0;
    }
}

/* Relaxation of the result of Boolean operations as one assembly: bodies
 * b[0..nb) (same dx, h and options) and operations pairs[3 q + (0, 1, 2)] =
 * (first operand, second operand, op).  The forces of Eq. 15 over the
 * particles of every body (one neighbour grid over all meshes' boxes), one
 * amax and so one dt, then each particle's own projection, subject to the
 * rules of every operation its body takes part in (apply_step_partners): a
 * body in several operations keeps to all of their sides. */
int oracle_boolean_relax_many(or_ctx *const *b, int32_t nb, const int32_t *pairs, int32_t np, int32_t n_iter)
{
    if (nb < 1) return -1;
    for (int32_t q = 0; q < np; q++) {
        const int32_t i = pairs[3 * q], j = pairs[3 * q + 1], op = pairs[3 * q + 2];
        if (i < 0 || i >= nb || j < 0 || j >= nb || i == j || op < 0 || op > 2) return -1;
    }
    int64_t n = 0;
    for (int32_t i = 0; i < nb; i++) {
        if (b[i]->h != b[0]->h || b[i]->dx != b[0]->dx || b[i]->fixed_features != b[0]->fixed_features ||
            b[i]->mobile_mask != b[0]->mobile_mask)
            return -1;
        n += b[i]->n;
    }
    /* each body's partners and their rules */
    const or_ctx **part = malloc(sizeof(*part) * OR_MAX_PARTNERS * nb);
    int *srule = malloc(sizeof(int) * OR_MAX_PARTNERS * nb), *vrule = malloc(sizeof(int) * OR_MAX_PARTNERS * nb);
    int *npart = calloc((size_t)nb, sizeof(int));
    for (int32_t q = 0; q < np; q++) {
        const int32_t ij[2] = {pairs[3 * q], pairs[3 * q + 1]};
        for (int e = 0; e < 2; e++) {
            const int32_t me = ij[e], other = ij[1 - e];
            if (npart[me] == OR_MAX_PARTNERS) {
                free(part);
                free(srule);
                free(vrule);
                free(npart);
                return -1;
            }
            const int k = OR_MAX_PARTNERS * me + npart[me]++;
            part[k] = b[other];
            boolean_rules(pairs[3 * q + 2], e == 0, &srule[k], &vrule[k]);
        }
    }
    double *X = malloc(sizeof(double) * 3 * (n ? n : 1));
    double *acc = malloc(sizeof(double) * 3 * (n ? n : 1));
    int32_t *cls = malloc(sizeof(int32_t) * (n ? n : 1));
    or_ctx g = *b[0];   /* b[0]'s parameters, the assembly's neighbour grid and particles */
    float bbmin[3] = {INFINITY, INFINITY, INFINITY}, bbmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t q = 0; q < nb; q++)
        for (int64_t i = 0; i < b[q]->nv; i++)
            for (int k = 0; k < 3; k++) {
                bbmin[k] = fminf(bbmin[k], b[q]->Vf[3 * i + k]);
                bbmax[k] = fmaxf(bbmax[k], b[q]->Vf[3 * i + k]);
            }
    grid_setup(bbmin, bbmax, b[0]->ng_cell, 1.0, 1, g.ng_o, &g.ng_inv, g.ng_n);
    g.row_rank = g.cell_order ? morton_rank_table(g.ng_n) : NULL;   /* the assembly grid's own table */
    if (g.cell_order && !g.row_rank) {
        free(X);
        free(acc);
        free(cls);
        free(part);
        free(srule);
        free(vrule);
        free(npart);
        return -1;
    }
    for (int32_t it = 0; it < n_iter; it++) {
        int64_t off = 0;
        for (int32_t q = 0; q < nb; q++) {
            memcpy(X + 3 * off, b[q]->X, sizeof(double) * 3 * b[q]->n);
            memcpy(cls + off, b[q]->cls, sizeof(int32_t) * b[q]->n);
            off += b[q]->n;
        }
        g.X = X;
        g.cls = cls;
        g.n = n;
        double amax = compute_forces(&g, X, acc, NULL);
        off = 0;
        for (int32_t q = 0; q < nb; q++) {
            b[q]->last_amax = amax;
            const int k = OR_MAX_PARTNERS * q;
            apply_step_partners(b[q], acc + 3 * off, amax, part + k, srule + k, vrule + k, npart[q]);
            off += b[q]->n;
        }
    }
    free(g.row_rank);
    free(X);
    free(acc);
    free(cls);
    free(part);
    free(srule);
    free(vrule);
    free(npart);
    return 0;
}

/* The same for the two bodies of one operation. */
int oracle_boolean_relax(or_ctx *a, or_ctx *b, int op, int32_t n_iter)
{
    or_ctx *m[2] = {a, b};
    const int32_t pair[3] = {0, 1, op};
    return oracle_boolean_relax_many(m, 2, pair, 1, n_iter);
}

void oracle_last_iteration(const or_ctx *c, double *amax, double *maxdisp, int64_t *reverts)
{
    if (amax) *amax = c->last_amax;
    if (maxdisp) *maxdisp = c->last_maxdisp;
    if (reverts) *reverts = c->last_reverts;
}

/* ------------------------------------------------------------------------ */
/* uniformity energy and its gradient                                        */
/* ------------------------------------------------------------------------ */
/* W0 per class: planar lattice for S, cubic for V, linear for F (3-D kernel
 * throughout). */
static double class_w0(const or_ctx *c, int32_t cl)
{
    int dim = cl == OR_S ? 2 : (cl == OR_F ? 1 : 3);
    return oracle_lattice_sum((double)c->dx, (double)c->h, dim);
}

void oracle_w0(const or_ctx *c, double *w0)
{
    for (int cl = 0; cl < 5; cl++) w0[cl] = class_w0(c, cl);
}

typedef struct {
    const or_ctx *c;
    const double *X;
    double rho;
} dens_acc;

static void dens_pair(void *user, int64_t i, int64_t j)
{
    dens_acc *da = user;
    double d[3];
    sub3(da->X + 3 * i, da->X + 3 * j, d);
    da->rho += oracle_W(sqrt(dot3(d, d)), (double)da->c->h);
}

/* kernel sum rho_i = W(0) + sum over masked neighbours of W(r_ij) */
static void densities(const or_ctx *c, const double *X, const or_kv *L, double *rho)
{
    double w00 = oracle_W(0.0, (double)c->h);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < c->n; i++) {
        dens_acc da = {c, X, w00};
        for_neighbours(c, X, c->cls, L, c->n, i, 1, dens_pair, &da);
        rho[i] = da.rho;
    }
}

void oracle_density(const or_ctx *c, double *rho)
{
    or_kv *L = build_cells(c, c->X, c->n);
    densities(c, c->X, L, rho);
    free(L);
}

typedef struct {
    const or_ctx *c;
    const double *X;
    const double *rho;
    const double *w0;
    double g[3];
} grad_acc;

/* pair (k, j) visited without a mask: the term of rho_k (if j acts on k and
 * k is counted) and the term of rho_j (if k acts on j and j is counted) */
static void grad_pair(void *user, int64_t k, int64_t j)
{
    grad_acc *ga = user;
    const or_ctx *c = ga->c;
    double coef = 0.0;
    int32_t ck = c->cls[k], cj = c->cls[j];
    if (is_mobile(c, ck) && acts_on(ck, cj)) coef += 2.0 * (ga->rho[k] - ga->w0[ck]);
    if (is_mobile(c, cj) && acts_on(cj, ck)) coef += 2.0 * (ga->rho[j] - ga->w0[cj]);
    if (coef == 0.0) return;
    double d[3];
    sub3(ga->X + 3 * k, ga->X + 3 * j, d);
    double r = sqrt(dot3(d, d));
    if (r <= 0.0) return;
    double w = oracle_dW(r, (double)c->h);
    for (int q = 0; q < 3; q++) ga->g[q] += coef * w * d[q] / r;
}

/* E = sum over mobile i of (rho_i - W0_{class i})^2 at positions X, and
 * dE/dX [n*3] (nullable). */
static double energy_at(const or_ctx *c, const double *X, double *gX)
{
    or_kv *L = build_cells(c, X, c->n);
    double *rho = malloc(sizeof(double) * (c->n ? c->n : 1));
    densities(c, X, L, rho);
    double w0[5];
    oracle_w0(c, w0);
    double E = 0.0;
    for (int64_t i = 0; i < c->n; i++)
        if (is_mobile(c, c->cls[i])) {
            double e = rho[i] - w0[c->cls[i]];
            E += e * e;
        }
    if (gX) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t k = 0; k < c->n; k++) {
            grad_acc ga = {c, X, rho, w0, {0, 0, 0}};
            for_neighbours(c, X, c->cls, L, c->n, k, 0, grad_pair, &ga);
            for (int q = 0; q < 3; q++) gX[3 * k + q] = ga.g[q];
        }
    }
    free(rho);
    free(L);
    return E;
}

double oracle_energy(const or_ctx *c, double *grad)
{
    return energy_at(c, c->X, grad);
}

/* Energy through the surface projection.  Surface particles with a
 * triangle are x = y - ((y - v_a) . n) n with n the unit normal of the
 * frozen triangle built from verts (the mesh when verts is NULL); every
 * other particle has x = y.  Returns E and the gradients w.r.t. y [n*3] and
 * w.r.t. the vertices [nv*3] (both nullable). */
double oracle_energy_projected(const or_ctx *c, const double *y, const double *verts, double *gy, double *gV)
{
    const double *Vv = verts ? verts : c->V;
    int64_t n = c->n;
    double *X = malloc(sizeof(double) * 3 * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        const double *yi = y + 3 * i;
        int32_t t = c->cons[i];
        if (c->cls[i] == OR_S && t >= 0) {
            const double *a = Vv + 3 * c->T[3 * t], *b = Vv + 3 * c->T[3 * t + 1], *cc = Vv + 3 * c->T[3 * t + 2];
            double e1[3], e2[3], m[3], ya[3];
            sub3(b, a, e1);
            sub3(cc, a, e2);
            cross3(e1, e2, m);
            double ml = sqrt(dot3(m, m)), nh[3] = {m[0] / ml, m[1] / ml, m[2] / ml};
            sub3(yi, a, ya);
            double s = dot3(ya, nh);
            for (int k = 0; k < 3; k++) X[3 * i + k] = yi[k] - s * nh[k];
        } else {
            memcpy(X + 3 * i, yi, sizeof(double) * 3);
        }
    }
    double *gX = (gy || gV) ? malloc(sizeof(double) * 3 * (n ? n : 1)) : NULL;
    double E = energy_at(c, X, gX);
    if (gV) memset(gV, 0, sizeof(double) * 3 * c->nv);
    if (gX) {
        for (int64_t i = 0; i < n; i++) {
            const double *g = gX + 3 * i, *yi = y + 3 * i;
            int32_t t = c->cons[i];
            if (!(c->cls[i] == OR_S && t >= 0)) {
                if (gy) memcpy(gy + 3 * i, g, sizeof(double) * 3);
                continue;
            }
            int32_t ia = c->T[3 * t], ib = c->T[3 * t + 1], ic = c->T[3 * t + 2];
            const double *a = Vv + 3 * ia, *b = Vv + 3 * ib, *cc = Vv + 3 * ic;
            double e1[3], e2[3], m[3], ya[3];
            sub3(b, a, e1);
            sub3(cc, a, e2);
            cross3(e1, e2, m);
            double ml = sqrt(dot3(m, m)), nh[3] = {m[0] / ml, m[1] / ml, m[2] / ml};
            sub3(yi, a, ya);
            double s = dot3(ya, nh), gn = dot3(g, nh);
            /* dx = dy - ds n - s dn with ds = (dy - da) . n + (y - a) . dn */
            if (gy)
                for (int k = 0; k < 3; k++) gy[3 * i + k] = g[k] - gn * nh[k];
            if (gV) {
                /* u . dn with u = -(gn (y - a) + s g); dn = (I - n n^T) dm / |m| */
                double u[3], ut[3];
                for (int k = 0; k < 3; k++) u[k] = -(gn * ya[k] + s * g[k]);
                double un = dot3(u, nh);
                for (int k = 0; k < 3; k++) ut[k] = (u[k] - un * nh[k]) / ml;
                double gb[3], gc[3];
                cross3(e2, ut, gb); /* d/d e1 of ut . (e1 x e2) */
                cross3(ut, e1, gc); /* d/d e2 */
                for (int k = 0; k < 3; k++) {
                    gV[3 * ib + k] += gb[k];
                    gV[3 * ic + k] += gc[k];
                    gV[3 * ia + k] += -gb[k] - gc[k] + gn * nh[k];
                }
            }
        }
        free(gX);
    }
    free(X);
    return E;
}

/* Energy-descent relaxation: the same limited step and projection as the
 * force form, with a = -dE/dx in place of the pressure force. */
int oracle_relax_energy(or_ctx *c, int32_t n_iter)
{
    double *g = malloc(sizeof(double) * 3 * (c->n ? c->n : 1));
    for (int32_t it = 0; it < n_iter; it++) {
        energy_at(c, c->X, g);
        double amax = 0.0;
        for (int64_t i = 0; i < c->n; i++) {
            for (int k = 0; k < 3; k++) g[3 * i + k] = is_mobile(c, c->cls[i]) ? -g[3 * i + k] : 0.0;
            double m = sqrt(dot3(g + 3 * i, g + 3 * i));
            if (m > amax) amax = m;
        }
        c->last_amax = amax;
        apply_step(c, g, amax);
    }
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* uniformity statistics                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *X;
    double rmin;
} min_acc;

static void min_pair(void *user, int64_t i, int64_t j)
{
    min_acc *ma = user;
    double d[3];
    sub3(ma->X + 3 * i, ma->X + 3 * j, d);
    double r = sqrt(dot3(d, d));
    if (r < ma->rmin) ma->rmin = r;
}

/* out[0..2]  mean kernel sum of S, V, F particles
 * out[3..5]  standard deviation of the kernel sum of S, V, F
 * out[6]     minimum masked pair distance over mobile particles / dx
 * out[7]     largest displacement of the last iteration / dx
 * out[8..10] number of S, V, F particles */
void oracle_stats(const or_ctx *c, double *out)
{
    double *rho = malloc(sizeof(double) * (c->n ? c->n : 1));
    or_kv *L = build_cells(c, c->X, c->n);
    densities(c, c->X, L, rho);
    double s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0}, cnt[3] = {0, 0, 0}, rmin = INFINITY;
    const int64_t n_own = c->n - c->n_ghost;   /* ghosts are another domain's */
    for (int64_t i = 0; i < n_own; i++) {
        int32_t cl = c->cls[i];
        if (cl > OR_F) continue;
        s1[cl] += rho[i];
        cnt[cl] += 1.0;
    }
    for (int k = 0; k < 3; k++) s1[k] = cnt[k] > 0 ? s1[k] / cnt[k] : 0.0;
    for (int64_t i = 0; i < n_own; i++) {
        int32_t cl = c->cls[i];
        if (cl > OR_F) continue;
        s2[cl] += (rho[i] - s1[cl]) * (rho[i] - s1[cl]);
    }
#pragma omp parallel for schedule(dynamic, 256) reduction(min : rmin)
    for (int64_t i = 0; i < c->n; i++) {
        if (!moves(c, i)) continue;
        min_acc ma = {c->X, INFINITY};
        for_neighbours(c, c->X, c->cls, L, c->n, i, 1, min_pair, &ma);
        if (ma.rmin < rmin) rmin = ma.rmin;
    }
    for (int k = 0; k < 3; k++) {
        out[k] = s1[k];
        out[3 + k] = cnt[k] > 0 ? sqrt(s2[k] / cnt[k]) : 0.0;
        out[8 + k] = cnt[k];
    }
    out[6] = rmin / (double)c->dx;
    out[7] = c->last_maxdisp / (double)c->dx;
    free(L);
    free(rho);
}

/* ------------------------------------------------------------------------ */
/* particle generation (Sec. 3.2)                                            */
/* ------------------------------------------------------------------------ */
/* centre of triangle cell (i, j, k), FP64 rounded to FP32 */
static void cell_centre(const or_ctx *c, int32_t i, int32_t j, int32_t k, float *out)
{
    int32_t idx[3] = {i, j, k};
    for (int a = 0; a < 3; a++) out[a] = (float)((double)c->tg_o[a] + ((double)idx[a] + 0.5) * (double)c->dx);
}

/* Ray parity of Fig. 6 for the cell centres of one grid column (i, j): the
 * +z ray starts at each centre displaced by (1.234567e-6, 2.345678e-6) dx in
 * x and y so that it never meets a mesh edge or vertex exactly.  Every
 * triangle the vertical line crosses is binned into some cell of the
 * column, so the column's triangles (each counted once) give all crossing
 * heights; a centre is inside when an odd number of them lie above it. */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

static void column_inside(const or_ctx *c, int32_t i, int32_t j, unsigned char *inside_col)
{
    const int32_t *n = c->tg_n;
    float p0[3];
    cell_centre(c, i, j, 0, p0);
    double qx = (double)p0[0] + 1.234567e-6 * (double)c->dx, qy = (double)p0[1] + 2.345678e-6 * (double)c->dx;
    /* triangles binned into the column's cells, each once */
    int64_t cap = 64, m = 0;
    int32_t *tri = malloc(sizeof(int32_t) * cap);
    for (int32_t k = 0; k < n[2]; k++) {
        int64_t key = (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
        for (int64_t p = lower_bound_i64(c->pair_key, c->npairs, key); p < c->npairs && c->pair_key[p] == key; p++) {
            if (m == cap) {
                cap *= 2;
                tri = realloc(tri, sizeof(int32_t) * cap);
            }
            tri[m++] = c->pair_tri[p];
        }
    }
    qsort(tri, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t q = 0; q < m; q++)
        if (q == 0 || tri[q] != tri[q - 1]) tri[u++] = tri[q];
    double *zc = malloc(sizeof(double) * (u ? u : 1));
    int64_t nz = 0;
    for (int64_t q = 0; q < u; q++) {
        int64_t t = tri[q];
        const double *a = c->V + 3 * c->T[3 * t], *b = c->V + 3 * c->T[3 * t + 1], *cc = c->V + 3 * c->T[3 * t + 2];
        double d = (b[0] - a[0]) * (cc[1] - a[1]) - (cc[0] - a[0]) * (b[1] - a[1]);
        if (d == 0.0) continue;
        double l1 = ((b[0] - qx) * (cc[1] - qy) - (cc[0] - qx) * (b[1] - qy)) / d;
        double l2 = ((cc[0] - qx) * (a[1] - qy) - (a[0] - qx) * (cc[1] - qy)) / d;
        double l3 = 1.0 - l1 - l2;
        if (l1 < 0 || l2 < 0 || l3 < 0) continue;
        zc[nz++] = l1 * a[2] + l2 * b[2] + l3 * cc[2];
    }
    for (int32_t k = 0; k < n[2]; k++) {
        float p[3];
        cell_centre(c, i, j, k, p);
        int64_t cross = 0;
        for (int64_t q = 0; q < nz; q++)
            if (zc[q] > (double)p[2]) cross++;
        inside_col[k] = (unsigned char)(cross & 1);
    }
    free(zc);
    free(tri);
}

/* Initial particles (Sec. 3.2, Fig. 9):
 *   features: the feature-line particles (F, constraint = the segment it
 *             lies on; P at singular points, constraint -1);
 *   surface:  every triangle cell holding triangles contributes its centre
 *             mapped to the nearest triangle of that cell whose foot is
 *             inside (smallest |plane distance|, ties to the lower index);
 *             a centre with no such triangle is discarded (S, constraint =
 *             the triangle);
 *   volume:   every cell without triangles whose centre is inside by ray
 *             parity (Fig. 6) contributes its centre: class V when band_cells
 *             <= 0 or when a cell with triangles lies within band_cells cells
 *             (Chebyshev), else I -- or nothing when inner_cells > 0 and no
 *             cell with triangles lies within band_cells + inner_cells.
 * Order: features, then surface cells by key, then volume cells by key.
 * Writes at most cap particles; returns the total count. */
int64_t oracle_map_particles(const or_ctx *c, int surface, int volume, int features, int band_cells, int inner_cells,
                             double *xyz, int32_t *cls, int32_t *cons, int64_t cap)
{
    int64_t cnt = 0;
    if (features) {
        int64_t nf = feature_particles_on_segments(c, (double)c->dx, NULL, NULL, NULL, 0);
        double *fx = malloc(sizeof(double) * 3 * (nf ? nf : 1));
        int32_t *fc = malloc(sizeof(int32_t) * (nf ? nf : 1));
        int32_t *fs = malloc(sizeof(int32_t) * (nf ? nf : 1));
        feature_particles_on_segments(c, (double)c->dx, fx, fc, fs, nf);
        for (int64_t i = 0; i < nf; i++, cnt++)
            if (cnt < cap) {
                memcpy(xyz + 3 * cnt, fx + 3 * i, sizeof(double) * 3);
                cls[cnt] = fc[i];
                cons[cnt] = fs[i];   /* F: the segment it lies on; P: -1 */
            }
        free(fx);
        free(fc);
        free(fs);
    }
    const int32_t *n = c->tg_n;
    if (surface) {
        for (int64_t q = 0; q < c->npairs;) {
            int64_t key = c->pair_key[q], e = q;
            while (e < c->npairs && c->pair_key[e] == key) e++;
            int32_t i = (int32_t)(key % n[0]), j = (int32_t)((key / n[0]) % n[1]), k = (int32_t)(key / ((int64_t)n[0] * n[1]));
            float ctr[3];
            cell_centre(c, i, j, k, ctr);
            float best = INFINITY;
            int64_t bt = -1;
            for (int64_t p = q; p < e; p++) {
                float d;
                int64_t t = c->pair_tri[p];
                if (!surface_candidate(c, t, ctr, &d)) continue;
                if (d < best || (d == best && t < bt)) {
                    best = d;
                    bt = t;
                }
            }
            if (bt >= 0) {
                if (cnt < cap) {
                    double y[3] = {ctr[0], ctr[1], ctr[2]};
                    plane_foot(c, bt, y, xyz + 3 * cnt);
                    cls[cnt] = OR_S;
                    cons[cnt] = (int32_t)bt;
                }
                cnt++;
            }
            q = e;
        }
    }
    if (volume) {
        const int64_t cells = (int64_t)n[0] * n[1] * n[2];
        unsigned char *occ = calloc((size_t)cells, 1), *ins = calloc((size_t)cells, 1);
        for (int64_t p = 0; p < c->npairs; p++) occ[c->pair_key[p]] = 1;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t col = 0; col < (int64_t)n[0] * n[1]; col++) {
            int32_t i = (int32_t)(col % n[0]), j = (int32_t)(col / n[0]);
            unsigned char *buf = malloc((size_t)n[2]);
            column_inside(c, i, j, buf);
            for (int32_t k = 0; k < n[2]; k++) ins[(int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k)] = buf[k];
            free(buf);
        }
        for (int32_t k = 0; k < n[2]; k++)
            for (int32_t j = 0; j < n[1]; j++)
                for (int32_t i = 0; i < n[0]; i++) {
                    int64_t key = (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
                    if (occ[key] || !ins[key]) continue;
                    int32_t cl = OR_V;
                    if (band_cells > 0) {
                        /* Chebyshev distance (in cells) to the nearest cell with triangles */
                        int32_t reach = inner_cells > 0 ? band_cells + inner_cells : band_cells, dmin = reach + 1;
                        for (int32_t dz = -reach; dz <= reach; dz++)
                            for (int32_t dy = -reach; dy <= reach; dy++)
                                for (int32_t dx = -reach; dx <= reach; dx++) {
                                    int32_t a = i + dx, b = j + dy, d = k + dz;
                                    if (a < 0 || b < 0 || d < 0 || a >= n[0] || b >= n[1] || d >= n[2]) continue;
                                    if (!occ[(int64_t)a + (int64_t)n[0] * ((int64_t)b + (int64_t)n[1] * d)]) continue;
                                    int32_t cd = abs(dx) > abs(dy) ? abs(dx) : abs(dy);
                                    if (abs(dz) > cd) cd = abs(dz);
                                    if (cd < dmin) dmin = cd;
                                }
                        if (dmin > band_cells) cl = OR_I;
                        if (inner_cells > 0 && dmin > band_cells + inner_cells) continue;
                    }
                    if (cnt < cap) {
                        float ctr[3];
                        cell_centre(c, i, j, k, ctr);
                        for (int a = 0; a < 3; a++) xyz[3 * cnt + a] = (double)ctr[a];
                        cls[cnt] = cl;
                        cons[cnt] = -1;
                    }
                    cnt++;
                }
        free(occ);
        free(ins);
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* C_compact interval form of a cell set and its Boolean algebra            */
/* (Sec. 3.1.3: C_compact begin / length; Sec. 3.2.3 and Fig. 10: union,    */
/* difference and intersection of two bodies' grid sets as intervals)       */
/* ------------------------------------------------------------------------ */
/* A cell set of a lattice (origin o, spacing d; cells (i, j, k) with
 * 0 <= i, j, k < 2^21) is the ascending list of its Morton codes (Eq. 9),
 * run-length encoded: C_compact begin = the first code of a run of
 * consecutive codes, length = the run's size.  Runs are maximal, so the next
 * begin lies at least one code past the end of a run. */

static int cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* the lattice cell holding point x: floor((x - o) / d) per axis in FP32;
 * -1 when a coordinate lies outside [0, 2^21) */
static int lattice_cell(const float *x, const float *o, float d, uint32_t *ijk)
{
    for (int a = 0; a < 3; a++) {
        const float t = floorf((x[a] - o[a]) / d);
        if (!(t >= 0.0f && t < 2097152.0f)) return -1;
        ijk[a] = (uint32_t)t;
    }
    return 0;
}

/* Morton code (Eq. 9) back to its cell: bit 3b + a of the code is bit b of
 * axis a */
static void morton3_decode(uint64_t code, uint32_t *ijk)
{
    ijk[0] = ijk[1] = ijk[2] = 0;
    for (int b = 0; b < 21; b++)
        for (int a = 0; a < 3; a++) ijk[a] |= (uint32_t)((code >> (3 * b + a)) & 1u) << b;
}

/* maximal runs of ascending codes (repeats allowed); returns the count and
 * writes at most cap runs */
static int64_t runs_of_codes(const uint64_t *code, int64_t n, uint64_t *begin, uint64_t *len, int64_t cap)
{
    int64_t r = 0;
    int64_t i = 0;
    while (i < n) {
        const uint64_t b = code[i];
        uint64_t e = b + 1;
        i++;
        while (i < n && code[i] <= e) {   /* a repeat (< e) or the next code (== e) */
            if (code[i] == e) e++;
            i++;
        }
        if (r < cap) {
            begin[r] = b;
            len[r] = e - b;
        }
        r++;
    }
    return r;
}

/* C_compact of the cells that hold the n points: the codes of their cells,
 * sorted, as maximal runs.  Returns the run count (at most cap written), -1
 * for a point outside the lattice or d not finite and > 0. */
int64_t oracle_lattice_intervals(const float *xyz, int64_t n, const float *o, float d, uint64_t *begin, uint64_t *len,
                                 int64_t cap)
{
    if (n < 0 || !(d > 0.0f) || !isfinite(d)) return -1;
    uint64_t *code = malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        uint32_t c[3];
        if (lattice_cell(xyz + 3 * i, o, d, c)) {
            free(code);
            return -1;
        }
        code[i] = oracle_morton3(c[0], c[1], c[2]);
    }
    qsort(code, (size_t)n, sizeof(uint64_t), cmp_u64);
    const int64_t r = runs_of_codes(code, n, begin, len, cap);
    free(code);
    return r;
}

typedef struct {
    uint64_t b, e;   /* [b, e) */
} or_run;

static int cmp_run(const void *a, const void *b)
{
    const or_run *x = a, *y = b;
    return x->b < y->b ? -1 : (x->b > y->b ? 1 : 0);
}

/* the same set as maximal runs in ascending order: empty runs dropped,
 * overlapping and touching runs joined.  Returns the count, -1 when a run's
 * end passes 2^63. */
static int64_t canonical_runs(const uint64_t *b, const uint64_t *l, int64_t n, or_run *out)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        if (l[i] == 0) continue;
        if (b[i] >= (1ull << 63) || l[i] > (1ull << 63) - b[i]) return -1;
        out[m].b = b[i];
        out[m].e = b[i] + l[i];
        m++;
    }
    qsort(out, (size_t)m, sizeof(or_run), cmp_run);
    int64_t k = 0;
    for (int64_t i = 0; i < m; i++) {
        if (k > 0 && out[i].b <= out[k - 1].e) {
            if (out[i].e > out[k - 1].e) out[k - 1].e = out[i].e;
        } else {
            out[k++] = out[i];
        }
    }
    return k;
}

/* is code p in the canonical runs r[0..n)?  (binary search for the last run
 * that begins at or before p) */
static int in_runs(const or_run *r, int64_t n, uint64_t p)
{
    int64_t lo = 0, hi = n;   /* first run with b > p */
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (r[mid].b <= p) lo = mid + 1;
        else hi = mid;
    }
    return lo > 0 && p < r[lo - 1].e;
}

/* Fig. 10's interval algebra: the cells c with op(c in A, c in B) -- union
 * (op 0), difference A - B (op 1), intersection (op 2) -- as maximal runs.
 * The inputs may be in any order, overlap, touch or hold empty runs.  Every
 * begin or end of an input run cuts the code line into pieces on which
 * membership in A and in B is constant; a piece is tested at its first code
 * and joined to the previous one when both are in.  Returns the run count
 * (at most cap written), -1 for an unknown op or a run past 2^63. */
int64_t oracle_interval_boolean(const uint64_t *ab, const uint64_t *al, int64_t na, const uint64_t *bb,
                                const uint64_t *bl, int64_t nb, int op, uint64_t *ob, uint64_t *ol, int64_t cap)
{
    if (op < 0 || op > 2 || na < 0 || nb < 0) return -1;
    or_run *A = malloc(sizeof(or_run) * (size_t)(na > 0 ? na : 1));
    or_run *B = malloc(sizeof(or_run) * (size_t)(nb > 0 ? nb : 1));
    const int64_t ma = canonical_runs(ab, al, na, A), mb = canonical_runs(bb, bl, nb, B);
    if (ma < 0 || mb < 0) {
        free(A);
        free(B);
        return -1;
    }
    const int64_t np = 2 * (ma + mb);
    uint64_t *pt = malloc(sizeof(uint64_t) * (size_t)(np > 0 ? np : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < ma; i++) {
        pt[k++] = A[i].b;
        pt[k++] = A[i].e;
    }
    for (int64_t i = 0; i < mb; i++) {
        pt[k++] = B[i].b;
        pt[k++] = B[i].e;
    }
    qsort(pt, (size_t)np, sizeof(uint64_t), cmp_u64);
    int64_t r = 0;
    int open = 0;   /* the previous piece was in the result */
    for (int64_t i = 0; i + 1 < np; i++) {
        if (pt[i] == pt[i + 1]) continue;   /* an empty piece */
        const int inA = in_runs(A, ma, pt[i]), inB = in_runs(B, mb, pt[i]);
        const int in = op == 0 ? (inA || inB) : (op == 1 ? (inA && !inB) : (inA && inB));
        if (in && open) {
            if (r - 1 < cap) ol[r - 1] = pt[i + 1] - ob[r - 1];
        } else if (in) {
            if (r < cap) {
                ob[r] = pt[i];
                ol[r] = pt[i + 1] - pt[i];
            }
            r++;
        }
        open = in;
    }
    free(pt);
    free(A);
    free(B);
    return r;
}

/* the cells of runs (in the given order, codes ascending within a run) as
 * their centres (float)(o + (i + 0.5) d) per axis, each coordinate evaluated
 * in FP64 and rounded once -- the generation's cell centres.  Returns the
 * cell count (at most cap written), -1 for a run past 2^63. */
int64_t oracle_interval_cells(const uint64_t *b, const uint64_t *l, int64_t n, const float *o, float d, float *xyz,
                              int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t r = 0; r < n; r++) {
        if (b[r] >= (1ull << 63) || l[r] > (1ull << 63) - b[r]) return -1;
        for (uint64_t c = b[r]; c < b[r] + l[r]; c++, cnt++) {
            if (cnt >= cap) continue;
            uint32_t ijk[3];
            morton3_decode(c, ijk);
            for (int a = 0; a < 3; a++)
                xyz[3 * cnt + a] = (float)((double)o[a] + ((double)ijk[a] + 0.5) * (double)d);
        }
    }
    return cnt;
}
