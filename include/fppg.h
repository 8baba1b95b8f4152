/*
 * fppg.h -- C ABI of the GB300 (sm_103a) relaxation library for
 * Feature-Preserving Particle Generation (FPPG, arXiv 2501.03056).
 *
 * The library relaxes surface, feature-line and volume particles of a body
 * given as an explicit triangle mesh (Sec. 3.1): every iteration rebuilds a
 * cell-key + radix-sort neighbour grid (Sec. 3.1.3), sums the pairwise
 * Wendland C2 kernel-gradient repulsion (Eq. 15 with Eqs. 16-17), takes the
 * limited step (Eqs. 22-25) and projects each particle back to its
 * constraint (Sec. 3.3.3, Sec. 3.3.4).  Everything runs in hand-written CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every call:
 *  - Return value: FPPG_OK (0) or one of the FPPG_ERR_* codes.  A failing
 *    call leaves a message in fppg_last_error(ctx).  No C++ exception crosses
 *    the ABI.
 *  - Pointers named *_host are host memory; pointers named *_dev are device
 *    memory of the current CUDA device.  Inputs are copied: the caller keeps
 *    ownership of every buffer it passes.  Outputs go to caller-allocated
 *    buffers whose capacity is passed explicitly.
 *  - Handles (fppg_ctx, fppg_batch) are owned by the library until the
 *    matching destroy call.
 *  - Work is enqueued on the stream given by fppg_set_stream (default: the
 *    legacy default stream).  Calls that return host data synchronise that
 *    stream before returning; fppg_relax and fppg_batch_relax do not.
 *  - Arrays of points are packed xyz triples (row-major [n][3]).
 *  - Particle classes: FPPG_S surface, FPPG_V volume (relaxes),
 *    FPPG_F feature line, FPPG_I innermost volume (fixed), FPPG_P singular
 *    feature point (fixed).
 */
#ifndef FPPG_H
#define FPPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FPPG_OK = 0,
    FPPG_ERR_ARG = 1,      /* invalid argument (null, size, index, NaN)      */
    FPPG_ERR_STATE = 2,    /* call out of order (e.g. relax before particles) */
    FPPG_ERR_OOM = 3,      /* device or host allocation failed               */
    FPPG_ERR_CUDA = 4,     /* a CUDA runtime call failed                     */
    FPPG_ERR_TIMEOUT = 5,  /* a device-side wait ran out of its budget       */
    FPPG_ERR_INTERNAL = 6  /* a device-side consistency check failed         */
};

enum { FPPG_S = 0, FPPG_V = 1, FPPG_F = 2, FPPG_I = 3, FPPG_P = 4 };

typedef struct fppg_ctx fppg_ctx;
typedef struct fppg_batch fppg_batch;

/* Uniformity statistics (fppg_stats). */
typedef struct {
    double mean_rho[3];      /* mean kernel sum of S, V, F particles           */
    double std_rho[3];       /* its standard deviation per class               */
    double min_pair_over_dx; /* smallest masked pair distance / dx (mobile)    */
    double max_disp_over_dx; /* largest move of the last iteration / dx        */
    int64_t count[3];        /* number of S, V, F particles                    */
} fppg_stats_t;

/* ---- body ----------------------------------------------------------------
 * fppg_create: upload a closed, outward-oriented triangle mesh (Sec. 3.1:
 * explicit STL-like geometry) and build its device structures:
 *   - per-triangle unit normals, in-plane edge normals, edge and
 *     angle-weighted vertex pseudonormals (FP64, stored FP32);
 *   - the triangle grid with cell size dx (Sec. 3.1.1), triangles binned to
 *     cells by the separating-axis triangle-box test (Sec. 3.1.2) on cells
 *     inflated by 1e-6 dx;
 *   - the compact cell list C_compact and the hash H of Eq. 10 with
 *     H_begin / H_length (Sec. 3.1.3);
 *   - the neighbour grid: cell 2h (1 + 2^-8), one cell of margin around the
 *     mesh bounding box.
 * verts_host: [nv][3] float; tris_host: [nt][3] int32 vertex indices in
 * [0, nv); dx: particle spacing; h: smoothing length (Wendland support 2h;
 * the paper uses h = 1.3 dx).  Errors: FPPG_ERR_ARG for empty meshes,
 * out-of-range indices, non-finite vertices or dx, h <= 0; FPPG_ERR_OOM. */
int fppg_create(const float *verts_host, int64_t nv, const int32_t *tris_host, int64_t nt, float dx, float h,
                fppg_ctx **out);
int fppg_destroy(fppg_ctx *ctx);
/* Last error message of ctx ("" when none); ctx may be NULL for errors of
 * fppg_create.  The string lives until the next call on ctx. */
const char *fppg_last_error(const fppg_ctx *ctx);
/* Stream (a cudaStream_t) on which all later work of ctx is enqueued. */
int fppg_set_stream(fppg_ctx *ctx, void *stream);
/* Feature particles never move when fixed != 0 (paper-literal boundary
 * role of feature lines, Sec. 2.2); by default they slide along their line. */
int fppg_set_fixed_features(fppg_ctx *ctx, int32_t fixed);
/* Classes that move (bit 1 << class of FPPG_S, FPPG_V, FPPG_F; I and P
 * never move); default all three, relaxed together.  The paper relaxes the
 * surface particles (Algorithm 1) and then the intermediate volume
 * particles "similarly" (Sec. 3.3.4): mask (1 << S) | (1 << F) for the
 * first stage, then (1 << V).  A class that does not move still acts on
 * the others.  Applies to fppg_relax and to batches created afterwards.
 * Errors: FPPG_ERR_ARG for bits outside S, V, F. */
int fppg_set_mobile_classes(fppg_ctx *ctx, int32_t mask);
/* Surface re-projection rule (A6): FPPG_PROJECT_CLOSEST (default, reading:
 * the closest projectable triangle over the 27 triangle cells of the trial
 * point) or FPPG_PROJECT_CASCADE (Sec. 3.3.3's order: a particle still on
 * its triangle stays there; else the closest projectable triangle of the
 * trial point's own cell, as in the mapping of Sec. 3.2.1; else over the
 * 27 cells; else revert).  Applies to fppg_relax, fppg_project_points and
 * batches created afterwards.  Errors: FPPG_ERR_ARG for another value. */
#define FPPG_PROJECT_CLOSEST 0
#define FPPG_PROJECT_CASCADE 1
int fppg_set_projection_rule(fppg_ctx *ctx, int32_t rule);

/* ---- features (Sec. 3.2.2) -------------------------------------------------
 * fppg_extract_features: edge-face map with v1 < v2 keys; an edge is a
 * feature when it has other than two faces or when the angle between the
 * two unit face normals exceeds dihedral_deg (dot < cos(dihedral_deg)),
 * both in FP64.  Singular points: feature degree 1 or more than 2.  Feature
 * lines: walks from singular points (ascending vertex id, incident edges in
 * ascending edge id), then closed loops from the lowest uncoloured edge.
 * Writes the feature-edge count to *n_edges (nullable). */
int fppg_extract_features(fppg_ctx *ctx, float dihedral_deg, int64_t *n_edges);
/* Feature edges as [n][2] vertex ids (v1 < v2), ascending (v1, v2) order.
 * Copies min(cap, n) edges; *n receives the total. */
int fppg_get_feature_edges(fppg_ctx *ctx, int32_t *edges_host, int64_t cap, int64_t *n);
/* Feature lines: line_nseg_host[l] segments each, closed flag per line,
 * seg_v_host [n_seg][2] vertex pairs in walk order.  Capacities in lines and
 * segments; totals through *n_lines and *n_seg. */
int fppg_get_feature_lines(fppg_ctx *ctx, int64_t *line_nseg_host, int32_t *closed_host, int64_t cap_lines,
                           int32_t *seg_v_host, int64_t cap_seg, int64_t *n_lines, int64_t *n_seg);

/* ---- particle generation (Sec. 3.2) ------------------------------------------
 * fppg_map_particles: replace the body's particles by the initial set of
 * Sec. 3.2, built on the triangle grid (cell dx):
 *   features   particles along the feature lines of fppg_extract_features,
 *              n = ceil(L / dx) pieces of length L / n, singular end points
 *              once (class P), the others F with constraint = the feature
 *              segment each was placed on (Sec. 3.2.2);
 *   surface    every cell holding triangles maps its centre to the nearest
 *              triangle of that cell whose orthogonal foot is inside (class S,
 *              constraint = that triangle); a centre with none is discarded
 *              (Sec. 3.2.1, Figs. 8-9);
 *   volume     every cell without triangles whose centre is inside by ray
 *              parity along +z (Fig. 6; the ray starts at the centre displaced
 *              by (1.234567e-6, 2.345678e-6) dx so it meets no edge or vertex
 *              exactly) gives a particle at its centre: class V, or I when
 *              band_cells > 0 and no cell with triangles lies within
 *              band_cells cells (Chebyshev) -- the three layers of Sec. 3.3.4;
 *              with inner_cells > 0 the innermost layer is inner_cells thick
 *              and deeper cells give no particle.
 * Order: feature, surface (cell key order), volume (cell key order).
 * *n_out (nullable) receives the count.  Errors: FPPG_ERR_INTERNAL when a
 * grid column meets more than 256 triangle entries (ray buffer). */
typedef struct {
    int32_t surface;
    int32_t volume;
    int32_t features;
    int32_t band_cells;
    int32_t inner_cells;
} fppg_map_opts;
int fppg_map_particles(fppg_ctx *ctx, const fppg_map_opts *opts, int64_t *n_out);

/* ---- particles --------------------------------------------------------------
 * fppg_set_particles: copy n particles (xyz_host [n][3] float, cls_host [n]
 * class codes) to the device; constraint ids start at -1 (the first
 * iteration then searches all triangles / feature segments of the body).
 * Errors: FPPG_ERR_ARG for a class outside 0..4 or non-finite coordinates. */
int fppg_set_particles(fppg_ctx *ctx, const float *xyz_host, const int32_t *cls_host, int64_t n);
/* Constraint ids per particle (cons_host [n]: local triangle for S, local
 * feature segment for F, -1 for none), e.g. to resume a saved state.
 * Errors: FPPG_ERR_STATE without particles, FPPG_ERR_ARG for n other than
 * the particle count or an id out of range for the particle's class. */
int fppg_set_constraints(fppg_ctx *ctx, const int32_t *cons_host, int64_t n);
/* Boolean operations on two bodies (Sec. 3.2.3 and Fig. 10: bodies combined
 * through their cell sets, by interval union, difference and intersection).
 * Reading on particles, with "inside" = the ray parity of Fig. 6 against
 * the other mesh (+z ray, FP64, from the particle displaced by
 * (1.234567e-6, 2.345678e-6) dx in x, y so that it meets no edge) and
 * "volume" = volume or innermost particle:
 *   FPPG_UNION         a keeps what is outside b; b keeps what is outside a
 *                      and its volume particles (one copy of the overlap);
 *   FPPG_DIFFERENCE    a - b: a keeps what is outside b; b keeps its
 *                      surface, feature and singular particles inside a
 *                      (the wall of the cavity);
 *   FPPG_INTERSECTION  a keeps what is inside b; b keeps its surface,
 *                      feature and singular particles inside a.
 * The two bodies become partners: they relax only inside one batch
 * (fppg_batch_create with both) as one assembly — one neighbour grid over
 * both boxes, so their particles repel each other, and one time step — and
 * a projected position must keep to the operation's side of the partner
 * (closest-feature sign of the partner's triangles within the 27 triangle
 * cells; none in range: the particle is where it started), else the
 * particle reverts: surface and feature particles of a union stay outside
 * the partner, of a difference outside b (a's) or inside a (b's, the
 * cavity wall), of an intersection inside the partner; volume particles of
 * a difference also stay outside b, of an intersection inside b.  The
 * curve where the surfaces meet gets feature particles from
 * fppg_boolean_curve (below).
 * Chains (Fig. 10 combines several bodies): a body may take part in up to
 * four operations, each applied to the particles its earlier ones left; it
 * keeps what every operation keeps and relaxes under the rules of all of
 * them.  Bodies joined by operations, directly or through others, form one
 * assembly (one neighbour grid over all their boxes, one time step) and
 * relax in one batch that holds all of them.  A cavity cut by several
 * overlapping bodies is their union: unite the cutters as well.  *n_a, *n_b
 * (nullable) receive the particle counts left.  Errors: FPPG_ERR_ARG for
 * the same handle twice, an unknown op, different dx / h / feature
 * setting, or a mesh that is not closed and consistently oriented;
 * FPPG_ERR_STATE without particles, when the two bodies are already in an
 * operation together, or when one of them is in four operations already.
 * fppg_relax on an operand afterwards returns FPPG_ERR_STATE, and so does
 * fppg_batch_create with an operand but not all of its partners.
 * fppg_union(a, b, ...) = fppg_boolean(a, b, FPPG_UNION, ...). */
#define FPPG_UNION 0
#define FPPG_DIFFERENCE 1
#define FPPG_INTERSECTION 2
int fppg_boolean(fppg_ctx *a, fppg_ctx *b, int32_t op, int64_t *n_a, int64_t *n_b);
int fppg_union(fppg_ctx *a, fppg_ctx *b, int64_t *n_a, int64_t *n_b);
/* The crease of a Boolean result (Sec. 3.2.3) as a feature line (Sec. 3.2.2):
 * the curve where a's surface crosses b's becomes feature lines of a, with
 * feature particles along them appended to a's particles, constraint = the
 * curve segment.  Call after fppg_boolean(a, b, ...) (either order of the
 * pair; the lines go to the first argument) and before fppg_batch_create;
 * in a chain, once per pair whose crease is wanted.
 * Set-up on the host, in FP64 with every operation rounded in the written
 * order:
 *   - pairs: every (a-triangle, b-triangle) pair whose closed bounding boxes
 *     overlap; the side of a vertex against the other triangle's plane
 *     (unnormalised normal (v1 - v0) x (v2 - v0), origin v0) is d >= 0; the
 *     two edges of each triangle whose ends lie on different sides cross
 *     the other plane at u + (v - u) du / (du - dv) (u < v vertex ids), a
 *     point named by the key (mesh, u, v, other triangle); the pair's
 *     segment is the overlap of the two triangles' crossing intervals along
 *     na x nb, kept when of positive length;
 *   - chains: segments in (a, b) order; ends with the same key join when
 *     exactly two share it; ends still free join the first free end of
 *     another segment (in segment, end order) within 2^-30 of a's largest
 *     bounding-box extent; open chains are walked from the free end of the
 *     first segment that has one, then loops from their first segment,
 *     leaving by the end of larger key;
 *   - the points join a's vertex list (rounded to FP32, after the mesh
 *     vertices; fppg_get_feature_lines gives the segments' vertex ids and
 *     fppg_get_curve_points their coordinates), each chain one feature line
 *     after a's own, with n = ceil(L / dx) feature particles placed as on
 *     a's own lines (open chains add their end points as singular points).
 * In the relaxation these particles move along their line and are exempt
 * from the pair's partner rule (they lie on both surfaces); the rules of
 * a's other operations still apply to them.  *n_added (nullable) receives
 * the particles added.  Errors: FPPG_ERR_ARG for the same handle twice or
 * more than 2^31 curve points; FPPG_ERR_STATE when b is not a's Boolean
 * partner, a has no particles, or the pair has its curve already;
 * FPPG_ERR_OOM.  On an error a keeps its own lines (after a failed
 * particle upload, like fppg_set_particles, no particles).  Extracting
 * features again drops the curve lines (their particles are then left
 * without a line: extract the features first, then add the curves). */
int fppg_boolean_curve(fppg_ctx *a, fppg_ctx *b, int64_t *n_added);
/* The intersection-curve points of ctx (FP32 xyz, the vertices after the
 * mesh's own) into xyz_host (capacity cap points, nullable); *n receives
 * their number. */
int fppg_get_curve_points(fppg_ctx *ctx, float *xyz_host, int64_t cap, int64_t *n);
/* Positions, classes and constraint ids (triangle for S, feature segment for
 * F, -1 otherwise) into caller buffers of capacity cap (each nullable);
 * *n_out receives the particle count.  Synchronises the stream. */
int fppg_get_particles(fppg_ctx *ctx, float *xyz_host, int32_t *cls_host, int32_t *cons_host, int64_t cap,
                       int64_t *n_out);

/* ---- relaxation (Algorithm 1) ----------------------------------------------
 * fppg_relax: n_iter Jacobi iterations of
 *   A1 cell keys  A2 stable radix sort  A3 gather + cell ranges
 *   A4 force a_i = -sum_j dW/dr(r_ij) e_ij over the masked neighbours
 *      (S <- S,F,P; V <- all; F <- F,P) and amax over mobile particles
 *   A5 step dr = a dt^2 with dt = 0.25 sqrt(h / amax) (largest move h/16),
 *      normal part removed for S (current triangle), tangential only for F
 *   A6 projection: S to the closest projectable triangle in the 3x3x3 cells
 *      around the trial point, else revert; F to the closest point of its
 *      line; V reverted when the pseudonormal sign says outside.
 * Enqueued on the stream; does not synchronise.  Errors: FPPG_ERR_STATE
 * without particles; FPPG_ERR_ARG for n_iter < 0. */
int fppg_relax(fppg_ctx *ctx, int32_t n_iter);
/* Spatial decomposition over several GPUs (one body split into slabs, one
 * per process; the exchanges are the caller's).  fppg_set_ghost_count marks
 * the last n_ghost particles of the set as ghosts: copies of particles a
 * neighbouring domain owns within 2h of the shared face.  A ghost acts on
 * its neighbours by its class (Eq. 15 with the class mask) but never moves,
 * gets no force and is left out of amax and fppg_stats.  fppg_set_particles
 * clears the count.  FPPG_ERR_ARG outside 0..n, FPPG_ERR_STATE without
 * particles.
 * One iteration of Algorithm 1 in two halves, so that the largest force can
 * be reduced over the domains between them (the time step of Eqs. 22-23 is
 * shared): fppg_relax_forces builds the grid and sums the forces (A1-A4) and
 * writes this domain's largest |a| over its moving particles to *amax_host;
 * fppg_relax_step takes the step with the given amax (every domain passes
 * the same, the maximum over all) and projects (A5-A6).  Both synchronise
 * the stream.  fppg_relax_step without a preceding fppg_relax_forces is
 * FPPG_ERR_STATE; amax must be finite and >= 0. */
int fppg_set_ghost_count(fppg_ctx *ctx, int64_t n_ghost);
int fppg_relax_forces(fppg_ctx *ctx, float *amax_host);
int fppg_relax_step(fppg_ctx *ctx, float amax);
/* Same iteration with the acceleration a = -dE/dx of the uniformity energy
 * (energy-descent relaxation). */
int fppg_relax_energy(fppg_ctx *ctx, int32_t n_iter);
/* Statistics of the current state; synchronises. */
int fppg_stats(fppg_ctx *ctx, fppg_stats_t *out);

/* ---- single steps of the path (parity and diagnostics) ---------------------
 * fppg_debug_grid: A1-A3 on the current state.  key_host [n]: cell key per
 * particle in id order; perm_host [n]: stable sort permutation (id of the
 * k-th particle in key order); cells/start/end: occupied cells ascending
 * with their [start, end) slot ranges (capacity cap_cells, count through
 * *n_cells).  Any output may be NULL. */
int fppg_debug_grid(fppg_ctx *ctx, uint32_t *key_host, uint32_t *perm_host, uint32_t *cells_host,
                    uint32_t *start_host, uint32_t *end_host, int64_t cap_cells, int64_t *n_cells);
/* A4 on the current state: acc_host [n][3] (id order, zero for fixed
 * particles), count_host [n] masked neighbour counts, *amax.  Nullable. */
int fppg_debug_forces(fppg_ctx *ctx, float *acc_host, int32_t *count_host, float *amax_host);
/* A6 alone on n given trial points y_host [n][3] with classes cls_host and
 * incoming constraints cons_host (nullable = all -1): writes x_host [n][3],
 * cons_out_host [n] and ok_host [n] (0 = not projectable / outside; x then
 * equals y). */
int fppg_project_points(fppg_ctx *ctx, const float *y_host, const int32_t *cls_host, const int32_t *cons_host,
                        int64_t n, float *x_host, int32_t *cons_out_host, int32_t *ok_host);

/* A6 bookkeeping: *queued = particles of the last iteration that went to
 * the triangle search (the others finished in the step: features, nothing
 * within reach, or a volume particle inside its inside certificate, i.e. a
 * ball that an earlier search found free of surface and inside a closed
 * mesh); *closed = 1 when every mesh edge has two faces of opposite
 * direction and no face is degenerate (certificates apply), else 0.
 * Either output may be NULL.  Synchronises. */
int fppg_debug_search(fppg_ctx *ctx, int64_t *queued, int32_t *closed);

/* Candidate lists of the triangle search: every cell within one cell of a
 * triangle cell (the dilated occupancy) stores the distinct triangles binned
 * into its 27 cells (Sec. 3.1.3's C_compact lists, merged once at
 * fppg_create), so a search reads one list instead of probing 27 cells
 * through the Eq. 10 hash.  *cells = cells with a list, *entries = total
 * list entries, *overflow = cells whose list was too long to merge (their
 * searches probe the cells).  Outputs nullable. */
int fppg_debug_cell_lists(fppg_ctx *ctx, int64_t *cells, int64_t *entries, int64_t *overflow);

/* Work of one force pass (A4) on the current state, summed over mobile
 * particles: candidates = particles in the 27 neighbour cells around each
 * particle (the search set of the cell grid, Sec. 3.1.3), pairs = masked
 * neighbours within 2h (Eq. 15), tested = candidates the force kernel
 * actually tests after cutting each grid row to the x-slabs within reach.
 * Any output may be NULL.  Synchronises. */
int fppg_work_counts(fppg_ctx *ctx, int64_t *candidates, int64_t *pairs, int64_t *tested);

/* ---- uniformity energy and its backward -------------------------------------
 * E = sum over mobile i of (rho_i - W0_{c_i})^2, rho_i = W(0) + sum over the
 * masked neighbours of W(r_ij); W0 the kernel sum of a perfect lattice of
 * the class (cubic for V, square for S, line for F).  Positions are
 * x = y - ((y - v_a) . n) n for S particles with a triangle (frozen
 * triangle, unit normal n from verts_dev) and x = y otherwise.
 * y_dev [n][3] float, verts_dev [nv][3] float (NULL = the body's mesh).
 * Writes *E_host; gy_dev [n][3] and gV_dev [nv][3] receive dE/dy and
 * dE/dverts when non-NULL (gV_dev is overwritten, not accumulated).
 * Synchronises the stream. */
int fppg_energy(fppg_ctx *ctx, const float *y_dev, const float *verts_dev, double *E_host, float *gy_dev,
                float *gV_dev);
/* Current positions [n][3] into a device buffer (for the energy). */
int fppg_copy_positions_dev(fppg_ctx *ctx, float *xyz_dev);

/* ---- batched form -------------------------------------------------------------
 * fppg_batch_create: one group over n bodies (each with particles set):
 * their particles are concatenated and every phase of an iteration runs as
 * one launch over all bodies, each keeping its own grids, mesh and amax.
 * The batch copies the bodies' state; fppg_batch_store writes it back. */
int fppg_batch_create(fppg_ctx *const *ctxs, int32_t n, fppg_batch **out);
int fppg_batch_destroy(fppg_batch *b);
int fppg_batch_set_stream(fppg_batch *b, void *stream);
/* n_iter iterations; use_graph != 0 captures graph_iters iterations into
 * one CUDA graph (built on first use) and replays it. */
int fppg_batch_relax(fppg_batch *b, int32_t n_iter, int32_t use_graph);
int fppg_batch_set_graph_iters(fppg_batch *b, int32_t graph_iters);
/* Copy the batch state back into its bodies, or reload it from them (after
 * fppg_set_particles on the bodies with unchanged particle counts). */
int fppg_batch_store(fppg_batch *b);
int fppg_batch_load(fppg_batch *b);
/* Autotuner: times `iters` iterations of the batch for every combination
 * of force-kernel block size (128, 256) and force-kernel variant (0 per-lane
 * rows, 1 shared-row union) with the warp search on 4 CTAs per SM; then,
 * with the fastest force kernel, the triangle search on 8 or 16 CTAs per SM
 * or -- search CTAs 0 -- one thread per queued particle on 16 CTAs per SM;
 * then, with the fastest of those, the two ways of ordering the cell keys
 * (a full stable sort, or the incremental repair of the previous order,
 * fppg_batch_set_incremental), then the two orders of the grid rows
 * (fppg_batch_set_cell_order), keeps the fastest and restores the particle
 * state afterwards.  The choice is cached per (particle-count bucket,
 * volume-particle share, GPU name) for the life of the process; a cached
 * choice is applied without timing.  Every variant, block size, search
 * grid and ordering gives the same bits; the Morton row order moves
 * particles between the force loop's two partial sums, so it agrees with
 * row-major rows up to FP32 rounding (a plain body set to the same row
 * order gives the batch's bits).  Outputs (nullable): chosen variant,
 * block size, search CTAs, ordering (1 incremental), row order and the
 * measured ms per iteration (0 when taken from the cache). */
int fppg_batch_autotune(fppg_batch *b, int32_t iters, int32_t *variant, int32_t *block, int32_t *search_ctas,
                        int32_t *incremental, int32_t *cell_order, double *ms_per_iter);
/* How the cell keys are put in order every iteration (Sec. 3.1.3): 0 a full
 * stable radix sort of every key; 1 the previous order repaired -- the
 * particles whose key changed since the last grid build are sorted alone and
 * merged with the others, which keep their order.  Both give the one order by
 * (key, particle id), so the results are the same bits; the incremental form
 * moves less data once few keys change per iteration (large groups start
 * with it).  Drops a captured graph.  FPPG_ERR_ARG for other values. */
int fppg_batch_set_incremental(fppg_batch *b, int32_t incremental);
/* The same for the single body of a handle (its fppg_relax, fppg_stats and
 * debug calls); a body of at least 2^21 particles starts incremental. */
int fppg_set_incremental(fppg_ctx *ctx, int32_t incremental);
/* Order of the neighbour grid's rows in the cell key (Sec. 3.1.3 sorts
 * particles by cell; Eq. 9 gives the Morton code of a cell):
 *   FPPG_ORDER_ROWS          key cell = x + nx (y + ny z) (row-major, default)
 *   FPPG_ORDER_MORTON_ROWS   key cell = x + nx rank(y, z), rank = the place
 *                            of row (y, z) in the order of its Morton code
 *                            (Eq. 9 over y and z: the bits interleaved, z's
 *                            above y's at every level)
 * x stays the fastest axis inside a row in both, so every grid row is one
 * range of keys (the force pass cuts each row to the x-slabs in reach); a
 * full 3-D Morton key would split a row into many ranges.  Both orders give
 * the same neighbours in the same order (each particle sums its rows in
 * stencil order and every row in x order), so the forces agree up to the
 * FP32 rounding of the two partial sums a row's slots are split between
 * (by the parity of their absolute position); the keys and the permutation
 * follow the order.  The rank table of every grid is built on first use
 * (FPPG_ERR_ARG above 2^26 rows).  The previous order of the keys is
 * forgotten.  fppg_set_cell_order for the body of a handle,
 * fppg_batch_set_cell_order for a batch (bodies of a batch take the
 * batch's order). */
#define FPPG_ORDER_ROWS 0
#define FPPG_ORDER_MORTON_ROWS 1
int fppg_set_cell_order(fppg_ctx *ctx, int32_t order);
int fppg_batch_set_cell_order(fppg_batch *b, int32_t order);
/* fppg_set_mobile_classes for every body of the batch (a captured graph
 * keeps working: the mask is read from device memory). */
int fppg_batch_set_mobile_classes(fppg_batch *b, int32_t mask);
/* The same choice made by hand: force variant 0 or 1, force block 128 or 256,
 * search CTAs per SM 1..64 for the warp form or 0 for the thread form
 * (FPPG_ERR_ARG otherwise).  Every choice gives the
 * same bits; only the speed differs.  Drops a captured graph. */
int fppg_batch_configure(fppg_batch *b, int32_t variant, int32_t block, int32_t search_ctas);
/* Kernel launches of one iteration of the batch (A1-A6, all bodies). */
int32_t fppg_batch_kernels_per_iter(const fppg_batch *b);
/* Particle count and the last error of the batch. */
int64_t fppg_batch_size(const fppg_batch *b);
const char *fppg_batch_last_error(const fppg_batch *b);
/* Phase timing of the graph form: fppg_batch_time_force(b, 1) puts CUDA
 * event records into the captured graph (dropping a graph captured
 * without them) around each iteration's grid build (A1-A3), force pass
 * (A4), step (A5, with the projections that need no search) and triangle
 * search (A6).  After a graph replay of fppg_batch_relax,
 * fppg_batch_phase_ms writes the device ms of the four phases, averaged
 * over the graph's iterations, into ms4[4] (in that order) and
 * fppg_batch_force_ms the force pass alone; FPPG_ERR_STATE when timing is
 * off or no graph has been captured.  Both synchronise the batch stream. */
int fppg_batch_time_force(fppg_batch *b, int32_t enable);
int fppg_batch_force_ms(fppg_batch *b, double *ms);
int fppg_batch_phase_ms(fppg_batch *b, double *ms4);

/* Test hook for the out-of-memory paths: the k-th device allocation the
 * library makes from now on (k = 0: the next one) fails as if the device
 * were out of memory, once; k = -1 cancels.  Not part of the method.  The
 * call that meets the failure returns FPPG_ERR_OOM and frees what it had
 * allocated; handles made before stay usable.  FPPG_ERR_ARG for k < -1. */
int fppg_debug_fail_allocation(int64_t k);

/* Streaming multiprocessors of the current CUDA device
 * (cudaDevAttrMultiProcessorCount) into *sms: the unit count behind the
 * ALU roofline of the force pass (SMs x 128 FP32 lanes x clock).  Not part
 * of the method.  FPPG_ERR_ARG for a null pointer, FPPG_ERR_CUDA when no
 * device is usable (message in fppg_last_error(NULL)). */
int fppg_device_sm_count(int32_t *sms);
/* Bounds checks.  A library built with -DFPPG_CHECKED (the `checked`
 * build of paper_2501_03056_gb300._build) checks, in the hot-path kernels,
 * every index it computes before using it: the sorted ids and fine keys of
 * the gather, each grid row's slot range of the force pass, the search
 * queue's slots and entries, the candidate triangles of the searches, the
 * compaction positions and merge splits of the incremental order.  A
 * failed check skips the access and ORs its code into a device word:
 * 1 gather, 2 slot range, 4 queue slot, 8 queue entry, 16 candidate
 * triangle, 32 merge split, 64 compaction position.  fppg_check_status
 * returns that word in *word and clears it (0 in the normal build, where
 * the checks compile away), and *checked (nullable) = 1 for the checked
 * build.  FPPG_ERR_ARG for word NULL; FPPG_ERR_CUDA when the word cannot be
 * read. */
int fppg_check_status(uint32_t *word, int32_t *checked);

/* ---- C_compact interval form of grid sets (Sec. 3.1.3, Sec. 3.2.3) --------
 * Sec. 3.1.3 stores a body's cells as C_compact begin / length, runs of
 * consecutive Morton codes (Eq. 9); Sec. 3.2.3 and Fig. 10 combine two
 * bodies' grid sets by union, difference and intersection of those
 * intervals.  A lattice is an origin o (3 floats, host) and a spacing d;
 * cell (i, j, k), 0 <= i, j, k < 2^21, has the Morton code with bit b of i,
 * j, k at bits 3b, 3b + 1, 3b + 2.  A run list is two device arrays of
 * uint64: begin (first code of a run) and len (its size).  The result of
 * every call is a set of maximal runs in ascending order (the next begin
 * lies at least one code past the end of a run).
 *
 * Each call enqueues its work on `stream` (a cudaStream_t, NULL = legacy
 * default), allocates its temporaries, and synchronises the stream to read
 * the result count into *n_out; it writes the result only when the count
 * fits cap (else FPPG_ERR_ARG with *n_out set: call again with room).
 * Errors (message in fppg_last_error(NULL)): FPPG_ERR_ARG for null buffers,
 * negative sizes, the cases below; FPPG_ERR_OOM; FPPG_ERR_CUDA. */

/* fppg_grid_lattice: the lattice of a body's generation (Sec. 3.2): the
 * triangle grid's origin (*origin_host, 3 floats) and spacing dx (*d_host).
 * fppg_map_particles puts one volume particle at the centre of every
 * interior cell of that lattice.  Bodies whose lattices coincide (the same
 * dx and origin) have grid sets that combine cell for cell.  FPPG_ERR_ARG
 * for a NULL argument. */
int fppg_grid_lattice(const fppg_ctx *ctx, float *origin_host, float *d_host);

/* fppg_lattice_intervals: C_compact of the cells that hold the n points
 * xyz_dev [n][3] (device): the cell of a point is floor((x - o) / d) per
 * axis in FP32; repeated cells count once.  n < 2^32.  FPPG_ERR_ARG for d
 * not finite and > 0 or a point outside the lattice. */
int fppg_lattice_intervals(const float *xyz_dev, int64_t n, const float *origin_host, float d, uint64_t *begin_dev,
                           uint64_t *len_dev, int64_t cap, int64_t *n_out, void *stream);

/* fppg_interval_boolean: the runs of the cells c with op(c in A, c in B),
 * op = FPPG_UNION, FPPG_DIFFERENCE (A - B) or FPPG_INTERSECTION (Fig. 10).
 * The input runs may come in any order, overlap, touch or be empty;
 * na + nb < 2^31.  FPPG_ERR_ARG for another op or a run ending past 2^63. */
int fppg_interval_boolean(const uint64_t *a_begin_dev, const uint64_t *a_len_dev, int64_t na,
                          const uint64_t *b_begin_dev, const uint64_t *b_len_dev, int64_t nb, int32_t op,
                          uint64_t *begin_dev, uint64_t *len_dev, int64_t cap, int64_t *n_out, void *stream);

/* fppg_interval_cells: the cells of n runs as their centres xyz_dev
 * [*n_out][3] (device), runs in the given order and codes ascending within
 * a run; each coordinate is (float)(o + (i + 0.5) d) evaluated in FP64 --
 * the generation's cell centres, so the runs of a body's volume particles
 * give those particles back bit for bit.  n < 2^32, fewer than 2^32 cells.
 * FPPG_ERR_ARG for d not finite and > 0, a run ending past 2^63 or a run of
 * 2^32 cells or more. */
int fppg_interval_cells(const uint64_t *begin_dev, const uint64_t *len_dev, int64_t n, const float *origin_host,
                        float d, float *xyz_dev, int64_t cap, int64_t *n_out, void *stream);

/* ---- allocation-free force pass ---------------------------------------------
 * fppg_forces_static: the neighbour grid and the force pass (A1-A4) for one
 * body, without a handle and without allocating any memory: for callers
 * that cannot call cudaMalloc -- applications whose device memory is owned
 * by their own pool allocator, and time-critical loops that must not pay
 * for an allocation or the device synchronisation it may cause.  The paper
 * has no counterpart; the result equals fppg_debug_forces of a body whose
 * mesh has the bounding box [bbmin, bbmax] (the neighbour-grid rule of
 * fppg_create).
 *
 * xyz_dev [n][3] float and cls_dev [n] int32 (device), n <= 65536; the box
 * must need at most 131072 grid cells of 2h (1 + 2^-8); acc_dev [n][3]
 * float (device) receives the accelerations in input order (zero for fixed
 * classes); *amax_host (nullable) the largest |a| over moving particles.
 * stream: a cudaStream_t (NULL = legacy default); the call synchronises it.
 *
 * Every temporary lives in one static device array of about 9.5 MB (the
 * per-particle arrays, 5 MiB, the start table of every fine key of the
 * grid, 4 MiB, and a few tens of KB of parameters, flags, radix histograms
 * and the start table's block starts) that each GPU loading the library holds until the process
 * exits.  The first call on
 * a device looks up that array's address (cudaGetSymbolAddress) -- make it
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them.
 *
 * Errors (message in fppg_last_error(NULL)): FPPG_ERR_ARG for n above the
 * limit, a box needing more cells, null buffers, h not finite and positive
 * or a class outside 0..4 (the output is then unspecified); FPPG_ERR_CUDA
 * when a CUDA call fails.  Non-finite coordinates give unspecified output. */
int fppg_forces_static(const float *xyz_dev, const int32_t *cls_dev, int64_t n, const float *bbmin_host,
                       const float *bbmax_host, float h, int32_t fixed_features, float *acc_dev, float *amax_host,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FPPG_H */
