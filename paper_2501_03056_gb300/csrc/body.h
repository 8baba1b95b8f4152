// One body (mesh + grids + feature lines) and the group runtime that relaxes
// one or many bodies with the same launches.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include "fppg_internal.cuh"

namespace fppg {

// largest cell count of one grid axis (2^20): every grid of the library has
// its cell keys in 32 bits, which no axis above this can reach anyway
constexpr int kGridAxisMax = 1 << 20;
// origin, 1 / cell and cell counts of a grid over [bbmin, bbmax]; false when
// an axis would need more than kGridAxisMax cells (or cell is not positive)
bool grid_setup(const float *bbmin, const float *bbmax, float cell, double shift, int margin, float *o, float *inv,
                int *n);

struct Body {
    int nv = 0, nt = 0;
    float dx = 0, h = 0;
    // triangle grid (cell dx, origin 2.5 cells below the box, 2 cells of margin)
    float tg_o[3] = {0, 0, 0};
    float tg_inv = 0;
    int tg_n[3] = {0, 0, 0};
    // neighbour grid (cell 2h (1 + 2^-8), 1 cell of margin)
    float ng_o[3] = {0, 0, 0};
    float ng_inv = 0, ng_cell = 0, R2 = 0;
    float edge_tol = 0;  // 2^-20 of the largest bounding-box extent
    bool closed = false; // every edge has two faces of opposite direction, none degenerate
    float bbmin[3] = {0, 0, 0}, bbmax[3] = {0, 0, 0};   // bounding box of the vertices
    int ng_n[3] = {0, 0, 0};
    // device mesh
    float *d_verts = nullptr;
    int32_t *d_tris = nullptr;
    float4 *geo = nullptr, *vx = nullptr, *pn = nullptr;
    double *nu = nullptr;        // FP64 unit normals (set-up only)
    uint64_t *ekey = nullptr;    // sorted edge keys v1 * nv + v2
    uint32_t *eval = nullptr;    // 3 t + k of each sorted edge entry
    uint2 *hrng = nullptr;
    int64_t hash_size = 0;
    uint4 *compact = nullptr;
    int64_t ncompact = 0;
    int32_t *tlist = nullptr;
    int64_t npairs = 0;
    uint32_t *occ = nullptr;     // occupancy bitmap, then its 27-cell dilation
    int64_t occ_words = 0;       // words of one bitmap
    // candidate lists: the distinct triangles of the 27 cells around every
    // dilated cell; drank[w] = set dilated bits before word w, coff[r] the
    // list start of the r-th dilated cell (bit 31: list too long, probe
    // the cells), coff[n_dil] the total
    uint32_t *drank = nullptr, *coff = nullptr;
    int32_t *cand = nullptr;
    int64_t n_dil = 0, n_cand = 0;
    // feature lines (host copies + device segments)
    bool has_features = false;
    std::vector<int32_t> fe;           // [nfe][2] sorted
    std::vector<int32_t> sing;         // singular vertices
    std::vector<int64_t> line_first, line_nseg;
    std::vector<int32_t> line_closed;
    std::vector<int32_t> seg_v;        // [nseg][2]
    std::vector<float> verts_host;     // FP32 mesh vertices, then the intersection-curve points
    std::vector<int32_t> tris_host;    // the triangles
    float4 *seg = nullptr;
    int2 *lines = nullptr;
    int nseg = 0, nlines = 0;
    int nseg_own = 0;                  // segments of the body's own lines; intersection-curve ones follow

    // feature particles of lines l0 .. l1 - 1 (l1 < 0: to the last line)
    void feature_particles(std::vector<float> &xyz, std::vector<int32_t> &cls, std::vector<int32_t> &seg,
                           int l0 = 0, int l1 = -1) const;
    // back to an earlier set of lines: the first nseg_keep segments and the
    // lines they form, verts_keep vertex coordinates (host side; the device
    // copy only holds more segments than are used)
    void drop_lines_after(int nseg_keep, size_t verts_keep, bool has_features_keep);
    int add_curve(const Body &other, std::vector<float> &xyz, std::vector<int32_t> &cls, std::vector<int32_t> &seg,
                  cudaStream_t s, std::string &err);
    int build_mesh(const float *verts_host, int64_t nv, const int32_t *tris_host, int64_t nt, float dx, float h,
                   cudaStream_t s, std::string &err);
    int extract_features(float deg, cudaStream_t s, std::string &err);
    void build_lines();
    // upload of the segments and lines; on a failed allocation the body is
    // left without features, or (keep_on_failure) with its old device copy
    int upload_lines(cudaStream_t s, std::string &err, bool keep_on_failure = false);
    void drop_features();   // forget every feature edge, line and segment
    void free_mesh();
    ~Body() { free_mesh(); }
};

// Host description of one body inside a group.
AsmParams make_params(const Body &b, uint32_t key_base, int p_begin, int p_end, int fixed_features);

// scratch of the energy and its backward (energy.cu), kept between calls
struct EnergyScratch {
    float4 *xs = nullptr, *vcon = nullptr;
    double *e_s = nullptr, *part = nullptr;
    uint32_t *vk[2] = {nullptr, nullptr}, *vi[2] = {nullptr, nullptr}, *hist = nullptr, *tot = nullptr;
    int64_t n = 0;   // particles it is sized for
    void release() {
        void *p[] = {xs, vcon, e_s, part, vk[0], vk[1], vi[0], vi[1], hist, tot};
        for (void *q : p)
            if (q) cudaFree(q);
        *this = EnergyScratch();
    }
};

struct Group {
    DevGroup d;
    EnergyScratch escr;
    std::vector<AsmParams> hp;    // host copy of the per-body parameters
    MeshView mesh{};
    bool owns_mesh = false;       // batches own concatenated copies
    // timing of the force kernel inside a relaxation (optional)
    bool time_force = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    // CUDA graph of graph_iters iterations
    int search_blocks = 152 * 8;  // persistent grid of the search
    bool search_thread = false;   // one thread (not one warp) per queued particle
    int force_block = 256;        // threads per block of the force kernel (multiple of 32, <= 256)
    int force_variant = 0;        // 0 per-lane rows, 1 shared-row union
    // order of the neighbour grid's rows: 0 row-major, 1 Morton (Eq. 9 over
    // (y, z)); the rank tables of every grid live in d.row_rank, body i's at
    // row_off[i]
    int cell_order = 0;
    std::vector<int64_t> row_off;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    cudaStream_t graph_stream = nullptr;

    int alloc_particles(int64_t N, std::string &err);   // on failure: nothing allocated, N = 0
    int alloc_particles_once(int64_t N, std::string &err);
    void release_particles();
    int alloc_order_state(std::string &err);
    void free_order_state();
    // forget the previous order (the next grid build sorts every key); used
    // when the incremental ordering is switched on
    void invalidate_order(cudaStream_t s);
    int upload_params(cudaStream_t s, std::string &err);
    // the rank tables of the grids of hp (built once), then every body's
    // parameters pointed at its table (order 1) or at none (order 0); the
    // previous order of the keys is forgotten.  Uploads the parameters.
    int set_cell_order(int order, cudaStream_t s, std::string &err);
    void free_all();
    ~Group() { free_all(); }
};

// an NVTX range for the life of the object (host side; shows the library's
// calls and phases on a timeline profiler; a few ns with no tool attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// the codes of the failed bounds checks of a checked build since the last
// call, cleared (0 in the normal build; 0xffffffff when it cannot be read)
uint32_t check_word_take();

// rank[y + ny z] of every grid row in the Morton order of Eq. 9 over (y, z):
// the bits of y and z interleaved, z's above y's at every level
void morton_row_ranks(int ny, int nz, std::vector<uint32_t> &rank);

// groups of at least this many particles start with the incremental ordering
constexpr int64_t kIncrementalMinN = 1 << 21;

// event records per timed iteration: before A1, after A3, A4, A5 and A6
constexpr int kPhaseEvents = 5;
// one relaxation iteration of every body of the group (A1-A6)
void iterate(Group &g, cudaStream_t s, bool energy_mode, int32_t *count_dbg = nullptr);
// A5-A6 (step, then the projections) after a grid build that returned buf
// and a force pass; amax is whatever the device holds
void step_and_project(Group &g, cudaStream_t s, int buf);
// particles [first_ghost, N) become ghosts, the others not (the ghost bit of w)
void tag_ghosts(Group &g, int64_t first_ghost, cudaStream_t s);
// A1-A3 only (keys, sort, gather + cell ranges); returns the buffer index
// holding the sorted keys / ids
int build_grid(Group &g, cudaStream_t s);
// the same on bare device arrays (no Group): A1-A3, A4, back to id order
int build_grid_dev(DevGroup &d, cudaStream_t s);
// kernel launches of one grid build (A1-A3)
int grid_kernels(const DevGroup &d);
void forces_dev(DevGroup &d, int block, int variant, cudaStream_t s, int32_t *count_s = nullptr,
                int32_t *tested_s = nullptr);
void unpermute_dev(DevGroup &d, int buf, cudaStream_t s, float *acc_out, const int32_t *count_s, int32_t *count_out);
// A4 into acc_s (and counts when non-null)
void forces(Group &g, cudaStream_t s, int32_t *count_s, int32_t *cand_s = nullptr, int32_t *tested_s = nullptr);
// energy-descent acceleration -dE/dx into acc_s
void energy_accel(Group &g, cudaStream_t s);
// debug helpers
void unpermute(Group &g, int buf, cudaStream_t s, float *acc_out, const int32_t *count_s, int32_t *count_out);
void project_points(Group &g, const float *y, const int32_t *cls, const int32_t *cons_in, int64_t n, float *x,
                    int32_t *cons_out, int32_t *ok, cudaStream_t s);
// uniformity statistics into host doubles (see fppg_stats_t)
int stats(Group &g, cudaStream_t s, double *mean, double *sd, double *minpair, double *maxdisp, int64_t *cnt,
          std::string &err);
// initial particles of Sec. 3.2 into the group (features, surface, volume)
int map_particles(Group &g, Body &b, int surface, int volume, int features, int band_cells, int inner_cells,
                  cudaStream_t s, int64_t *n_out, std::vector<int32_t> &cls_host, std::string &err);
// Boolean union: inside[i] (device) = ray parity (Fig. 6, FP64) of point i
// against body 0 of group `other`
void ray_parity(const Group &other, const float4 *pos, int64_t n, int32_t *inside, cudaStream_t s);
// energy and gradients (positions y, vertex coordinates verts of body 0)
int energy(Group &g, const Body &b, const float *y_dev, const float *verts_dev, double *E, float *gy, float *gV,
           cudaStream_t s, std::string &err);

} // namespace fppg
