// The relaxation hot path (Algorithm 1, Sec. 3.3) for a group of bodies.
//
// Per iteration, all bodies at once:
//   k_keys          A1  cell key per particle (FP32 rule, no contraction);
//                       zeroes the per-body amax / max-move
//   radix sort      A2  stable (key, id) sort, 8-bit digits
//   k_gather        A3  positions and constraint ids in key order
//   start table     A3  the dense table of the first slot of every fine key,
//                       from the sorted keys (block starts, then a binary
//                       search per fine key inside its block's slots)
//   k_force         A4  Eq. 15 over the 3 x 3 rows of 3 cells around the
//                       particle (each row is one contiguous slot range),
//                       amax per body by a labelled warp max + atomicMax
//   k_step          A5  limited step and tangential part; feature particles,
//                       and particles with no triangle within reach, finish
//                       here; the others are queued
//   k_search        A6  one warp per queued particle, its lanes over the 27
//                       triangle cells: projection or revert; positions are
//                       written back in id order
#include <cfloat>

#include "body.h"

namespace fppg {

#ifdef FPPG_CHECKED
// the codes of the failed bounds checks since the last fppg_check_status
__device__ uint32_t g_check_word = 0u;
__device__ bool fppg_check_failed(uint32_t code) {
    atomicOr(&g_check_word, code);
    return false;
}
#endif

uint32_t check_word_take() {
#ifdef FPPG_CHECKED
    uint32_t w = 0u;
    const uint32_t zero = 0u;
    if (cudaMemcpyFromSymbol(&w, g_check_word, sizeof(w)) != cudaSuccess) return 0xffffffffu;
    cudaMemcpyToSymbol(g_check_word, &zero, sizeof(zero));
    return w;
#else
    return 0u;
#endif
}

namespace {

constexpr int TPB = 256;

inline unsigned nblocks(int64_t n, int t = TPB) { return (unsigned)std::max<int64_t>((n + t - 1) / t, 1); }

__device__ inline float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ inline float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ inline float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ inline float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// max of v (>= 0) over the lanes that share `label`, added to dst[label] by
// one lane (dst starts every iteration at 0, so a max of 0 needs no atomic)
__device__ inline void labelled_max(uint32_t *dst, int label, float v) {
    uint32_t peers = __match_any_sync(0xffffffffu, label);
    uint32_t m = __reduce_max_sync(peers, __float_as_uint(v));
    if ((uint32_t)(__ffs(peers) - 1) == (threadIdx.x & 31u) && m) atomicMax(dst + label, m);
}

// The same over a whole block (every thread must call it): a warp whose
// lanes share one label leaves (label, max) in shared memory and thread 0
// adds one atomic per run of equal labels over the warps; a warp that
// mixes labels uses labelled_max.  On one large body this turns one
// same-address atomic per warp into one per block.
template <int WARPS>
__device__ inline void block_labelled_max(uint32_t *dst, int label, float v, int *s_lab, uint32_t *s_max) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lab0 = __shfl_sync(0xffffffffu, label, 0);
    if (__all_sync(0xffffffffu, label == lab0)) {
        const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
        if (lane == 0) {
            s_lab[w] = lab0;
            s_max[w] = m;
        }
    } else {
        labelled_max(dst, label, v);
        if (lane == 0) {
            s_lab[w] = -1;
            s_max[w] = 0u;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run_l = -1;
        uint32_t run_m = 0u;
        for (int q = 0; q < WARPS; q++) {
            if (s_lab[q] != run_l) {
                if (run_m) atomicMax(dst + run_l, run_m);
                run_l = s_lab[q];
                run_m = 0u;
            }
            if (run_l >= 0) run_m = max(run_m, s_max[q]);
        }
        if (run_m) atomicMax(dst + run_l, run_m);
    }
}

// ---- A1 ----------------------------------------------------------------------
__global__ void __launch_bounds__(TPB) k_keys(const float4 *__restrict__ pos, int64_t N,
                                              const AsmParams *__restrict__ P, uint32_t *__restrict__ key,
                                              uint32_t *__restrict__ amax, uint32_t *__restrict__ maxdisp, int B,
                                              uint32_t *__restrict__ work_count) {
    int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i < B) {
        amax[i] = 0u;
        maxdisp[i] = 0u;
    }
    if (i == 0) {
        work_count[0] = 0u;
        work_count[1] = 0u;
    }
    if (i >= N) return;
    float4 p = pos[i];
    const AsmParams &A = P[body_of(p.w)];
    const int fx = fine_coord(p.x, A.ng_o[0], A.ng_inv, A.ng_n[0]);
    const int cy = cell_coord(p.y, A.ng_o[1], A.ng_inv, A.ng_n[1]);
    const int cz = cell_coord(p.z, A.ng_o[2], A.ng_inv, A.ng_n[2]);
    key[i] = kSlabs * A.key_base + (uint32_t)fx +
             kSlabs * (uint32_t)A.ng_n[0] * grid_row(A, cy, cz);
}

// ---- A1-A2, incremental form ---------------------------------------------------
// A particle moves at most h / 16 per iteration, so from one grid build to
// the next only a few per cent of the fine keys change (under 1 % once the
// relaxation settles).  The incremental form keeps the last (key, id) order
// and repairs it: the particles whose key changed are sorted alone (radix,
// count on the device), the others keep their relative order, and the two
// sorted lists are merged by (key, id).  The result is the one order by
// (key, id), the same permutation as the stable sort of every key; with a
// stale or foreign previous order every key counts as changed and the
// repair is a full sort.

// The flags of both compactions are bits (bit i & 31 of word i >> 5: 1/32 of
// the bytes of a flag array, small enough to stay in L2).  A block handles a
// tile of kOrdTile items, kOrdItems per thread at stride TPB (item tile0 +
// TPB j + thread): fewer, longer blocks than one item per thread, whose
// launch cost would exceed the work of these light passes.  Word j of warp w
// holds items tile0 + TPB j + 32 w + (0..31); every tile counts its set
// bits.  One exclusive scan of the 2 x tiles counts (the changed tiles by
// id, then the kept tiles by previous slot) places every tile; inside a tile
// a bit's rank is the set bits of the earlier words and lanes.
constexpr int kOrdItems = 8, kOrdTile = TPB * kOrdItems, kOrdWords = kOrdItems * (TPB / 32);
static_assert(kOrdWords == 64, "tile_ranks scans two word counts per lane");
static_assert(kOrdTile == 2048, "the order state (Group::alloc_order_state) has tiles of 2048");

// the word counts of a tile, summed: its number of set bits
__device__ inline void store_tile_count(uint32_t cnt, int64_t N, uint32_t *__restrict__ tile_cnt, uint32_t *wcnt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wcnt[w] = cnt;
    __syncthreads();
    if (threadIdx.x == 0 && (int64_t)blockIdx.x * kOrdTile < N) {
        uint32_t t = 0;
        for (int q = 0; q < TPB / 32; q++) t += wcnt[q];
        tile_cnt[blockIdx.x] = t;
    }
}

// key of every particle (the rule of k_keys), compared with the key it had
// at the last grid build: the changed bits by id and their tile counts;
// key_id updated
__global__ void __launch_bounds__(TPB) k_keys_inc(const float4 *__restrict__ pos, int64_t N,
                                                  const AsmParams *__restrict__ P, uint32_t *__restrict__ key_id,
                                                  uint32_t *__restrict__ chg_bits, uint32_t *__restrict__ tile_cnt,
                                                  uint32_t *__restrict__ amax, uint32_t *__restrict__ maxdisp, int B,
                                                  uint32_t *__restrict__ work_count) {
    __shared__ uint32_t wcnt[TPB / 32];
    const int64_t g = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (g < B) {
        amax[g] = 0u;
        maxdisp[g] = 0u;
    }
    if (g == 0) {
        work_count[0] = 0u;
        work_count[1] = 0u;
    }
    const int64_t i0 = (int64_t)blockIdx.x * kOrdTile + threadIdx.x;
    float4 p[kOrdItems];
    uint32_t old[kOrdItems];
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        const int64_t i = i0 + (int64_t)j * TPB;
        p[j] = i < N ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        old[j] = i < N ? key_id[i] : 0u;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        const int64_t i = i0 + (int64_t)j * TPB;
        bool changed = false;
        if (i < N) {
            const AsmParams &A = P[body_of(p[j].w)];
            const int fx = fine_coord(p[j].x, A.ng_o[0], A.ng_inv, A.ng_n[0]);
            const int cy = cell_coord(p[j].y, A.ng_o[1], A.ng_inv, A.ng_n[1]);
            const int cz = cell_coord(p[j].z, A.ng_o[2], A.ng_inv, A.ng_n[2]);
            const uint32_t k = kSlabs * A.key_base + (uint32_t)fx +
                               kSlabs * (uint32_t)A.ng_n[0] * grid_row(A, cy, cz);
            changed = k != old[j];
            if (changed) key_id[i] = k;
        }
        const uint32_t word = __ballot_sync(~0u, changed);
        if ((threadIdx.x & 31) == 0 && i < N) chg_bits[i >> 5] = word;   // i is a multiple of 32 in lane 0
        cnt += __popc(word);
    }
    store_tile_count(cnt, N, tile_cnt, wcnt);
}

// the kept bits by previous slot (the particle in slot k kept its key) and
// their tile counts
__global__ void __launch_bounds__(TPB) k_keep_bits(const uint32_t *__restrict__ prev_id,
                                                   const uint32_t *__restrict__ chg_bits, int64_t N,
                                                   uint32_t *__restrict__ keep_bits,
                                                   uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wcnt[TPB / 32];
    const int64_t k0 = (int64_t)blockIdx.x * kOrdTile + threadIdx.x;
    uint32_t id[kOrdItems];
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        const int64_t k = k0 + (int64_t)j * TPB;
        id[j] = k < N ? prev_id[k] : 0u;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        const int64_t k = k0 + (int64_t)j * TPB;
        const bool kept = k < N && FPPG_CHECK(id[j] < N, kChkCompact) &&
                          !((chg_bits[id[j] >> 5] >> (id[j] & 31)) & 1u);
        const uint32_t word = __ballot_sync(~0u, kept);
        if ((threadIdx.x & 31) == 0 && k < N) keep_bits[k >> 5] = word;
        cnt += __popc(word);
    }
    store_tile_count(cnt, N, tile_cnt, wcnt);
}

// this thread's words of a tile (word j of its warp) and, for each, the rank
// of its own bit among the tile's set bits in item order (j, then warp, then
// lane); sc: kOrdWords shared words
__device__ inline void tile_ranks(const uint32_t *__restrict__ bits, int64_t tile0, int64_t N,
                                  uint32_t (&word)[kOrdItems], uint32_t (&rank)[kOrdItems], uint32_t *sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        const int64_t i0 = tile0 + (int64_t)j * TPB + 32 * w;
        word[j] = i0 < N ? bits[i0 >> 5] : 0u;
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < kOrdItems; j++) sc[j * (TPB / 32) + w] = __popc(word[j]);
    __syncthreads();
    if (w == 0) {
        // exclusive scan of the 64 word counts, two per lane
        const uint32_t a = sc[2 * lane], b = sc[2 * lane + 1];
        uint32_t v = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(~0u, v, o);
            if (lane >= o) v += t;
        }
        const uint32_t ex = v - a - b;
        sc[2 * lane] = ex;
        sc[2 * lane + 1] = ex + a;
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) rank[j] = sc[j * (TPB / 32) + w] + __popc(word[j] & lt);
}

// the changed particles, in id order: (key, id) at their positions
__global__ void __launch_bounds__(TPB) k_compact_changed(const uint32_t *__restrict__ chg_bits,
                                                         const uint32_t *__restrict__ tile_pos,
                                                         const uint32_t *__restrict__ key_id, int64_t N,
                                                         uint32_t *__restrict__ ck, uint32_t *__restrict__ cv) {
    __shared__ uint32_t sc[kOrdWords];
    const int64_t tile0 = (int64_t)blockIdx.x * kOrdTile;
    uint32_t word[kOrdItems], rank[kOrdItems];
    tile_ranks(chg_bits, tile0, N, word, rank, sc);
    const uint32_t p0 = tile_pos[blockIdx.x];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        if (!((word[j] >> lane) & 1u)) continue;
        const int64_t i = tile0 + (int64_t)j * TPB + threadIdx.x;
        const uint32_t p = p0 + rank[j];
        if (!FPPG_CHECK(p < N, kChkCompact)) continue;
        ck[p] = key_id[i];
        cv[p] = (uint32_t)i;
    }
}

// the kept slots of the previous order, compacted (still sorted); the kept
// tiles' positions follow the changed tiles' (nb tiles of each), so they
// start at the number of changed particles, tile_pos[nb]
__global__ void __launch_bounds__(TPB) k_compact_kept(const uint32_t *__restrict__ keep_bits,
                                                      const uint32_t *__restrict__ tile_pos, int64_t nb,
                                                      const uint32_t *__restrict__ prev_key,
                                                      const uint32_t *__restrict__ prev_id, int64_t N,
                                                      uint32_t *__restrict__ uk, uint32_t *__restrict__ uv) {
    __shared__ uint32_t sc[kOrdWords];
    const int64_t tile0 = (int64_t)blockIdx.x * kOrdTile;
    uint32_t word[kOrdItems], rank[kOrdItems];
    tile_ranks(keep_bits, tile0, N, word, rank, sc);
    const uint32_t p0 = tile_pos[nb + blockIdx.x] - tile_pos[nb];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kOrdItems; j++) {
        if (!((word[j] >> lane) & 1u)) continue;
        const int64_t k = tile0 + (int64_t)j * TPB + threadIdx.x;
        const uint32_t p = p0 + rank[j];
        if (!FPPG_CHECK(p < N, kChkCompact)) continue;
        uk[p] = prev_key[k];
        uv[p] = prev_id[k];
    }
}

// counts[0] = changed particles, counts[1] = kept slots, from the scan of
// the 2 nb tile counts
__global__ void k_order_counts(const uint32_t *__restrict__ tile_cnt, const uint32_t *__restrict__ tile_pos,
                               int64_t nb, uint32_t *__restrict__ counts) {
    const uint32_t c = tile_pos[nb];
    counts[0] = c;
    counts[1] = tile_pos[2 * nb - 1] + tile_cnt[2 * nb - 1] - c;
}

// merge of the kept list u (U items) and the sorted changed list c (C
// items), U + C = N, in (key, id) order; ids are distinct, so the order is
// strict and the merge unique
constexpr int kMergeThreads = 256, kMergeItems = 8, kMergeTile = kMergeThreads * kMergeItems;

__device__ inline bool kv_less(uint32_t ka, uint32_t ia, uint32_t kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// split[b]: how many u items the first min(b tile, N) outputs take
__global__ void k_merge_splits(const uint32_t *__restrict__ uk, const uint32_t *__restrict__ uv,
                               const uint32_t *__restrict__ ck, const uint32_t *__restrict__ cv,
                               const uint32_t *__restrict__ counts, int64_t N, int nblk,
                               uint32_t *__restrict__ split) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblk) return;
    const int64_t C = counts[0], U = counts[1];
    const int64_t d = min((int64_t)b * kMergeTile, N);
    int64_t lo = max((int64_t)0, d - C), hi = min(d, U);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t j = d - 1 - mid;
        if (kv_less(uk[mid], uv[mid], ck[j], cv[j])) lo = mid + 1;
        else hi = mid;
    }
    split[b] = (uint32_t)lo;
}

// one tile of kMergeTile outputs per block: its u and c items staged in
// shared memory, then kMergeItems outputs per thread
__global__ void __launch_bounds__(kMergeThreads) k_merge(const uint32_t *__restrict__ uk,
                                                         const uint32_t *__restrict__ uv,
                                                         const uint32_t *__restrict__ ck,
                                                         const uint32_t *__restrict__ cv,
                                                         const uint32_t *__restrict__ split, int64_t N,
                                                         uint32_t *__restrict__ out_key,
                                                         uint32_t *__restrict__ out_id) {
    __shared__ uint32_t sk[kMergeTile], si[kMergeTile];
    const int64_t d0 = (int64_t)blockIdx.x * kMergeTile, d1 = min(d0 + kMergeTile, N);
    const int64_t i0 = split[blockIdx.x], i1 = split[blockIdx.x + 1];
    const int64_t j0 = d0 - i0, j1 = d1 - i1;
    // (nu + nc = d1 - d0 <= kMergeTile: the staging fits when both are >= 0)
    if (!FPPG_CHECK(i0 <= i1 && j0 <= j1 && j0 >= 0, kChkMerge)) return;
    const int nu = (int)(i1 - i0), nc = (int)(j1 - j0), n = nu + nc;
    {
        // all loads of a thread issued before the first store (one round trip)
        uint32_t lk[kMergeItems], li[kMergeItems];
#pragma unroll
        for (int r = 0; r < kMergeItems; r++) {
            const int q = (int)threadIdx.x + r * kMergeThreads;
            lk[r] = li[r] = 0u;
            if (q < nu) {
                lk[r] = uk[i0 + q];
                li[r] = uv[i0 + q];
            } else if (q < n) {
                lk[r] = ck[j0 + q - nu];
                li[r] = cv[j0 + q - nu];
            }
        }
#pragma unroll
        for (int r = 0; r < kMergeItems; r++) {
            const int q = (int)threadIdx.x + r * kMergeThreads;
            if (q < n) {
                sk[q] = lk[r];
                si[q] = li[r];
            }
        }
    }
    __syncthreads();
    const int dt = min((int)threadIdx.x * kMergeItems, n);
    int lo = max(0, dt - nc), hi = min(dt, nu);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int j = dt - 1 - mid;
        if (kv_less(sk[mid], si[mid], sk[nu + j], si[nu + j])) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = dt - lo;
    uint32_t rk[kMergeItems], ri[kMergeItems];
#pragma unroll
    for (int q = 0; q < kMergeItems; q++) {
        if (dt + q < n) {
            const bool take_u = j >= nc || (i < nu && kv_less(sk[i], si[i], sk[nu + j], si[nu + j]));
            const int src = take_u ? i++ : nu + j++;
            rk[q] = sk[src];
            ri[q] = si[src];
        }
    }
    // the tile's outputs back through shared memory, then stored coalesced
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMergeItems; q++)
        if (dt + q < n) {
            sk[dt + q] = rk[q];
            si[dt + q] = ri[q];
        }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += kMergeThreads) {
        out_key[d0 + q] = sk[q];
        out_id[d0 + q] = si[q];
    }
}

// ---- A3 ----------------------------------------------------------------------
// Positions in key order (also as slot pairs) and the constraint ids in key
// order.
__global__ void __launch_bounds__(TPB) k_gather(const uint32_t *__restrict__ id_s, const float4 *__restrict__ pos,
                                                int64_t N, float4 *__restrict__ pos_s, float4 *__restrict__ pos_p,
                                                const int32_t *__restrict__ cons, int32_t *__restrict__ cons_s) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool valid = k < N;
    uint32_t id = valid ? id_s[k] : 0u;
    if (valid && !FPPG_CHECK(id < N, kChkGather)) id = 0u;
    const float4 q = valid ? pos[id] : make_float4(0.f, 0.f, 0.f, 0.f);
    // the constraint ids in key order too, for the step
    if (valid && cons_s) cons_s[k] = cons[id];
    // slot-pair copy: pair m = slots 2m and 2m + 1 as {x0, x1, y0, y1} at
    // pos_p[m] and {z0, z1, w0, w1} at pos_p[(N + 1) / 2 + m]; the two slots
    // sit in neighbouring lanes, which swap their points and write one half
    // each; past the last slot a lane holds a finite point of no class, the
    // padding of an odd count
    const float ox = __shfl_xor_sync(0xffffffffu, q.x, 1), oy = __shfl_xor_sync(0xffffffffu, q.y, 1);
    const float oz = __shfl_xor_sync(0xffffffffu, q.z, 1), ow = __shfl_xor_sync(0xffffffffu, q.w, 1);
    if ((k & 1) == 0) {
        if (valid) pos_p[k >> 1] = make_float4(q.x, ox, q.y, oy);
    } else if (k <= N) {
        pos_p[(N + 1) / 2 + (k >> 1)] = make_float4(oz, q.z, ow, q.w);
    }
    if (valid) pos_s[k] = q;
}

// The dense start table of the fine keys, from the sorted keys themselves:
// fstart[f] = the first slot whose fine key is >= f, for f in [0, F] (so
// fstart[F] = N).  The fine keys are cut into blocks of kStartBlock.
// k_key_block_starts: slot k starts the blocks (b(k - 1), b(k)] (b = key /
// kStartBlock; block -1 before the first slot, the block count after the
// last), so each block's first slot is written once, by the slot whose key
// step crosses it.  k_fine_starts: one CTA per block; the block's slots
// [bstart[b], bstart[b + 1]) hold every key of the block, and each thread
// finds its fine key's lower bound among them by binary search, in shared
// memory when the slots fit.  Every entry is written once: no counts,
// atomics or scans.  (Tiles of 4096 fine keys with a 16-key walk per
// thread measured slower: the table of the largest workload, 63 MB, stays
// in L2 either way, and the short per-thread search keeps more loads in
// flight.)
constexpr int kStartStage = 4096;

__global__ void __launch_bounds__(TPB) k_key_block_starts(const uint32_t *__restrict__ key_s, int64_t N,
                                                          int64_t nblk, uint32_t *__restrict__ bstart) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k > N) return;
    int64_t b0 = k == 0 ? -1 : (int64_t)(key_s[k - 1] / kStartBlock);
    int64_t b1 = k == N ? nblk : (int64_t)(key_s[k] / kStartBlock);
    if (!FPPG_CHECK(b0 < nblk && b1 <= nblk, kChkGather)) {   // a key past the fine-key count
        b0 = min(b0, nblk - 1);
        b1 = min(b1, nblk);
    }
    for (int64_t b = b0 + 1; b <= b1; b++) bstart[b] = (uint32_t)k;
}

__global__ void __launch_bounds__(kStartBlock) k_fine_starts(const uint32_t *__restrict__ key_s,
                                                             const uint32_t *__restrict__ bstart, int64_t F1,
                                                             uint32_t *__restrict__ fstart) {
    __shared__ uint32_t s_key[kStartStage];
    const int64_t b = blockIdx.x;
    const uint32_t lo = bstart[b], hi = bstart[b + 1];
    const uint32_t len = hi > lo ? hi - lo : 0u;
    const bool staged = len <= (uint32_t)kStartStage;
    if (staged)
        for (uint32_t i = threadIdx.x; i < len; i += kStartBlock) s_key[i] = key_s[lo + i];
    __syncthreads();
    const int64_t f = b * kStartBlock + threadIdx.x;
    if (f >= F1) return;
    uint32_t a = 0u, c = len;   // first of the block's slots with key >= f
    while (a < c) {
        const uint32_t m = (a + c) >> 1;
        if ((int64_t)(staged ? s_key[m] : key_s[lo + m]) < f) a = m + 1u;
        else c = m;
    }
    fstart[f] = lo + a;
}

// ---- A4 ----------------------------------------------------------------------
// a_i = -sum_j dW/dr(r_ij) e_ij = force_scale * sum_j (1 - r_ij / 2h)^3 (x_i - x_j)
//
// Each lane owns one particle (key order) and scans the 3 x 3 grid rows
// around it; per row it walks one contiguous slot range: the x-slabs of the
// row's stencil cells that lie within the reach sqrt((2h)^2 - gap_y^2 -
// gap_z^2) of it (rows out of reach are skipped).  Candidates come two at a
// time from the slot-pair copy pos_p ({x0, x1, y0, y1}, {z0, z1, w0, w1}),
// so one float4 load gives the packed FP32x2 operands; each packed
// operation is per component identical to the scalar round-to-nearest one,
// so the neighbour test r^2 = (dx dx + dy dy) + dz dz < (2h)^2 decides
// exactly as the scalar rule.  The loop works on q - p (the exact negation
// of p - q) and accumulates without branches into two partial sums.
//
// Variant 0 walks each lane's own ranges.  Variant 1 (shared row): when
// every moving lane of a warp lies in the same grid row of the same body,
// the lanes' ranges for one row offset lie in a single grid row and the
// warp walks their union in lockstep (broadcast loads); a candidate outside
// a lane's own range is out of its reach and fails the test.
// The particle itself adds (1 - 0)^3 * 0 = 0, so no self test is needed.
// Slots are paired by absolute parity (even -> .x, odd -> .y) with the range
// [s, e) applied as a mask, so every accepted neighbour lands in the same
// partial sum, in the same order, in every variant.
// COUNT adds, per particle, the accepted neighbours (self excluded) and the
// slots of its own ranges (candidates tested).
// r = sqrt(r^2) by sqrt_approx (exactly 0 at 0, so the particle itself
// needs no guard)

struct PairAcc {
    float2 ax, ay, az;
    int cnt;
};

// One slot pair (2m, 2m + 1).  EDGE: the pair may hold a slot outside the
// range [s, e) (the first and last pair of a range), which is masked out.
// The weight is clamped at zero, max(1 - r / 2h, 0)^3, instead of testing
// r^2 < (2h)^2: a pair beyond 2h adds exactly 0, one within rounding of 2h a
// weight below 1e-18; unless every class acts on the lane (ALL) the class
// mask selects.  The counting form keeps the exact FP32 test.
// pos_p holds the {x, y} halves of the slot pairs, pos_b the {z, w} halves;
// where every class acts on the lane (ALL) the class bits are not needed and
// only {z0, z1} is read: 24 bytes per slot pair instead of 32.
template <bool ALL, bool COUNT, bool EDGE>
__device__ inline void pair_step(const float4 *__restrict__ pos_p, const float4 *__restrict__ pos_b, uint32_t m,
                                 uint32_t s, uint32_t e, const float2 npx, const float2 npy, const float2 npz,
                                 uint32_t mbits, float R2, float hih, PairAcc &acc, uint32_t self) {
    const uint32_t j = 2 * m;
    const bool has0 = !EDGE || j >= s, has1 = !EDGE || j + 1 < e;
    const float4 A = pos_p[m];
    float4 B;
    if (ALL) {
        const float2 z = *reinterpret_cast<const float2 *>(pos_b + m);
        B = make_float4(z.x, z.y, 0.f, 0.f);
    } else {
        B = pos_b[m];
    }
    const float2 dx = __fadd2_rn(make_float2(A.x, A.y), npx);     // q - p
    const float2 dy = __fadd2_rn(make_float2(A.z, A.w), npy);
    const float2 dz = __fadd2_rn(make_float2(B.x, B.y), npz);
    float2 w;
    if (!COUNT) {
        // r^2 with fused multiply-adds and the weight max(1 - r / 2h, 0)^3
        // from a saturating FMA: no decision is taken on r^2 here (a slot
        // beyond 2h weighs exactly 0, one within rounding of 2h below 1e-18)
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 t = make_float2(__saturatef(fmaf(sqrt_approx(r2.x), -hih, 1.f)),
                                     __saturatef(fmaf(sqrt_approx(r2.y), -hih, 1.f)));
        w = __fmul2_rn(__fmul2_rn(t, t), t);
        bool k0 = has0, k1 = has1;
        if (!ALL) {
            k0 = k0 && (mbits & __float_as_uint(B.z)) != 0u;
            k1 = k1 && (mbits & __float_as_uint(B.w)) != 0u;
        }
        if (EDGE || !ALL) {
            w.x = k0 ? w.x : 0.f;
            w.y = k1 ? w.y : 0.f;
        }
    } else {
        // the counting form: the exact FP32 test r^2 = (dx dx + dy dy) + dz dz
        // < (2h)^2 without contraction decides each neighbour
        const float2 r2 = __fadd2_rn(__fadd2_rn(__fmul2_rn(dx, dx), __fmul2_rn(dy, dy)), __fmul2_rn(dz, dz));
        const float2 r = make_float2(sqrt_approx(r2.x), sqrt_approx(r2.y));
        const float2 t = __ffma2_rn(r, make_float2(-hih, -hih), make_float2(1.f, 1.f));   // 1 - r / 2h
        bool t0 = has0 && r2.x < R2, t1 = has1 && r2.y < R2;
        if (!ALL) {
            t0 = t0 && (mbits & __float_as_uint(B.z)) != 0u;
            t1 = t1 && (mbits & __float_as_uint(B.w)) != 0u;
        }
        if (COUNT) acc.cnt += (int)(t0 && j != self) + (int)(t1 && j + 1 != self);
        w = __fmul2_rn(__fmul2_rn(t, t), t);
        w.x = t0 ? w.x : 0.f;
        w.y = t1 ? w.y : 0.f;
    }
    acc.ax = __ffma2_rn(w, dx, acc.ax);
    acc.ay = __ffma2_rn(w, dy, acc.ay);
    acc.az = __ffma2_rn(w, dz, acc.az);
}

// the slot pairs [s >> 1, (e + 1) >> 1) of range [s, e): the first and last
// pair masked, the ones between without a range test
template <bool ALL, bool COUNT>
__device__ inline void force_range2(const float4 *__restrict__ pos_p, const float4 *__restrict__ pos_b,
                                    const float2 npx, const float2 npy, const float2 npz, uint32_t mbits, float R2,
                                    float hih, uint32_t s, uint32_t e, PairAcc &acc, uint32_t self) {
    if (s >= e) return;
    uint32_t m = s >> 1;
    const uint32_t m1 = (e + 1) >> 1;
    pair_step<ALL, COUNT, true>(pos_p, pos_b, m, s, e, npx, npy, npz, mbits, R2, hih, acc, self);
    if (m + 1 >= m1) return;
    for (m = m + 1; m + 1 < m1; m++)
        pair_step<ALL, COUNT, false>(pos_p, pos_b, m, s, e, npx, npy, npz, mbits, R2, hih, acc, self);
    pair_step<ALL, COUNT, true>(pos_p, pos_b, m1 - 1, s, e, npx, npy, npz, mbits, R2, hih, acc, self);
}

template <int VARIANT, bool COUNT, bool MORTON>
// (at most 48 registers: five 256-thread blocks per SM)
__global__ void __launch_bounds__(TPB, 5)
    k_force(const float4 *__restrict__ pos_s, const float4 *__restrict__ pos_p, int64_t N,
            const AsmParams *__restrict__ P, const uint32_t *__restrict__ fstart, float4 *__restrict__ acc_s,
            uint32_t *__restrict__ amax, int32_t *__restrict__ count_s, int32_t *__restrict__ tested_s) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = k < N;
    const float4 p = active ? pos_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int cls = active ? cls_of(p.w) : kClsI;
    const int b = active ? body_of(p.w) : 0;
    const AsmParams &A = P[b];
    const bool mob = active && is_mobile(cls, A) && !is_ghost(p.w);
    // the counting form also counts the neighbours of fixed particles
    const uint32_t mbits = (mob || (COUNT && active)) ? acts_on_bits(cls) : 0u;
    const int nx = A.ng_n[0], ny = A.ng_n[1], nz = A.ng_n[2];
    const GridPoint g = grid_point(A, p.x, p.y, p.z);
    const int cy = g.c[1], cz = g.c[2];
    const float R2 = A.R2, hih = A.half_inv_h;
    const float2 npx = make_float2(-p.x, -p.x), npy = make_float2(-p.y, -p.y), npz = make_float2(-p.z, -p.z);
    const float4 *pos_b = pos_p + (N + 1) / 2;
    // every class acts on every moving lane (volume targets): no mask test
    const bool all_cls = __all_sync(0xffffffffu, mbits == 0u || mbits == 0x1Fu);
    bool shared_row = false;
    if (VARIANT == 1) {
        const uint32_t mover = __ballot_sync(0xffffffffu, mbits != 0u);
        const int leader = mover ? __ffs(mover) - 1 : 0;
        const uint32_t rowkey = A.key_base + (uint32_t)nx * grid_row_of<MORTON>(A, cy, cz);
        const uint32_t lead_row = __shfl_sync(0xffffffffu, rowkey, leader);
        shared_row = __all_sync(0xffffffffu, mbits == 0u || rowkey == lead_row);
    }
    PairAcc acc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0};
    int tested = 0;
    for (int dz = -1; dz <= 1; dz++) {
        const int z = cz + dz;
        const float gz = row_gap(g.t[2], cz, dz, g.slack);
        for (int dy = -1; dy <= 1; dy++) {
            const int y = cy + dy;
            uint32_t s = 0xffffffffu, e = 0u;
            if (mbits && z >= 0 && z < nz && y >= 0 && y < ny) {
                const uint32_t row = A.key_base + (uint32_t)nx * grid_row_of<MORTON>(A, y, z);
                row_slots(A, fstart, g, row_gap(g.t[1], cy, dy, g.slack), gz, row, s, e);
                if (!FPPG_CHECK(e == 0u || (s <= e && e <= (uint64_t)N), kChkRange)) {
                    s = 0xffffffffu;
                    e = 0u;
                }
            }
            if (COUNT && e > s) tested += (int)(e - s);
            if (VARIANT == 1 && shared_row) {
                s = __reduce_min_sync(0xffffffffu, s);
                e = __reduce_max_sync(0xffffffffu, e);
            }
            if (all_cls)
                force_range2<true, COUNT>(pos_p, pos_b, npx, npy, npz, mbits, R2, hih, s, e, acc, (uint32_t)k);
            else
                force_range2<false, COUNT>(pos_p, pos_b, npx, npy, npz, mbits, R2, hih, s, e, acc, (uint32_t)k);
        }
    }
    float fx = 0.f, fy = 0.f, fz = 0.f, mag = 0.f;
    if (mob) {
        // the sums hold q - p: negate
        fx = -(acc.ax.x + acc.ax.y) * A.force_scale;
        fy = -(acc.ay.x + acc.ay.y) * A.force_scale;
        fz = -(acc.az.x + acc.az.y) * A.force_scale;
        mag = sqrtf(fx * fx + fy * fy + fz * fz);
    }
    if (active) acc_s[k] = make_float4(fx, fy, fz, mag);
    if (COUNT && active) {
        count_s[k] = acc.cnt;
        if (tested_s) tested_s[k] = mob ? tested : 0;
    }
    labelled_max(amax, A.amax_slot, mag);
}

// Masked neighbour count (self excluded) and the number of candidates in the
// particle's own 27 cells (the full stencil, no reach cut), per particle in
// key order (diagnostics).
__global__ void __launch_bounds__(TPB) k_count(const float4 *__restrict__ pos_s, int64_t N,
                                               const AsmParams *__restrict__ P, const uint32_t *__restrict__ fstart,
                                               int32_t *__restrict__ count_s, int32_t *__restrict__ cand_s) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    const float4 p = pos_s[k];
    const int cls = cls_of(p.w);
    const AsmParams &A = P[body_of(p.w)];
    const uint32_t mbits = acts_on_bits(cls);
    const int nx = A.ng_n[0], ny = A.ng_n[1], nz = A.ng_n[2];
    const int cx = cell_coord(p.x, A.ng_o[0], A.ng_inv, nx);
    const int cy = cell_coord(p.y, A.ng_o[1], A.ng_inv, ny);
    const int cz = cell_coord(p.z, A.ng_o[2], A.ng_inv, nz);
    int cnt = 0, cand = 0;
    for (int z = max(cz - 1, 0); z <= min(cz + 1, nz - 1); z++)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, ny - 1); y++) {
            const uint32_t row = A.key_base + (uint32_t)nx * grid_row(A, y, z);
            uint32_t s, e;
            cells_slots(fstart, row, max(cx - 1, 0), min(cx + 1, nx - 1), s, e);
            if (e > s) cand += (int)(e - s);
            for (uint32_t j = s; j < e; j++) {
                const float4 q = pos_s[j];
                const float r2 = dist2_rn(p.x - q.x, p.y - q.y, p.z - q.z);
                if (r2 < A.R2 && (int64_t)j != k && (mbits & __float_as_uint(q.w)) != 0u) cnt++;
            }
        }
    if (count_s) count_s[k] = cnt;
    if (cand_s) cand_s[k] = is_mobile(cls, A) && !is_ghost(p.w) ? cand : 0;
}

// ---- A6 helpers -------------------------------------------------------------

// closest point on a triangle by barycentric regions (Ericson, Real-Time
// Collision Detection, 2005); region 0 face, 1 + k edge (v_k, v_k+1),
// 4 + k vertex k
__device__ inline float3 closest_on_triangle(float3 p, float3 a, float3 b, float3 c, int &region) {
    const float3 ab = b - a, ac = c - a, ap = p - a;
    const float d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) {
        region = 4;
        return a;
    }
    const float3 bp = p - b;
    const float d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.f && d4 <= d3) {
        region = 5;
        return b;
    }
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        region = 1;
        return a + (d1 / (d1 - d3)) * ab;
    }
    const float3 cp = p - c;
    const float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.f && d5 <= d6) {
        region = 6;
        return c;
    }
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        region = 3;
        return a + (d2 / (d2 - d6)) * ac;
    }
    const float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        region = 2;
        return b + ((d4 - d3) / ((d4 - d3) + (d5 - d6))) * (c - b);
    }
    const float den = 1.f / (va + vb + vc);
    region = 0;
    return a + (vb * den) * ab + (vc * den) * ac;
}

// Warp-cooperative search of the 27 triangle cells around y (every lane
// holds the same y).  Lane c < 27 owns cell c of the block: its occupancy
// bit, its hash lookup (Eq. 10) and its triangles; the warp then reduces to
// the overall best with ties to the lower triangle index, so the choice is
// the same as a serial scan of the 27 cells.
//   surface: smallest |plane distance| among triangles whose foot is inside
//            (edge functions >= 0); returns the triangle or -1
//   volume:  closest triangle; returns inside (sign of (y - c) . psi <= 0)
//            or true when no triangle is near
struct CellRange {
    uint32_t beg, len;
};

__device__ inline CellRange lane_cell(const MeshView &M, const AsmParams &A, float3 y, int lane) {
    CellRange r{0u, 0u};
    if (lane >= 27) return r;
    const int x = cell_coord(y.x, A.tg_o[0], A.tg_inv, A.tg_n[0]) + lane % 3 - 1;
    const int yy = cell_coord(y.y, A.tg_o[1], A.tg_inv, A.tg_n[1]) + (lane / 3) % 3 - 1;
    const int z = cell_coord(y.z, A.tg_o[2], A.tg_inv, A.tg_n[2]) + lane / 9 - 1;
    if (x < 0 || yy < 0 || z < 0 || x >= A.tg_n[0] || yy >= A.tg_n[1] || z >= A.tg_n[2]) return r;
    if (!test_bit(M.occ, A.occ_off, tri_key(A, x, yy, z))) return r;
    tri_cell(M, A, x, yy, z, r.beg, r.len);
    return r;
}

// lexicographic (value, index) minimum over the warp; every lane gets it
__device__ inline void warp_argmin(float &v, int &t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int ot = __shfl_xor_sync(0xffffffffu, t, o);
        if (ov < v || (ov == v && ot < t)) {
            v = ov;
            t = ot;
        }
    }
}

// The candidate triangles of the 27 cells are gathered into a per-warp list
// in shared memory (an exclusive scan of the cells' list lengths gives each
// cell its place), then all 32 lanes test the list together.  A list longer
// than the buffer is tested by the lanes cell by cell instead.
constexpr int kSearchBuf = 160;   // triangle ids per warp

__device__ inline int gather_candidates(const MeshView &M, const CellRange r, int32_t *buf) {
    const int lane = threadIdx.x & 31;
    uint32_t off = r.len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, off, 31);
    off -= r.len;
    if (total <= (uint32_t)kSearchBuf)
        for (uint32_t q = 0; q < r.len; q++) buf[off + q] = M.tlist[r.beg + q];
    __syncwarp();
    return (int)total;
}

template <typename Test>
__device__ inline void for_candidates(const MeshView &M, const CellRange r, int32_t *buf, Test &&test) {
    const int lane = threadIdx.x & 31;
    const int total = gather_candidates(M, r, buf);
    if (total <= kSearchBuf) {
        for (int q = lane; q < total; q += 32) test(buf[q]);
    } else {
        for (uint32_t e = r.beg; e < r.beg + r.len; e++) test(M.tlist[e]);
    }
    __syncwarp();
}

// Surface candidate test: the foot of y on the plane of triangle t lies
// inside it (every in-plane edge distance >= -edge_tol: Fig. 8 with a
// tolerance, so a foot on a shared edge belongs to both triangles); *d gets
// the signed plane distance
__device__ inline bool surface_candidate(const MeshView &M, const AsmParams &A, int t, float3 y, float &d) {
    const float4 *g = M.geo + 5 * (size_t)(A.tri_off + t);
    const float3 u = y - f3(g[0]);
    const float tol = -A.edge_tol;
    const float4 m0 = g[2];
    if (dot3(u, f3(m0)) < tol) return false;
    const float4 m1 = g[3];
    if (dot3(u, f3(m1)) - m1.w < tol) return false;
    const float4 m2 = g[4];
    if (dot3(u, f3(m2)) - m2.w < tol) return false;
    d = dot3(u, f3(g[1]));
    return true;
}

// The same decision, with every edge evaluated: *emin gets the smallest
// in-plane edge distance of the foot (negative outside), so a triangle that
// is not projectable at y stays so within -emin - edge_tol of y (the edge
// distances are 1-Lipschitz in y: unit in-plane edge normals)
__device__ inline bool surface_candidate_margin(const MeshView &M, const AsmParams &A, int t, float3 y, float &d,
                                                float &emin) {
    const float4 *g = M.geo + 5 * (size_t)(A.tri_off + t);
    const float3 u = y - f3(g[0]);
    const float tol = -A.edge_tol;
    const float4 m0 = g[2], m1 = g[3], m2 = g[4];
    const float e0 = dot3(u, f3(m0));
    const float e1 = dot3(u, f3(m1)) - m1.w;
    const float e2 = dot3(u, f3(m2)) - m2.w;
    emin = fminf(e0, fminf(e1, e2));
    if (e0 < tol || e1 < tol || e2 < tol) return false;
    d = dot3(u, f3(g[1]));
    return true;
}

// Surface certificate (not in the paper; it changes no decision): when
// exactly one candidate is projectable at y, every other candidate of y's
// triangle cell stays non-projectable within the smallest -emin - edge_tol
// over them, so for a trial point in the same cell and within that radius
// the choice is the particle's own triangle if it is projectable there, and
// the step takes it without the search.  Radius shrunk by 2^-10 relative and
// 2^-12 dx for the FP32 rounding of the edge distances; 0: no certificate.
__device__ inline float surface_cert_radius(const AsmParams &A, int n_projectable, float r_other) {
    if (n_projectable != 1 || !(r_other < FLT_MAX)) return 0.f;
    return fmaxf(r_other * (1.f - 0x1p-10f) - A.dx * 0x1p-12f, 0.f);
}

// closest projectable triangle (smallest |plane distance|, ties to the lower
// index) among those binned into the 27 cells around y, or into y's own
// cell alone (own_cell); -1 when none
// The candidate triangles of the 27 cells around y's cell from that cell's
// list (built with the mesh: the distinct triangles of the 27 cells): 1 with
// [beg, end) into M.cand; 2 when the list was too long to build (probe the
// cells); 0 when no triangle lies in the 27 cells.  Warp-uniform.
// The same as a range of triangle cell c: [beg, end) into M.cand, (0, 0)
// for no triangle, (kProbeCells, kProbeCells) for a list too long to build.
// The step computes it for every particle it queues, so that the search
// starts from the list instead of the chain bitmap -> rank -> list start.
constexpr uint32_t kProbeCells = 0xffffffffu;

__device__ inline uint2 cand_range(const MeshView &M, const AsmParams &A, uint32_t c) {
    const uint32_t w = M.occ[A.dil_off + (c >> 5)];
    if (!((w >> (c & 31u)) & 1u)) return make_uint2(0u, 0u);
    const uint32_t r = M.drank[A.drank_off + (c >> 5)] + __popc(w & ((1u << (c & 31u)) - 1u));
    const uint32_t o0 = M.coff[A.coff_off + r], o1 = M.coff[A.coff_off + r + 1];
    if (o0 >> 31) return make_uint2(kProbeCells, kProbeCells);
    return make_uint2(A.cand_off + o0, A.cand_off + (o1 & 0x7fffffffu));
}

__device__ inline uint32_t tri_cell_of(const AsmParams &A, float3 y) {
    return tri_key(A, cell_coord(y.x, A.tg_o[0], A.tg_inv, A.tg_n[0]), cell_coord(y.y, A.tg_o[1], A.tg_inv, A.tg_n[1]),
                   cell_coord(y.z, A.tg_o[2], A.tg_inv, A.tg_n[2]));
}

// pre: the range of y's cell when the caller has it (nullptr: look it up)
__device__ inline int cell_candidates(const MeshView &M, const AsmParams &A, float3 y, uint32_t &beg, uint32_t &end,
                                      const uint2 *pre = nullptr) {
    const uint2 r = pre ? *pre : cand_range(M, A, tri_cell_of(A, y));
    if (r.x == kProbeCells) return 2;
    if (r.y <= r.x) return 0;
    beg = r.x;
    end = r.y;
    return 1;
}

// every candidate triangle of the 27 cells around y, spread over the lanes
template <typename Test>
__device__ inline void for_27_candidates(const MeshView &M, const AsmParams &A, float3 y, int32_t *buf,
                                         Test &&test, const uint2 *pre = nullptr) {
    const int lane = threadIdx.x & 31;
    uint32_t beg = 0, end = 0;
    const int kind = cell_candidates(M, A, y, beg, end, pre);
    auto checked = [&](int t) {
        if (FPPG_CHECK(t >= 0 && t < A.nt, kChkTri)) test(t);
    };
    if (kind == 1) {
        for (uint32_t q = beg + lane; q < end; q += 32) checked(M.cand[q]);
    } else if (kind == 2) {
        const CellRange r = lane_cell(M, A, y, lane);
        for_candidates(M, r, buf, checked);
    }
}

__device__ int warp_project_surface(const MeshView &M, const AsmParams &A, float3 y, float &dist, int32_t *buf,
                                    bool own_cell = false, const uint2 *pre = nullptr, float *cert_r = nullptr) {
    const int lane = threadIdx.x & 31;
    float best = FLT_MAX;
    int bt = 0x7fffffff;
    float bd = 0.f;
    int nproj = 0;
    float rother = FLT_MAX;
    auto test = [&](int t) {
        float d;
        if (cert_r) {
            float emin;
            if (!surface_candidate_margin(M, A, t, y, d, emin)) {
                rother = fminf(rother, -emin - A.edge_tol);
                return;
            }
            nproj++;
        } else if (!surface_candidate(M, A, t, y, d)) {
            return;
        }
        const float ad = fabsf(d);
        if (ad < best || (ad == best && t < bt)) {
            best = ad;
            bt = t;
            bd = d;
        }
    };
    if (own_cell) {
        // the cell that holds y alone: lane 13 probes the centre cell
        CellRange r = lane_cell(M, A, y, lane);
        if (lane != 13) r = CellRange{0u, 0u};
        for_candidates(M, r, buf, test);
    } else {
        for_27_candidates(M, A, y, buf, test, pre);
    }
    float v = best;
    int t = bt;
    warp_argmin(v, t);
    // the signed distance of the winner, from a lane that holds it
    const uint32_t own = __ballot_sync(0xffffffffu, bt == t && best == v);
    dist = __shfl_sync(0xffffffffu, bd, own ? __ffs(own) - 1 : 0);
    if (cert_r) {
        const int total = __reduce_add_sync(0xffffffffu, nproj);
        float r = rother;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fminf(r, __shfl_xor_sync(0xffffffffu, r, o));
        *cert_r = surface_cert_radius(A, total, r);
    }
    return t == 0x7fffffff ? -1 : t;
}

// Surface re-projection of trial point y of a particle on triangle c: the
// closest projectable triangle over the 27 cells, or with A.cascade the
// cascade of Sec. 3.3.3 (still on triangle c: stay; else the closest
// projectable one of y's own cell; else over the 27 cells).  -1: revert.
__device__ int warp_surface_choice(const MeshView &M, const AsmParams &A, float3 y, int c, float &dist,
                                   int32_t *buf, const uint2 *pre = nullptr, float *cert_r = nullptr) {
    if (A.cascade) {
        if (c >= 0 && c < A.nt) {
            float d = 0.f;
            const bool on = surface_candidate(M, A, c, y, d);   // every lane, same answer
            if (on) {
                dist = d;
                return c;
            }
        }
        const int t = warp_project_surface(M, A, y, dist, buf, true);
        if (t >= 0) return t;
    }
    return warp_project_surface(M, A, y, dist, buf, false, pre, A.cascade ? nullptr : cert_r);
}

// distance from y to the faces of the 3 x 3 x 3 triangle-cell block around
// its cell (0 when y lies outside the grid): no triangle outside the block
// comes closer than this
__device__ inline float block_margin(const AsmParams &A, float3 y) {
    const float v[3] = {y.x, y.y, y.z};
    float m = FLT_MAX;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float t = __fmul_rn(__fsub_rn(v[k], A.tg_o[k]), A.tg_inv);
        const float c = (float)cell_coord(v[k], A.tg_o[k], A.tg_inv, A.tg_n[k]);
        m = fminf(m, fminf(t - (c - 1.f), (c + 2.f) - t));
    }
    return fmaxf(m, 0.f) / A.tg_inv;
}

// Closest-feature sign (reading: closest point over the 27 triangle cells,
// sign of the angle-weighted pseudonormal): 1 inside, 0 outside, -1 when no
// triangle lies in range.  *clear gets a lower bound of the distance from y
// to the surface, valid when inside.
__device__ int warp_closest_sign(const MeshView &M, const AsmParams &A, float3 y, int32_t *buf, float &clear,
                                 const uint2 *pre = nullptr) {
    const int lane = threadIdx.x & 31;
    float best = FLT_MAX;
    int bt = 0x7fffffff, breg = 0;
    float3 bcp = make_float3(0.f, 0.f, 0.f);
    for_27_candidates(M, A, y, buf, [&](int t) {
        const size_t g = (size_t)(A.tri_off + t);
        const float3 n = f3(M.geo[5 * g + 1]);
        if (n.x == 0.f && n.y == 0.f && n.z == 0.f) return;   // degenerate
        int reg;
        const float3 cp = closest_on_triangle(y, f3(M.vx[3 * g]), f3(M.vx[3 * g + 1]), f3(M.vx[3 * g + 2]), reg);
        const float3 w = y - cp;
        const float dd = dot3(w, w);
        if (dd < best || (dd == best && t < bt)) {
            best = dd;
            bt = t;
            breg = reg;
            bcp = cp;
        }
    }, pre);
    float v = best;
    int t = bt;
    warp_argmin(v, t);
    const float blk = block_margin(A, y);
    clear = fmaxf(fminf(t == 0x7fffffff ? FLT_MAX : sqrtf(v), blk) * (1.f - 0x1p-10f) - A.dx * 0x1p-16f, 0.f);
    if (t == 0x7fffffff) return -1;
    const uint32_t own = __ballot_sync(0xffffffffu, bt == t && best == v);
    const int src = __ffs(own) - 1;
    int inside = 0;
    if (lane == src) {
        const size_t g = (size_t)(A.tri_off + bt);
        const float3 psi = breg == 0 ? f3(M.geo[5 * g + 1]) : f3(M.pn[6 * g + breg - 1]);
        inside = dot3(y - bcp, psi) <= 0.f;
    }
    return __shfl_sync(0xffffffffu, inside, src);
}

// Volume test of a particle of the body: the closest-feature sign, inside
// when no triangle is in range (a step is below a cell)
__device__ inline bool warp_volume_inside(const MeshView &M, const AsmParams &A, float3 y, int32_t *buf,
                                          float &clear, const uint2 *pre = nullptr) {
    return warp_closest_sign(M, A, y, buf, clear, pre) != 0;
}

// Boolean partner rule (1 stay outside, 2 stay inside, 0 none) for point x:
// with no partner triangle in range the particle is where it started
__device__ inline bool warp_partner_ok(const MeshView &M, const AsmParams &Q, int rule, float3 x, int32_t *buf) {
    if (rule == 0) return true;
    float unused;
    const int t = warp_closest_sign(M, Q, x, buf, unused);
    return rule == 1 ? t != 1 : t != 0;
}

// closest point of the particle's feature line (all lines of the body when
// it has none yet); ties to the lower segment
__device__ bool project_feature(const MeshView &M, const AsmParams &A, float3 y, int cons, float3 &x, int &seg) {
    if (A.nseg <= 0) return false;
    int s0 = 0, s1 = A.nseg;
    if (cons >= 0 && cons < A.nseg) {
        const int line = __float_as_int(M.seg[3 * (size_t)(A.seg_off + cons)].w);
        const int2 L = M.lines[A.line_off + line];
        s0 = L.x;
        s1 = L.x + L.y;
    }
    float best = FLT_MAX;
    int bs = -1;
    float3 bq = y;
    for (int s = s0; s < s1; s++) {
        const float4 *sg = M.seg + 3 * (size_t)(A.seg_off + s);
        const float3 a = f3(sg[0]), e = f3(sg[1]) - a;
        const float ee = dot3(e, e);
        float t = ee > 0.f ? dot3(y - a, e) / ee : 0.f;
        t = fminf(fmaxf(t, 0.f), 1.f);
        const float3 q = a + t * e;
        const float3 w = y - q;
        const float dd = dot3(w, w);
        if (dd < best) {
            best = dd;
            bs = s;
            bq = q;
        }
    }
    x = bq;
    seg = bs;
    return bs >= 0;
}

// some triangle of body Q within the 27 triangle cells of x (its dilated
// occupancy bit)
__device__ inline bool near_body(const MeshView &M, const AsmParams &Q, float3 x) {
    return test_bit(M.occ, Q.dil_off,
                    tri_key(Q, cell_coord(x.x, Q.tg_o[0], Q.tg_inv, Q.tg_n[0]),
                            cell_coord(x.y, Q.tg_o[1], Q.tg_inv, Q.tg_n[1]),
                            cell_coord(x.z, Q.tg_o[2], Q.tg_inv, Q.tg_n[2])));
}

// ---- A5 + A6 -------------------------------------------------------------------
// k_step: one thread per particle (key order): the limited step and its
// tangential part, then the cases that need no triangle search -- feature
// particles (their own line), volume particles with no triangle in the 27
// cells (accepted), surface particles with none (reverted).  Every other
// particle is queued with its trial point for k_search.
__global__ void __launch_bounds__(TPB, 5) k_step(const float4 *__restrict__ pos_s, const float4 *__restrict__ acc_s,
                                              const uint32_t *__restrict__ id_s, int64_t N,
                                              const AsmParams *__restrict__ P, const uint32_t *__restrict__ amax,
                                              float4 *__restrict__ pos, int32_t *__restrict__ cons, MeshView M,
                                              uint32_t *__restrict__ maxdisp, int4 *__restrict__ work,
                                              uint2 *__restrict__ work_r, uint32_t *__restrict__ work_count,
                                              const float4 *__restrict__ cert, const int32_t *__restrict__ cons_s) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    const bool active = k < N;
    // the particle's streams are read together, before its class is known
    // (one round trip to memory instead of two)
    const float4 p = active ? pos_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 a = active ? acc_s[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t i = active ? id_s[k] : 0u;
    const int c = active ? cons_s[k] : -1;
    const int cls = active ? cls_of(p.w) : kClsI;
    const int b = active ? body_of(p.w) : 0;
    const AsmParams &A = P[b];
    float disp = 0.f;
    bool queue = false;
    uint2 rng = make_uint2(0u, 0u);   // candidate list of the trial point's triangle cell
    float3 y = f3(p);
    if (active && is_mobile(cls, A) && !is_ghost(p.w)) {
        const float am = __uint_as_float(amax[A.amax_slot]);
        const float sc = am > 0.f ? A.step_h / am : 0.f;     // dt^2 with dt = 0.25 sqrt(h / amax)
        float3 dr = make_float3(a.x * sc, a.y * sc, a.z * sc);
        if (cls == kClsS && c >= 0 && c < A.nt) {
            const float3 n = f3(M.geo[5 * (size_t)(A.tri_off + c) + 1]);
            dr = dr - dot3(dr, n) * n;
        } else if (cls == kClsF && c >= 0 && c < A.nseg) {
            const float3 tau = f3(M.seg[3 * (size_t)(A.seg_off + c) + 2]);
            dr = dot3(dr, tau) * tau;
        }
        const float3 p3 = f3(p);
        y = p3 + dr;
        if (cls == kClsF) {
            float3 x;
            int cn;
            if (project_feature(M, A, y, c, x, cn)) {
                // a partner's triangles within reach: the search tests that
                // partner's rule on the projection (a particle on the
                // intersection curve with a partner lies on both surfaces:
                // no rule of that partner)
                bool near_partner = false;
                for (int q = 0; q < A.npart && !near_partner; q++)
                    if (A.partner_surf[q] != 0 && !(cn >= A.curve_lo[q] && cn < A.curve_hi[q]))
                        near_partner = near_body(M, P[A.partner[q]], x);
                if (near_partner) {
                    queue = true;
                } else {
                    pos[i] = make_float4(x.x, x.y, x.z, p.w);
                    cons[i] = cn;
                    const float3 w = x - p3;
                    disp = sqrtf(dot3(w, w));
                }
            }
        } else {
            const int cx = cell_coord(y.x, A.tg_o[0], A.tg_inv, A.tg_n[0]);
            const int cy = cell_coord(y.y, A.tg_o[1], A.tg_inv, A.tg_n[1]);
            const int cz = cell_coord(y.z, A.tg_o[2], A.tg_inv, A.tg_n[2]);
            bool certified = false;
            bool near_partner = false;
            // some triangle of the body within the 27 triangle cells of y
            const bool near_own = test_bit(M.occ, A.dil_off, tri_key(A, cx, cy, cz));
            if (cls == kClsV && A.vol_rules) {
                for (int q = 0; q < A.npart && !near_partner; q++)
                    if (A.partner_vol[q] != 0) near_partner = near_body(M, P[A.partner[q]], y);
            } else if (cls == kClsV && A.closed && near_own) {
                // (with no triangle near, the volume test accepts anyway: the
                // certificate is not read)
                // inside a ball that an earlier search found free of surface
                // and inside the body: the volume test would accept
                const float4 cc = cert[i];
                const float3 w = y - f3(cc);
                certified = cc.w > 0.f && sqrtf(dot3(w, w)) + cc.w * 0x1p-6f + A.dx * 0x1p-10f < cc.w;
            }
            bool surf_cert = false;
            float3 xs = y;
            if (cls == kClsS && c >= 0 && c < A.nt && !A.cascade) {
                // inside a ball where an earlier search found exactly one
                // projectable candidate of the same triangle cell: the own
                // triangle is the choice when it is projectable here, and lies
                // this close (so it is a candidate of this cell); with no
                // Boolean partner's triangle near the foot the partner rules
                // hold as they would in the search
                const float4 cc = cert[i];
                const float3 w = y - f3(cc);
                if (cc.w < 0.f && sqrtf(dot3(w, w)) < -cc.w &&
                    tri_key(A, cell_coord(cc.x, A.tg_o[0], A.tg_inv, A.tg_n[0]),
                            cell_coord(cc.y, A.tg_o[1], A.tg_inv, A.tg_n[1]),
                            cell_coord(cc.z, A.tg_o[2], A.tg_inv, A.tg_n[2])) == tri_key(A, cx, cy, cz)) {
                    float d;
                    if (surface_candidate(M, A, c, y, d) && fabsf(d) <= A.dx * 0x1p-10f) {
                        surf_cert = true;
                        xs = y - d * f3(M.geo[5 * (size_t)(A.tri_off + c) + 1]);
                        for (int q = 0; q < A.npart && surf_cert; q++)
                            if (A.partner_surf[q] != 0 && near_body(M, P[A.partner[q]], xs)) surf_cert = false;
                    }
                }
            }
            if (certified) {
                pos[i] = make_float4(y.x, y.y, y.z, p.w);
                disp = sqrtf(dot3(dr, dr));
            } else if (surf_cert) {
                pos[i] = make_float4(xs.x, xs.y, xs.z, p.w);
                const float3 w = xs - p3;
                disp = sqrtf(dot3(w, w));
            } else if (near_partner || near_own) {
                queue = true;
                rng = cand_range(M, A, tri_key(A, cx, cy, cz));
            } else if (cls == kClsV) {       // nothing near: inside, accept
                pos[i] = make_float4(y.x, y.y, y.z, p.w);
                disp = sqrtf(dot3(dr, dr));
            }                                // S with nothing near: revert
        }
    }
    // warp-aggregated append to the search queue: surface and feature
    // particles from the front (count work_count[0]), volume particles from
    // the back (work_count[1]), so that a warp of the thread-per-particle
    // search meets one kind of test
    const bool qv = queue && cls == kClsV, qs = queue && cls != kClsV;
    const uint32_t ms = __ballot_sync(0xffffffffu, qs), mv = __ballot_sync(0xffffffffu, qv);
    if (ms | mv) {
        const int lane = threadIdx.x & 31;
        const int ls = ms ? __ffs(ms) - 1 : 0, lv = mv ? __ffs(mv) - 1 : 0;
        uint32_t bs = 0u, bv = 0u;
        if (ms && lane == ls) bs = atomicAdd(work_count, (uint32_t)__popc(ms));
        if (mv && lane == lv) bv = atomicAdd(work_count + 1, (uint32_t)__popc(mv));
        bs = __shfl_sync(0xffffffffu, bs, ls);
        bv = __shfl_sync(0xffffffffu, bv, lv);
        const int4 it = make_int4((int)k, __float_as_int(y.x), __float_as_int(y.y), __float_as_int(y.z));
        if (qs) {
            const uint32_t q = bs + __popc(ms & lanemask_lt());
            if (FPPG_CHECK(q < N, kChkQueue)) {
                work[q] = it;
                work_r[q] = rng;
            }
        }
        if (qv) {
            const int64_t q = N - 1 - (int64_t)(bv + __popc(mv & lanemask_lt()));
            if (FPPG_CHECK(q >= 0 && q < N, kChkQueue)) {
                work[q] = it;
                work_r[q] = rng;
            }
        }
    }
    __shared__ int s_lab[TPB / 32];
    __shared__ uint32_t s_max[TPB / 32];
    block_labelled_max<TPB / 32>(maxdisp, b, disp, s_lab, s_max);
}

// entry e of the two-ended search queue: the nf front entries first, then
// the back ones from slot N - 1 downwards
__device__ inline int64_t queue_slot(uint32_t nf, int64_t N, uint32_t e) {
    return e < nf ? (int64_t)e : N - 1 - (int64_t)(e - nf);
}


// k_search: one warp per queued particle (grid-stride over the queue):
// surface particles go to the closest projectable triangle or revert,
// volume particles are accepted when the pseudonormal sign says inside.
__global__ void __launch_bounds__(TPB) k_search(const float4 *__restrict__ pos_s,
                                                const uint32_t *__restrict__ id_s,
                                                const AsmParams *__restrict__ P, float4 *__restrict__ pos,
                                                int32_t *__restrict__ cons, MeshView M,
                                                uint32_t *__restrict__ maxdisp, const int4 *__restrict__ work,
                                                const uint2 *__restrict__ work_r,
                                                const uint32_t *__restrict__ work_count, int64_t N,
                                                float4 *__restrict__ cert) {
    __shared__ int32_t sbuf[TPB / 32][kSearchBuf];
    int32_t *buf = sbuf[threadIdx.x / 32];
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (TPB / 32);
    const uint32_t nf = work_count[0], n = nf + work_count[1];
    // lane 0's running max move of body run_b, added when the body changes
    // (the queue is in key order, so a warp meets few bodies)
    int run_b = -1;
    uint32_t run = 0u;
    for (uint32_t e = (blockIdx.x * TPB + threadIdx.x) / 32; e < n; e += warps) {
        const int64_t qs = queue_slot(nf, N, e);
        if (!FPPG_CHECK(qs >= 0 && qs < N, kChkQueue)) continue;
        const int4 it = work[qs];
        const uint2 rng = work_r[qs];
        if (!FPPG_CHECK(it.x >= 0 && it.x < N, kChkEntry)) continue;
        const float3 y = make_float3(__int_as_float(it.y), __int_as_float(it.z), __int_as_float(it.w));
        const float4 p = pos_s[it.x];
        const int cls = cls_of(p.w), b = body_of(p.w);
        const AsmParams &A = P[b];
        float3 x = y;
        int tri = -2;
        float clear = 0.f;
        bool ok;
        if (cls == kClsS) {
            float d;
            tri = warp_surface_choice(M, A, y, A.cascade ? cons[id_s[it.x]] : -1, d, buf, &rng, &clear);
            ok = tri >= 0;
            if (ok) x = y - d * f3(M.geo[5 * (size_t)(A.tri_off + tri) + 1]);
        } else if (cls == kClsF) {
            // a feature particle of a union member near the partner: its
            // projection again, then the partner test below
            int cn = -1, okf = 0;
            if (lane == 0) okf = project_feature(M, A, y, cons[id_s[it.x]], x, cn) ? 1 : 0;
            okf = __shfl_sync(0xffffffffu, okf, 0);
            x = make_float3(__shfl_sync(0xffffffffu, x.x, 0), __shfl_sync(0xffffffffu, x.y, 0),
                            __shfl_sync(0xffffffffu, x.z, 0));
            tri = __shfl_sync(0xffffffffu, cn, 0);
            ok = okf != 0;
        } else {
            ok = warp_volume_inside(M, A, y, buf, clear, &rng);
        }
        // Boolean operations: the partner rule of the particle's class
        for (int q = 0; q < A.npart && ok; q++)
            if (!(cls == kClsF && tri >= A.curve_lo[q] && tri < A.curve_hi[q]))
                ok = warp_partner_ok(M, P[A.partner[q]], cls == kClsV ? A.partner_vol[q] : A.partner_surf[q], x,
                                     buf);
        if (ok && lane == 0) {
            const uint32_t i = id_s[it.x];
            pos[i] = make_float4(x.x, x.y, x.z, p.w);
            if (tri >= 0) cons[i] = tri;
            if (cls == kClsV && A.closed && !A.vol_rules) cert[i] = make_float4(y.x, y.y, y.z, clear);
            // surface certificates carry a negative radius (never taken for an inside one)
            if (cls == kClsS && clear > 0.f) cert[i] = make_float4(y.x, y.y, y.z, -clear);
            const float3 w = x - f3(p);
            if (b != run_b) {
                if (run) atomicMax(maxdisp + run_b, run);
                run_b = b;
                run = 0u;
            }
            run = max(run, __float_as_uint(sqrtf(dot3(w, w))));
        }
    }
    if (lane == 0 && run) atomicMax(maxdisp + run_b, run);
}

// ---- the same search, one thread per queued particle --------------------------
// Each thread walks its particle's candidate list alone: no lanes idle on a
// short list, and 32 particles' dependent loads are in flight per warp.
// The candidate set and the comparisons (smallest distance, ties to the
// lower index) are those of the warp form, so the choices are identical.

// every candidate triangle of the 27 cells around y, one after another
template <typename Test>
__device__ inline void each_27_candidate(const MeshView &M, const AsmParams &A, float3 y, Test &&test,
                                         const uint2 *pre = nullptr) {
    uint32_t beg = 0, end = 0;
    const int kind = cell_candidates(M, A, y, beg, end, pre);
    auto checked = [&](int t) {
        if (FPPG_CHECK(t >= 0 && t < A.nt, kChkTri)) test(t);
    };
    if (kind == 1) {
        for (uint32_t q = beg; q < end; q++) checked(M.cand[q]);
    } else if (kind == 2) {
        for (int c = 0; c < 27; c++) {
            const CellRange r = lane_cell(M, A, y, c);
            for (uint32_t e = r.beg; e < r.beg + r.len; e++) checked(M.tlist[e]);
        }
    }
}

__device__ int thread_project_surface(const MeshView &M, const AsmParams &A, float3 y, float &dist,
                                      bool own_cell = false, const uint2 *pre = nullptr, float *cert_r = nullptr) {
    float best = FLT_MAX, bd = 0.f;
    int bt = 0x7fffffff;
    int nproj = 0;
    float rother = FLT_MAX;
    auto test = [&](int t) {
        float d;
        if (cert_r) {
            float emin;
            if (!surface_candidate_margin(M, A, t, y, d, emin)) {
                rother = fminf(rother, -emin - A.edge_tol);
                return;
            }
            nproj++;
        } else if (!surface_candidate(M, A, t, y, d)) {
            return;
        }
        const float ad = fabsf(d);
        if (ad < best || (ad == best && t < bt)) {
            best = ad;
            bt = t;
            bd = d;
        }
    };
    if (own_cell) {
        const CellRange r = lane_cell(M, A, y, 13);   // the centre cell
        for (uint32_t e = r.beg; e < r.beg + r.len; e++) test(M.tlist[e]);
    } else {
        each_27_candidate(M, A, y, test, pre);
    }
    dist = bd;
    if (cert_r) *cert_r = surface_cert_radius(A, nproj, rother);
    return bt == 0x7fffffff ? -1 : bt;
}

__device__ int thread_surface_choice(const MeshView &M, const AsmParams &A, float3 y, int c, float &dist,
                                     const uint2 *pre = nullptr, float *cert_r = nullptr) {
    if (A.cascade) {
        if (c >= 0 && c < A.nt) {
            float d = 0.f;
            if (surface_candidate(M, A, c, y, d)) {
                dist = d;
                return c;
            }
        }
        const int t = thread_project_surface(M, A, y, dist, true);
        if (t >= 0) return t;
    }
    return thread_project_surface(M, A, y, dist, false, pre, A.cascade ? nullptr : cert_r);
}

__device__ int thread_closest_sign(const MeshView &M, const AsmParams &A, float3 y, float &clear,
                                   const uint2 *pre = nullptr) {
    float best = FLT_MAX;
    int bt = 0x7fffffff, breg = 0;
    float3 bcp = make_float3(0.f, 0.f, 0.f);
    each_27_candidate(M, A, y, [&](int t) {
        const size_t g = (size_t)(A.tri_off + t);
        const float3 n = f3(M.geo[5 * g + 1]);
        if (n.x == 0.f && n.y == 0.f && n.z == 0.f) return;   // degenerate
        int reg;
        const float3 cp = closest_on_triangle(y, f3(M.vx[3 * g]), f3(M.vx[3 * g + 1]), f3(M.vx[3 * g + 2]), reg);
        const float3 w = y - cp;
        const float dd = dot3(w, w);
        if (dd < best || (dd == best && t < bt)) {
            best = dd;
            bt = t;
            breg = reg;
            bcp = cp;
        }
    }, pre);
    const float blk = block_margin(A, y);
    clear = fmaxf(fminf(bt == 0x7fffffff ? FLT_MAX : sqrtf(best), blk) * (1.f - 0x1p-10f) - A.dx * 0x1p-16f, 0.f);
    if (bt == 0x7fffffff) return -1;
    const size_t g = (size_t)(A.tri_off + bt);
    const float3 psi = breg == 0 ? f3(M.geo[5 * g + 1]) : f3(M.pn[6 * g + breg - 1]);
    return dot3(y - bcp, psi) <= 0.f ? 1 : 0;
}

__device__ inline bool thread_partner_ok(const MeshView &M, const AsmParams &Q, int rule, float3 x) {
    if (rule == 0) return true;
    float unused;
    const int t = thread_closest_sign(M, Q, x, unused);
    return rule == 1 ? t != 1 : t != 0;
}

// k_search_thread: one thread per queued particle; the warps stride over the
// queue together so that the per-body max move is reduced once per warp.
// At most 64 registers (four blocks, 32 warps per SM): the kernel waits on
// dependent loads, and more particles in flight hide more of them (at 75
// registers and 24 warps it took 0.509 against 0.441 ms per iteration on
// the vehicle shell)
__global__ void __launch_bounds__(TPB, 4) k_search_thread(const float4 *__restrict__ pos_s,
                                                       const uint32_t *__restrict__ id_s,
                                                       const AsmParams *__restrict__ P, float4 *__restrict__ pos,
                                                       int32_t *__restrict__ cons, MeshView M,
                                                       uint32_t *__restrict__ maxdisp,
                                                       const int4 *__restrict__ work,
                                                       const uint2 *__restrict__ work_r,
                                                       const uint32_t *__restrict__ work_count, int64_t N,
                                                       float4 *__restrict__ cert) {
    const uint32_t nf = work_count[0], n = nf + work_count[1];
    const uint32_t stride = gridDim.x * TPB;
    // this thread's running max move of body run_b, added when the body
    // changes and once at the end (the queue is in key order: few changes)
    int run_b = 0;
    float run = 0.f;
    for (uint32_t e0 = blockIdx.x * TPB + (threadIdx.x & ~31u); e0 < n; e0 += stride) {
        const uint32_t e = e0 + (threadIdx.x & 31u);
        int b = 0;
        float disp = 0.f;
        if (e < n) {
            const int64_t qs = queue_slot(nf, N, e);
            const bool entry_ok = FPPG_CHECK(qs >= 0 && qs < N, kChkQueue) &&
                                  FPPG_CHECK(work[qs].x >= 0 && work[qs].x < N, kChkEntry);
            if (!entry_ok) continue;
            const int4 it = work[qs];
            const uint2 rng = work_r[qs];
            const float3 y = make_float3(__int_as_float(it.y), __int_as_float(it.z), __int_as_float(it.w));
            const float4 p = pos_s[it.x];
            const int cls = cls_of(p.w);
            b = body_of(p.w);
            const AsmParams &A = P[b];
            const uint32_t i = id_s[it.x];
            float3 x = y;
            int tri = -2;
            float clear = 0.f;
            bool ok;
            if (cls == kClsS) {
                float d;
                tri = thread_surface_choice(M, A, y, A.cascade ? cons[i] : -1, d, &rng, &clear);
                ok = tri >= 0;
                if (ok) x = y - d * f3(M.geo[5 * (size_t)(A.tri_off + tri) + 1]);
            } else if (cls == kClsF) {
                int cn = -1;
                ok = project_feature(M, A, y, cons[i], x, cn);
                tri = cn;
            } else {
                ok = thread_closest_sign(M, A, y, clear, &rng) != 0;
            }
            for (int q = 0; q < A.npart && ok; q++)
                if (!(cls == kClsF && tri >= A.curve_lo[q] && tri < A.curve_hi[q]))
                    ok = thread_partner_ok(M, P[A.partner[q]], cls == kClsV ? A.partner_vol[q] : A.partner_surf[q],
                                           x);
            if (ok) {
                pos[i] = make_float4(x.x, x.y, x.z, p.w);
                if (tri >= 0) cons[i] = tri;
                if (cls == kClsV && A.closed && !A.vol_rules) cert[i] = make_float4(y.x, y.y, y.z, clear);
                // surface certificates carry a negative radius (never taken for an inside one)
                if (cls == kClsS && clear > 0.f) cert[i] = make_float4(y.x, y.y, y.z, -clear);
                const float3 w = x - f3(p);
                disp = sqrtf(dot3(w, w));
            }
            if (b != run_b) {
                if (run > 0.f) atomicMax(maxdisp + run_b, __float_as_uint(run));
                run_b = b;
                run = 0.f;
            }
            run = fmaxf(run, disp);
        }
    }
    labelled_max(maxdisp, run_b, run);
}

// ---- diagnostics --------------------------------------------------------------
__global__ void k_unpermute(const float4 *__restrict__ acc_s, const uint32_t *__restrict__ id_s, int64_t N,
                            float *__restrict__ acc, const int32_t *__restrict__ cnt_s, int32_t *__restrict__ cnt) {
    int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    uint32_t i = id_s[k];
    if (acc) {
        float4 a = acc_s[k];
        acc[3 * (size_t)i] = a.x;
        acc[3 * (size_t)i + 1] = a.y;
        acc[3 * (size_t)i + 2] = a.z;
    }
    if (cnt) cnt[i] = cnt_s[k];
}

__global__ void k_project_points(const float *__restrict__ y, const int32_t *__restrict__ cls,
                                  const int32_t *__restrict__ cons_in, int64_t n, const AsmParams *__restrict__ P,
                                  MeshView M, float *__restrict__ x, int32_t *__restrict__ cons_out,
                                  int32_t *__restrict__ ok) {
    __shared__ int32_t sbuf[TPB / 32][kSearchBuf];
    int32_t *buf = sbuf[threadIdx.x / 32];
    const int64_t i = ((int64_t)blockIdx.x * TPB + threadIdx.x) / 32;   // one warp per point
    const int lane = threadIdx.x & 31;
    if (i >= n) return;                                                    // whole warp
    const AsmParams &A = P[0];
    const float3 yy = make_float3(y[3 * i], y[3 * i + 1], y[3 * i + 2]);
    float3 xx = yy;
    const int c = cons_in ? cons_in[i] : -1;
    int cn = c;
    bool r = true;
    const int cl = cls[i];
    if (cl == kClsS) {
        float d;
        const int t = warp_surface_choice(M, A, yy, c, d, buf);
        r = t >= 0;
        if (r) {
            xx = yy - d * f3(M.geo[5 * (size_t)(A.tri_off + t) + 1]);
            cn = t;
        }
    } else if (cl == kClsV) {
        float clear;
        r = warp_volume_inside(M, A, yy, buf, clear);
    } else if (cl == kClsF) {
        r = project_feature(M, A, yy, c, xx, cn);
    }
    if (!r) {
        xx = yy;
        cn = c;
    }
    if (lane == 0) {
        x[3 * i] = xx.x;
        x[3 * i + 1] = xx.y;
        x[3 * i + 2] = xx.z;
        cons_out[i] = cn;
        ok[i] = r ? 1 : 0;
    }
}

// ---- statistics -------------------------------------------------------------------
// kernel sum rho = W(0) + sum of W over masked neighbours; per-class sums in
// FP64; smallest masked pair distance over mobile particles
__global__ void __launch_bounds__(TPB) k_density(const float4 *__restrict__ pos_s, int64_t N,
                                                 const AsmParams *__restrict__ P, const uint32_t *__restrict__ fstart,
                                                 float *__restrict__ rho_s, uint32_t *__restrict__ minpair) {
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    const float4 p = pos_s[k];
    const int cls = cls_of(p.w);
    const AsmParams &A = P[body_of(p.w)];
    const uint32_t mbits = acts_on_bits(cls);
    const int nx = A.ng_n[0], ny = A.ng_n[1], nz = A.ng_n[2];
    const int cx = cell_coord(p.x, A.ng_o[0], A.ng_inv, nx);
    const int cy = cell_coord(p.y, A.ng_o[1], A.ng_inv, ny);
    const int cz = cell_coord(p.z, A.ng_o[2], A.ng_inv, nz);
    float rho = 0.f, rmin2 = FLT_MAX;
    for (int z = max(cz - 1, 0); z <= min(cz + 1, nz - 1); z++)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, ny - 1); y++) {
            const uint32_t row = A.key_base + (uint32_t)nx * grid_row(A, y, z);
            uint32_t s, e;
            cells_slots(fstart, row, max(cx - 1, 0), min(cx + 1, nx - 1), s, e);
            for (uint32_t j = s; j < e; j++) {
                const float4 q = pos_s[j];
                const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
                const float r2 = dist2_rn(dx, dy, dz);
                if (r2 < A.R2 && (int64_t)j != k && (mbits & __float_as_uint(q.w)) != 0u) {
                    const float r = sqrtf(r2);
                    const float qh = r * A.half_inv_h;   // q / 2
                    const float t = 1.f - qh;
                    rho += t * t * t * t * (4.f * qh + 1.f);
                    rmin2 = fminf(rmin2, r2);
                }
            }
        }
    rho_s[k] = A.alpha * (rho + 1.f);
    if (is_mobile(cls, A) && !is_ghost(p.w) && rmin2 < FLT_MAX) atomicMin(minpair, __float_as_uint(sqrtf(rmin2)));
}

__global__ void k_class_sums(const float4 *__restrict__ pos_s, const float *__restrict__ rho_s, int64_t N,
                             const double *__restrict__ mean, double *__restrict__ sums) {
    // sums[0..2] sum rho, [3..5] sum (rho - mean)^2 when mean != null, [6..8] count
    const int64_t k = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (k >= N) return;
    const float w = pos_s[k].w;
    int c = cls_of(w);
    if (c > kClsF || is_ghost(w)) return;
    double r = rho_s[k];
    if (mean) {
        double d = r - mean[c];
        atomicAdd(sums + 3 + c, d * d);
    } else {
        atomicAdd(sums + c, r);
        atomicAdd(sums + 6 + c, 1.0);
    }
}

} // namespace

// ---- host driver ----------------------------------------------------------------
// A1-A2 of the incremental form; the order ends in key[0] / id[0], which is
// also the previous order it starts from
static void order_incremental(DevGroup &d, cudaStream_t s) {
    const int64_t N = d.N;
    const int64_t nb = nblocks(N, kOrdTile);
    k_keys_inc<<<std::max<unsigned>(nb, nblocks(d.B)), TPB, 0, s>>>(d.pos, N, d.params, d.key_id, d.chg_bits,
                                                                     d.tile_cnt, d.amax, d.maxdisp, d.B,
                                                                     d.work_count);
    if (N == 0) return;
    k_keep_bits<<<nb, TPB, 0, s>>>(d.id[0], d.chg_bits, N, d.keep_bits, d.tile_cnt + nb);
    exclusive_scan_u32(d.tile_cnt, d.tile_pos, 2 * nb, nullptr, d.scan_tmp_n, scan_tmp_elems(2 * nb), s);
    k_order_counts<<<1, 1, 0, s>>>(d.tile_cnt, d.tile_pos, nb, d.counts);
    k_compact_changed<<<nb, TPB, 0, s>>>(d.chg_bits, d.tile_pos, d.key_id, N, d.ck[0], d.cv[0]);
    const int cb = radix_sort_u32_dev(d.ck, d.cv, N, d.counts, d.key_bits, d.hist, d.totals, s);
    k_compact_kept<<<nb, TPB, 0, s>>>(d.keep_bits, d.tile_pos, nb, d.key[0], d.id[0], N, d.uk, d.uv);
    const int nblk = (int)((N + kMergeTile - 1) / kMergeTile);
    k_merge_splits<<<(nblk + 1 + 255) / 256, 256, 0, s>>>(d.uk, d.uv, d.ck[cb], d.cv[cb], d.counts, N, nblk,
                                                          d.split);
    k_merge<<<nblk, kMergeThreads, 0, s>>>(d.uk, d.uv, d.ck[cb], d.cv[cb], d.split, N, d.key[0], d.id[0]);
}

int build_grid_dev(DevGroup &d, cudaStream_t s) {
    int buf = 0;
    if (d.incremental) {
        order_incremental(d, s);
    } else {
        k_keys<<<nblocks(std::max<int64_t>(d.N, d.B)), TPB, 0, s>>>(d.pos, d.N, d.params, d.key[0], d.amax,
                                                                     d.maxdisp, d.B, d.work_count);
        buf = radix_sort_u32(d.key, d.id, true, d.N, d.key_bits, d.hist, d.totals, s);
    }
    k_gather<<<nblocks(d.N), TPB, 0, s>>>(d.id[buf], d.pos, d.N, d.pos_s, d.pos_p, d.cons, d.cons_s);
    // the start table from the sorted keys
    const int64_t F1 = kSlabs * d.total_cells + 1;
    const int64_t nblk = start_blocks(F1);
    k_key_block_starts<<<nblocks(d.N + 1), TPB, 0, s>>>(d.key[buf], d.N, nblk, d.bstart);
    k_fine_starts<<<(unsigned)nblk, kStartBlock, 0, s>>>(d.key[buf], d.bstart, F1, d.fstart);
    return buf;
}

int grid_kernels(const DevGroup &d) {
    const int tail = 3;    // gather, block starts, fine-key starts
    if (!d.incremental) return 1 + 3 * d.passes + tail;
    // keys, keep bits, the scan of the tile counts and the counts, 2
    // compactions, the changed list's radix passes, merge splits and merge
    return 2 + scan_launches(2 * (int64_t)nblocks(d.N, kOrdTile)) + 1 + 2 + 3 * d.passes + 2 + tail;
}

int build_grid(Group &g, cudaStream_t s) { return build_grid_dev(g.d, s); }

void forces_dev(DevGroup &d, int tb, int variant, cudaStream_t s, int32_t *count_s, int32_t *tested_s) {
    const unsigned nbk = (unsigned)std::max<int64_t>((d.N + tb - 1) / tb, 1);
#define FPPG_FORCE(V, C, M)                                                                                    \
    k_force<V, C, M><<<nbk, tb, 0, s>>>(d.pos_s, d.pos_p, d.N, d.params, d.fstart, d.acc_s, d.amax, count_s,        \
                                        tested_s)
    if (d.morton_rows) {
        if (count_s) {
            if (variant == 1) FPPG_FORCE(1, true, true);
            else FPPG_FORCE(0, true, true);
        } else {
            if (variant == 1) FPPG_FORCE(1, false, true);
            else FPPG_FORCE(0, false, true);
        }
    } else if (count_s) {
        if (variant == 1) FPPG_FORCE(1, true, false);
        else FPPG_FORCE(0, true, false);
    } else {
        if (variant == 1) FPPG_FORCE(1, false, false);
        else FPPG_FORCE(0, false, false);
    }
#undef FPPG_FORCE
}

void forces(Group &g, cudaStream_t s, int32_t *count_s, int32_t *cand_s, int32_t *tested_s) {
    DevGroup &d = g.d;
    forces_dev(d, g.force_block, g.force_variant, s, count_s, tested_s);
    if (cand_s)
        k_count<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.fstart, nullptr, cand_s);
}

void iterate(Group &g, cudaStream_t s, bool energy_mode, int32_t *count_dbg) {
    DevGroup &d = g.d;
    if (d.N == 0) return;
    // phase timing: events before A1, after A3, after A4, after A5 and after A6
    const bool timed = g.time_force && g.ev_used + kPhaseEvents <= (int)g.ev.size();
    // inside a stream capture the records must be external so that they
    // become event-record nodes whose timestamps can be read after a replay
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (timed) cudaStreamIsCapturing(s, &cap);
    const unsigned flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (timed) cudaEventRecordWithFlags(g.ev[g.ev_used], s, flags);
    int buf;
    {
        NvtxRange r("A1-A3 grid");
        buf = build_grid(g, s);
    }
    if (timed) cudaEventRecordWithFlags(g.ev[g.ev_used + 1], s, flags);
    {
        NvtxRange r("A4 force");
        if (energy_mode) energy_accel(g, s);
        else forces(g, s, count_dbg);
    }
    if (timed) cudaEventRecordWithFlags(g.ev[g.ev_used + 2], s, flags);
    NvtxRange r("A5-A6 step and search");
    k_step<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.acc_s, d.id[buf], d.N, d.params, d.amax, d.pos, d.cons, g.mesh,
                                         d.maxdisp, d.work, queue_ranges(d), d.work_count, d.cert, d.cons_s);
    if (timed) cudaEventRecordWithFlags(g.ev[g.ev_used + 3], s, flags);
    if (g.search_thread)
        k_search_thread<<<g.search_blocks, TPB, 0, s>>>(d.pos_s, d.id[buf], d.params, d.pos, d.cons, g.mesh,
                                                        d.maxdisp, d.work, queue_ranges(d), d.work_count, d.N,
                                                        d.cert);
    else
        k_search<<<g.search_blocks, TPB, 0, s>>>(d.pos_s, d.id[buf], d.params, d.pos, d.cons, g.mesh, d.maxdisp,
                                                 d.work, queue_ranges(d), d.work_count, d.N, d.cert);
    if (timed) {
        cudaEventRecordWithFlags(g.ev[g.ev_used + 4], s, flags);
        g.ev_used += kPhaseEvents;
    }
}

void step_and_project(Group &g, cudaStream_t s, int buf) {
    DevGroup &d = g.d;
    if (d.N == 0) return;
    k_step<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.acc_s, d.id[buf], d.N, d.params, d.amax, d.pos, d.cons, g.mesh,
                                         d.maxdisp, d.work, queue_ranges(d), d.work_count, d.cert, d.cons_s);
    if (g.search_thread)
        k_search_thread<<<g.search_blocks, TPB, 0, s>>>(d.pos_s, d.id[buf], d.params, d.pos, d.cons, g.mesh,
                                                        d.maxdisp, d.work, queue_ranges(d), d.work_count, d.N,
                                                        d.cert);
    else
        k_search<<<g.search_blocks, TPB, 0, s>>>(d.pos_s, d.id[buf], d.params, d.pos, d.cons, g.mesh, d.maxdisp,
                                                 d.work, queue_ranges(d), d.work_count, d.N, d.cert);
}

namespace {
__global__ void k_tag_ghosts(float4 *__restrict__ pos, int64_t n, int64_t first_ghost) {
    const int64_t i = (int64_t)blockIdx.x * TPB + threadIdx.x;
    if (i >= n) return;
    const uint32_t w = __float_as_uint(pos[i].w);
    pos[i].w = __uint_as_float(i >= first_ghost ? (w | kGhostBit) : (w & ~kGhostBit));
}
} // namespace

void tag_ghosts(Group &g, int64_t first_ghost, cudaStream_t s) {
    if (g.d.N > 0) k_tag_ghosts<<<nblocks(g.d.N), TPB, 0, s>>>(g.d.pos, g.d.N, first_ghost);
}

void unpermute_dev(DevGroup &d, int buf, cudaStream_t s, float *acc_out, const int32_t *count_s,
                   int32_t *count_out) {
    k_unpermute<<<nblocks(d.N), TPB, 0, s>>>(d.acc_s, d.id[buf], d.N, acc_out, count_s, count_out);
}

void unpermute(Group &g, int buf, cudaStream_t s, float *acc_out, const int32_t *count_s, int32_t *count_out) {
    unpermute_dev(g.d, buf, s, acc_out, count_s, count_out);
}

void project_points(Group &g, const float *y, const int32_t *cls, const int32_t *cons_in, int64_t n, float *x,
                    int32_t *cons_out, int32_t *ok, cudaStream_t s) {
    k_project_points<<<nblocks(32 * n), TPB, 0, s>>>(y, cls, cons_in, n, g.d.params, g.mesh, x, cons_out, ok);
}

int stats(Group &g, cudaStream_t s, double *mean, double *sd, double *minpair, double *maxdisp, int64_t *cnt,
          std::string &err) {
    DevGroup &d = g.d;
    double *sums = nullptr;
    uint32_t *mp = nullptr;
    float *rho = nullptr;
    if (dev_malloc(&sums, 12 * sizeof(double)) != cudaSuccess || dev_malloc(&mp, 8) != cudaSuccess ||
        dev_malloc(&rho, sizeof(float) * std::max<int64_t>(d.N, 1)) != cudaSuccess) {
        err = "stats: out of device memory";
        cudaFree(sums);
        cudaFree(mp);
        return 3;
    }
    cudaMemsetAsync(sums, 0, 12 * sizeof(double), s);
    uint32_t big = 0x7f7fffffu;
    cudaMemcpyAsync(mp, &big, 4, cudaMemcpyHostToDevice, s);
    uint32_t md = 0;
    cudaMemcpyAsync(&md, d.maxdisp, 4, cudaMemcpyDeviceToHost, s);
    if (d.N > 0) {
        build_grid(g, s);
        k_density<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, d.N, d.params, d.fstart, rho, mp);
        k_class_sums<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, rho, d.N, nullptr, sums);
    }
    double h[12];
    cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int c = 0; c < 3; c++) mean[c] = h[6 + c] > 0 ? h[c] / h[6 + c] : 0.0;
    cudaMemcpyAsync(sums + 9, mean, 3 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (d.N > 0) k_class_sums<<<nblocks(d.N), TPB, 0, s>>>(d.pos_s, rho, d.N, sums + 9, sums);
    uint32_t mph = 0;
    cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&mph, mp, 4, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    for (int c = 0; c < 3; c++) {
        sd[c] = h[6 + c] > 0 ? std::sqrt(h[3 + c] / h[6 + c]) : 0.0;
        cnt[c] = (int64_t)h[6 + c];
    }
    float mpf, mdf;
    memcpy(&mpf, &mph, 4);
    memcpy(&mdf, &md, 4);
    const float dx = g.hp[0].dx;
    *minpair = mph == big ? INFINITY : (double)mpf / dx;
    *maxdisp = (double)mdf / dx;
    cudaFree(sums);
    cudaFree(mp);
    cudaFree(rho);
    if (e != cudaSuccess) {
        err = std::string("stats: ") + cudaGetErrorString(e);
        return 4;
    }
    return 0;
}

} // namespace fppg
