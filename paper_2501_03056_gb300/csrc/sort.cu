// Stable LSD radix sort of (key, value) pairs and an exclusive scan.
//
// Sec. 3.1.3 sorts the cell list by key with a radix sort; here every pass
// handles one 8-bit digit in three launches:
//   upsweep     per-tile digit histogram (warp-aggregated shared atomics)
//   digit scan  one CTA per digit scans the per-tile counts, digit-major
//   downsweep   stable rank of every item inside its tile (warp match +
//               per-warp counters), staging through shared memory so that
//               global writes are contiguous runs per digit
// No CTA waits on another CTA, so nothing here can spin.
#include <cstdint>
#include <algorithm>
#include <cstring>

#include "fppg_internal.cuh"

namespace fppg {

namespace {

constexpr int RT = 256;               // threads per CTA
constexpr int RW = RT / 32;           // warps per CTA
// RC 32-item chunks per warp, a tile of RW * RC * 32 items per CTA: 4096,
// 2048 or 1024, the largest that still gives every SM four tiles
constexpr int kMinTile = RW * 4 * 32;

__device__ inline uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// inclusive scan over the 256 threads of a CTA; wsum: RW shared words
__device__ inline uint32_t block_incl_scan(uint32_t v, uint32_t *wsum, uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < RW ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < RW) wsum[lane] = s;
    }
    __syncthreads();
    uint32_t r = v + (w > 0 ? wsum[w - 1] : 0u);
    if (total) *total = wsum[RW - 1];
    __syncthreads();
    return r;
}

// DB-bit digits (ND = 2^DB values; the passes use DB = 8): the upsweep
// counts them per tile in shared memory
// n_dev (nullable): the item count is read from device memory (at most n),
// so that a captured graph can sort a list whose length it does not know;
// tiles past it count nothing and write nothing (the digit scan and the
// downsweep stop at the last tile that holds items)
template <typename K, int RC, int DB>
__global__ void __launch_bounds__(RT) k_upsweep(const K *__restrict__ keys, int64_t n, int shift,
                                                uint32_t *__restrict__ hist, int n_tiles,
                                                const uint32_t *__restrict__ n_dev) {
    constexpr int TILE = RW * RC * 32, ND = 1 << DB;
    __shared__ uint32_t cnt[ND];
    if (n_dev) n = min(n, (int64_t)*n_dev);
    const int n_act = (int)min((int64_t)n_tiles, (n + TILE - 1) / TILE);   // tiles past the count: none
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < n_act; tile += gridDim.x) {
        for (int d = threadIdx.x; d < ND; d += RT) cnt[d] = 0;
        __syncthreads();
        const int64_t base = (int64_t)tile * TILE + w * (RC * 32) + l;
#pragma unroll 4
        for (int c = 0; c < RC; c++) {
            int64_t idx = base + c * 32;
            bool valid = idx < n;
            uint32_t d = valid ? (uint32_t)((keys[idx] >> shift) & (K)(ND - 1)) : (uint32_t)ND;
            uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && (uint32_t)(__ffs(peers) - 1) == (uint32_t)l) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
        }
        __syncthreads();
        for (int d = threadIdx.x; d < ND; d += RT) hist[(int64_t)d * n_tiles + tile] = cnt[d];
        __syncthreads();   // cnt is zeroed again for the next tile
    }
}

// one CTA per digit: exclusive scan of its row of per-tile counts, over the
// tiles that hold items (n_dev: the item count on the device, else n)
__global__ void __launch_bounds__(RT) k_digit_scan(uint32_t *__restrict__ hist, int n_tiles,
                                                   uint32_t *__restrict__ totals, int64_t n, int tile,
                                                   const uint32_t *__restrict__ n_dev) {
    __shared__ uint32_t wsum[RW];
    if (n_dev) n = min(n, (int64_t)*n_dev);
    const int n_act = (int)min((int64_t)n_tiles, (n + tile - 1) / tile);
    uint32_t *row = hist + (int64_t)blockIdx.x * n_tiles;
    uint32_t carry = 0;
    for (int start = 0; start < n_act; start += RT) {
        int idx = start + threadIdx.x;
        uint32_t v = idx < n_act ? row[idx] : 0u, tot;
        uint32_t inc = block_incl_scan(v, wsum, &tot);
        if (idx < n_act) row[idx] = carry + inc - v;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <typename K, bool IOTA, int RC, int DB>
__global__ void __launch_bounds__(RT) k_downsweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                  K *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                                  int shift, const uint32_t *__restrict__ hist,
                                                  const uint32_t *__restrict__ totals, int n_tiles,
                                                  const uint32_t *__restrict__ n_dev) {
    constexpr int TILE = RW * RC * 32, ND = 1 << DB, KD = ND / RT;
    if (n_dev) n = min(n, (int64_t)*n_dev);
    const int n_act = (int)min((int64_t)n_tiles, (n + TILE - 1) / TILE);   // tiles past the count: none
    extern __shared__ __align__(16) unsigned char smem[];
    K *skey = reinterpret_cast<K *>(smem);
    uint32_t *sval = reinterpret_cast<uint32_t *>(smem + sizeof(K) * TILE);
    uint32_t(*wcnt)[ND] = reinterpret_cast<uint32_t(*)[ND]>(smem + (sizeof(K) + 4) * TILE);
    uint32_t *dstart = reinterpret_cast<uint32_t *>(smem + (sizeof(K) + 4) * TILE + RW * ND * 4);
    uint32_t *gbase = dstart + ND;
    uint32_t *wsum = gbase + ND;

    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < n_act; tile += gridDim.x) {
        for (int i = threadIdx.x; i < RW * ND; i += RT) (&wcnt[0][0])[i] = 0;
        __syncthreads();

        const int64_t tile0 = (int64_t)tile * TILE;
        const int64_t base = tile0 + w * (RC * 32) + l;
        K k[RC];
        uint32_t v[RC], rank[RC];
        const uint32_t lt = lanemask_lt();
#pragma unroll
        for (int c = 0; c < RC; c++) {
            int64_t idx = base + c * 32;
            bool valid = idx < n;
            k[c] = valid ? kin[idx] : (K)0;
            v[c] = valid ? (IOTA ? (uint32_t)idx : vin[idx]) : 0u;
            uint32_t d = valid ? (uint32_t)((k[c] >> shift) & (K)(ND - 1)) : (uint32_t)ND;
            uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t before = valid ? wcnt[w][d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0u) wcnt[w][d] = before + __popc(peers);
            __syncwarp();
            rank[c] = before + __popc(peers & lt);
        }
        __syncthreads();
        // thread t owns digits t KD .. t KD + KD - 1: per-warp exclusive offsets,
        // the tile count and the global start of each
        uint32_t cnt_d[KD], tot_d[KD], s_cnt = 0, s_tot = 0;
#pragma unroll
        for (int j = 0; j < KD; j++) {
            const int d = threadIdx.x * KD + j;
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < RW; ww++) {
                uint32_t t = wcnt[ww][d];
                wcnt[ww][d] = run;
                run += t;
            }
            cnt_d[j] = run;
            s_cnt += run;
            tot_d[j] = totals[d];
            s_tot += tot_d[j];
        }
        uint32_t tmp;
        uint32_t loc = block_incl_scan(s_cnt, wsum, &tmp) - s_cnt;
        uint32_t dig = block_incl_scan(s_tot, wsum, &tmp) - s_tot;
#pragma unroll
        for (int j = 0; j < KD; j++) {
            const int d = threadIdx.x * KD + j;
            dstart[d] = loc;
            gbase[d] = dig + hist[(int64_t)d * n_tiles + tile] - loc;
            loc += cnt_d[j];
            dig += tot_d[j];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < RC; c++) {
            int64_t idx = base + c * 32;
            if (idx < n) {
                uint32_t dd = (uint32_t)((k[c] >> shift) & (K)(ND - 1));
                uint32_t p = dstart[dd] + wcnt[w][dd] + rank[c];
                skey[p] = k[c];
                sval[p] = v[c];
            }
        }
        __syncthreads();
        const int tile_n = (int)min((int64_t)TILE, n - tile0);
        for (int j = threadIdx.x; j < tile_n; j += RT) {
            K kk = skey[j];
            uint32_t dd = (uint32_t)((kk >> shift) & (K)(ND - 1));
            uint32_t o = gbase[dd] + (uint32_t)j;
            kout[o] = kk;
            vout[o] = sval[j];
        }
        __syncthreads();   // the staging and the counters are reused by the next tile
    }
}

template <typename K, int RC, int DB>
size_t downsweep_smem() {
    return (sizeof(K) + 4) * (size_t)(RW * RC * 32) + RW * (4 << DB) + 2 * (4 << DB) + RW * 4;
}

template <typename K, int RC, int DB>
void set_smem_attr() {
    cudaFuncSetAttribute(k_downsweep<K, true, RC, DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)downsweep_smem<K, RC, DB>());
    cudaFuncSetAttribute(k_downsweep<K, false, RC, DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)downsweep_smem<K, RC, DB>());
}

// grid: CTAs of the sweeps (at most the tiles; each CTA takes every grid-th
// tile)
template <typename K, int RC, int DB>
int radix_passes(K *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int passes, uint32_t *hist,
                 uint32_t *totals, cudaStream_t s, const uint32_t *n_dev, int grid) {
    constexpr int TILE = RW * RC * 32;
    const int n_tiles = (int)((n + TILE - 1) / TILE);
    const int g = std::max(1, std::min(grid, n_tiles));
    int cur = 0;
    for (int p = 0; p < passes; p++) {
        const int shift = DB * p;
        k_upsweep<K, RC, DB><<<g, RT, 0, s>>>(keys[cur], n, shift, hist, n_tiles, n_dev);
        k_digit_scan<<<1 << DB, RT, 0, s>>>(hist, n_tiles, totals, n, TILE, n_dev);
        if (p == 0 && iota_vals)
            k_downsweep<K, true, RC, DB><<<g, RT, downsweep_smem<K, RC, DB>(), s>>>(
                keys[cur], nullptr, keys[cur ^ 1], vals[cur ^ 1], n, shift, hist, totals, n_tiles, n_dev);
        else
            k_downsweep<K, false, RC, DB><<<g, RT, downsweep_smem<K, RC, DB>(), s>>>(
                keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift, hist, totals, n_tiles, n_dev);
        cur ^= 1;
    }
    return cur;
}

template <typename K, int DB>
int radix_sort_db(K *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int passes, uint32_t *hist,
                  uint32_t *totals, cudaStream_t s, int sms, const uint32_t *n_dev) {
    // a count on the device (usually far below n): the smallest tiles, taken
    // by at most 8 CTAs per SM in turn, so that neither the CTAs of the
    // tiles past the count nor a long walk through a few large tiles set
    // the time
    if (n_dev) return radix_passes<K, 4, DB>(keys, vals, iota_vals, n, passes, hist, totals, s, n_dev, 8 * sms);
    // else the largest tile that still gives every SM four tiles (latency
    // hiding), one CTA per tile
    const int64_t want = 4 * (int64_t)sms;
    if ((n + 4095) / 4096 >= want)
        return radix_passes<K, 16, DB>(keys, vals, iota_vals, n, passes, hist, totals, s, nullptr, INT32_MAX);
    if ((n + 2047) / 2048 >= want)
        return radix_passes<K, 8, DB>(keys, vals, iota_vals, n, passes, hist, totals, s, nullptr, INT32_MAX);
    return radix_passes<K, 4, DB>(keys, vals, iota_vals, n, passes, hist, totals, s, nullptr, INT32_MAX);
}

// once per key type and process (thread-safe static initialisation): the
// downsweeps' shared-memory limits on the current device and its SM count
template <typename K>
int sort_setup_sms() {
    static const int sms = [] {
        set_smem_attr<K, 4, 8>();
        set_smem_attr<K, 8, 8>();
        set_smem_attr<K, 16, 8>();
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        return v;
    }();
    return sms;
}

template <typename K>
int radix_sort_impl(K *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int bits, uint32_t *hist,
                    uint32_t *totals, cudaStream_t s) {
    if (n <= 0) return 0;
    const int sms = sort_setup_sms<K>();
    int db = 8;
    const int passes = radix_pass_plan(bits, &db);
    return radix_sort_db<K, 8>(keys, vals, iota_vals, n, passes, hist, totals, s, sms, nullptr);
}

// ---- exclusive scan (set-up work) -----------------------------------------
// 16 entries per thread, 4096 per block; entries move as 16-byte vectors
// when both arrays are 16-byte aligned (VEC), else one by one.  CLEAR: the
// input is set to 0 once read (a count array made ready for its next
// accumulation).  in == out is allowed (each thread reads its entries
// before it writes them).
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_BLOCK = RT * SCAN_ITEMS;

template <bool CLEAR>
__global__ void __launch_bounds__(RT) k_scan_block(uint32_t *in, uint32_t *out, int64_t n,
                                                   uint32_t *__restrict__ block_sums, bool vec) {
    __shared__ uint32_t wsum[RW];
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], s = 0;
    const bool whole = vec && base + SCAN_ITEMS <= n;
    if (whole) {
        uint4 *q = reinterpret_cast<uint4 *>(in + base);
#pragma unroll
        for (int c = 0; c < SCAN_ITEMS / 4; c++) {
            const uint4 a = q[c];
            v[4 * c] = a.x;
            v[4 * c + 1] = a.y;
            v[4 * c + 2] = a.z;
            v[4 * c + 3] = a.w;
            if (CLEAR) q[c] = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            v[i] = base + i < n ? in[base + i] : 0u;
            if (CLEAR && base + i < n) in[base + i] = 0u;
        }
    }
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) s += v[i];
    uint32_t tot;
    uint32_t run = block_incl_scan(s, wsum, &tot) - s;
    if (whole) {
        uint4 *o = reinterpret_cast<uint4 *>(out + base);
#pragma unroll
        for (int c = 0; c < SCAN_ITEMS / 4; c++) {
            uint4 a;
            a.x = run;
            run += v[4 * c];
            a.y = run;
            run += v[4 * c + 1];
            a.z = run;
            run += v[4 * c + 2];
            a.w = run;
            run += v[4 * c + 3];
            o[c] = a;
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; i++) {
            if (base + i < n) out[base + i] = run;
            run += v[i];
        }
    }
    if (threadIdx.x == 0 && block_sums) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(RT) k_scan_add(uint32_t *__restrict__ out, int64_t n,
                                                 const uint32_t *__restrict__ offs, bool vec) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    const uint32_t o = offs[blockIdx.x];
    if (vec && base + SCAN_ITEMS <= n) {
        uint4 *q = reinterpret_cast<uint4 *>(out + base);
#pragma unroll
        for (int c = 0; c < SCAN_ITEMS / 4; c++) {
            uint4 a = q[c];
            a.x += o;
            a.y += o;
            a.z += o;
            a.w += o;
            q[c] = a;
        }
    } else {
        for (int i = 0; i < SCAN_ITEMS; i++)
            if (base + i < n) out[base + i] += o;
    }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

__global__ void k_scan_total(const uint32_t *in, const uint32_t *out, int64_t n, uint32_t *total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

} // namespace

// tiles of the smallest tile size: room for the histogram of any choice
int64_t radix_tiles(int64_t n) { return (n + kMinTile - 1) / kMinTile; }

// passes for keys of `bits` bits, in 8-bit digits.  (10-bit digits would
// save a pass for 17-20 and 25-30 bit keys, but measured slower: with 1024
// buckets a tile scatters about one key per digit, and the 1024-CTA digit
// scan costs more than the pass saved.)
int radix_pass_plan(int bits, int *digit_bits) {
    *digit_bits = 8;
    return bits <= 0 ? 0 : (bits + 7) / 8;
}

int radix_sort_u32(uint32_t *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int bits, uint32_t *hist,
                   uint32_t *totals, cudaStream_t s) {
    return radix_sort_impl<uint32_t>(keys, vals, iota_vals, n, bits, hist, totals, s);
}

int radix_sort_u32_dev(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max, const uint32_t *n_dev, int bits,
                       uint32_t *hist, uint32_t *totals, cudaStream_t s) {
    if (n_max <= 0) return 0;
    const int sms = sort_setup_sms<uint32_t>();
    int db = 8;
    const int passes = radix_pass_plan(bits, &db);
    return radix_sort_db<uint32_t, 8>(keys, vals, false, n_max, passes, hist, totals, s, sms, n_dev);
}

int radix_sort_u64(uint64_t *keys[2], uint32_t *vals[2], bool iota_vals, int64_t n, int bits, uint32_t *hist,
                   uint32_t *totals, cudaStream_t s) {
    return radix_sort_impl<uint64_t>(keys, vals, iota_vals, n, bits, hist, totals, s);
}


// The last element of `in` is read after the scan to form the total, so
// `out` must not alias `in` when total_dev is requested.
template <bool CLEAR>
static void scan_impl(uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, int64_t tmp_elems, cudaStream_t s) {
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    const bool vec = aligned16(in) && aligned16(out);
    if (nb == 1) {
        k_scan_block<CLEAR><<<1, RT, 0, s>>>(in, out, n, nullptr, vec);
    } else {
        uint32_t *sums = tmp;
        k_scan_block<CLEAR><<<(unsigned)nb, RT, 0, s>>>(in, out, n, sums, vec);
        scan_impl<false>(sums, sums, nb, tmp + nb + 1, tmp_elems - nb - 1, s);
        k_scan_add<<<(unsigned)nb, RT, 0, s>>>(out, n, sums, vec);
    }
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total_dev, uint32_t *tmp,
                        int64_t tmp_elems, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
        return;
    }
    scan_impl<false>(const_cast<uint32_t *>(in), out, n, tmp, tmp_elems, s);   // not written without CLEAR
    if (total_dev) k_scan_total<<<1, 1, 0, s>>>(in, out, n, total_dev);
}

void exclusive_scan_u32_clear(uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp, int64_t tmp_elems,
                              cudaStream_t s) {
    if (n > 0) scan_impl<true>(in, out, n, tmp, tmp_elems, s);
}

// block sums of every level (with one spare entry each): at most this many
int64_t scan_tmp_elems(int64_t n) {
    int64_t tot = 0;
    while (n > SCAN_BLOCK) {
        n = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
        tot += n + 1;
    }
    return tot + 1;
}

int scan_launches(int64_t n) {
    if (n <= 0) return 0;
    const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    return nb == 1 ? 1 : 2 + scan_launches(nb);
}

int scan_clear_launches(int64_t n) { return scan_launches(n); }

} // namespace fppg
