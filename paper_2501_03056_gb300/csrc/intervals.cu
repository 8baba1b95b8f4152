// C_compact interval form of a lattice cell set and its Boolean algebra.
//
// Sec. 3.1.3 stores the cells of a body as C_compact begin / length: runs of
// consecutive Morton codes (Eq. 9).  Sec. 3.2.3 and Fig. 10 combine two
// bodies' grid sets by union, difference and intersection of those
// intervals.  Three entry points, all on device buffers and the caller's
// stream:
//
//   fppg_lattice_intervals  points -> the codes of their lattice cells,
//                           radix-sorted, as maximal runs (a run starts
//                           where a code exceeds its predecessor + 1;
//                           repeats continue a run)
//   fppg_interval_boolean   two run lists -> op(A, B) as maximal runs: every
//                           run contributes a +1 event at its begin and a -1
//                           event at its end; the events are radix-sorted by
//                           code, the coverage of A and of B is the scan of
//                           their deltas, and a result run starts or ends
//                           where op(coverA > 0, coverB > 0) changes between
//                           consecutive distinct codes
//   fppg_interval_cells     run list -> the centres of its cells, one thread
//                           per cell (binary search in the scan of the run
//                           lengths)
//
// Each call computes its result count, reads it back (synchronising the
// stream), and writes the result only when it fits the caller's capacity.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/fppg.h"
#include "body.h"

namespace fppg {
void set_global_error(const char *msg);
}

using namespace fppg;

namespace {

constexpr uint64_t kCodeLimit = 1ull << 63;      // codes of cells below 2^21 per axis
constexpr float kAxisCells = 2097152.0f;         // 2^21

// Eq. 9: bit b of axis a goes to bit 3b + a of the code (x lowest)
__device__ inline uint64_t morton_encode(uint32_t i, uint32_t j, uint32_t k) {
    uint64_t c = 0;
    for (int b = 0; b < 21; b++)
        c |= ((uint64_t)((i >> b) & 1u) << (3 * b)) | ((uint64_t)((j >> b) & 1u) << (3 * b + 1)) |
             ((uint64_t)((k >> b) & 1u) << (3 * b + 2));
    return c;
}

__device__ inline void morton_decode(uint64_t c, uint32_t &i, uint32_t &j, uint32_t &k) {
    i = j = k = 0u;
    for (int b = 0; b < 21; b++) {
        i |= (uint32_t)((c >> (3 * b)) & 1u) << b;
        j |= (uint32_t)((c >> (3 * b + 1)) & 1u) << b;
        k |= (uint32_t)((c >> (3 * b + 2)) & 1u) << b;
    }
}

// the lattice cell of each point, floor((x - o) / d) per axis in FP32, as
// its Morton code; a point outside [0, 2^21) cells raises the error word
__global__ void k_cell_codes(const float *__restrict__ xyz, int64_t n, float3 o, float d,
                             uint64_t *__restrict__ code, uint32_t *__restrict__ err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float x[3] = {xyz[3 * t], xyz[3 * t + 1], xyz[3 * t + 2]};
    const float oo[3] = {o.x, o.y, o.z};
    uint32_t c[3];
    bool ok = true;
    for (int a = 0; a < 3; a++) {
        const float f = floorf(__fdiv_rn(__fsub_rn(x[a], oo[a]), d));
        ok = ok && f >= 0.0f && f < kAxisCells;
        c[a] = ok ? (uint32_t)f : 0u;
    }
    if (!ok) atomicOr(err, 1u);
    code[t] = ok ? morton_encode(c[0], c[1], c[2]) : 0ull;
}

// 1 where a sorted code starts a run (the first, or more than one past the
// previous code)
__global__ void k_run_starts(const uint64_t *__restrict__ code, int64_t n, uint32_t *__restrict__ start) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    start[t] = (t == 0 || code[t] > code[t - 1] + 1ull) ? 1u : 0u;
}

// begin of run r at its first code, its end (last code + 1) into len[r]
__global__ void k_run_write(const uint64_t *__restrict__ code, int64_t n, const uint32_t *__restrict__ start,
                            const uint32_t *__restrict__ pos, uint64_t *__restrict__ begin, uint64_t *__restrict__ len) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t r = pos[t] + start[t] - 1u;
    if (start[t]) begin[r] = code[t];
    if (t == n - 1 || start[t + 1]) len[r] = code[t] + 1ull;
}

// len[r] held the end of run r: the length
__global__ void k_end_to_len(const uint64_t *__restrict__ begin, int64_t m, uint64_t *__restrict__ len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < m) len[r] -= begin[r];
}

// event e of the two run lists: e < 2 na belongs to A's run e / 2, the rest
// to B's run (e - 2 na) / 2; even events are begins, odd ones ends
__global__ void k_events(const uint64_t *__restrict__ ab, const uint64_t *__restrict__ al, int64_t na,
                         const uint64_t *__restrict__ bb, const uint64_t *__restrict__ bl, int64_t E,
                         uint64_t *__restrict__ key, uint32_t *__restrict__ err) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const bool inB = e >= 2 * na;
    const int64_t r = (inB ? e - 2 * na : e) >> 1;
    const uint64_t b = inB ? bb[r] : ab[r], l = inB ? bl[r] : al[r];
    const bool ok = b < kCodeLimit && l <= kCodeLimit - b;
    if (!ok) atomicOr(err, 1u);
    key[e] = ok ? ((e & 1) ? b + l : b) : 0ull;
}

// coverage deltas of the sorted events (two's complement in uint32)
__global__ void k_deltas(const uint32_t *__restrict__ ev, int64_t E, int64_t na, uint32_t *__restrict__ dA,
                         uint32_t *__restrict__ dB) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E) return;
    const uint32_t e = ev[t];
    const uint32_t d = (e & 1u) ? 0xffffffffu : 1u;
    const bool inB = (int64_t)e >= 2 * na;
    dA[t] = inB ? 0u : d;
    dB[t] = inB ? d : 0u;
}

__device__ inline bool in_result(int op, const uint32_t *cA, const uint32_t *dA, const uint32_t *cB,
                                 const uint32_t *dB, int64_t t) {
    const bool a = (int32_t)(cA[t] + dA[t]) > 0, b = (int32_t)(cB[t] + dB[t]) > 0;
    return op == FPPG_UNION ? (a || b) : (op == FPPG_DIFFERENCE ? (a && !b) : (a && b));
}

// 1 at the last event of a code where the result changes: the state after
// the previous code's events against the state after this code's
__global__ void k_changes(const uint64_t *__restrict__ key, int64_t E, int op, const uint32_t *__restrict__ cA,
                          const uint32_t *__restrict__ dA, const uint32_t *__restrict__ cB,
                          const uint32_t *__restrict__ dB, uint32_t *__restrict__ mark) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E) return;
    uint32_t m = 0u;
    if (t == E - 1 || key[t + 1] != key[t]) {
        int64_t s = t;
        while (s > 0 && key[s - 1] == key[t]) s--;
        const bool before = s > 0 && in_result(op, cA, dA, cB, dB, s - 1);
        m = before != in_result(op, cA, dA, cB, dB, t) ? 1u : 0u;
    }
    mark[t] = m;
}

// changes alternate start, end, start, ...: change q is the begin (q even)
// or the end (q odd) of result run q / 2
__global__ void k_change_write(const uint64_t *__restrict__ key, int64_t E, const uint32_t *__restrict__ mark,
                               const uint32_t *__restrict__ pos, uint64_t *__restrict__ begin,
                               uint64_t *__restrict__ len) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= E || !mark[t]) return;
    const uint32_t q = pos[t];
    if (q & 1u) len[q >> 1] = key[t];
    else begin[q >> 1] = key[t];
}

// run lengths as uint32 for the scan, their exact sum, and the range checks
__global__ void k_lengths(const uint64_t *__restrict__ b, const uint64_t *__restrict__ l, int64_t n,
                          uint32_t *__restrict__ len32, unsigned long long *__restrict__ sum,
                          uint32_t *__restrict__ err) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t x = l[r];
    const bool ok = b[r] < kCodeLimit && x <= kCodeLimit - b[r] && x < (1ull << 32);
    if (!ok) atomicOr(err, 1u);
    len32[r] = ok ? (uint32_t)x : 0u;
    if (ok && x) atomicAdd(sum, (unsigned long long)x);
}

// cell c of the runs: the last run whose first cell index is <= c (runs of
// length 0 share their index with the next run and are never chosen), its
// code, and the cell centre (float)(o + (i + 0.5) d) evaluated in FP64
__global__ void k_cells(const uint64_t *__restrict__ b, const uint32_t *__restrict__ off, int64_t n, int64_t total,
                        double3 o, double d, float *__restrict__ xyz) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;   // first run with off > c
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if ((int64_t)off[mid] <= c) lo = mid + 1;
            else hi = mid;
        }
        const int64_t r = lo - 1;
        uint32_t ijk[3];
        morton_decode(b[r] + (uint64_t)(c - (int64_t)off[r]), ijk[0], ijk[1], ijk[2]);
        const double oo[3] = {o.x, o.y, o.z};
        for (int a = 0; a < 3; a++)
            xyz[3 * c + a] = __double2float_rn(__dadd_rn(oo[a], __dmul_rn(__dadd_rn((double)ijk[a], 0.5), d)));
    }
}

unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>((n + 255) / 256, 1); }

// device temporaries of one call, freed on every exit
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    bool get(T **p, int64_t n) {
        void *q = nullptr;
        if (dev_malloc_raw(&q, sizeof(T) * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) return false;
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return true;
    }
};

int err_out(int code, const char *msg) {
    set_global_error(msg);
    return code;
}

// the count words and error word back on the host
int read_back(cudaStream_t s, const void *dev, void *host, size_t bytes) {
    if (cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FPPG_ERR_CUDA;
    return FPPG_OK;
}

} // namespace

extern "C" int fppg_lattice_intervals(const float *xyz_dev, int64_t n, const float *origin_host, float d,
                                      uint64_t *begin_dev, uint64_t *len_dev, int64_t cap, int64_t *n_out,
                                      void *stream) {
    if (!n_out || !origin_host || n < 0 || n > 0xffffffffll || cap < 0 || (n > 0 && !xyz_dev) ||
        (cap > 0 && (!begin_dev || !len_dev)))
        return err_out(FPPG_ERR_ARG, "fppg_lattice_intervals: null buffer or size out of range");
    if (!(d > 0.f) || !std::isfinite(d) || !std::isfinite(origin_host[0]) || !std::isfinite(origin_host[1]) ||
        !std::isfinite(origin_host[2]))
        return err_out(FPPG_ERR_ARG, "fppg_lattice_intervals: origin and d must be finite, d > 0");
    *n_out = 0;
    if (n == 0) return FPPG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch S;
    uint64_t *code[2];
    uint32_t *val[2], *hist, *tot, *start, *pos, *tmp, *words;
    const int64_t tmp_elems = scan_tmp_elems(n);
    if (!S.get(&code[0], n) || !S.get(&code[1], n) || !S.get(&val[0], n) || !S.get(&val[1], n) ||
        !S.get(&hist, kMaxDigits * std::max<int64_t>(radix_tiles(n), 1)) || !S.get(&tot, kMaxDigits) ||
        !S.get(&start, n) || !S.get(&pos, n) || !S.get(&tmp, tmp_elems) || !S.get(&words, 2))
        return err_out(FPPG_ERR_OOM, "fppg_lattice_intervals: out of device memory");
    if (cudaMemsetAsync(words, 0, 2 * sizeof(uint32_t), s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_lattice_intervals: memset failed");
    k_cell_codes<<<nblk(n), 256, 0, s>>>(xyz_dev, n, make_float3(origin_host[0], origin_host[1], origin_host[2]), d,
                                         code[0], words + 1);
    const int cb = radix_sort_u64(code, val, true, n, 63, hist, tot, s);
    k_run_starts<<<nblk(n), 256, 0, s>>>(code[cb], n, start);
    exclusive_scan_u32(start, pos, n, words, tmp, tmp_elems, s);
    uint32_t host[2] = {0u, 0u};
    if (cudaGetLastError() != cudaSuccess || read_back(s, words, host, sizeof(host)))
        return err_out(FPPG_ERR_CUDA, "fppg_lattice_intervals: a launch failed");
    if (host[1]) return err_out(FPPG_ERR_ARG, "fppg_lattice_intervals: a point lies outside the lattice");
    *n_out = host[0];
    if ((int64_t)host[0] > cap) return err_out(FPPG_ERR_ARG, "fppg_lattice_intervals: capacity below the run count");
    k_run_write<<<nblk(n), 256, 0, s>>>(code[cb], n, start, pos, begin_dev, len_dev);
    k_end_to_len<<<nblk(host[0]), 256, 0, s>>>(begin_dev, host[0], len_dev);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_lattice_intervals: a launch failed");
    return FPPG_OK;
}

extern "C" int fppg_interval_boolean(const uint64_t *a_begin_dev, const uint64_t *a_len_dev, int64_t na,
                                     const uint64_t *b_begin_dev, const uint64_t *b_len_dev, int64_t nb, int32_t op,
                                     uint64_t *begin_dev, uint64_t *len_dev, int64_t cap, int64_t *n_out,
                                     void *stream) {
    if (!n_out || na < 0 || nb < 0 || na + nb > 0x7fffffffll || cap < 0 || (na > 0 && (!a_begin_dev || !a_len_dev)) ||
        (nb > 0 && (!b_begin_dev || !b_len_dev)) || (cap > 0 && (!begin_dev || !len_dev)))
        return err_out(FPPG_ERR_ARG, "fppg_interval_boolean: null buffer or size out of range");
    if (op != FPPG_UNION && op != FPPG_DIFFERENCE && op != FPPG_INTERSECTION)
        return err_out(FPPG_ERR_ARG, "fppg_interval_boolean: unknown op");
    *n_out = 0;
    const int64_t E = 2 * (na + nb);
    if (E == 0) return FPPG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch S;
    uint64_t *key[2];
    uint32_t *ev[2], *hist, *tot, *dA, *dB, *cA, *cB, *mark, *pos, *tmp, *words;
    const int64_t tmp_elems = scan_tmp_elems(E);
    if (!S.get(&key[0], E) || !S.get(&key[1], E) || !S.get(&ev[0], E) || !S.get(&ev[1], E) ||
        !S.get(&hist, kMaxDigits * std::max<int64_t>(radix_tiles(E), 1)) || !S.get(&tot, kMaxDigits) ||
        !S.get(&dA, E) || !S.get(&dB, E) || !S.get(&cA, E) || !S.get(&cB, E) || !S.get(&mark, E) ||
        !S.get(&pos, E) || !S.get(&tmp, tmp_elems) || !S.get(&words, 2))
        return err_out(FPPG_ERR_OOM, "fppg_interval_boolean: out of device memory");
    if (cudaMemsetAsync(words, 0, 2 * sizeof(uint32_t), s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_interval_boolean: memset failed");
    k_events<<<nblk(E), 256, 0, s>>>(a_begin_dev, a_len_dev, na, b_begin_dev, b_len_dev, E, key[0], words + 1);
    const int kb = radix_sort_u64(key, ev, true, E, 64, hist, tot, s);
    k_deltas<<<nblk(E), 256, 0, s>>>(ev[kb], E, na, dA, dB);
    exclusive_scan_u32(dA, cA, E, nullptr, tmp, tmp_elems, s);
    exclusive_scan_u32(dB, cB, E, nullptr, tmp, tmp_elems, s);
    k_changes<<<nblk(E), 256, 0, s>>>(key[kb], E, op, cA, dA, cB, dB, mark);
    exclusive_scan_u32(mark, pos, E, words, tmp, tmp_elems, s);
    uint32_t host[2] = {0u, 0u};
    if (cudaGetLastError() != cudaSuccess || read_back(s, words, host, sizeof(host)))
        return err_out(FPPG_ERR_CUDA, "fppg_interval_boolean: a launch failed");
    if (host[1]) return err_out(FPPG_ERR_ARG, "fppg_interval_boolean: a run ends past 2^63");
    const int64_t m = host[0] / 2;
    *n_out = m;
    if (m > cap) return err_out(FPPG_ERR_ARG, "fppg_interval_boolean: capacity below the run count");
    k_change_write<<<nblk(E), 256, 0, s>>>(key[kb], E, mark, pos, begin_dev, len_dev);
    k_end_to_len<<<nblk(m), 256, 0, s>>>(begin_dev, m, len_dev);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_interval_boolean: a launch failed");
    return FPPG_OK;
}

extern "C" int fppg_interval_cells(const uint64_t *begin_dev, const uint64_t *len_dev, int64_t n,
                                   const float *origin_host, float d, float *xyz_dev, int64_t cap, int64_t *n_out,
                                   void *stream) {
    if (!n_out || !origin_host || n < 0 || n > 0xffffffffll || cap < 0 || (n > 0 && (!begin_dev || !len_dev)) ||
        (cap > 0 && !xyz_dev))
        return err_out(FPPG_ERR_ARG, "fppg_interval_cells: null buffer or size out of range");
    if (!(d > 0.f) || !std::isfinite(d) || !std::isfinite(origin_host[0]) || !std::isfinite(origin_host[1]) ||
        !std::isfinite(origin_host[2]))
        return err_out(FPPG_ERR_ARG, "fppg_interval_cells: origin and d must be finite, d > 0");
    *n_out = 0;
    if (n == 0) return FPPG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch S;
    uint32_t *len32, *off, *tmp, *err;
    unsigned long long *sum;
    const int64_t tmp_elems = scan_tmp_elems(n);
    if (!S.get(&len32, n) || !S.get(&off, n) || !S.get(&tmp, tmp_elems) || !S.get(&err, 1) || !S.get(&sum, 1))
        return err_out(FPPG_ERR_OOM, "fppg_interval_cells: out of device memory");
    if (cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_interval_cells: memset failed");
    k_lengths<<<nblk(n), 256, 0, s>>>(begin_dev, len_dev, n, len32, sum, err);
    exclusive_scan_u32(len32, off, n, nullptr, tmp, tmp_elems, s);
    uint32_t herr = 0u;
    unsigned long long total = 0ull;
    if (cudaGetLastError() != cudaSuccess || read_back(s, err, &herr, sizeof(herr)) ||
        read_back(s, sum, &total, sizeof(total)))
        return err_out(FPPG_ERR_CUDA, "fppg_interval_cells: a launch failed");
    if (herr) return err_out(FPPG_ERR_ARG, "fppg_interval_cells: a run ends past 2^63 or holds 2^32 cells or more");
    if (total >= (1ull << 32)) return err_out(FPPG_ERR_ARG, "fppg_interval_cells: 2^32 cells or more");
    *n_out = (int64_t)total;
    if ((int64_t)total > cap) return err_out(FPPG_ERR_ARG, "fppg_interval_cells: capacity below the cell count");
    if (total > 0) {
        const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)total + 255) / 256, 65536);
        k_cells<<<grid, 256, 0, s>>>(begin_dev, off, n, (int64_t)total,
                                     make_double3(origin_host[0], origin_host[1], origin_host[2]), (double)d, xyz_dev);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return err_out(FPPG_ERR_CUDA, "fppg_interval_cells: a launch failed");
    return FPPG_OK;
}
