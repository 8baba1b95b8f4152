// fppg_forces_static: the neighbour grid and force pass (A1-A4) on caller
// buffers, with every temporary in one file-scope device array, so the call
// allocates nothing.
//
// It exists for callers that cannot call cudaMalloc themselves or through
// this library: applications whose device memory is owned entirely by their
// own pool allocator (a stray cudaMalloc would bypass its accounting and can
// fail once the pool holds the device), and time-critical loops that must
// not pay for an allocation or for the implicit device synchronisation that
// cudaMalloc / cudaFree may perform.  The paper has no counterpart.
//
// The scratch below is a plain __device__ array: every GPU that loads the
// library holds it (about 9.5 MB) until the process exits.  In host code its
// name is only a host-side stand-in, not a device address, so the address is
// looked up with cudaGetSymbolAddress once per device (on the first call
// made with that device current; make that first call before any stream
// capture) and passed to the kernels.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/fppg.h"
#include "body.h"

namespace fppg {
namespace {

constexpr int64_t kStaticMaxN = 65536;       // particles per call
constexpr int64_t kStaticMaxCells = 131072;  // neighbour-grid cells
constexpr int64_t kStaticMaxTiles = (kStaticMaxN + 1023) / 1024;  // tiles of the smallest radix tile

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// byte offsets inside the scratch array
constexpr size_t kOffParams = 0;
constexpr size_t kOffFlags = kOffParams + align256(sizeof(AsmParams));        // (unused), amax, maxdisp, queue (2), error
constexpr size_t kOffTotals = kOffFlags + 256;
constexpr size_t kOffHist = kOffTotals + align256(kMaxDigits * 4);
constexpr size_t kOffPos = kOffHist + align256(kMaxDigits * 4 * kStaticMaxTiles);
constexpr size_t kOffKey0 = kOffPos + align256(16 * kStaticMaxN);
constexpr size_t kOffKey1 = kOffKey0 + align256(4 * kStaticMaxN);
constexpr size_t kOffId0 = kOffKey1 + align256(4 * kStaticMaxN);
constexpr size_t kOffId1 = kOffId0 + align256(4 * kStaticMaxN);
constexpr size_t kOffPosS = kOffId1 + align256(4 * kStaticMaxN);
constexpr size_t kOffPosP = kOffPosS + align256(16 * kStaticMaxN);
constexpr size_t kOffAccS = kOffPosP + align256(16 * (kStaticMaxN + 1));
constexpr int64_t kStaticMaxFine = kSlabs * kStaticMaxCells + 1;   // fine keys + 1
constexpr size_t kOffFstart = kOffAccS + align256(16 * kStaticMaxN);
constexpr size_t kOffBstart = kOffFstart + align256(4 * kStaticMaxFine);
constexpr size_t kScratchBytes = kOffBstart + align256(4 * (start_blocks(kStaticMaxFine) + 1));

__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_addr_mu;
unsigned char *g_addr[64] = {nullptr};

// positions and one-hot classes of body 0; a class outside 0..4 raises the
// error word and becomes a fixed particle
__global__ void k_pack_static(const float *__restrict__ xyz, const int32_t *__restrict__ cls, int64_t n,
                              float4 *__restrict__ pos, uint32_t *__restrict__ error) {
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    int c = cls[i];
    if (c < 0 || c > 4) {
        atomicOr(error, 1u);
        c = kClsI;
    }
    pos[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __uint_as_float(class_bit(c)));
}

} // namespace
} // namespace fppg

namespace fppg {
void set_global_error(const char *msg);
}

using namespace fppg;

extern "C" int fppg_forces_static(const float *xyz_dev, const int32_t *cls_dev, int64_t n, const float *bbmin_host,
                                  const float *bbmax_host, float h, int32_t fixed_features, float *acc_dev,
                                  float *amax_host, void *stream) {
    if (n < 0 || n > kStaticMaxN) {
        set_global_error("fppg_forces_static: n must be in [0, 65536] (static scratch limit)");
        return FPPG_ERR_ARG;
    }
    if ((n > 0 && (!xyz_dev || !cls_dev || !acc_dev)) || !bbmin_host || !bbmax_host || !(h > 0.f) ||
        !std::isfinite(h)) {
        set_global_error("fppg_forces_static: null buffer or h not finite and positive");
        return FPPG_ERR_ARG;
    }
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(bbmin_host[k]) || !std::isfinite(bbmax_host[k]) || bbmin_host[k] > bbmax_host[k]) {
            set_global_error("fppg_forces_static: bounding box not finite or inverted");
            return FPPG_ERR_ARG;
        }
    // neighbour grid of the body: the rule of fppg_create
    AsmParams A;
    memset(&A, 0, sizeof(A));
    const float R = 2.0f * h;
    const float cell = (float)((double)R * (1.0 + 1.0 / 256.0));
    // each axis is bounded (2^20) before the product, so the product cannot
    // wrap; it is then taken in FP64 against the scratch limit
    const bool axes_ok = grid_setup(bbmin_host, bbmax_host, cell, 1.0, 1, A.ng_o, &A.ng_inv, A.ng_n);
    const double cells_d = (double)A.ng_n[0] * (double)A.ng_n[1] * (double)A.ng_n[2];
    if (!axes_ok || !(cells_d <= (double)kStaticMaxCells)) {
        set_global_error("fppg_forces_static: the box needs more than 131072 grid cells of 2h (static scratch limit)");
        return FPPG_ERR_ARG;
    }
    const double hd = (double)h;
    A.h = h;
    A.R2 = (float)((double)R * (double)R);
    A.slab_r2 = slab_reach2(A.R2, A.ng_inv);
    A.half_inv_h = (float)(1.0 / (2.0 * hd));
    A.force_scale = (float)(5.0 * (21.0 / (16.0 * M_PI * hd * hd * hd)) / (hd * hd));
    A.step_h = (float)(hd / 16.0);
    A.fixed_features = fixed_features ? 1 : 0;
    A.mobile = (1 << kClsS) | (1 << kClsV) | (1 << kClsF);
    A.npart = 0;
    A.amax_slot = 0;
    A.p_end = (int)n;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_global_error("fppg_forces_static: no current CUDA device");
        return FPPG_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) {
                char msg[200];
                snprintf(msg, sizeof(msg), "fppg_forces_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                set_global_error(msg);
                return FPPG_ERR_CUDA;
            }
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *flags = (uint32_t *)(base + kOffFlags);
    DevGroup d;
    d.B = 1;
    d.N = n;
    const int64_t cells = (int64_t)cells_d;
    d.total_cells = cells;
    d.key_bits = fine_key_bits(cells);
    int digit_bits = 8;
    d.passes = radix_pass_plan(d.key_bits, &digit_bits);
    d.n_tiles = (int)std::max<int64_t>(radix_tiles(n), 1);
    d.params = (AsmParams *)(base + kOffParams);
    d.pos = (float4 *)(base + kOffPos);
    d.key[0] = (uint32_t *)(base + kOffKey0);
    d.key[1] = (uint32_t *)(base + kOffKey1);
    d.id[0] = (uint32_t *)(base + kOffId0);
    d.id[1] = (uint32_t *)(base + kOffId1);
    d.pos_s = (float4 *)(base + kOffPosS);
    d.pos_p = (float4 *)(base + kOffPosP);
    d.acc_s = (float4 *)(base + kOffAccS);
    d.fstart = (uint32_t *)(base + kOffFstart);
    d.bstart = (uint32_t *)(base + kOffBstart);
    d.amax = flags + 1;
    d.maxdisp = flags + 2;
    d.work_count = flags + 3;   // two words: front and back of the search queue
    d.hist = (uint32_t *)(base + kOffHist);
    d.totals = (uint32_t *)(base + kOffTotals);
    uint32_t *error = flags + 5;
    // the error word and amax start at zero on every call
    if (cudaMemcpyAsync(d.params, &A, sizeof(A), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(error, 0, sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(d.amax, 0, sizeof(uint32_t), s) != cudaSuccess) {
        set_global_error("fppg_forces_static: could not set up the scratch");
        return FPPG_ERR_CUDA;
    }
    if (n > 0) {
        k_pack_static<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(xyz_dev, cls_dev, n, d.pos, error);
        const int buf = build_grid_dev(d, s);
        forces_dev(d, 256, 0, s);
        unpermute_dev(d, buf, s, acc_dev, nullptr, nullptr);
        // a launch that failed to start is not reported by the synchronise
        // below: ask for it here
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            char msg[200];
            snprintf(msg, sizeof(msg), "fppg_forces_static: launch failed: %s", cudaGetErrorString(le));
            set_global_error(msg);
            cudaStreamSynchronize(s);
            return FPPG_ERR_CUDA;
        }
    }
    uint32_t err_h = 0, amax_h = 0;
    cudaMemcpyAsync(&err_h, error, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&amax_h, d.amax, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "fppg_forces_static: %s", cudaGetErrorString(e));
        set_global_error(msg);
        return FPPG_ERR_CUDA;
    }
    if (err_h) {
        set_global_error("fppg_forces_static: a class outside 0..4 (treated as fixed)");
        return FPPG_ERR_ARG;
    }
    if (amax_host) memcpy(amax_host, &amax_h, sizeof(float));
    return FPPG_OK;
}
