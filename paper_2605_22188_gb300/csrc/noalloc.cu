// The batched product G = R X for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: code that runs while
// a CUDA graph is being captured, plug-ins that must draw every byte from a
// host application's own device pool, and processes that must not grow
// their device footprint once a serving loop is up.  For them this file
// provides kglm_xtr_noalloc_f32, the split-K product of kglm_xtr whose
// partial tiles and tile counters live in a file-scope device array instead
// of a context's scratch.  The array is part of the library image: every GPU
// that loads the library holds KGLM_XTR_NOALLOC_SCRATCH_FLOATS floats plus
// KGLM_XTR_NOALLOC_MAX_TILES counters until the process exits.
#include <mutex>

#include "common.cuh"
#include "engine.h"
#include "kglm.h"

namespace {

static __device__ __align__(256) float g_xtr_part[KGLM_XTR_NOALLOC_SCRATCH_FLOATS];
static __device__ __align__(256) int g_xtr_counters[KGLM_XTR_NOALLOC_MAX_TILES];

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    float* part = nullptr;
    int* counters = nullptr;
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

}  // namespace

extern "C" kglm_status kglm_xtr_noalloc_f32(int32_t m, int32_t n, int32_t p, const float* R, const float* Xt,
                                             float* G, void* stream) {
    if (m < 1 || n < 1 || p < 1 || !R || !Xt || !G) return KGLM_EINVAL;
    const int64_t tr = kglm::gemm_tile_rows_f32(), tc = kglm::gemm_tile_cols_f32();
    const int64_t tiles = (((int64_t)m + tr - 1) / tr) * (((int64_t)p + tc - 1) / tc);
    if (tiles > KGLM_XTR_NOALLOC_MAX_TILES) return KGLM_EINVAL;   // beyond the fixed scratch
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return KGLM_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // an error left pending by earlier work on this thread is not this call's:
    // report it without clearing it and without launching
    if (cudaPeekAtLastError() != cudaSuccess) return KGLM_ECUDA;
    DeviceScratch ds;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_dev[dev].part == nullptr) {
            // first call on this device: device addresses of the file-scope
            // arrays (host code only holds stand-ins for them), counters to 0.
            // Not under stream capture: the set-up must run, not be recorded.
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
                cudaGetLastError();
                return KGLM_ECUDA;
            }
            if (cap != cudaStreamCaptureStatusNone) return KGLM_EINVAL;
            float* part = nullptr;
            int* counters = nullptr;
            if (cudaGetSymbolAddress((void**)&part, g_xtr_part) != cudaSuccess ||
                cudaGetSymbolAddress((void**)&counters, g_xtr_counters) != cudaSuccess ||
                cudaMemsetAsync(counters, 0, sizeof(int) * KGLM_XTR_NOALLOC_MAX_TILES, st) != cudaSuccess) {
                cudaGetLastError();
                return KGLM_ECUDA;
            }
            g_dev[dev].part = part;
            g_dev[dev].counters = counters;
        }
        ds = g_dev[dev];
    }
    kglm::GemmScratch scr{ds.part, sizeof(float) * (size_t)KGLM_XTR_NOALLOC_SCRATCH_FLOATS, ds.counters,
                          KGLM_XTR_NOALLOC_MAX_TILES};
    kglm::gemm_nt_f32_clamped(st, m, p, n, R, n, Xt, n, G, p, scr);
    if (cudaGetLastError() != cudaSuccess) return KGLM_ECUDA;
    return KGLM_OK;
}
