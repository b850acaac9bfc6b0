// mcmi_exclusive_scan_noalloc: the row-offset scan of the CSR assembly with
// its scratch in a fixed device array, for callers that cannot allocate.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where
// they need row offsets: code that runs between other work on a latency
// budget, where an allocation could block on the driver or fragment a pool;
// programs whose device memory is handed out once up front by their own
// arena; or callers that own every byte of a fixed-size device heap.  This
// entry point runs the same scan kernels as the build path, but their
// scratch (one 8-byte partial sum per 2048-element tile) lives in the
// file-scope array below instead of a stream-ordered allocation.
#include <cstdio>
#include <mutex>

#include "kernels.h"
#include "mcmi.h"

namespace {

// 16384 tiles of 2048 counts: up to 33,554,432 elements per call.  The array
// (128 KB + 8 B) stays resident on every device that loads this library
// until the process exits.
constexpr int64_t kNoAllocMaxTiles = 16384;
constexpr int64_t kNoAllocTile = 2048;   // elements per scan tile (256 threads x 8)
constexpr int64_t kNoAllocMaxN = kNoAllocMaxTiles * kNoAllocTile;

static __device__ __align__(256) int64_t g_scan_scratch[kNoAllocMaxTiles + 1];

std::mutex g_mu;
int64_t *g_scratch_ptr[128] = {};   // device address of g_scan_scratch, per device

mcmi_status fail(mcmi_status st, const char *msg)
{
    mcmi::set_error_message(msg);   // reported by mcmi_last_error()
    return st;
}

}  // namespace

extern "C" mcmi_status mcmi_exclusive_scan_noalloc(const int32_t *counts, int64_t n, int64_t *offsets,
                                                   void *stream)
{
    char msg[256];
    if (n < 0 || (n > 0 && !counts) || !offsets) {
        snprintf(msg, sizeof(msg), "mcmi_exclusive_scan_noalloc: bad argument (n=%lld, NULL array?)", (long long)n);
        return fail(MCMI_ERR_ARG, msg);
    }
    if (n > kNoAllocMaxN) {
        snprintf(msg, sizeof(msg), "mcmi_exclusive_scan_noalloc: n=%lld exceeds the fixed scratch limit of %lld elements",
                 (long long)n, (long long)kNoAllocMaxN);
        return fail(MCMI_ERR_ARG, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        snprintf(msg, sizeof(msg), "mcmi_exclusive_scan_noalloc: no usable current device (%s)", cudaGetErrorString(e));
        return fail(MCMI_ERR_CUDA, msg);
    }
    int64_t *scratch = nullptr;
    {
        // one-time set-up per device, with that device current: look up the
        // device address of the fixed array (a query, not an allocation).
        // The address stays valid while the device's primary context lives;
        // a cudaDeviceReset in this process would leave it stale (the header
        // tells callers not to use this entry point after one).
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scan_scratch);
            if (e != cudaSuccess || !ptr) {
                snprintf(msg, sizeof(msg), "mcmi_exclusive_scan_noalloc: cudaGetSymbolAddress failed (%s)",
                         cudaGetErrorString(e));
                return fail(MCMI_ERR_CUDA, msg);
            }
            g_scratch_ptr[dev] = static_cast<int64_t *>(ptr);
        }
        scratch = g_scratch_ptr[dev];
    }
    // every tile sum is written by the first kernel before it is read, so the
    // array needs no clearing between calls
    e = mcmi::scan_counts(counts, n, offsets, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "mcmi_exclusive_scan_noalloc: launch failed (%s)", cudaGetErrorString(e));
        return fail(MCMI_ERR_CUDA, msg);
    }
    return MCMI_OK;
}
