// fk_noalloc.cu -- grid orthant counts without any device allocation.
//
// fk_ecdf_grid allocates its scratch (the histogram and the per-axis pass
// buffers) with cudaMallocAsync when the caller passes no workspace, and
// stages host arrays through temporary device buffers.  Some callers may not
// allocate at all once they are running: real-time loops that forbid
// allocation after start-up (cudaMalloc can synchronise the device and take
// unbounded time), and host applications or plugin frameworks that own the
// whole device memory budget and do not let a library allocate behind their
// back.  For them this file provides fk_ecdf_grid_counts_noalloc, which runs
// the same grid kernels with its scratch in a fixed array that is part of the
// library image.
#include <mutex>

#include "fk_internal.cuh"
#include "fk_nvtx.cuh"

namespace fk {

// Size of the static scratch.  It is reserved on every GPU that loads the
// library and stays reserved until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  The symbol's
// name in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached: the first call on a
// device does this set-up and should come before any stream capture.
fk_status noalloc_scratch(void** out) {
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FK_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return FK_OK;
}
}  // namespace
}  // namespace fk

using namespace fk;

extern "C" {

fk_status fk_ecdf_grid_counts_noalloc(const void* x, fk_dtype xdtype, int64_t N, int d, const double* z_axes,
                                      const int64_t* M, const uint32_t* orthant_mask, int64_t* out,
                                      fk_stream_t stream) {
    FK_RANGE("fk_ecdf_grid_counts_noalloc");
    cudaStream_t st = (cudaStream_t)stream;
    if (xdtype != FK_F32 && xdtype != FK_F64) return set_error(FK_ERR_INVALID_ARG, "xdtype must be FK_F32 or FK_F64");
    if (d < 1 || d > 8) return set_error(FK_ERR_UNSUPPORTED, "d must be in [1, 8]");
    if (N < 0 || N >= ((int64_t)1 << 32)) return set_error(FK_ERR_UNSUPPORTED, "N must be in [0, 2^32)");
    if (!M) return set_error(FK_ERR_INVALID_ARG, "M is NULL");
    for (int k = 0; k < d; ++k)
        if (M[k] < 1) return set_error(FK_ERR_INVALID_ARG, "M[%d] must be >= 1", k);
    // Cap the histogram's cell count before any size arithmetic: the histogram
    // alone takes 4 bytes per cell, so a grid with more cells than the scratch
    // holds 4-byte entries can never fit.  Checked factor by factor (no
    // product is formed that could wrap), which also bounds every product the
    // planner forms below (pass buffers <= 2^7 cells, outputs <= 2^8 cells).
    const int64_t kMaxCells = (int64_t)(kNoAllocScratchBytes / 4);
    int64_t cells = 1;
    for (int k = 0; k < d; ++k) {
        if (M[k] + 1 > kMaxCells / cells)
            return set_error(FK_ERR_UNSUPPORTED,
                             "grid too large: its histogram exceeds the %zu-byte static scratch of "
                             "fk_ecdf_grid_counts_noalloc",
                             kNoAllocScratchBytes);
        cells *= M[k] + 1;
    }
    if (!z_axes || !out || (N > 0 && !x)) return set_error(FK_ERR_INVALID_ARG, "NULL array argument");
    // Host arrays would need staging buffers, i.e. an allocation.
    if (!is_device_pointer(z_axes) || !is_device_pointer(out) || (N > 0 && !is_device_pointer(x)))
        return set_error(FK_ERR_INVALID_ARG, "fk_ecdf_grid_counts_noalloc needs device pointers for x, z_axes, out");
    // Scratch needed by the grid kernels for this shape (a host-only plan).
    Arena plan;
    int dummy = 0;
    grid_run(nullptr, xdtype, N, d, nullptr, nullptr, M, nullptr, nullptr, FK_PATH_MIXED, plan, st, &dummy);
    if (plan.used > kNoAllocScratchBytes)
        return set_error(FK_ERR_UNSUPPORTED,
                         "grid needs %zu bytes of scratch; the static scratch of fk_ecdf_grid_counts_noalloc "
                         "holds %zu bytes",
                         plan.used, kNoAllocScratchBytes);
    void* scratch = nullptr;
    FK_TRY(noalloc_scratch(&scratch));
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    Arena ar;
    ar.sizing = false;
    ar.base = (char*)scratch;
    ar.cap = kNoAllocScratchBytes;
    ar.used = 0;
    // grid_run zeroes the histogram it accumulates into on every call.
    return grid_run(x, xdtype, N, d, nullptr, z_axes, M, orthant_mask, out, FK_PATH_MIXED, ar, st, errw);
}

}  // extern "C"
