// fk_api.cu -- extern "C" entry points of fastecdf.h: argument validation,
// host/device staging of the caller's arrays, workspace handling, dispatch.
#include <algorithm>
#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "fk_dc_ops.cuh"
#include "fk_nvtx.cuh"

namespace fk {
fk_status kde_backward_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                           const double* h, unsigned flags, const double* g, double* gw, double* gz, double* gh,
                           fk_path path, Arena& ar, cudaStream_t st);
fk_status loo_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* h, double* L,
                  double* gh, fk_path path, Arena& ar, cudaStream_t st);

fk_status kde_grid_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* z_dev,
                       const int64_t* M, const double* h, double* out, fk_path path, Arena& ar, cudaStream_t st,
                       int* err_word);
fk_status grid_interp_run(const double* f, int d, const double* z_dev, const int64_t* M, const void* q, fk_dtype qd,
                          int64_t nq, double* out, Arena& ar, cudaStream_t st, int* err_word);

fk_status uniform_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                      const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st);
fk_status matern32_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                       const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st);
fk_status hmatrix_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                      const double* R, const double* hd, unsigned flags, double* out, fk_path path, Arena& ar,
                      cudaStream_t st);
fk_status loclin_run(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                     const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st);

fk_status batched_run(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h, int64_t* ecdf_out,
                      double* kde_out, fk_path path, const BatchCfg& cfg, Arena& ar, cudaStream_t st);

static thread_local char g_msg[512] = "no error";

fk_status set_error(fk_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

fk_status cuda_error(cudaError_t e, const char* where) {
    return set_error(FK_ERR_CUDA, "CUDA error %d (%s) at %s", (int)e, cudaGetErrorString(e), where);
}

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked host memory (cudaHostAlloc / cudaHostRegister): copies to and
// from it are asynchronous on the stream.
static bool is_pinned_host_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct ProfRec { int fam; double bytes; double mem; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_free_events;
bool profiling_on() { return g_prof_on.load(std::memory_order_relaxed); }
cudaEvent_t prof_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void prof_record(int family, double work, double bytes, cudaEvent_t a, cudaEvent_t b) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(ProfRec{family, work, bytes, a, b});
}

// The per-device error word: kernels record the first device-side error here
// (atomicCAS from 0); fk_device_status reads and clears it.
__device__ int g_fk_err_word = 0;

fk_status device_error_word(int** ptr) {
    FK_CUDA(cudaGetSymbolAddress((void**)ptr, g_fk_err_word));
    return FK_OK;
}

// Library-owned stream-ordered memory pool of each device, for staging
// buffers and internal workspaces.  Freed blocks stay in the pool for the next
// call (the default pool would hand them back to the driver at every
// synchronisation and map them again); fk_release_cached_memory() trims it.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static fk_status lib_pool(cudaMemPool_t* out) {
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(FK_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        FK_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = UINT64_MAX;
        FK_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return FK_OK;
}

static fk_status pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    FK_TRY(lib_pool(&pool));
    FK_CUDA(cudaMallocFromPoolAsync(p, bytes, pool, st));
    return FK_OK;
}

// Stages caller arrays that live in host memory through device buffers.  The
// staging buffers are allocated and freed in stream order.  If every host
// array of the call is page-locked the copies stay asynchronous and so does
// the call; a pageable host array makes the call wait for its host outputs.
struct Stager {
    cudaStream_t st;
    std::vector<void*> allocs;
    struct Out { void* dev; void* host; size_t bytes; };
    std::vector<Out> outs;
    bool any_pageable = false;
    explicit Stager(cudaStream_t s) : st(s) {}
    ~Stager() {
        for (void* p : allocs) cudaFreeAsync(p, st);
    }
    // input array: returns a device pointer holding the same bytes
    fk_status in(const void* p, size_t bytes, const void** dev) {
        *dev = p;
        if (!p || bytes == 0 || is_device_pointer(p)) return FK_OK;
        if (!is_pinned_host_pointer(p)) any_pageable = true;
        void* d = nullptr;
        FK_TRY(pool_alloc(&d, bytes, st));
        allocs.push_back(d);
        FK_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, st));
        *dev = d;
        return FK_OK;
    }
    // output array: device pointer to write; host copies back in finish()
    fk_status out(void* p, size_t bytes, void** dev) {
        *dev = p;
        if (!p || bytes == 0 || is_device_pointer(p)) return FK_OK;
        if (!is_pinned_host_pointer(p)) any_pageable = true;
        void* d = nullptr;
        FK_TRY(pool_alloc(&d, bytes, st));
        allocs.push_back(d);
        outs.push_back(Out{d, p, bytes});
        *dev = d;
        return FK_OK;
    }
    fk_status finish() {
        for (auto& o : outs)
            FK_CUDA(cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, st));
        if (any_pageable) FK_CUDA(cudaStreamSynchronize(st));
        return FK_OK;
    }
};

// Workspace: caller scratch, or a stream-ordered allocation of the planned size.
struct Workspace {
    cudaStream_t st;
    void* owned = nullptr;
    explicit Workspace(cudaStream_t s) : st(s) {}
    ~Workspace() {
        if (owned) cudaFreeAsync(owned, st);
    }
    fk_status bind(Arena& ar, void* ws, size_t ws_bytes, size_t need) {
        ar.sizing = false;
        ar.used = 0;
        if (ws) {
            if (ws_bytes < need)
                return set_error(FK_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, need);
            if (((uintptr_t)ws & 255u) != 0)
                return set_error(FK_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
            ar.base = (char*)ws;
            ar.cap = ws_bytes;
            return FK_OK;
        }
        if (need > 0) FK_TRY(pool_alloc(&owned, need, st));
        ar.base = (char*)owned;
        ar.cap = need;
        return FK_OK;
    }
};

static size_t dtype_size(fk_dtype t) { return t == FK_F64 ? 8 : 4; }

static fk_status check_common(const void* x, fk_dtype xd, int64_t N, int d, fk_path path) {
    if (xd != FK_F32 && xd != FK_F64) return set_error(FK_ERR_INVALID_ARG, "xdtype must be FK_F32 or FK_F64");
    if (path != FK_PATH_MIXED && path != FK_PATH_FP64) return set_error(FK_ERR_INVALID_ARG, "unknown precision path");
    if (N < 0) return set_error(FK_ERR_INVALID_ARG, "N must be >= 0");
    if (N > 0 && !x) return set_error(FK_ERR_INVALID_ARG, "x is NULL");
    if (d < 1) return set_error(FK_ERR_INVALID_ARG, "d must be >= 1");
    return FK_OK;
}

}  // namespace fk

using namespace fk;

extern "C" {

const char* fk_last_error(void) { return g_msg; }

const char* fk_version(void) { return "fastecdf-gb300 0.1 (sm_103a)"; }

uint64_t fk_kernel_launches(void) { return (uint64_t)g_launches.load(); }

void fk_profile_enable(int on) { g_prof_on.store(on != 0); }

void fk_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) { g_free_events.push_back(r.a); g_free_events.push_back(r.b); }
    g_prof.clear();
}

fk_status fk_profile_read_bytes(int family, double* bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double by = 0.0;
    for (auto& r : g_prof)
        if (r.fam == family) by += r.mem;
    if (bytes) *bytes = by;
    return FK_OK;
}

fk_status fk_profile_read(int family, double* total_ms, uint64_t* launches, double* alg_bytes) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double ms = 0.0, by = 0.0;
    uint64_t cnt = 0;
    for (auto& r : g_prof) {
        if (r.fam != family) continue;
        FK_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        FK_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        by += r.bytes;
        ++cnt;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    if (alg_bytes) *alg_bytes = by;
    return FK_OK;
}

fk_status fk_release_cached_memory(void) {
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (dev >= 0 && dev < 64) p = g_pool[dev];
    }
    if (p) FK_CUDA(cudaMemPoolTrimTo(p, 0));
    return FK_OK;
}

fk_status fk_device_status(fk_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int* w = nullptr;
    FK_TRY(device_error_word(&w));
    FK_CUDA(cudaStreamSynchronize(st));
    int v = 0;
    FK_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    int zero = 0;
    FK_CUDA(cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice));
    switch (v) {
        case 0: return FK_OK;
        case DEV_TIMEOUT: return set_error(FK_ERR_TIMEOUT, "a bounded device wait ran out");
        case DEV_AXIS: return set_error(FK_ERR_INVALID_ARG, "grid axis not strictly increasing (device check)");
        case DEV_NONFINITE: return set_error(FK_ERR_NONFINITE, "non-finite coordinate in x or z (device check)");
        default: return set_error(FK_ERR_CUDA, "device error code %d", v);
    }
}

fk_status fk_debug_lookback_timeout(int64_t n, fk_stream_t stream) {
    FK_TRY(radix_lookback_timeout_probe(n, (cudaStream_t)stream));
    return fk_device_status(stream);
}

// ------------------------------------------------------------------ grid path
static fk_status grid_validate(const void* x, fk_dtype xd, int64_t N, int d, const int64_t* M,
                               fk_path path) {
    FK_TRY(check_common(x, xd, N, d, path));
    if (d > 8) return set_error(FK_ERR_UNSUPPORTED, "ecdf_grid supports d <= 8");
    if (!M) return set_error(FK_ERR_INVALID_ARG, "M is NULL");
    int64_t cells = 1;
    for (int k = 0; k < d; ++k) {
        if (M[k] < 1) return set_error(FK_ERR_INVALID_ARG, "M[%d] must be >= 1", k);
        if (cells > ((int64_t)1 << 40) / (M[k] + 1)) return set_error(FK_ERR_UNSUPPORTED, "grid too large");
        cells *= (M[k] + 1);
    }
    if (N >= ((int64_t)1 << 32)) return set_error(FK_ERR_UNSUPPORTED, "N must be < 2^32 on the grid path");
    return FK_OK;
}

size_t fk_ecdf_grid_workspace(int64_t N, int d, const int64_t* M, int weighted, fk_path path) {
    if (grid_validate((const void*)1, FK_F32, N, d, M, path) != FK_OK) return 0;
    Arena ar;
    int one = 0;
    grid_run(nullptr, FK_F32, N, d, weighted ? (const void*)1 : nullptr, nullptr, M, nullptr,
             nullptr, path, ar, 0, &one);
    return ar.used;
}

fk_status fk_ecdf_grid(const void* x, fk_dtype xd, int64_t N, int d, const void* y,
                       const double* z_axes, const int64_t* M, const uint32_t* orthant_mask,
                       void* out, fk_path path, void* ws, size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_ecdf_grid");
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(grid_validate(x, xd, N, d, M, path));
    if (!z_axes) return set_error(FK_ERR_INVALID_ARG, "z_axes is NULL");
    if (!out) return set_error(FK_ERR_INVALID_ARG, "out is NULL");   // a grid has >= 1 point
    int64_t ztot = 0, gpts = 1;
    for (int k = 0; k < d; ++k) { ztot += M[k]; gpts *= M[k]; }
    // host-side monotonicity check when the axes are host memory
    if (!is_device_pointer(z_axes)) {
        int64_t off = 0;
        for (int k = 0; k < d; ++k) {
            for (int64_t j = 0; j < M[k]; ++j) {
                double v = z_axes[off + j];
                if (!(v == v) || (j > 0 && !(z_axes[off + j - 1] < v)))
                    return set_error(FK_ERR_INVALID_ARG, "grid axis %d not strictly increasing at %lld", k, (long long)j);
            }
            off += M[k];
        }
    }
    int nsel = 0;
    for (int o = 0; o < (1 << d); ++o)
        if (!orthant_mask || ((orthant_mask[o >> 5] >> (o & 31)) & 1u)) ++nsel;
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xd_p = nullptr, *yd_p = nullptr, *zd_p = nullptr;
    void* od_p = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xd_p));
    FK_TRY(sg.in(y, (size_t)N * ds, &yd_p));
    FK_TRY(sg.in(z_axes, (size_t)ztot * sizeof(double), &zd_p));
    FK_TRY(sg.out(out, (size_t)nsel * gpts * 8, &od_p));
    Arena plan;
    int dummy = 0;
    grid_run(nullptr, xd, N, d, y, nullptr, M, nullptr, nullptr, path, plan, st, &dummy);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    FK_TRY(grid_run(xd_p, xd, N, d, yd_p, (const double*)zd_p, M, orthant_mask, od_p, path, ar, st, errw));
    return sg.finish();
}

static fk_status check_h(const double* h, int d) {
    if (!h) return set_error(FK_ERR_INVALID_ARG, "h is NULL");
    for (int k = 0; k < d; ++k)
        if (!(h[k] > 0.0) || !(h[k] < 1e300)) return set_error(FK_ERR_INVALID_ARG, "h[%d] must be finite and > 0", k);
    return FK_OK;
}

// host-side strict monotonicity of host-resident axes
static fk_status check_axes_host(const double* z_axes, int d, const int64_t* M) {
    if (is_device_pointer(z_axes)) return FK_OK;
    int64_t off = 0;
    for (int k = 0; k < d; ++k) {
        for (int64_t j = 0; j < M[k]; ++j) {
            const double v = z_axes[off + j];
            if (!(v == v) || (j > 0 && !(z_axes[off + j - 1] < v)))
                return set_error(FK_ERR_INVALID_ARG, "grid axis %d not strictly increasing at %lld", k, (long long)j);
        }
        off += M[k];
    }
    return FK_OK;
}

size_t fk_kde_grid_workspace(int64_t N, int d, const int64_t* M, fk_path path) {
    if (grid_validate((const void*)1, FK_F32, N, d, M, path) != FK_OK) return 0;
    Arena ar;
    int one = 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    kde_grid_run(nullptr, FK_F32, N, d, nullptr, nullptr, M, h, nullptr, path, ar, 0, &one);
    return ar.used;
}

fk_status fk_kde_grid(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* z_axes,
                      const int64_t* M, const double* h, double* out, fk_path path, void* ws, size_t ws_bytes,
                      fk_stream_t stream) {
    FK_RANGE("fk_kde_grid");
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(grid_validate(x, xd, N, d, M, path));
    FK_TRY(check_h(h, d));
    if (!z_axes) return set_error(FK_ERR_INVALID_ARG, "z_axes is NULL");
    if (!out) return set_error(FK_ERR_INVALID_ARG, "out is NULL");
    FK_TRY(check_axes_host(z_axes, d, M));
    int64_t ztot = 0, gpts = 1;
    for (int k = 0; k < d; ++k) { ztot += M[k]; gpts *= M[k]; }
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *wp = nullptr, *zp = nullptr;
    void* op = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(w, (size_t)N * ds, &wp));
    FK_TRY(sg.in(z_axes, (size_t)ztot * sizeof(double), &zp));
    FK_TRY(sg.out(out, (size_t)gpts * 8, &op));
    Arena plan;
    int dummy = 0;
    kde_grid_run(nullptr, xd, N, d, w, nullptr, M, h, nullptr, path, plan, st, &dummy);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    FK_TRY(kde_grid_run(xp, xd, N, d, wp, (const double*)zp, M, h, (double*)op, path, ar, st, errw));
    return sg.finish();
}

size_t fk_grid_interp_workspace(void) {
    Arena ar;
    int one = 0;
    int64_t M[1] = {1};
    grid_interp_run(nullptr, 1, nullptr, M, nullptr, FK_F64, 0, nullptr, ar, 0, &one);
    return ar.used;
}

fk_status fk_grid_interp(const double* f, int d, const double* z_axes, const int64_t* M, const void* q,
                         fk_dtype qd, int64_t Q, double* out, void* ws, size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_grid_interp");
    cudaStream_t st = (cudaStream_t)stream;
    if (qd != FK_F32 && qd != FK_F64) return set_error(FK_ERR_INVALID_ARG, "qdtype must be FK_F32 or FK_F64");
    if (d < 1 || d > 8) return set_error(FK_ERR_UNSUPPORTED, "grid_interp supports d in [1, 8]");
    if (!M || !z_axes || !f) return set_error(FK_ERR_INVALID_ARG, "f, z_axes and M must be given");
    if (Q < 0) return set_error(FK_ERR_INVALID_ARG, "Q must be >= 0");
    if (Q > 0 && (!q || !out)) return set_error(FK_ERR_INVALID_ARG, "q and out must be given");
    int64_t ztot = 0, gpts = 1;
    for (int k = 0; k < d; ++k) {
        if (M[k] < 1) return set_error(FK_ERR_INVALID_ARG, "M[%d] must be >= 1", k);
        ztot += M[k];
        gpts *= M[k];
    }
    FK_TRY(check_axes_host(z_axes, d, M));
    Stager sg(st);
    const void *fp = nullptr, *zp = nullptr, *qp = nullptr;
    void* op = nullptr;
    FK_TRY(sg.in(f, (size_t)gpts * 8, &fp));
    FK_TRY(sg.in(z_axes, (size_t)ztot * sizeof(double), &zp));
    FK_TRY(sg.in(q, (size_t)Q * d * dtype_size(qd), &qp));
    FK_TRY(sg.out(out, (size_t)Q * 8, &op));
    Arena plan;
    int dummy = 0;
    grid_interp_run(nullptr, d, nullptr, M, nullptr, qd, Q, nullptr, plan, st, &dummy);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    FK_TRY(grid_interp_run((const double*)fp, d, (const double*)zp, M, qp, qd, Q, (double*)op, ar, st, errw));
    return sg.finish();
}

// ------------------------------------------------------------------ sample-point path
// max_d: 8 for orthant counts (inclusion-exclusion over dominance counts),
// 6 for the weighted orthant sums, the KDE and Nadaraya-Watson (2^(d-1)
// channels per sweep), 4 for what needs per-orthant terms or signed sums (the
// adjoint and the leave-one-out likelihood).
static fk_status points_validate(const void* x, fk_dtype xd, int64_t N, int d, const void* z, int64_t M,
                                 fk_path path, bool doubled, int max_d = 6) {
    FK_TRY(check_common(x, xd, N, d, path));
    if (d > max_d)
        return set_error(FK_ERR_UNSUPPORTED, "this sample-point call supports d <= %d (counts: d <= 8)", max_d);
    if (z && M < 0) return set_error(FK_ERR_INVALID_ARG, "M must be >= 0");
    const int64_t items = z ? N + M : (doubled ? 2 * N : N);
    if (items >= ((int64_t)1 << dc::kItemBits))
        return set_error(FK_ERR_UNSUPPORTED, "too many items (%lld) for the sample-point path", (long long)items);
    return FK_OK;
}


size_t fk_ecdf_points_workspace(int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path) {
    const void* z = sample_points ? nullptr : (const void*)1;
    if (points_validate((const void*)1, FK_F32, N, d, z, M, path, true, weighted ? 6 : 8) != FK_OK) return 0;
    size_t best = 0;
    for (int t = 0; t < 2; ++t) {   // size for both dtypes (FP64 keys are wider)
        Arena ar;
        points_orthant(nullptr, t ? FK_F64 : FK_F32, N, d, weighted ? (const void*)1 : nullptr, z, M, nullptr,
                       nullptr, path, ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

static fk_status ecdf_points_impl(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z,
                                  int64_t M, const uint32_t* mask, void* out, fk_path path, void* ws,
                                  size_t ws_bytes, fk_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(points_validate(x, xd, N, d, z, M, path, true, y ? 6 : 8));
    const int64_t m_out = z ? M : N;
    int nsel = 0;
    for (int o = 0; o < (1 << d); ++o)
        if (!mask || ((mask[o >> 5] >> (o & 31)) & 1u)) ++nsel;
    if (nsel == 0 || m_out == 0) return FK_OK;          // nothing to write
    if (!out) return set_error(FK_ERR_INVALID_ARG, "out is NULL");
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *yp = nullptr, *zp = nullptr;
    void* op = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(y, (size_t)N * ds, &yp));
    FK_TRY(sg.in(z, z ? (size_t)M * d * ds : 0, &zp));
    FK_TRY(sg.out(out, (size_t)nsel * m_out * 8, &op));
    if (z && !zp) zp = z;
    Arena plan;
    points_orthant(nullptr, xd, N, d, y, z, M, mask, nullptr, path, plan, st);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    FK_TRY(points_orthant(xp, xd, N, d, yp, zp, M, mask, op, path, ar, st));
    return sg.finish();
}

fk_status fk_ecdf_points(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                         const uint32_t* orthant_mask, void* out, fk_path path, void* ws, size_t ws_bytes,
                         fk_stream_t stream) {
    FK_RANGE("fk_ecdf_points");
    return ecdf_points_impl(x, xd, N, d, y, z, M, orthant_mask, out, path, ws, ws_bytes, stream);
}

fk_status fk_esf_points(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                        void* out, fk_path path, void* ws, size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_esf_points");
    if (d < 1 || d > 8) return set_error(FK_ERR_UNSUPPORTED, "d out of range");
    uint32_t mask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int o = (1 << d) - 1;
    mask[o >> 5] = 1u << (o & 31);
    return ecdf_points_impl(x, xd, N, d, y, z, M, mask, out, path, ws, ws_bytes, stream);
}

size_t fk_kde_laplace_workspace(int64_t N, int d, int64_t M, int sample_points, int want_terms, fk_path path) {
    const void* z = sample_points ? nullptr : (const void*)1;
    if (points_validate((const void*)1, FK_F32, N, d, z, M, path, false) != FK_OK) return 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    size_t best = 0;
    for (int t = 0; t < 2; ++t) {
        Arena ar;
        points_kernel(nullptr, t ? FK_F64 : FK_F32, N, d, (const void*)1, z, M, h, 0, 1, nullptr,
                      want_terms ? (double*)1 : nullptr, path, ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

size_t fk_kreg_laplace_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path) {
    const void* z = sample_points ? nullptr : (const void*)1;
    if (points_validate((const void*)1, FK_F32, N, d, z, M, path, false) != FK_OK) return 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    size_t best = 0;
    for (int t = 0; t < 2; ++t) {
        Arena ar;
        points_kernel(nullptr, t ? FK_F64 : FK_F32, N, d, (const void*)1, z, M, h, 0, 2, nullptr, nullptr, path,
                      ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

static fk_status kernel_impl(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                             const double* h, unsigned flags, int nw, double* out, double* terms, fk_path path,
                             void* ws, size_t ws_bytes, fk_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(points_validate(x, xd, N, d, z, M, path, false));
    FK_TRY(check_h(h, d));
    if ((flags & FK_LOO) && z) return set_error(FK_ERR_INVALID_ARG, "FK_LOO needs z == NULL");
    const int64_t m_out = z ? M : N;
    if (m_out == 0) return FK_OK;                        // nothing to write
    if (!out) return set_error(FK_ERR_INVALID_ARG, "out is NULL");
    if (nw == 2 && !w && N > 0) return set_error(FK_ERR_INVALID_ARG, "y is NULL");
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *wp = nullptr, *zp = nullptr;
    void *op = nullptr, *tp = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(w, (size_t)N * ds, &wp));
    FK_TRY(sg.in(z, z ? (size_t)M * d * ds : 0, &zp));
    FK_TRY(sg.out(out, (size_t)m_out * 8, &op));
    FK_TRY(sg.out(terms, terms ? ((size_t)1 << d) * m_out * 8 : 0, &tp));
    Arena plan;
    points_kernel(nullptr, xd, N, d, w, z, M, h, flags, nw, nullptr, terms, path, plan, st);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    FK_TRY(points_kernel(xp, xd, N, d, wp, zp, M, h, flags, nw, (double*)op, (double*)tp, path, ar, st));
    return sg.finish();
}

fk_status fk_kde_laplace(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                         const double* h, unsigned flags, double* out, double* orthant_terms, fk_path path,
                         void* ws, size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_kde_laplace");
    return kernel_impl(x, xd, N, d, w, z, M, h, flags, 1, out, orthant_terms, path, ws, ws_bytes, stream);
}

fk_status fk_kreg_laplace(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                          const double* h, unsigned flags, double* out, fk_path path, void* ws, size_t ws_bytes,
                          fk_stream_t stream) {
    FK_RANGE("fk_kreg_laplace");
    return kernel_impl(x, xd, N, d, y, z, M, h, flags, 2, out, nullptr, path, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ adjoints
size_t fk_kde_laplace_backward_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path) {
    const void* z = sample_points ? nullptr : (const void*)1;
    if (points_validate((const void*)1, FK_F32, N, d, z, M, path, false, 4) != FK_OK) return 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    // the plan differs with and without weights (terms vs signed sums): the larger
    size_t best = 0;
    for (int t = 0; t < 4; ++t) {
        Arena ar;
        // plans pass placeholders: x must be non-NULL, the transposed pass at
        // explicit targets takes it as its target array
        kde_backward_run((const void*)1, (t & 1) ? FK_F64 : FK_F32, N, d, (t & 2) ? (const void*)1 : nullptr, z, M, h, 0,
                         nullptr, (double*)1, sample_points ? nullptr : (double*)1, (double*)1, path, ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

fk_status fk_kde_laplace_backward(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                                  int64_t M, const double* h, unsigned flags, const double* grad_out,
                                  double* grad_w, double* grad_z, double* grad_h, fk_path path, void* ws,
                                  size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_kde_laplace_backward");
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(points_validate(x, xd, N, d, z, M, path, false, 4));
    FK_TRY(check_h(h, d));
    if ((flags & FK_LOO) && z) return set_error(FK_ERR_INVALID_ARG, "FK_LOO needs z == NULL");
    if (grad_z && !z) return set_error(FK_ERR_INVALID_ARG, "grad_z needs explicit targets z");
    const int64_t m_out = z ? M : N;
    if (m_out > 0 && !grad_out) return set_error(FK_ERR_INVALID_ARG, "grad_out is NULL");
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *wp = nullptr, *zp = nullptr, *gp = nullptr;
    void *gwp = nullptr, *gzp = nullptr, *ghp = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(w, (size_t)N * ds, &wp));
    FK_TRY(sg.in(z, z ? (size_t)M * d * ds : 0, &zp));
    FK_TRY(sg.in(grad_out, (size_t)m_out * 8, &gp));
    FK_TRY(sg.out(grad_w, (size_t)N * 8, &gwp));
    FK_TRY(sg.out(grad_z, z ? (size_t)M * d * 8 : 0, &gzp));
    FK_TRY(sg.out(grad_h, (size_t)d * 8, &ghp));
    Arena plan;
    kde_backward_run((const void*)1, xd, N, d, w, z, M, h, flags, nullptr, (double*)grad_w, (double*)grad_z,
                     (double*)grad_h, path, plan, st);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    if (N == 0 || m_out == 0) {
        if (gwp && N) FK_CUDA(cudaMemsetAsync(gwp, 0, (size_t)N * 8, st));
        if (gzp && M) FK_CUDA(cudaMemsetAsync(gzp, 0, (size_t)M * d * 8, st));
        if (ghp) FK_CUDA(cudaMemsetAsync(ghp, 0, (size_t)d * 8, st));
        return sg.finish();
    }
    FK_TRY(kde_backward_run(xp, xd, N, d, wp, zp, M, h, flags, (const double*)gp, (double*)gwp, (double*)gzp,
                            (double*)ghp, path, ar, st));
    return sg.finish();
}

size_t fk_loo_laplace_workspace(int64_t N, int d, fk_path path) {
    if (points_validate((const void*)1, FK_F32, N, d, nullptr, 0, path, false, 4) != FK_OK) return 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    size_t best = 0;
    for (int t = 0; t < 4; ++t) {
        Arena ar;
        loo_run((const void*)1, (t & 1) ? FK_F64 : FK_F32, N, d, (t & 2) ? (const void*)1 : nullptr, h, (double*)1,
                (double*)1, path, ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

fk_status fk_loo_laplace(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* h,
                         double* loglik, double* grad_h, fk_path path, void* ws, size_t ws_bytes,
                         fk_stream_t stream) {
    FK_RANGE("fk_loo_laplace");
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(points_validate(x, xd, N, d, nullptr, 0, path, false, 4));
    FK_TRY(check_h(h, d));
    if (N < 2) return set_error(FK_ERR_INVALID_ARG, "leave-one-out needs N >= 2");
    if (!loglik) return set_error(FK_ERR_INVALID_ARG, "loglik is NULL");
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *wp = nullptr;
    void *lp = nullptr, *ghp = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(w, (size_t)N * ds, &wp));
    FK_TRY(sg.out(loglik, 8, &lp));
    FK_TRY(sg.out(grad_h, (size_t)d * 8, &ghp));
    Arena plan;
    loo_run((const void*)1, xd, N, d, w, h, (double*)loglik, grad_h, path, plan, st);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    FK_TRY(loo_run(xp, xd, N, d, wp, h, (double*)lp, (double*)ghp, path, ar, st));
    return sg.finish();
}

// ------------------------------------------------------------------ other kernels, full H, local linear
// Which estimator an extra-kernel call runs (one validation and staging path for all four).
enum KFam { KF_UNIFORM = 0, KF_MATERN = 1, KF_HMATRIX = 2, KF_LOCLIN = 3 };

static fk_status kfam_run(int fam, const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                          int64_t M, const double* h, const double* R, unsigned flags, double* out, fk_path path,
                          Arena& ar, cudaStream_t st) {
    switch (fam) {
        case KF_UNIFORM: return uniform_run(x, xd, N, d, w, z, M, h, flags, out, path, ar, st);
        case KF_MATERN: return matern32_run(x, xd, N, d, w, z, M, h, flags, out, path, ar, st);
        case KF_HMATRIX: return hmatrix_run(x, xd, N, d, w, z, M, R, h, flags, out, path, ar, st);
        default: return loclin_run(x, xd, N, d, w, z, M, h, flags, out, path, ar, st);
    }
}

// Validation shared by the four calls; m_items is the item count of the
// sample-point engine run they make (the uniform kernel's corner targets).
static fk_status kfam_validate(int fam, const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                               int64_t M, fk_path path) {
    FK_TRY(check_common(x, xd, N, d, path));
    if (z && M < 0) return set_error(FK_ERR_INVALID_ARG, "M must be >= 0");
    const int max_d = (fam == KF_UNIFORM && !w) ? 8 : 4;
    if (d > max_d) return set_error(FK_ERR_UNSUPPORTED, "this call supports d <= %d", max_d);
    const int64_t m = z ? M : N;
    const int64_t items = (fam == KF_UNIFORM) ? N + ((int64_t)1 << d) * m : N + (z ? M : 0);
    if (items >= ((int64_t)1 << dc::kItemBits))
        return set_error(FK_ERR_UNSUPPORTED, "too many items (%lld) for the sample-point path", (long long)items);
    if (fam == KF_LOCLIN && path != FK_PATH_FP64)
        return set_error(FK_ERR_UNSUPPORTED, "locally linear regression needs FK_PATH_FP64");
    return FK_OK;
}

// Cyclic Jacobi eigendecomposition of a symmetric d x d matrix (d <= 8):
// H = V diag(ev) V^T, V row-major with the eigenvectors as columns.
static void jacobi_eigen(const double* H, int d, double* V, double* ev) {
    double A[8][8];
    for (int p = 0; p < d; ++p)
        for (int q = 0; q < d; ++q) {
            A[p][q] = 0.5 * (H[p * d + q] + H[q * d + p]);
            V[p * d + q] = (p == q) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < d; ++p) {
            diag += A[p][p] * A[p][p];
            for (int q = p + 1; q < d; ++q) off += A[p][q] * A[p][q];
        }
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                if (A[p][q] == 0.0) continue;
                // rotation angle phi with cot(2 phi) = theta zeroes A[p][q]
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {     // A <- A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {     // A <- J^T A
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) {     // V <- V J
                    const double vkp = V[k * d + p], vkq = V[k * d + q];
                    V[k * d + p] = c * vkp - s * vkq;
                    V[k * d + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int p = 0; p < d; ++p) ev[p] = A[p][p];
}

fk_status fk_hmatrix_factor(const double* H, int d, double* R, double* h) {
    FK_RANGE("fk_hmatrix_factor");
    if (d < 1 || d > 8) return set_error(FK_ERR_UNSUPPORTED, "d out of range");
    if (!H || !R || !h) return set_error(FK_ERR_INVALID_ARG, "NULL argument");
    double amax = 0.0;
    for (int e = 0; e < d * d; ++e) {
        if (!std::isfinite(H[e])) return set_error(FK_ERR_NONFINITE, "H has a non-finite entry");
        amax = std::max(amax, fabs(H[e]));
    }
    for (int p = 0; p < d; ++p)
        for (int q = p + 1; q < d; ++q)
            if (fabs(H[p * d + q] - H[q * d + p]) > 1e-12 * amax)
                return set_error(FK_ERR_INVALID_ARG, "H is not symmetric");
    double ev[8];
    jacobi_eigen(H, d, R, ev);
    for (int p = 0; p < d; ++p) {
        if (!(ev[p] > 0.0)) return set_error(FK_ERR_INVALID_ARG, "H is not positive definite");
        h[p] = sqrt(ev[p]);
    }
    return FK_OK;
}

static size_t kfam_workspace(int fam, int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path) {
    const void* z = sample_points ? nullptr : (const void*)1;
    const void* w = weighted ? (const void*)1 : nullptr;
    if (kfam_validate(fam, (const void*)1, FK_F32, N, d, w, z, M, path) != FK_OK) return 0;
    double h[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    double R[64] = {0};
    size_t best = 0;
    for (int t = 0; t < 2; ++t) {
        Arena ar;
        kfam_run(fam, (const void*)1, t ? FK_F64 : FK_F32, N, d, w, z, M, h, R, 0, nullptr, path, ar, 0);
        if (ar.used > best) best = ar.used;
    }
    return best;
}

static fk_status kfam_impl(int fam, const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                           int64_t M, const double* h, const double* H, unsigned flags, double* out, fk_path path,
                           void* ws, size_t ws_bytes, fk_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    FK_TRY(kfam_validate(fam, x, xd, N, d, w, z, M, path));
    double R[64], hd[8];
    if (fam == KF_HMATRIX) {
        if (!H) return set_error(FK_ERR_INVALID_ARG, "H is NULL");
        FK_TRY(fk_hmatrix_factor(H, d, R, hd));
        h = hd;
    } else {
        FK_TRY(check_h(h, d));
    }
    if ((flags & FK_LOO) && z) return set_error(FK_ERR_INVALID_ARG, "FK_LOO needs z == NULL");
    if ((flags & FK_LOO) && N < 2) return set_error(FK_ERR_INVALID_ARG, "leave-one-out needs N >= 2");
    if (fam == KF_LOCLIN && !w && N > 0) return set_error(FK_ERR_INVALID_ARG, "y is NULL");
    const int64_t m_out = z ? M : N;
    if (m_out == 0) return FK_OK;                        // nothing to write
    if (!out) return set_error(FK_ERR_INVALID_ARG, "out is NULL");
    const size_t ds = dtype_size(xd);
    Stager sg(st);
    const void *xp = nullptr, *wp = nullptr, *zp = nullptr;
    void* op = nullptr;
    FK_TRY(sg.in(x, (size_t)N * d * ds, &xp));
    FK_TRY(sg.in(w, (size_t)N * ds, &wp));
    FK_TRY(sg.in(z, z ? (size_t)M * d * ds : 0, &zp));
    FK_TRY(sg.out(out, (size_t)m_out * 8, &op));
    if (N == 0) {
        FK_CUDA(cudaMemsetAsync(op, 0, (size_t)m_out * 8, st));
        return sg.finish();
    }
    Arena plan;
    kfam_run(fam, (const void*)1, xd, N, d, w, z, M, h, R, flags, nullptr, path, plan, st);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, plan.used));
    FK_TRY(kfam_run(fam, xp, xd, N, d, wp, zp, M, h, R, flags, (double*)op, path, ar, st));
    return sg.finish();
}

size_t fk_kde_uniform_workspace(int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path) {
    return kfam_workspace(KF_UNIFORM, N, d, M, sample_points, weighted, path);
}
fk_status fk_kde_uniform(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                         const double* h, unsigned flags, double* out, fk_path path, void* ws, size_t ws_bytes,
                         fk_stream_t stream) {
    FK_RANGE("fk_kde_uniform");
    return kfam_impl(KF_UNIFORM, x, xd, N, d, w, z, M, h, nullptr, flags, out, path, ws, ws_bytes, stream);
}
size_t fk_kde_matern32_workspace(int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path) {
    return kfam_workspace(KF_MATERN, N, d, M, sample_points, weighted, path);
}
fk_status fk_kde_matern32(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                          const double* h, unsigned flags, double* out, fk_path path, void* ws, size_t ws_bytes,
                          fk_stream_t stream) {
    FK_RANGE("fk_kde_matern32");
    return kfam_impl(KF_MATERN, x, xd, N, d, w, z, M, h, nullptr, flags, out, path, ws, ws_bytes, stream);
}
size_t fk_kde_laplace_hmatrix_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path) {
    return kfam_workspace(KF_HMATRIX, N, d, M, sample_points, 1, path);
}
fk_status fk_kde_laplace_hmatrix(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                                 int64_t M, const double* H, unsigned flags, double* out, fk_path path, void* ws,
                                 size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_kde_laplace_hmatrix");
    return kfam_impl(KF_HMATRIX, x, xd, N, d, w, z, M, nullptr, H, flags, out, path, ws, ws_bytes, stream);
}
size_t fk_kreg_loclin_laplace_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path) {
    return kfam_workspace(KF_LOCLIN, N, d, M, sample_points, 1, path);
}
fk_status fk_kreg_loclin_laplace(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z,
                                 int64_t M, const double* h, unsigned flags, double* out, fk_path path, void* ws,
                                 size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_kreg_loclin_laplace");
    return kfam_impl(KF_LOCLIN, x, xd, N, d, y, z, M, h, nullptr, flags, out, path, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ batching
static fk_status batched_validate(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, fk_path path) {
    if (count < 0 || (count > 0 && !sets)) return set_error(FK_ERR_INVALID_ARG, "bad dataset list");
    if (xd != FK_F32 && xd != FK_F64) return set_error(FK_ERR_INVALID_ARG, "xdtype must be FK_F32 or FK_F64");
    if (path != FK_PATH_MIXED && path != FK_PATH_FP64) return set_error(FK_ERR_INVALID_ARG, "unknown precision path");
    if (!(what & (FK_BATCH_ECDF | FK_BATCH_KDE))) return set_error(FK_ERR_INVALID_ARG, "nothing requested");
    for (int b = 0; b < count; ++b) {
        if (sets[b].d < 1 || sets[b].d > 4) return set_error(FK_ERR_UNSUPPORTED, "dataset %d: d must be in [1, 4]", b);
        if (sets[b].N < 0 || 2 * sets[b].N >= ((int64_t)1 << 25))
            return set_error(FK_ERR_UNSUPPORTED, "dataset %d: N out of range", b);
        if (sets[b].N > 0 && !sets[b].x) return set_error(FK_ERR_INVALID_ARG, "dataset %d: x is NULL", b);
    }
    return FK_OK;
}

static fk_status batch_cfg(const fk_batch_config* c, BatchCfg& out) {
    out = BatchCfg{};
    if (!c) return FK_OK;
    if (c->streams < 1 || c->streams > 8) return set_error(FK_ERR_INVALID_ARG, "streams must be 1..8");
    if (c->coarsen < 0 || c->coarsen > 2) return set_error(FK_ERR_INVALID_ARG, "coarsen must be 0..2");
    if (c->kernel_tile < 0 || c->kernel_tile > 1) return set_error(FK_ERR_INVALID_ARG, "kernel_tile must be 0 or 1");
    if (c->count_tile < 0 || c->count_tile > 2) return set_error(FK_ERR_INVALID_ARG, "count_tile must be 0..2");
    out.streams = c->streams;
    out.coarsen = c->coarsen;
    out.kernel_tile = c->kernel_tile;
    out.count_tile = c->count_tile;
    return FK_OK;
}

static size_t batched_plan(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, fk_path path,
                           const BatchCfg& c) {
    Arena ar;
    batched_run(sets, count, xd, what, 1.0, nullptr, nullptr, path, c, ar, 0);
    return ar.used;
}

void fk_batched_config_default(fk_batch_config* cfg) {
    if (!cfg) return;
    const BatchCfg d;
    cfg->streams = d.streams;
    cfg->coarsen = d.coarsen;
    cfg->kernel_tile = d.kernel_tile;
    cfg->count_tile = d.count_tile;
}

size_t fk_batched_workspace_ex(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, fk_path path,
                               const fk_batch_config* cfg) {
    BatchCfg c;
    if (batch_cfg(cfg, c) != FK_OK) return 0;
    if (batched_validate(sets, count, xd, what, path) != FK_OK) return 0;
    return batched_plan(sets, count, xd, what, path, c);
}

size_t fk_batched_workspace(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, fk_path path) {
    return fk_batched_workspace_ex(sets, count, xd, what, path, nullptr);
}

static fk_status batched_check(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h,
                               int64_t* ecdf_out, double* kde_out, fk_path path) {
    FK_TRY(batched_validate(sets, count, xd, what, path));
    if ((what & FK_BATCH_KDE) && !(h > 0.0 && h < 1e300)) return set_error(FK_ERR_INVALID_ARG, "h must be > 0");
    if ((what & FK_BATCH_ECDF) && !ecdf_out) return set_error(FK_ERR_INVALID_ARG, "ecdf_out is NULL");
    if ((what & FK_BATCH_KDE) && !kde_out) return set_error(FK_ERR_INVALID_ARG, "kde_out is NULL");
    for (int b = 0; b < count; ++b)
        if ((sets[b].x && !is_device_pointer(sets[b].x)) || (sets[b].y && !is_device_pointer(sets[b].y)))
            return set_error(FK_ERR_INVALID_ARG, "fk_batched needs device pointers (dataset %d)", b);
    if ((ecdf_out && !is_device_pointer(ecdf_out)) || (kde_out && !is_device_pointer(kde_out)))
        return set_error(FK_ERR_INVALID_ARG, "fk_batched needs device output pointers");
    return FK_OK;
}

fk_status fk_batched_ex(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h, int64_t* ecdf_out,
                        double* kde_out, fk_path path, const fk_batch_config* cfg, void* ws, size_t ws_bytes,
                        fk_stream_t stream) {
    FK_RANGE("fk_batched_ex");
    cudaStream_t st = (cudaStream_t)stream;
    BatchCfg c;
    FK_TRY(batch_cfg(cfg, c));
    FK_TRY(batched_check(sets, count, xd, what, h, ecdf_out, kde_out, path));
    const size_t need = batched_plan(sets, count, xd, what, path, c);
    Workspace wsp(st);
    Arena ar;
    FK_TRY(wsp.bind(ar, ws, ws_bytes, need));
    return batched_run(sets, count, xd, what, h, ecdf_out, kde_out, path, c, ar, st);
}

fk_status fk_batched(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h, int64_t* ecdf_out,
                     double* kde_out, fk_path path, void* ws, size_t ws_bytes, fk_stream_t stream) {
    FK_RANGE("fk_batched");
    return fk_batched_ex(sets, count, xd, what, h, ecdf_out, kde_out, path, nullptr, ws, ws_bytes, stream);
}

// The autotuner's candidate values per dimension.
static const int kTuneStreams[] = {1, 2, 4, 8};
static const int kTuneCoarsen[] = {0, 1, 2};
static const int kTuneCountTile[] = {0, 1, 2};
static const int kTuneKernelTile[] = {0, 1};

size_t fk_batched_autotune_workspace(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, fk_path path) {
    if (batched_validate(sets, count, xd, what, path) != FK_OK) return 0;
    size_t mx = 0;
    BatchCfg c;
    for (int s : kTuneStreams)
        for (int co : kTuneCoarsen)
            for (int ct : kTuneCountTile)
                for (int kt : kTuneKernelTile) {
                    c.streams = s;
                    c.coarsen = co;
                    c.count_tile = ct;
                    c.kernel_tile = kt;
                    mx = std::max(mx, batched_plan(sets, count, xd, what, path, c));
                }
    return mx;
}

fk_status fk_batched_autotune(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h,
                              int64_t* ecdf_out, double* kde_out, fk_path path, void* ws, size_t ws_bytes,
                              fk_stream_t stream, fk_batch_config* best, double* best_ms) {
    FK_RANGE("fk_batched_autotune");
    cudaStream_t st = (cudaStream_t)stream;
    if (!best) return set_error(FK_ERR_INVALID_ARG, "best is NULL");
    FK_TRY(batched_check(sets, count, xd, what, h, ecdf_out, kde_out, path));
    cudaEvent_t ea = nullptr, eb = nullptr;
    FK_CUDA(cudaEventCreate(&ea));
    FK_CUDA(cudaEventCreate(&eb));
    // one candidate: warm-up run, then the best of two timed runs
    auto trial = [&](const BatchCfg& c, double* ms) -> fk_status {
        const size_t need = batched_plan(sets, count, xd, what, path, c);
        Workspace wsp(st);
        Arena ar;
        FK_TRY(wsp.bind(ar, ws, ws_bytes, need));
        FK_TRY(batched_run(sets, count, xd, what, h, ecdf_out, kde_out, path, c, ar, st));
        double bestt = 1e300;
        for (int r = 0; r < 2; ++r) {
            ar.used = 0;
            FK_CUDA(cudaEventRecord(ea, st));
            FK_TRY(batched_run(sets, count, xd, what, h, ecdf_out, kde_out, path, c, ar, st));
            FK_CUDA(cudaEventRecord(eb, st));
            FK_CUDA(cudaEventSynchronize(eb));
            float t = 0.f;
            FK_CUDA(cudaEventElapsedTime(&t, ea, eb));
            bestt = std::min(bestt, (double)t);
        }
        *ms = bestt;
        return FK_OK;
    };
    BatchCfg cur;
    double cur_ms = 0.0;
    fk_status rc = trial(cur, &cur_ms);
    // coordinate descent, one dimension at a time
    auto descend = [&](int BatchCfg::*field, const int* vals, int nv) {
        const int start = cur.*field;
        for (int i = 0; i < nv && rc == FK_OK; ++i) {
            if (vals[i] == start) continue;
            BatchCfg c = cur;
            c.*field = vals[i];
            double ms = 0.0;
            rc = trial(c, &ms);
            if (rc == FK_OK && ms < cur_ms) {
                cur = c;
                cur_ms = ms;
            }
        }
    };
    if (rc == FK_OK) descend(&BatchCfg::streams, kTuneStreams, 4);
    if (rc == FK_OK) descend(&BatchCfg::coarsen, kTuneCoarsen, 3);
    if (rc == FK_OK && (what & FK_BATCH_ECDF)) descend(&BatchCfg::count_tile, kTuneCountTile, 3);
    if (rc == FK_OK && (what & FK_BATCH_KDE)) descend(&BatchCfg::kernel_tile, kTuneKernelTile, 2);
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (rc != FK_OK) return rc;
    best->streams = cur.streams;
    best->coarsen = cur.coarsen;
    best->kernel_tile = cur.kernel_tile;
    best->count_tile = cur.count_tile;
    if (best_ms) *best_ms = cur_ms;
    return FK_OK;
}

// Busy time of a family: the length of the union of its launches' intervals
// (launches of concurrent streams overlap, so their summed durations exceed
// the time the family kept the GPU busy).  Times are taken relative to the
// first recorded start event of the session.
fk_status fk_profile_busy(int family, double* busy_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!busy_ms) return set_error(FK_ERR_INVALID_ARG, "busy_ms is NULL");
    *busy_ms = 0.0;
    if (g_prof.empty()) return FK_OK;
    const cudaEvent_t ref = g_prof.front().a;
    std::vector<std::pair<double, double>> iv;
    for (auto& r : g_prof) {
        if (r.fam != family) continue;
        FK_CUDA(cudaEventSynchronize(r.b));
        float t0 = 0.f, t1 = 0.f;
        FK_CUDA(cudaEventElapsedTime(&t0, ref, r.a));
        FK_CUDA(cudaEventElapsedTime(&t1, ref, r.b));
        iv.emplace_back((double)t0, (double)t1);
    }
    std::sort(iv.begin(), iv.end());
    double total = 0.0, cs = 0.0, ce = 0.0;
    bool open = false;
    for (auto& v : iv) {
        if (!open) { cs = v.first; ce = v.second; open = true; continue; }
        if (v.first > ce) { total += ce - cs; cs = v.first; ce = v.second; }
        else if (v.second > ce) ce = v.second;
    }
    if (open) total += ce - cs;
    *busy_ms = total;
    return FK_OK;
}

}  // extern "C"
