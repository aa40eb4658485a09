// fk_internal.cuh -- shared internals of the fastecdf library (not part of the ABI).
#pragma once

#include <mutex>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/fastecdf.h"

namespace fk {

// ------------------------------------------------------------------ errors
fk_status set_error(fk_status st, const char* fmt, ...);
fk_status cuda_error(cudaError_t e, const char* where);

#define FK_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t fk_e_ = (call);                                     \
        if (fk_e_ != cudaSuccess) return ::fk::cuda_error(fk_e_, #call); \
    } while (0)

#define FK_TRY(call)                        \
    do {                                    \
        fk_status fk_s_ = (call);           \
        if (fk_s_ != FK_OK) return fk_s_;   \
    } while (0)

// Every kernel launch site is followed by FK_LAUNCH_CHECK(), which also counts it.
void note_launch();
#define FK_LAUNCH_CHECK()          \
    do {                           \
        ::fk::note_launch();       \
        FK_CUDA(cudaGetLastError()); \
    } while (0)

// Optional CUDA-event timing of kernel families (fk_profile_*).
enum ProfFamily : int { PF_MERGE_SWEEP = 0, PF_MERGE_TOTALS = 1, PF_MERGE_PLAIN = 2, PF_GRID_PASS = 3,
                        PF_GRID_HIST = 4, PF_RADIX = 5, PF_GATHER = 6, PF_LOCAL = 7, PF_KLOCAL = 8,
                        PF_COUNT = 9 };
// Arithmetic of the kernel-sum sweep per item and merge level (family PF_KLOCAL):
// two compensated additions into the running sums and two scaled compensated
// additions into the target's sum, 10 + 1 operations each.
constexpr double kKernelOpsPerItemLevel = 44.0;
bool profiling_on();
void prof_record(int family, double work, double bytes, cudaEvent_t a, cudaEvent_t b);
cudaEvent_t prof_event();
struct ProfScope {
    int fam;
    double bytes;     // the family's work (bytes, or operations for PF_KLOCAL)
    double mem;       // algorithmic bytes (== bytes unless given)
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(int f, double b, cudaStream_t s, double m = -1.0) : fam(f), bytes(b), mem(m < 0.0 ? b : m), st(s) {
        if (profiling_on()) {
            a = prof_event();
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b2 = prof_event();
            cudaEventRecord(b2, st);
            prof_record(fam, bytes, mem, a, b2);
        }
    }
};

// Device-side error codes recorded in the per-device error word.
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BOUNDS = 2, DEV_AXIS = 3, DEV_NONFINITE = 4 };

// Records a non-finite input coordinate (NaN or +-inf) in the error word; the
// first error recorded since the last fk_device_status is kept.  Called by
// the kernels that first read each coordinate, so no extra pass over x.
__device__ __forceinline__ void note_nonfinite(int* err) {
    if (err && *(volatile int*)err == 0) atomicCAS(err, 0, (int)DEV_NONFINITE);
}

// Concurrent parts of one call (fk_streams.cu): begin() forks up to k-1
// library-owned streams from `main` (s[0] == main), end() (or the destructor)
// joins them back; ev[] are events of the pool the caller may use meanwhile.
// Pool 0 serves the batched groups, pool 1 the parts inside one operation,
// pool 2 the merge levels inside such a part.
constexpr int kPoolStreams = 8;
constexpr int kPoolAux = 16;     // extra events a fork may use between begin() and end()
constexpr int kPools = 3;
struct StreamFork {
    cudaStream_t s[kPoolStreams] = {};
    cudaEvent_t ev[kPoolAux] = {};
    int n = 1;
    fk_status begin(int pool, cudaStream_t main, int k);
    fk_status end();
    ~StreamFork();
    cudaStream_t st = nullptr;
    int pool = 0;
    int dev_ = 0;
    int slot_ = 0;
    bool forked = false;
    std::unique_lock<std::mutex> lock;
};

// Launch configuration of the batched path (the autotuner's search space).
struct BatchCfg {
    int streams = 1;       // groups run concurrently on this many streams (1..8)
    int coarsen = 0;       // group padded sizes rounded up to multiples of coarsen+1 levels (0..2)
    int kernel_tile = 0;   // tile-local kernel-sum levels: 0 default tile, 1 half tile
    int count_tile = 0;    // tile-local counting levels: 0 2048, 1 1024, 2 4096 items
};

// ------------------------------------------------------------------ workspace arena
// A bump allocator over caller scratch.  In sizing mode (base == nullptr) it
// only accumulates the total so that the same plan code gives the size.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    bool sizing = true;
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = count * sizeof(T);
        used = off + ((bytes + 255) & ~size_t(255));
        if (sizing) return nullptr;
        if (used > cap) return nullptr;
        return reinterpret_cast<T*>(base + off);
    }
    bool overflow() const { return !sizing && used > cap; }
};

// ------------------------------------------------------------------ launch helpers
constexpr int kSMs = 152;
inline unsigned grid_for(int64_t n, int per_block) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ------------------------------------------------------------------ value types
// FF: unevaluated sum hi + lo of two floats (compensated FP32).
struct FF { float hi, lo; };

__device__ __forceinline__ FF ff_zero() { return FF{0.f, 0.f}; }

// Knuth two-sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    float hi = s + e;
    return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e += a.lo;
    float hi = s + e;
    return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_from_double(double v) {
    float hi = (float)v;
    return FF{hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Exact powers of two built from the exponent field: k <= 0 flushes below
// the normal range to zero; the _any forms saturate above it to infinity.
// (A clamp and a shift: no compare-and-select.)
__device__ __forceinline__ float pow2f_le0(int k) { return __int_as_float((max(k, -127) + 127) << 23); }
__device__ __forceinline__ double pow2d_le0(int k) {
    return __longlong_as_double((long long)(max(k, -1023) + 1023) << 52);
}
__device__ __forceinline__ float pow2f_any(int k) { return __int_as_float((min(max(k, -127), 128) + 127) << 23); }
__device__ __forceinline__ double pow2d_any(int k) {
    return __longlong_as_double((long long)(min(max(k, -1023), 1024) + 1023) << 52);
}

// Shifted compensated value (hi + lo) * 2^e; the zero value has e = kEmin.
constexpr int kEmin = -(1 << 28);
struct SFF { float hi, lo; int e; };
__device__ __forceinline__ SFF sff_zero() { return SFF{0.f, 0.f, kEmin}; }
// A zero value always carries kEmin: a zero with a large shift would
// otherwise raise the shift of every sum it joins and flush the sum.
__device__ __forceinline__ SFF sff_term(float m, int s) { return SFF{m, 0.f, m != 0.f ? s : kEmin}; }
__device__ __forceinline__ SFF sff_add(SFF a, SFF b) {
    int e = max(a.e, b.e);
    float sa = pow2f_le0(a.e - e), sb = pow2f_le0(b.e - e);
    FF r = ff_add(FF{a.hi * sa, a.lo * sa}, FF{b.hi * sb, b.lo * sb});
    return SFF{r.hi, r.lo, r.hi != 0.f ? e : kEmin};
}
// Shifted plain FP32 value m * 2^e (short sums: tile-local walks and scans).
struct SF { float m; int e; };
__device__ __forceinline__ SF sf_zero() { return SF{0.f, kEmin}; }
__device__ __forceinline__ SF sf_term(float m, int s) { return SF{m, m != 0.f ? s : kEmin}; }
__device__ __forceinline__ SF sf_add(SF a, SF b) {
    const int e = max(a.e, b.e);
    return SF{a.m * pow2f_le0(a.e - e) + b.m * pow2f_le0(b.e - e), e};
}
// Shifted FP64 value m * 2^e.
struct SD { double m; int e; };
__device__ __forceinline__ SD sd_zero() { return SD{0.0, kEmin}; }
// Zero test on the two 32-bit halves: integer instructions only (an FP64
// compare would take the FP64 pipe, the scarce one on this part).
__device__ __forceinline__ bool f64_nonzero(double v) {
    return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) != 0;
}
__device__ __forceinline__ SD sd_term(double m, int s) { return SD{m, f64_nonzero(m) ? s : kEmin}; }
// m * 2^k by an integer add to the exponent field (no FP64 instruction):
// m normal or zero; results below the normal range flush to zero, above it
// saturate to infinity.
__device__ __forceinline__ double ldexp_i(double m, int k) {
    const int hi = __double2hiint(m), lo = __double2loint(m);
    const int eb = (hi >> 20) & 0x7ff;
    const int nb = eb + k;
    if (eb == 0 || nb <= 0) return 0.0;
    if (nb >= 0x7ff) return __hiloint2double((hi & (int)0x80000000) | 0x7ff00000, 0);
    return __hiloint2double((int)((unsigned)hi + ((unsigned)k << 20)), lo);
}
// One FP64 addition: the operand with the smaller shift is rescaled by an
// exponent add.  (No zero test on the result: a sum that cancels to exactly
// zero keeps its shift, which only matters if far smaller values follow.)
__device__ __forceinline__ SD sd_add(SD a, SD b) {
    const bool ag = a.e >= b.e;
    const double big = ag ? a.m : b.m, small = ag ? b.m : a.m;
    const int eb = ag ? a.e : b.e, es = ag ? b.e : a.e;
    return SD{big + ldexp_i(small, max(es - eb, -4096)), eb};
}

// Full-warp shuffles for every accumulator type.
__device__ __forceinline__ uint32_t shfl_up_any(uint32_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint32_t shfl_down_any(uint32_t v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint32_t shfl_idx_any(uint32_t v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double shfl_up_any(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down_any(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_idx_any(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ FF shfl_up_any(FF v, int o) {
    return FF{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ FF shfl_down_any(FF v, int o) {
    return FF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ FF shfl_idx_any(FF v, int l) {
    return FF{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}

__device__ __forceinline__ double dc_as_f64(double v) { return v; }
__device__ __forceinline__ double dc_as_f64(FF v) { return ff_to_double(v); }

// Per-item, per-axis exponent factor e^{+-v/h} = m_plus * 2^s, m_minus * 2^-s.
struct FacF { float mp, mm; int s; };
struct FacD { double mp, mm; int s; int pad; };

// ------------------------------------------------------------------ host helpers
bool is_device_pointer(const void* p);
fk_status device_error_word(int** ptr);   // address of the current device's error word

// scan.cu
// Exclusive scan of n uint32 values (in may equal out).  `tmp` needs
// scan_u32_tmp_words(n) words.
size_t scan_u32_tmp_words(int64_t n);
fk_status scan_u32_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                             cudaStream_t st);

// sort.cu -- stable LSD radix sort of (key, value) pairs.
size_t radix_sort_tmp_bytes(int64_t n, int key_bits);
fk_status radix_lookback_timeout_probe(int64_t n, cudaStream_t st);
fk_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                               uint32_t* vals_alt, int64_t n, int key_bits, void* tmp,
                               size_t tmp_bytes, cudaStream_t st, bool* result_in_alt);
fk_status radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                               uint32_t* vals_alt, int64_t n, int key_bits, void* tmp,
                               size_t tmp_bytes, cudaStream_t st, bool* result_in_alt);

// grid.cu
fk_status grid_run(const void* x, fk_dtype xd, int64_t N, int d, const void* y,
                   const double* z_dev, const int64_t* M, const uint32_t* mask, void* out,
                   fk_path path, Arena& ar, cudaStream_t st, int* err_word);

}  // namespace fk
