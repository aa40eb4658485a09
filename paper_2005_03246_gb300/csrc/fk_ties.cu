// fk_ties.cu -- exact tie handling for the one-item-per-point layout at the
// sample points.
//
// Every point is one item that is both a source and a target.  The stable
// rank transform orders equal coordinates by point index on every axis, so
// the divide-and-conquer engine puts source i on the <= side of target j's
// axis k exactly when x_ik < x_jk, or x_ik == x_jk and i < j.  The definition
// (eq. ECDFdelta read as in eq. Laplacian decomposition nD: x_k <= z_k on the
// <= side) wants x_ik <= x_jk.  The two differ only for pairs that tie on
// some axis with the later point (i > j) as the source: those pairs sit in
// the tie groups of the sorted axes, and each is corrected here once, at the
// first axis of the subset on which it ties.  The engine never pairs an item
// with itself; the self term (x_j <= x_j on every axis) is added in the
// combine.
#include "fk_dc_ops.cuh"

namespace fk {
namespace {

// The rank transform's sort key of a coordinate (-0 and +0 are one value).
__device__ __forceinline__ uint64_t okey(float v) {
    if (v == 0.0f) v = 0.0f;
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t okey(double v) {
    if (v == 0.0) v = 0.0;
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_sorted_from_pos(const uint32_t* __restrict__ P, int64_t n, uint32_t* __restrict__ sorted) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n) sorted[P[it]] = (uint32_t)it;
}

// stats[0] += pairs inside the tie groups of axis a; stats[1] = 1 if a group
// is longer than kTieGroupMax.  The first position of each group counts it
// (each thread reads at most kTieGroupMax + 1 keys).
template <class T>
__global__ void k_tie_stats(const T* __restrict__ x, int d, int a, const uint32_t* __restrict__ sorted, int64_t n,
                            unsigned long long* __restrict__ stats) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint64_t kp = okey(x[(int64_t)sorted[p] * d + a]);
    if (p > 0 && okey(x[(int64_t)sorted[p - 1] * d + a]) == kp) return;
    int64_t q = p + 1;
    while (q < n && q - p <= kTieGroupMax && okey(x[(int64_t)sorted[q] * d + a]) == kp) ++q;
    const int64_t L = q - p;
    if (L > kTieGroupMax) {
        atomicOr(stats + 1, 1ull);
        return;
    }
    if (L > 1) atomicAdd(stats, (unsigned long long)(L * (L - 1) / 2));
}

// Comparison masks of point i against the keys kj of point j: bit b of
// le / gt / eq is x_ib <= / > / == x_jb.
template <class T>
__device__ __forceinline__ void masks_of(const T* x, int d, uint32_t i, const uint64_t (&kj)[8], uint32_t& le,
                                         uint32_t& gt, uint32_t& eq) {
    le = gt = eq = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b < d) {
            const uint64_t ki = okey(x[(int64_t)i * d + b]);
            le |= (ki <= kj[b] ? 1u : 0u) << b;
            gt |= (ki > kj[b] ? 1u : 0u) << b;
            eq |= (ki == kj[b] ? 1u : 0u) << b;
        }
    }
}

struct CTabW { uint32_t* c[256]; };

// Counts: for target j at sorted position p of axis a, the later members i of
// its tie group, for every subset A containing a on which x_i <= x_j and
// whose axes below a do not tie (those pairs are counted at that axis).
template <class T>
__global__ void k_tie_fix_counts(const T* __restrict__ x, int d, int a, const uint32_t* __restrict__ sorted,
                                 int64_t n, CTabW ct) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t j = sorted[p];
    uint64_t kj[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) kj[b] = (b < d) ? okey(x[(int64_t)j * d + b]) : 0ull;
    const uint32_t abit = 1u << a;
    for (int64_t q = p + 1; q < n && q - p <= kTieGroupMax; ++q) {
        const uint32_t i = sorted[q];
        if (okey(x[(int64_t)i * d + a]) != kj[a]) break;
        uint32_t le, gt, eq;
        masks_of(x, d, i, kj, le, gt, eq);
        const uint32_t rest = le & ~(eq & (abit - 1u)) & ~abit;
        uint32_t S = 0;
        while (true) {       // every subset S of rest: A = S | a (if an orthant reads C_A)
            uint32_t* c = ct.c[S | abit];
            if (c) atomicAdd(c + j, 1u);
            if (S == rest) break;
            S = (S - rest) & rest;
        }
    }
}

}  // namespace

fk_status tie_check(const void* x, fk_dtype xd, int d, int64_t n, const uint32_t* const* P, uint32_t* sorted,
                    unsigned long long* stats, cudaStream_t st, bool* fallback) {
    FK_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st));
    const unsigned g = grid_for(n, 256);
    for (int a = 0; a < d; ++a) {
        k_sorted_from_pos<<<g, 256, 0, st>>>(P[a], n, sorted);
        FK_LAUNCH_CHECK();
        if (xd == FK_F32) k_tie_stats<float><<<g, 256, 0, st>>>((const float*)x, d, a, sorted, n, stats);
        else k_tie_stats<double><<<g, 256, 0, st>>>((const double*)x, d, a, sorted, n, stats);
        FK_LAUNCH_CHECK();
    }
    unsigned long long hs[2] = {0, 0};
    FK_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    FK_CUDA(cudaStreamSynchronize(st));
    *fallback = hs[1] != 0 || hs[0] > (unsigned long long)(4 * n + 4096);
    return FK_OK;
}

// Cs[A] is NULL for the subsets no selected orthant reads; those are skipped.
fk_status tie_fix_counts(const void* x, fk_dtype xd, int d, int64_t n, const uint32_t* const* P, uint32_t* sorted,
                         uint32_t* const* Cs, cudaStream_t st) {
    CTabW cw = {};
    for (int A = 1; A < (1 << d); ++A) cw.c[A] = Cs[A];
    const unsigned g = grid_for(n, 256);
    for (int a = 0; a < d; ++a) {
        k_sorted_from_pos<<<g, 256, 0, st>>>(P[a], n, sorted);
        FK_LAUNCH_CHECK();
        if (xd == FK_F32) k_tie_fix_counts<float><<<g, 256, 0, st>>>((const float*)x, d, a, sorted, n, cw);
        else k_tie_fix_counts<double><<<g, 256, 0, st>>>((const double*)x, d, a, sorted, n, cw);
        FK_LAUNCH_CHECK();
    }
    return FK_OK;
}

}  // namespace fk
