// fk_dc_ops.cuh -- declarations shared by the divide-and-conquer translation
// units (engine instantiations and the operation orchestration).
#pragma once

#include "fk_dc_drv.cuh"

namespace fk {
namespace dc {

struct HVec { double v[8]; };
struct SelMap { int n; int o[256]; };   // output row r <- internal orthant o[r]

// Instantiated sweeps (one per accumulation policy); CLSB is d_eff - 2.
#define FK_DC_SWEEP_DECL(NAME, POL)                                                              \
    fk_status NAME(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top,    \
                   const POL& pol, Arena& ar, cudaStream_t st, int levels = -1, int opts = 0);
FK_DC_SWEEP_DECL(sweep_w64, PolW64)
FK_DC_SWEEP_DECL(sweep_wff, PolWFF)
FK_DC_SWEEP_DECL(sweep_kf1, PolKF<1>)
FK_DC_SWEEP_DECL(sweep_kf2, PolKF<2>)
FK_DC_SWEEP_DECL(sweep_kd1, PolKD<1>)
FK_DC_SWEEP_DECL(sweep_kd2, PolKD<2>)
#undef FK_DC_SWEEP_DECL

// d = 5 and 6 (3 and 4 enclosing class bits, 16 and 32 channels): one-channel
// policies only, instantiated in fk_dc_d5.cu and fk_dc_d6.cu; the others refuse.
#define FK_DC_SWEEP_HD_DECL(POL)                                                                 \
    fk_status sweep_d5(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top, \
                       const POL& pol, Arena& ar, cudaStream_t st, int levels, int opts);        \
    fk_status sweep_d6(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top, \
                       const POL& pol, Arena& ar, cudaStream_t st, int levels, int opts);
FK_DC_SWEEP_HD_DECL(PolW64)
FK_DC_SWEEP_HD_DECL(PolWFF)
FK_DC_SWEEP_HD_DECL(PolKF<1>)
FK_DC_SWEEP_HD_DECL(PolKD<1>)
#undef FK_DC_SWEEP_HD_DECL
template <class POL>
fk_status sweep_d5(int, int64_t, const uint32_t* const*, const uint32_t*, const POL&, Arena&, cudaStream_t, int,
                   int) {
    return set_error(FK_ERR_UNSUPPORTED, "two-channel kernel sums at the sample points support d <= 4");
}
template <class POL>
fk_status sweep_d6(int, int64_t, const uint32_t* const*, const uint32_t*, const POL&, Arena&, cudaStream_t, int,
                   int) {
    return set_error(FK_ERR_UNSUPPORTED, "two-channel kernel sums at the sample points support d <= 4");
}

#define FK_DC_SWEEP_DEF(NAME, POL)                                                               \
    fk_status NAME(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top,    \
                   const POL& pol, Arena& ar, cudaStream_t st, int levels, int opts) {         \
        switch (d_eff) {                                                                        \
            case 2: return dc_sweep<POL, 0>(d_eff, n, P, seq_top, pol, ar, st, levels, opts);   \
            case 3: return dc_sweep<POL, 1>(d_eff, n, P, seq_top, pol, ar, st, levels, opts);   \
            case 4: return dc_sweep<POL, 2>(d_eff, n, P, seq_top, pol, ar, st, levels, opts);   \
            case 5: return sweep_d5(d_eff, n, P, seq_top, pol, ar, st, levels, opts);           \
            case 6: return sweep_d6(d_eff, n, P, seq_top, pol, ar, st, levels, opts);           \
            default: return set_error(FK_ERR_UNSUPPORTED, "sample-point path supports d <= 6"); \
        }                                                                                       \
    }

}  // namespace dc

// Exact orthant counts by inclusion-exclusion over dominance counts (fk_dom.cu).
fk_status dom_orthant_counts(int d, int64_t n, int64_t n_src, int64_t tgt_off, int64_t n_tgt,
                             const uint32_t* const* P, const uint32_t* mask, int64_t* out, Arena& ar,
                             cudaStream_t st);
// The same at the sample points with one item per point (each a source and a
// target).  Synchronises `st` once, after the tie statistics: if a tie group
// on some axis is too long for the tie correction, sets *fallback and
// computes nothing (the caller then uses the source/target-copy layout).  In
// sizing mode *fallback is left as passed.
fk_status dom_self_counts(int d, int64_t n, const uint32_t* const* P, const void* x, fk_dtype xd,
                          const uint32_t* mask, int64_t* out, Arena& ar, cudaStream_t st, bool* fallback);
// Ties at the sample points with one item per point (fk_ties.cu).  The rank
// transform orders equal coordinates by point index on every axis, so the
// engine pairs source i with target j (i != j) on the <= side of an axis
// exactly when x_i < x_j there, or x_i == x_j and i < j.
// tie_check: tie statistics of the d sorted axes, read back once (it
// synchronises `st`); *fallback is set when a tie group is longer than
// kTieGroupMax points, or the tied pairs exceed the correction's budget.
// `sorted` [n] and `stats` [2] are scratch.
constexpr int kTieGroupMax = 64;
fk_status tie_check(const void* x, fk_dtype xd, int d, int64_t n, const uint32_t* const* P, uint32_t* sorted,
                    unsigned long long* stats, cudaStream_t st, bool* fallback);
// Counts: adds to C_A[j] (Cs[A], A a bitmask over the d axes) the sources i > j
// with x_i <= x_j on A and a tie on some axis of A, each pair once per A.
fk_status tie_fix_counts(const void* x, fk_dtype xd, int d, int64_t n, const uint32_t* const* P, uint32_t* sorted,
                         uint32_t* const* Cs, cudaStream_t st);

// Batched form: items in segments of 2^segE slots described by seg (see
// dc::ItemMap); the counts of target t go to out_base[b] + r * n_b + (t - t0_b)
// for dataset b (targets numbered by dataset), every orthant r < 2^d.
struct BatchOut {
    const int64_t* tbase;   // [nb + 1] first global target of each dataset (device)
    const int64_t* obase;   // [nb] output offset of each dataset (device)
    int nb;
};
// count_tile: tile of the tile-local counting levels (0: 2048, 1: 1024, 2: 4096).
fk_status dom_orthant_counts_seg(int d, int64_t n, const int64_t* seg, int segE, int64_t n_tgt,
                                 const uint32_t* const* P, BatchOut bo, int64_t* out, Arena& ar,
                                 cudaStream_t st, int count_tile = 0);

// Operations (fk_dc_common.cu).  All pointers are device pointers.
fk_status points_orthant(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z,
                         int64_t M, const uint32_t* mask, void* out, fk_path path, Arena& ar,
                         cudaStream_t st);
// `wd` is the dtype of w (default: that of x).  sgn >= 0: signed sums for the
// gradients -- nw must be 2 (weights w and 1) and every contribution carries
// the sign delta_sgn of its orthant; out[i][t] = C * (signed sum of channel i)
// with no self term (a pair at distance 0 on axis sgn contributes nothing to
// the gradients).
fk_status points_kernel(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z,
                        int64_t M, const double* h, unsigned flags, int nw, double* out, double* terms,
                        fk_path path, Arena& ar, cudaStream_t st, fk_dtype wd = (fk_dtype)-1, int sgn = -1);

}  // namespace fk
