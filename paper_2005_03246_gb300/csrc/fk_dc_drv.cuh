// fk_dc_drv.cuh -- accumulation policies and the host recursion of the
// divide-and-conquer engine (see fk_dc.cuh for the formulation).
#pragma once

#include "fk_dc.cuh"

namespace fk {
namespace dc {

// Which items are sources and which are targets.
//   sample points, orthant sums : items [0,N) sources, [N,2N) target copies
//   sample points, kernel sums  : items [0,N) are both (the self pair is added
//                                 separately, or dropped for leave-one-out)
//   explicit targets            : items [0,N) sources, [N,N+M) targets
//   batched layout (seg != nullptr): the items form segments of 2^segE slots,
//                                 one dataset per segment; seg[4s..4s+3] =
//                                 {sources, first target slot, targets,
//                                 global index of the first target}; the other
//                                 slots are padding (neither role).
struct ItemMap {
    int64_t n_src, tgt_off, n_tgt;
    const int64_t* seg;
    int segE;
    __device__ __forceinline__ bool is_src(uint32_t it) const {
        if (!seg) return (int64_t)it < n_src;
        const int64_t loc = it & ((1u << segE) - 1u);
        return loc < seg[4 * (int64_t)(it >> segE)];
    }
    __device__ __forceinline__ bool is_tgt(uint32_t it) const {
        if (!seg) return (int64_t)it >= tgt_off && (int64_t)it < tgt_off + n_tgt;
        const int64_t s = it >> segE, loc = it & ((1u << segE) - 1u);
        return loc >= seg[4 * s + 1] && loc < seg[4 * s + 1] + seg[4 * s + 2];
    }
    __device__ __forceinline__ int64_t tgt_index(uint32_t it) const {
        if (!seg) return (int64_t)it - tgt_off;
        const int64_t s = it >> segE, loc = it & ((1u << segE) - 1u);
        return seg[4 * s + 3] + loc - seg[4 * s + 1];
    }
};

// Orthant index receiving the forward sum of a target with position bits pb
// (bit 0: half on axis 1, bit j: side on axis j+1).  A target on the upper
// side of an axis receives from sources below it (delta = +1, bit clear);
// the backward sum (delta_0 = -1) goes to the same index | 1.
__device__ __forceinline__ uint32_t fwd_orthant(uint32_t pb, uint32_t pbmask) {
    return ((~pb) & pbmask) << 1;
}

// ------------------------------------------------------------------ orthant sums
struct PolCount : ItemMap {
    typedef uint32_t V;
    static constexpr int kSrcBytes = 0, kTgtBytes = 16, kTgtFacBytes = 0;
    static constexpr int kLocalT = 4096;
    static constexpr bool kUnitWeights = true;
    static constexpr bool kCanFold = false;      // sums stay per orthant
    static constexpr bool kRecords = false;
    static constexpr int kFoldT = kLocalT, kNW = 1;
    typedef float M;
    typedef float FA;
    struct LW { uint32_t unused; };
    uint32_t* acc;        // [2^d][n_tgt]
    uint32_t pbmask;
    __device__ static V zero() { return 0u; }
    __device__ static V one() { return 1u; }
    __device__ static V from_lw(LW) { return 1u; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ void local_weights(uint32_t, uint32_t, LW*) const {}
    __device__ void flush(uint32_t item, uint32_t cls, const V* loc) const {
        const int64_t t = tgt_index(item);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!loc[j]) continue;
            const uint32_t o = fwd_orthant((uint32_t)(j >> 1) | (cls << 1), pbmask) | (uint32_t)(j & 1);
            acc[(int64_t)o * n_tgt + t] += loc[j];
        }
    }
    __device__ void src_weights(uint32_t, int, V& f, V& b) const { f = 1u; b = 1u; }
    __device__ void prep_item(uint32_t, uint32_t) const {}
    __device__ void target(uint32_t item, uint32_t pb, V f, V b) const {
        const int64_t t = tgt_index(item);
        const uint32_t o = fwd_orthant(pb, pbmask);
        acc[(int64_t)o * n_tgt + t] += f;
        acc[(int64_t)(o | 1u) * n_tgt + t] += b;
    }
};

struct PolW64 : ItemMap {
    typedef double V;
    static constexpr int kSrcBytes = 8, kTgtBytes = 32, kTgtFacBytes = 0;
    static constexpr int kLocalT = 2048;
    static constexpr bool kUnitWeights = false;
    static constexpr bool kCanFold = false;      // sums stay per orthant
    static constexpr bool kRecords = false;
    static constexpr int kFoldT = kLocalT, kNW = 1;
    typedef float M;
    typedef float FA;
    typedef double LW;
    const double* w;      // [n_src]
    double* acc;          // [2^d][n_tgt]
    uint32_t pbmask;
    __device__ static V zero() { return 0.0; }
    __device__ static V one() { return 1.0; }
    __device__ static V from_lw(LW v) { return v; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ void local_weights(uint32_t item, uint32_t, LW* o) const {
        const double v = w[item];
        o[0] = o[1] = o[2] = o[3] = v;
    }
    __device__ void flush(uint32_t item, uint32_t cls, const V* loc) const {
        const int64_t t = tgt_index(item);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t o = fwd_orthant((uint32_t)(j >> 1) | (cls << 1), pbmask) | (uint32_t)(j & 1);
            acc[(int64_t)o * n_tgt + t] += loc[j];
        }
    }
    __device__ void src_weights(uint32_t item, int, V& f, V& b) const { f = b = w[item]; }
    __device__ void prep_item(uint32_t, uint32_t) const {}
    __device__ void target(uint32_t item, uint32_t pb, V f, V b) const {
        const int64_t t = tgt_index(item);
        const uint32_t o = fwd_orthant(pb, pbmask);
        acc[(int64_t)o * n_tgt + t] += f;
        acc[(int64_t)(o | 1u) * n_tgt + t] += b;
    }
};

struct PolWFF : ItemMap {
    typedef FF V;
    static constexpr int kSrcBytes = 8, kTgtBytes = 32, kTgtFacBytes = 0;
    static constexpr int kLocalT = 2048;
    static constexpr bool kUnitWeights = false;
    static constexpr bool kCanFold = false;      // sums stay per orthant
    static constexpr bool kRecords = false;
    static constexpr int kFoldT = kLocalT, kNW = 1;
    typedef float M;
    typedef float FA;
    typedef FF LW;
    const FF* w;          // [n_src] weights split into hi + lo
    FF* acc;              // [2^d][n_tgt]
    uint32_t pbmask;
    __device__ static V zero() { return ff_zero(); }
    __device__ static V one() { return FF{1.f, 0.f}; }
    __device__ static V from_lw(LW v) { return v; }
    __device__ static V add(V a, V b) { return ff_add(a, b); }
    __device__ void local_weights(uint32_t item, uint32_t, LW* o) const {
        const FF v = w[item];
        o[0] = o[1] = o[2] = o[3] = v;
    }
    __device__ void flush(uint32_t item, uint32_t cls, const V* loc) const {
        const int64_t t = tgt_index(item);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t o = fwd_orthant((uint32_t)(j >> 1) | (cls << 1), pbmask) | (uint32_t)(j & 1);
            acc[(int64_t)o * n_tgt + t] = ff_add(acc[(int64_t)o * n_tgt + t], loc[j]);
        }
    }
    __device__ void src_weights(uint32_t item, int, V& f, V& b) const { f = b = w[item]; }
    __device__ void prep_item(uint32_t, uint32_t) const {}
    __device__ void target(uint32_t item, uint32_t pb, V f, V b) const {
        const int64_t t = tgt_index(item);
        const uint32_t o = fwd_orthant(pb, pbmask);
        acc[(int64_t)o * n_tgt + t] = ff_add(acc[(int64_t)o * n_tgt + t], f);
        acc[(int64_t)(o | 1u) * n_tgt + t] = ff_add(acc[(int64_t)(o | 1u) * n_tgt + t], b);
    }
};

// ------------------------------------------------------------------ kernel sums
// Exponent factors e^{+-v/h} are stored per item and axis as an FP64-computed
// mantissa (rounded to FP32 on the mixed path) and a power-of-two shift, and
// the product over the enclosing axes (chosen by the item's side bits, the
// same factor in the source and the target role) as `base`.  A forward
// contribution is then  (sum_s w_s B_s E1_s E0+_s) * B_t E1_t E0-_t  with
// every factor pair bounded by 1, the shifted form of eq. (Laplacian
// decomposition nD) with the shift taken at the split of each level.
struct BaseF { float m; int s; };
struct BaseD { double m; int s; int pad; };

template <int NW>
struct SFFn { SFF v[NW]; };
template <int NW>
struct SFn_ { SF v[NW]; };
template <int NW>
struct SDn { SD v[NW]; };

// Mixed path: FP32 compensated bulk sums, FP64 exponent arithmetic.
template <int NW>
struct PolKF : ItemMap {
    typedef SFFn<NW> V;
    static constexpr int kSrcBytes = 36, kTgtBytes = 16 * NW, kTgtFacBytes = 32;
    static constexpr int kLocalT = NW == 1 ? 2048 : 1024;
    static constexpr bool kUnitWeights = false;
    struct LW { float m[NW]; int s; };
    const float* w;           // [n_src] weights (kreg: y), or nullptr for 1
    const FacF* fac;          // [d][n_items]
    int64_t n_items;
    int nbase;                // number of enclosing axes (d - 2)
    BaseF* base;              // [n_items]
    double* acc;              // [NW][n_tgt] (FP64: flushes of concurrent sorts add atomically)
    FF* terms;                // optional [2^d][n_tgt]
    uint32_t pbmask;
    int sgn = -1;             // >= 0: every contribution signed by delta_sgn (see signs())
    __device__ static V zero() {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sff_zero();
        return r;
    }
    __device__ static V add(V a, V b) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sff_add(a.v[i], b.v[i]);
        return r;
    }
    __device__ static V one() {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = SFF{1.f, 0.f, 0};
        return r;
    }
    __device__ static V from_lw(const LW& l) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sff_term(l.m[i], l.s);
        return r;
    }
    // folded local form (targets turn their sums into kernel values)
    static constexpr bool kCanFold = true;
    static constexpr int kFoldT = NW == 1 ? 4096 : 2048, kNW = NW;
    static constexpr bool kRecords = true;    // longer levels on streamed records
    static constexpr bool kFastLocal = true;  // tile-local levels may run on scaled FP32 values
    typedef float M;
    typedef FF FA;
    // Tile-local running sums and scans: plain FP32 mantissa with a shift.
    // A tile-local sum has at most 8 serial terms plus a scan tree of at most
    // 12 levels, so its relative rounding error stays near 1e-6; the target's
    // sum over all levels is compensated.
    struct LOps {
        typedef SFn_<NW> V;
        __device__ static V zero() {
            V r;
#pragma unroll
            for (int i = 0; i < NW; ++i) r.v[i] = sf_zero();
            return r;
        }
        __device__ static V add(V a, V b) {
            V r;
#pragma unroll
            for (int i = 0; i < NW; ++i) r.v[i] = sf_add(a.v[i], b.v[i]);
            return r;
        }
    };
    __device__ static FA fa_zero() { return ff_zero(); }
    // source weights of an element: channel 0 carries wt (0 without a source
    // role), channel 1 (two-channel sums) carries 1 for sources only
    __device__ static typename LOps::V fold_src(float m, int s, float wt, bool src) {
        typename LOps::V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sf_term(((NW == 2 && i == 1) ? (src ? 1.f : 0.f) : wt) * m, s);
        return r;
    }
    // kernel values v * (m 2^s) per weight channel, and a += cf + cb
    __device__ static void fold_value(const typename LOps::V& v, float m, int s, float* c) {
#pragma unroll
        for (int i = 0; i < NW; ++i) c[i] = v.v[i].m * m * pow2f_any(v.v[i].e + s);
    }
    __device__ static void fold_add(FA* a, const float* cf, const float* cb, float sf, float sb) {
#pragma unroll
        for (int i = 0; i < NW; ++i) a[i] = ff_add_f(ff_add_f(a[i], sf * cf[i]), sb * cb[i]);
    }
    // Signs of a target's forward and backward contributions for the signed
    // sums of axis sgn: +1 for orthants with delta_sgn = +1 (the source at or
    // below the target on that axis), -1 otherwise; 1 when unsigned.
    __device__ void signs(int half, uint32_t cls, float& sf, float& sb) const {
        if (sgn < 0) { sf = sb = 1.f; return; }
        if (sgn == 0) { sf = 1.f; sb = -1.f; return; }
        const int up = (sgn == 1) ? half : (int)((cls >> (sgn - 2)) & 1u);
        sf = sb = up ? 1.f : -1.f;
    }
    // the same for the compensated sums of the longer merge levels
    __device__ static V fold_src_g(float m, int s, float wt, bool src) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sff_term(((NW == 2 && i == 1) ? (src ? 1.f : 0.f) : wt) * m, s);
        return r;
    }
    __device__ static void fold_value_g(const V& v, float m, int s, float* c) {
#pragma unroll
        for (int i = 0; i < NW; ++i) c[i] = (v.v[i].hi + v.v[i].lo) * m * pow2f_any(v.v[i].e + s);
    }
    // the four products B E1^{h} E0^{dir} (index 2h + dir) and the weight
    __device__ void fold_item(uint32_t item, uint32_t cls, float* fm, int* fs, float& wt) const {
        const BaseF B = base_of(item, cls);
        const FacF e1 = fac[(int64_t)1 * n_items + item];
        const FacF e0 = fac[item];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            fm[j] = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mm : e0.mp);
            fs[j] = B.s + (h ? -e1.s : e1.s) + (dir ? -e0.s : e0.s);
        }
        wt = (w && is_src(item)) ? w[item] : 1.f;   // the caller zeroes it for non-sources
    }
    __device__ void fold_flush(uint32_t item, const FA* a) const {
        const int64_t t = tgt_index(item);
#pragma unroll
        for (int i = 0; i < NW; ++i) atomicAdd(acc + (int64_t)i * n_tgt + t, (double)a[i].hi + (double)a[i].lo);
    }
    __device__ BaseF base_of(uint32_t item, uint32_t cls) const {
        float m = 1.f;
        int s = 0;
        for (int j = 0; j < nbase; ++j) {
            const FacF f = fac[(int64_t)(j + 2) * n_items + item];
            const bool up = (cls >> j) & 1u;
            m *= up ? f.mm : f.mp;
            s += up ? -f.s : f.s;
        }
        return BaseF{m, s};
    }
    __device__ void prep_item(uint32_t item, uint32_t cls) const { base[item] = base_of(item, cls); }
    // source weights w B E1^{+-} E0^{+-} for (half, direction) = (j >> 1, j & 1)
    __device__ void local_weights(uint32_t item, uint32_t cls, LW* o) const {
        const BaseF B = base_of(item, cls);
        const FacF e1 = fac[(int64_t)1 * n_items + item];
        const FacF e0 = fac[item];
        const float w0 = w ? w[item] : 1.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            const float mm = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mm : e0.mp);
            LW l;
            l.s = B.s + (h ? -e1.s : e1.s) + (dir ? -e0.s : e0.s);
#pragma unroll
            for (int i = 0; i < NW; ++i) l.m[i] = ((NW == 2 && i == 1) ? 1.f : w0) * mm;
            o[j] = l;
        }
    }
    // target factors B E1^{+-} E0^{-+} applied once to the four local sums
    __device__ void flush(uint32_t item, uint32_t cls, const V* loc) const {
        const int64_t t = tgt_index(item);
        const BaseF B = base_of(item, cls);
        const FacF e1 = fac[(int64_t)1 * n_items + item];
        const FacF e0 = fac[item];
        FF a[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) a[i] = ff_zero();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            const float tf = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mp : e0.mm);
            const int ts = B.s + (h ? -e1.s : e1.s) + (dir ? e0.s : -e0.s);
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const float c = (loc[j].v[i].hi + loc[j].v[i].lo) * tf * pow2f_any(loc[j].v[i].e + ts);
                a[i] = ff_add_f(a[i], c);
                if (i == 0 && terms) {
                    const uint32_t o = fwd_orthant((uint32_t)h | (cls << 1), pbmask) | (uint32_t)dir;
                    terms[(int64_t)o * n_tgt + t] = ff_add_f(terms[(int64_t)o * n_tgt + t], c);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NW; ++i) acc[(int64_t)i * n_tgt + t] += (double)a[i].hi + (double)a[i].lo;
    }
    __device__ void src_weights(uint32_t item, int half, V& f, V& b) const {
        const FacF e1 = fac[(int64_t)1 * n_items + item];
        const FacF e0 = fac[item];
        const BaseF B = base[item];
        const float m1 = half ? e1.mm : e1.mp;
        const int s1 = half ? -e1.s : e1.s;
        const float mb = B.m * m1;
        const float w0 = w ? w[item] : 1.f;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const float wi = (NW == 2 && i == 1) ? 1.f : w0;
            f.v[i] = sff_term(wi * mb * e0.mp, B.s + s1 + e0.s);
            b.v[i] = sff_term(wi * mb * e0.mm, B.s + s1 - e0.s);
        }
    }
    __device__ void target(uint32_t item, uint32_t pb, V f, V b) const {
        const int64_t t = tgt_index(item);
        const FacF e1 = fac[(int64_t)1 * n_items + item];
        const FacF e0 = fac[item];
        const BaseF B = base[item];
        const int half = pb & 1u;
        const float m1 = half ? e1.mm : e1.mp;
        const int s1 = half ? -e1.s : e1.s;
        const float tf = B.m * m1 * e0.mm;            // forward: E0^-(t)
        const int sf = B.s + s1 - e0.s;
        const float tb = B.m * m1 * e0.mp;            // backward: E0^+(t)
        const int sb = B.s + s1 + e0.s;
        const uint32_t o = fwd_orthant(pb, pbmask);
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const float cf = (f.v[i].hi + f.v[i].lo) * tf * pow2f_any(f.v[i].e + sf);
            const float cb = (b.v[i].hi + b.v[i].lo) * tb * pow2f_any(b.v[i].e + sb);
            float gf, gb;
            signs(half, pb >> 1, gf, gb);
            acc[(int64_t)i * n_tgt + t] += (double)(gf * cf) + (double)(gb * cb);
            if (i == 0 && terms) {
                terms[(int64_t)o * n_tgt + t] = ff_add_f(terms[(int64_t)o * n_tgt + t], cf);
                terms[(int64_t)(o | 1u) * n_tgt + t] = ff_add_f(terms[(int64_t)(o | 1u) * n_tgt + t], cb);
            }
        }
    }
};

// All-FP64 path.
template <int NW>
struct PolKD : ItemMap {
    typedef SDn<NW> V;
    static constexpr int kSrcBytes = 72, kTgtBytes = 16 * NW, kTgtFacBytes = 64;
    static constexpr int kLocalT = NW == 1 ? 1024 : 512;
    static constexpr bool kUnitWeights = false;
    struct LW { double m[NW]; int s; int pad; };
    const double* w;
    const FacD* fac;
    int64_t n_items;
    int nbase;
    BaseD* base;
    double* acc;
    double* terms;
    uint32_t pbmask;
    int sgn = -1;             // >= 0: every contribution signed by delta_sgn (see signs())
    __device__ static V zero() {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sd_zero();
        return r;
    }
    __device__ static V add(V a, V b) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sd_add(a.v[i], b.v[i]);
        return r;
    }
    __device__ static V one() {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = SD{1.0, 0};
        return r;
    }
    __device__ static V from_lw(const LW& l) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sd_term(l.m[i], l.s);
        return r;
    }
    // folded local form (targets turn their sums into kernel values)
    static constexpr bool kCanFold = true;
    static constexpr int kFoldT = NW == 1 ? 2048 : 1024, kNW = NW;
    static constexpr bool kFastLocal = false;
    // longer levels gather the factors per item (measured faster on the FP64
    // path, whose cost is FP64 arithmetic rather than memory latency)
    static constexpr bool kRecords = false;
    typedef double M;
    typedef double FA;
    struct LOps {   // tile-local sums: the same shifted FP64 values
        typedef SDn<NW> V;
        __device__ static V zero() { return PolKD::zero(); }
        __device__ static V add(V a, V b) { return PolKD::add(a, b); }
    };
    __device__ static FA fa_zero() { return 0.0; }
    __device__ static V fold_src(double m, int s, double wt, bool src) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = sd_term(((NW == 2 && i == 1) ? (src ? 1.0 : 0.0) : wt) * m, s);
        return r;
    }
    __device__ static void fold_value(const V& v, double m, int s, double* c) {
#pragma unroll
        for (int i = 0; i < NW; ++i) c[i] = ldexp_i(v.v[i].m * m, max(v.v[i].e + s, -4096));
    }
    __device__ static void fold_add(FA* a, const double* cf, const double* cb, double sf, double sb) {
#pragma unroll
        for (int i = 0; i < NW; ++i) a[i] += sf * cf[i] + sb * cb[i];
    }
    __device__ void signs(int half, uint32_t cls, double& sf, double& sb) const {
        if (sgn < 0) { sf = sb = 1.0; return; }
        if (sgn == 0) { sf = 1.0; sb = -1.0; return; }
        const int up = (sgn == 1) ? half : (int)((cls >> (sgn - 2)) & 1u);
        sf = sb = up ? 1.0 : -1.0;
    }
    __device__ static V fold_src_g(double m, int s, double wt, bool src) { return fold_src(m, s, wt, src); }
    __device__ static void fold_value_g(const V& v, double m, int s, double* c) { fold_value(v, m, s, c); }
    __device__ void fold_item(uint32_t item, uint32_t cls, double* fm, int* fs, double& wt) const {
        const BaseD B = base_of(item, cls);
        const FacD e1 = fac[(int64_t)1 * n_items + item];
        const FacD e0 = fac[item];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            fm[j] = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mm : e0.mp);
            fs[j] = B.s + (h ? -e1.s : e1.s) + (dir ? -e0.s : e0.s);
        }
        wt = (w && is_src(item)) ? w[item] : 1.0;
    }
    __device__ void fold_flush(uint32_t item, const FA* a) const {
        const int64_t t = tgt_index(item);
#pragma unroll
        for (int i = 0; i < NW; ++i) atomicAdd(acc + (int64_t)i * n_tgt + t, a[i]);
    }
    __device__ BaseD base_of(uint32_t item, uint32_t cls) const {
        double m = 1.0;
        int s = 0;
        for (int j = 0; j < nbase; ++j) {
            const FacD f = fac[(int64_t)(j + 2) * n_items + item];
            const bool up = (cls >> j) & 1u;
            m *= up ? f.mm : f.mp;
            s += up ? -f.s : f.s;
        }
        return BaseD{m, s, 0};
    }
    __device__ void prep_item(uint32_t item, uint32_t cls) const { base[item] = base_of(item, cls); }
    __device__ void local_weights(uint32_t item, uint32_t cls, LW* o) const {
        const BaseD B = base_of(item, cls);
        const FacD e1 = fac[(int64_t)1 * n_items + item];
        const FacD e0 = fac[item];
        const double w0 = w ? w[item] : 1.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            const double mm = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mm : e0.mp);
            LW l;
            l.s = B.s + (h ? -e1.s : e1.s) + (dir ? -e0.s : e0.s);
            l.pad = 0;
#pragma unroll
            for (int i = 0; i < NW; ++i) l.m[i] = ((NW == 2 && i == 1) ? 1.0 : w0) * mm;
            o[j] = l;
        }
    }
    __device__ void flush(uint32_t item, uint32_t cls, const V* loc) const {
        const int64_t t = tgt_index(item);
        const BaseD B = base_of(item, cls);
        const FacD e1 = fac[(int64_t)1 * n_items + item];
        const FacD e0 = fac[item];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = j >> 1, dir = j & 1;
            const double tf = B.m * (h ? e1.mm : e1.mp) * (dir ? e0.mp : e0.mm);
            const int ts = B.s + (h ? -e1.s : e1.s) + (dir ? e0.s : -e0.s);
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const double c = ldexp_i(loc[j].v[i].m * tf, max(loc[j].v[i].e + ts, -4096));
                acc[(int64_t)i * n_tgt + t] += c;
                if (i == 0 && terms) {
                    const uint32_t o = fwd_orthant((uint32_t)h | (cls << 1), pbmask) | (uint32_t)dir;
                    terms[(int64_t)o * n_tgt + t] += c;
                }
            }
        }
    }
    __device__ void src_weights(uint32_t item, int half, V& f, V& b) const {
        const FacD e1 = fac[(int64_t)1 * n_items + item];
        const FacD e0 = fac[item];
        const BaseD B = base[item];
        const double m1 = half ? e1.mm : e1.mp;
        const int s1 = half ? -e1.s : e1.s;
        const double mb = B.m * m1;
        const double w0 = w ? w[item] : 1.0;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const double wi = (NW == 2 && i == 1) ? 1.0 : w0;
            f.v[i] = sd_term(wi * mb * e0.mp, B.s + s1 + e0.s);
            b.v[i] = sd_term(wi * mb * e0.mm, B.s + s1 - e0.s);
        }
    }
    __device__ void target(uint32_t item, uint32_t pb, V f, V b) const {
        const int64_t t = tgt_index(item);
        const FacD e1 = fac[(int64_t)1 * n_items + item];
        const FacD e0 = fac[item];
        const BaseD B = base[item];
        const int half = pb & 1u;
        const double m1 = half ? e1.mm : e1.mp;
        const int s1 = half ? -e1.s : e1.s;
        const double tf = B.m * m1 * e0.mm;
        const int sf = B.s + s1 - e0.s;
        const double tb = B.m * m1 * e0.mp;
        const int sb = B.s + s1 + e0.s;
        const uint32_t o = fwd_orthant(pb, pbmask);
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const double cf = ldexp_i(f.v[i].m * tf, max(f.v[i].e + sf, -4096));
            const double cb = ldexp_i(b.v[i].m * tb, max(b.v[i].e + sb, -4096));
            double gf, gb;
            signs(half, pb >> 1, gf, gb);
            acc[(int64_t)i * n_tgt + t] += gf * cf + gb * cb;
            if (i == 0 && terms) {
                terms[(int64_t)o * n_tgt + t] += cf;
                terms[(int64_t)(o | 1u) * n_tgt + t] += cb;
            }
        }
    }
};

// ------------------------------------------------------------------ gathers
typedef ClassSpecK ClassSpec;

// ------------------------------------------------------------------ driver
struct DCBuffers {
    uint32_t* k[2];   // inner sort ping-pong keys
    uint32_t* m[2];   // inner sort ping-pong metas
    void* totals;
    void* carries;
    int64_t* co;      // merge-path co-ranks of a level, shared by its totals and sweep passes
    // folded kernel sums: record arrays (fm, fs, wt, fa) of each ping-pong side
    void* rec[2][4];
    // kernel sums: per-item base factors of this buffer set's sorts (levels
    // sorted concurrently have different class bits), and, for the policies
    // whose longer levels update target sums in place, a private accumulator
    // (summed into the caller's after the sweep)
    void* base;
    double* acc;
};
template <class Pol>
FoldRecs<Pol> fold_recs(const DCBuffers& b, int q) {
    return FoldRecs<Pol>{(typename Pol::M*)b.rec[q][0], (int*)b.rec[q][1], (typename Pol::M*)b.rec[q][2],
                         (typename Pol::FA*)b.rec[q][3]};
}

// host-side common pieces (fk_dc_common.cu)
fk_status plain_merge_level(const MergeArgs& a, cudaStream_t st);
fk_status gather_outer(const uint32_t* seq, int64_t n, const uint32_t* Pkey, uint32_t* key,
                       uint32_t* meta, cudaStream_t st);
fk_status record_index(const uint32_t* seq, int64_t n, int E, uint32_t* idx, cudaStream_t st);
fk_status iota_u32(uint32_t* a, int64_t n, cudaStream_t st);
fk_status add_f64(double* dst, const double* src, int64_t n, cudaStream_t st);   // dst += src
inline int ceil_log2(int64_t n) {
    int e = 0;
    while (((int64_t)1 << e) < n) ++e;
    return e;
}

// Option bits of the sweeps (chosen by the batched autotuner).
enum : int { OPT_HALF_TILE = 1 };

template <class Pol, int CLSB, bool FOLD, bool HALF>
fk_status local_levels_t(const uint32_t* seq, int64_t n, int E, const uint32_t* P0, const ClassSpec& cs,
                         const Pol& pol, DCBuffers& b, int& L0, cudaStream_t st) {
    typedef LocalCfg<Pol, CLSB, FOLD, HALF> Cfg;
    int lt = 0;
    while ((1 << (lt + 1)) <= Cfg::T) ++lt;
    L0 = E < lt ? E : lt;
    constexpr size_t smem = Cfg::bytes;
    static_assert(smem <= 227 * 1024, "tile does not fit in shared memory");
    static bool attr_set = false;
    if (!attr_set) {
        if constexpr (FOLD)
            FK_CUDA(cudaFuncSetAttribute(k_local_fold<Pol, CLSB, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        else
            FK_CUDA(cudaFuncSetAttribute(k_local_sweep<Pol, CLSB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        attr_set = true;
    }
    const double lbytes = 4.0 * n + (double)pol.n_src * Pol::kSrcBytes +
                          (double)pol.n_tgt * (Pol::kTgtBytes + Pol::kTgtFacBytes) + (E > L0 ? 8.0 * n : 0.0);
    ProfScope ps(Pol::kCanFold ? PF_KLOCAL : PF_LOCAL,
                 Pol::kCanFold ? (double)n * L0 * kKernelOpsPerItemLevel : lbytes, st, lbytes);
    if constexpr (FOLD)
        k_local_fold<Pol, CLSB, HALF><<<grid_for(n, Cfg::T), Cfg::NT, smem, st>>>(
            seq, n, P0, cs, L0, pol, b.k[0], b.m[0], E > L0 ? 1 : 0, (E > L0 && Pol::kRecords) ? 1 : 0,
            fold_recs<Pol>(b, 0));
    else
        k_local_sweep<Pol, CLSB><<<grid_for(n, Cfg::T), Cfg::NT, smem, st>>>(seq, n, P0, cs, L0, pol, b.k[0], b.m[0],
                                                                           E > L0 ? 1 : 0);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

template <class Pol, int CLSB, bool FOLD>
fk_status local_levels(const uint32_t* seq, int64_t n, int E, const uint32_t* P0, const ClassSpec& cs,
                       const Pol& pol, DCBuffers& b, int& L0, int opts, cudaStream_t st) {
    if constexpr (FOLD && Pol::kNW == 1) {
        if (opts & OPT_HALF_TILE) return local_levels_t<Pol, CLSB, FOLD, true>(seq, n, E, P0, cs, pol, b, L0, st);
    }
    return local_levels_t<Pol, CLSB, FOLD, false>(seq, n, E, P0, cs, pol, b, L0, st);
}

// Merge levels L0..E-1 of the folded kernel sums on records.
template <class Pol, int CLSB>
fk_status fold_levels(int64_t n, int E, int L0, const Pol& pol, DCBuffers& b, cudaStream_t st) {
    typedef typename Pol::V V;
    constexpr int NCH = 2 << CLSB;
    constexpr int MTILE = MT * MergeItems<Pol, CLSB>::value;
    const unsigned ctas = grid_for(n, MTILE);
    // algorithmic bytes of one level: key, meta and the record in and out
    const double rec_bytes = 8.0 + 8.0 * sizeof(typename Pol::M) + 16.0 + Pol::kNW * sizeof(typename Pol::FA);
    int cur = 0;
    for (int m = L0; m < E; ++m) {
        MergeArgs a{b.k[cur], b.m[cur], b.k[cur ^ 1], b.m[cur ^ 1], n, m};
        const FoldRecs<Pol> rin = fold_recs<Pol>(b, cur), rout = fold_recs<Pol>(b, cur ^ 1);
        const int last = (m == E - 1) ? 1 : 0;
        const int64_t R2 = (int64_t)2 << m;
        const V* carries = nullptr;
        if (R2 > MTILE) a.co = b.co;          // the totals pass finds the co-ranks
        if (R2 > MTILE) {
            {
                ProfScope ps(PF_MERGE_TOTALS, (rec_bytes - Pol::kNW * sizeof(typename Pol::FA)) * n, st);
                k_merge_fold<Pol, CLSB, PH_TOTALS><<<ctas, MT, 0, st>>>(a, rin, rout, pol, (V*)b.totals, nullptr,
                                                                       last);
                FK_LAUNCH_CHECK();
            }
            const int64_t per = R2 / MTILE;
            const int64_t nblk = ((int64_t)ctas + per - 1) / per;
            k_carries<Pol, NCH, MTILE><<<grid_for(nblk * NCH * 2 * 32, 256), 256, 0, st>>>((const V*)b.totals,
                                                                              (V*)b.carries, n, m);
            FK_LAUNCH_CHECK();
            carries = (const V*)b.carries;
        }
        a.co_read = 1;                        // and the sweep reuses them
        ProfScope ps(PF_MERGE_SWEEP, rec_bytes * n * (last ? 0.5 : 1.0) + (last ? 8.0 * pol.n_tgt : 0.0), st);
        k_merge_fold<Pol, CLSB, PH_SWEEP><<<ctas, MT, 0, st>>>(a, rin, rout, pol, nullptr, carries, last);
        FK_LAUNCH_CHECK();
        cur ^= 1;
    }
    return FK_OK;
}

template <class Pol, int CLSB>
fk_status inner_sort(const uint32_t* seq, int64_t n, int E, const uint32_t* P0, const ClassSpec& cs,
                     const Pol& pol, DCBuffers& b, int opts, cudaStream_t st) {
    typedef typename Pol::V V;
    constexpr int NCH = 2 << CLSB;
    // tile-local levels (gather fused into the tile load)
    int L0 = 0;
    if constexpr (Pol::kCanFold && CLSB >= 3) {
        // d > 4: folded sums only (per-orthant terms would take 2^d channels
        // of target state per item)
        if (pol.terms) return set_error(FK_ERR_UNSUPPORTED, "per-orthant kernel terms support d <= 4");
        FK_TRY((local_levels<Pol, CLSB, true>(seq, n, E, P0, cs, pol, b, L0, opts, st)));
        if constexpr (Pol::kRecords) return fold_levels<Pol, CLSB>(n, E, L0, pol, b, st);
    } else if constexpr (Pol::kCanFold) {
        if (!pol.terms) {
            FK_TRY((local_levels<Pol, CLSB, true>(seq, n, E, P0, cs, pol, b, L0, opts, st)));
            if constexpr (Pol::kRecords) return fold_levels<Pol, CLSB>(n, E, L0, pol, b, st);
        } else {
            FK_TRY((local_levels<Pol, CLSB, false>(seq, n, E, P0, cs, pol, b, L0, opts, st)));
        }
    } else {
        FK_TRY((local_levels<Pol, CLSB, false>(seq, n, E, P0, cs, pol, b, L0, opts, st)));
    }
    if constexpr (Pol::kCanFold && Pol::kRecords && CLSB >= 3) {
        return FK_OK;   // not reached: the folded records handled every level above
    } else {
    int cur = 0;
    constexpr int MTILE = MT * MergeItems<Pol, CLSB>::value;
    const unsigned ctas = grid_for(n, MTILE);
    // algorithmic bytes of one sweep merge: keys+metas in and out, source
    // weights read once, target accumulators read and written once
    const double sweep_bytes = 16.0 * n + (double)pol.n_src * Pol::kSrcBytes + (double)pol.n_tgt * Pol::kTgtBytes +
                               (pol.tgt_off > 0 ? (double)pol.n_tgt * Pol::kTgtFacBytes : 0.0);
    for (int m = L0; m < E; ++m) {
        MergeArgs a{b.k[cur], b.m[cur], b.k[cur ^ 1], b.m[cur ^ 1], n, m};
        const int64_t R2 = (int64_t)2 << m;
        if (R2 > MTILE) {
            a.co = b.co;                      // found by the totals pass, reused by the sweep
            {
                ProfScope ps(PF_MERGE_TOTALS, 8.0 * n + (double)pol.n_src * Pol::kSrcBytes, st);
                k_merge<Pol, CLSB, PH_TOTALS><<<ctas, MT, 0, st>>>(a, pol, (V*)b.totals, nullptr);
                FK_LAUNCH_CHECK();
            }
            const int64_t per = R2 / MTILE;
            const int64_t nblk = ((int64_t)ctas + per - 1) / per;
            k_carries<Pol, NCH, MTILE><<<grid_for(nblk * NCH * 2 * 32, 256), 256, 0, st>>>((const V*)b.totals,
                                                                              (V*)b.carries, n, m);
            FK_LAUNCH_CHECK();
            a.co_read = 1;
            ProfScope ps(PF_MERGE_SWEEP, sweep_bytes, st);
            k_merge<Pol, CLSB, PH_SWEEP><<<ctas, MT, 0, st>>>(a, pol, nullptr, (const V*)b.carries);
            FK_LAUNCH_CHECK();
        } else {
            ProfScope ps(PF_MERGE_SWEEP, sweep_bytes, st);
            k_merge<Pol, CLSB, PH_SWEEP><<<ctas, MT, 0, st>>>(a, pol, nullptr, nullptr);
            FK_LAUNCH_CHECK();
        }
        cur ^= 1;
    }
    return FK_OK;
    }
}

// Recursion over the tree axes.  `seq` holds the items sorted by P_k inside
// nodes of size 2^E.  For k == 1 the innermost sweep sort runs directly; for
// k >= 2 the axis-k tree is a merge sort of seq by P_{k-1} whose level l
// states (nodes of 2^{l+1} sorted by P_{k-1}) each start the recursion one
// axis lower with the side bit l of the axis-k index added to the class.
struct OuterBuffers {
    uint32_t* k[kPoolStreams + 1];   // level states: ping-pong, or a ring of S + 1 (concurrent levels)
    uint32_t* m[kPoolStreams + 1];
    uint32_t* idx;    // index of every item inside its axis-k node
    // axis 2 with concurrent levels, for the policies whose longer levels add
    // to the target sums in place (no atomics): the nested launch's private
    // accumulator, summed into the caller's after the sweep
    double* nacc;
};

// Inner sorts of concurrent levels: streams used at the lowest tree axis.
constexpr int kSweepStreams = 4;
enum : int { OPT_SERIAL = 2 };   // option bit: no concurrent levels (the batched path)

template <class Pol>
__host__ int sweep_streams(const Pol& pol, int opts) {
    if constexpr (Pol::kCanFold) {
        // folded sums flush atomically; per-orthant terms and orthant sums do not
        return (!pol.terms && !(opts & OPT_SERIAL)) ? kSweepStreams : 1;
    }
    return 1;
}

template <class Pol, int CLSB>
fk_status recurse(int k, const uint32_t* seq, int64_t n, int E, const uint32_t* const* P,
                  ClassSpec cs, const Pol& pol, OuterBuffers* ob, DCBuffers* ib, int S, int opts,
                  cudaStream_t st) {
    if (k == 1) return inner_sort<Pol, CLSB>(seq, n, E, P[0], cs, pol, ib[0], opts, st);
    OuterBuffers& o = ob[k];
    const uint32_t* idx = P[k];
    if (o.idx) {
        FK_TRY(record_index(seq, n, E, o.idx, st));
        idx = o.idx;
    }
    FK_TRY(gather_outer(seq, n, P[k - 1], o.k[0], o.m[0], st));
    // Outer levels of axis 2 whose nodes fit a tile (folded sums): their inner
    // sorts run in one launch of k_nested_fold, beside the merges and the
    // inner sorts of the longer levels (on a stream of its own when the levels
    // run concurrently; its flushes are atomic, and it gets a private
    // accumulator where the longer levels update target sums in place).
    int l0 = 0;
    if constexpr (Pol::kCanFold && CLSB <= 2) {
        if (k == 2 && !pol.terms) {
            int lt = 0;
            while ((2 << lt) <= NFT) ++lt;
            l0 = E < lt ? E : lt;
        }
    }
    auto launch_nested = [&](cudaStream_t s2, const Pol& pl) -> fk_status {
        if constexpr (Pol::kCanFold && CLSB <= 2) {
            typedef NestedCfg<Pol, CLSB> NC;
            static bool attr_set = false;
            if (!attr_set) {
                FK_CUDA(cudaFuncSetAttribute(k_nested_fold<Pol, CLSB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)NC::bytes));
                attr_set = true;
            }
            const double lbytes = 4.0 * n + (double)pol.n_src * Pol::kSrcBytes +
                                  (double)pol.n_tgt * (Pol::kTgtBytes + Pol::kTgtFacBytes);
            ProfScope ps(PF_KLOCAL, (double)n * (l0 * (l0 + 1) / 2) * kKernelOpsPerItemLevel, s2, l0 * lbytes);
            k_nested_fold<Pol, CLSB><<<grid_for(n, NFT), NFN, NC::bytes, s2>>>(seq, n, P[0], P[1], cs, l0, pl);
            FK_LAUNCH_CHECK();
        }
        return FK_OK;
    };
    auto class_of_level = [&](int l) {
        ClassSpec c2 = cs;
        // the enclosing axes keep their bits; axis k contributes bit (k - 2)
        c2.idx[k - 2] = idx;
        c2.lvl[k - 2] = l;
        if (c2.nb < k - 1) c2.nb = k - 1;
        return c2;
    };
    if (k == 2 && S > 1) {
        // The merges of axis 2 run on the caller's stream, ahead of the inner
        // sorts, which run on S forked streams (buffers per stream); the level
        // states form a ring of S + 1, and a merge waits for the inner sort
        // that last read the state it overwrites.
        const int R = S + 1;
        StreamFork fork;
        FK_TRY(fork.begin(2, st, S + (l0 > 0 ? 1 : 0)));
        cudaEvent_t ready = fork.ev[0];
        cudaEvent_t* done = fork.ev + 1;
        fk_status rc = FK_OK;
        if (l0 > 0) {
            Pol pn = pol;
            if constexpr (Pol::kCanFold) {
                if (o.nacc) pn.acc = o.nacc;
            }
            rc = launch_nested(fork.s[S], pn);
        }
        for (int l = 0; l < E && rc == FK_OK; ++l) {
            const int in = l % R, out = (l + 1) % R;
            if (l >= R) {
                const cudaError_t e = cudaStreamWaitEvent(st, done[(l - R) % R], 0);
                if (e != cudaSuccess) { rc = cuda_error(e, "level wait"); break; }
            }
            MergeArgs a{o.k[in], o.m[in], o.k[out], o.m[out], n, l};
            rc = plain_merge_level(a, st);
            if (rc != FK_OK) break;
            if (l < l0) {
                // inner sort done by k_nested_fold: nothing reads this state
                const cudaError_t e = cudaEventRecord(done[l % R], st);
                if (e != cudaSuccess) rc = cuda_error(e, "level done");
                continue;
            }
            const int q = l % S;
            cudaError_t e = cudaEventRecord(ready, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(fork.s[q], ready, 0);
            if (e != cudaSuccess) { rc = cuda_error(e, "level fork"); break; }
            Pol pq = pol;
            if constexpr (Pol::kCanFold) {
                pq.base = (decltype(pq.base))ib[q].base;
                if (ib[q].acc) pq.acc = ib[q].acc;
            }
            rc = inner_sort<Pol, CLSB>(o.m[out], n, l + 1, P[0], class_of_level(l), pq, ib[q], opts, fork.s[q]);
            if (rc != FK_OK) break;
            e = cudaEventRecord(done[l % R], fork.s[q]);
            if (e != cudaSuccess) rc = cuda_error(e, "level done");
        }
        const fk_status rj = fork.end();
        return rc != FK_OK ? rc : rj;
    }
    if (l0 > 0) FK_TRY(launch_nested(st, pol));
    int cur = 0;
    for (int l = 0; l < E; ++l) {
        MergeArgs a{o.k[cur], o.m[cur], o.k[cur ^ 1], o.m[cur ^ 1], n, l};
        FK_TRY(plain_merge_level(a, st));
        cur ^= 1;
        if (l < l0) continue;   // inner sort done by k_nested_fold
        FK_TRY((recurse<Pol, CLSB>(k - 1, o.m[cur], n, l + 1, P, class_of_level(l), pol, ob, ib, S, opts, st)));
    }
    return FK_OK;
}

// Plans (sizing) and runs the whole sweep for a given policy.  P[0..d_eff-1]
// are the per-axis positions, seq_top the items sorted by P[d_eff-1].
template <class Pol, int CLSB>
fk_status dc_sweep(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top,
                   const Pol& pol, Arena& ar, cudaStream_t st, int levels = -1, int opts = 0) {
    typedef typename Pol::V V;
    constexpr int NCH = 2 << CLSB;
    const int S = d_eff >= 3 ? sweep_streams(pol, opts) : 1;
    OuterBuffers ob[8] = {};
    for (int k = 2; k < d_eff; ++k) {
        const int nb = (k == 2 && S > 1) ? S + 1 : 2;
        for (int q = 0; q < nb; ++q) { ob[k].k[q] = ar.take<uint32_t>(n); ob[k].m[q] = ar.take<uint32_t>(n); }
        ob[k].idx = (k < d_eff - 1) ? ar.take<uint32_t>(n) : nullptr;
    }
    if constexpr (Pol::kCanFold && !Pol::kRecords && CLSB <= 2) {
        if (d_eff >= 3 && S > 1 && !pol.terms) ob[2].nacc = ar.take<double>((size_t)Pol::kNW * pol.n_tgt);
    }
    DCBuffers ib[kPoolStreams] = {};
    const int64_t ctas = (n + kMergeTileMin - 1) / kMergeTileMin;   // at most, whatever the tile
    for (int s = 0; s < S; ++s) {
        for (int q = 0; q < 2; ++q) { ib[s].k[q] = ar.take<uint32_t>(n); ib[s].m[q] = ar.take<uint32_t>(n); }
        ib[s].totals = ar.take<V>((size_t)ctas * 2 * NCH);
        ib[s].carries = ar.take<V>((size_t)ctas * 2 * NCH);
        ib[s].co = ar.take<int64_t>((size_t)ctas * 2);
        for (int q = 0; q < 2; ++q)
            for (int j = 0; j < 4; ++j) ib[s].rec[q][j] = nullptr;
        ib[s].base = nullptr;
        ib[s].acc = nullptr;
        if constexpr (Pol::kCanFold) {
            if (S > 1 && !Pol::kRecords) {
                ib[s].base = ar.take<char>((size_t)n * sizeof(*pol.base));
                if (s > 0) ib[s].acc = ar.take<double>((size_t)Pol::kNW * pol.n_tgt);
            }
        }
        if constexpr (Pol::kCanFold && Pol::kRecords) {
            for (int q = 0; q < 2; ++q) {
                ib[s].rec[q][0] = ar.take<typename Pol::M>((size_t)4 * n);
                ib[s].rec[q][1] = ar.take<int>((size_t)4 * n);
                ib[s].rec[q][2] = ar.take<typename Pol::M>((size_t)n);
                ib[s].rec[q][3] = ar.take<typename Pol::FA>((size_t)Pol::kNW * n);
            }
        }
    }
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (dominance sweep)");
    if (n <= 1) return FK_OK;
    ClassSpec cs = {};
    const int E = levels >= 0 ? levels : ceil_log2(n);
    // for k == d_eff-1 the axis index is P[d_eff-1] itself (idx == nullptr above)
    if (d_eff - 1 >= 2) ob[d_eff - 1].idx = nullptr;
    for (int s = 1; s < S; ++s)
        if (ib[s].acc) FK_CUDA(cudaMemsetAsync(ib[s].acc, 0, sizeof(double) * Pol::kNW * pol.n_tgt, st));
    if (ob[2].nacc) FK_CUDA(cudaMemsetAsync(ob[2].nacc, 0, sizeof(double) * Pol::kNW * pol.n_tgt, st));
    FK_TRY((recurse<Pol, CLSB>(d_eff - 1, seq_top, n, E, P, cs, pol, ob, ib, S, opts, st)));
    if constexpr (Pol::kCanFold) {
        for (int s = 1; s < S; ++s)
            if (ib[s].acc) FK_TRY(add_f64(pol.acc, ib[s].acc, Pol::kNW * pol.n_tgt, st));
        if (ob[2].nacc) FK_TRY(add_f64(pol.acc, ob[2].nacc, Pol::kNW * pol.n_tgt, st));
    }
    return FK_OK;
}

}  // namespace dc
}  // namespace fk
