// fk_dc.cuh -- divide-and-conquer dominance sums at the sample points.
//
// Sec. 2.2 (Algorithms 2-5) and Appendix D (Algorithms 8-12) of the paper
// compute, for every target, the sum of the source weights lying in each of
// the 2^d orthants, by splitting on the last axis, recursing on both halves,
// and merging the cross pairs one dimension lower, down to a one-dimensional
// sweep (Merge1D).  This file re-expresses that recursion as nested bottom-up
// merge sorts so that every step is a data-parallel pass:
//
//  * items are sources and targets (a point evaluated at the sample points is
//    one source item plus one target item, so that the <= / > relation on tied
//    coordinates is decided by ordering sources before targets);
//  * P_k[item] is the item's position in the order of axis k (coordinate, then
//    source-before-target): a source s precedes a target t in that order iff
//    x_k(s) <= z_k(t), so every orthant relation becomes "precedes/follows";
//  * the tree of axis k (k >= 2) is a bottom-up merge sort of the axis-k order
//    by key P_{k-1}: after level l its runs are the level-l nodes (size
//    2^{l+1}) already sorted for the next axis, which is exactly the split of
//    Algorithm 3/4 with the children's sub-permutations phi_{l,m};
//  * at the innermost tree axis (axis 1) the merge sort is by key P_0 and each
//    merge of a left run C with a right run D is the Merge1D sweep: a target in
//    D adds the weights of the C sources before it (delta_0 = +1) and after it
//    (delta_0 = -1); a target in C does the same with the D sources.  Only
//    pairs on opposite sides at every enclosing level are cross pairs; the side
//    bits ("class") of the enclosing axes travel in the item's meta word and a
//    target reads the channel of the complementary class.
//
// One kernel (k_merge) implements all merges; its sweep uses per-channel
// forward and backward scans so that no suffix is ever formed by subtraction.
#pragma once

#include "fk_internal.cuh"

namespace fk {
namespace dc {

constexpr int MT = 256;            // threads per CTA
constexpr int MI = 8;              // outputs per thread
constexpr int MTILE = MT * MI;     // outputs per CTA
constexpr int kItemBits = 26;      // meta = item | cls << 26
constexpr uint32_t kItemMask = (1u << kItemBits) - 1u;

struct MergeArgs {
    const uint32_t* key_in;
    const uint32_t* meta_in;
    uint32_t* key_out;
    uint32_t* meta_out;
    int64_t n;
    int logR;     // input runs of length R = 2^logR, output runs 2R
};

// ------------------------------------------------------------ generic shuffles
template <class T>
__device__ __forceinline__ T shfl_up_t(const T& v, int o, int width) {
    static_assert(sizeof(T) % 4 == 0, "shuffle of non-word type");
    T r;
    const uint32_t* p = reinterpret_cast<const uint32_t*>(&v);
    uint32_t* q = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) q[i] = __shfl_up_sync(0xffffffffu, p[i], o, width);
    return r;
}
template <class T>
__device__ __forceinline__ T shfl_down_t(const T& v, int o, int width) {
    T r;
    const uint32_t* p = reinterpret_cast<const uint32_t*>(&v);
    uint32_t* q = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) q[i] = __shfl_down_sync(0xffffffffu, p[i], o, width);
    return r;
}

// Merge path: number of elements taken from A among the first q outputs of a
// stable merge (A first on ties) of sorted A[0,la) and B[0,lb).
template <class Acc>
__device__ __forceinline__ int64_t merge_path(Acc A, int64_t la, Acc B, int64_t lb, int64_t q) {
    int64_t lo = q > lb ? q - lb : 0;
    int64_t hi = q < la ? q : la;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (A(mid) <= B(q - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Warp-cooperative merge path over global memory: each step probes 32
// candidate split points at once, so a search over R elements takes about
// log_32(R) dependent round trips instead of log_2(R).  All 32 lanes must
// call it; every lane returns the same value.
__device__ __forceinline__ int64_t merge_path_warp(const uint32_t* __restrict__ A, int64_t la,
                                                   const uint32_t* __restrict__ B, int64_t lb, int64_t q) {
    const int lane = threadIdx.x & 31;
    int64_t lo = q > lb ? q - lb : 0;
    int64_t hi = q < la ? q : la;
    // invariant: the answer p (smallest p with A[p] > B[q-1-p], or hi) lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t span = hi - lo;
        const int64_t p = lo + (span * (lane + 1)) / 33;
        const bool f = A[p] <= B[q - 1 - p];           // true below the answer
        const unsigned m = __ballot_sync(0xffffffffu, f);
        // last lane with f true -> the answer is above its probe
        const int last = 31 - __clz((int)m);            // -1 when m == 0
        const int64_t nlo = (m == 0u) ? lo : lo + (span * (last + 1)) / 33 + 1;
        const int64_t nhi = (m == 0xffffffffu) ? hi : lo + (span * (last + 2)) / 33;
        lo = nlo;
        hi = nhi;
    }
    // final range of at most 32 candidates: one probe per lane
    const int64_t p = lo + lane;
    const bool f = (p < hi) && (A[p] <= B[q - 1 - p]);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    return lo + __popc(m);
}

struct GAcc {
    const uint32_t* p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct SAcc {
    const uint32_t* p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};

// Class bits of an item for the innermost sort: bit j = bit lvl[j] of idx[j][item].
struct ClassSpecK {
    const uint32_t* idx[6];
    int lvl[6];
    int nb;
};
__device__ __forceinline__ uint32_t class_of_k(const ClassSpecK& cs, uint32_t item) {
    uint32_t c = 0;
    for (int j = 0; j < cs.nb; ++j) c |= ((cs.idx[j][item] >> cs.lvl[j]) & 1u) << j;
    return c;
}

__device__ __forceinline__ int64_t mpd(int64_t p) { return p + (p >> 5); }
struct MAccP {
    const uint32_t* p;
    int base;
    __device__ uint32_t operator()(int64_t i) const { return p[mpd(base + i)]; }
};

// Phases of k_merge.
enum { PH_PLAIN = 0, PH_TOTALS = 1, PH_SWEEP = 2 };

// Scan of per-thread channel values over segments of `ts` consecutive threads
// (ts a power of two, 1 < ts <= MT).  On return fe/be hold the exclusive
// prefix (forward) and exclusive suffix (backward) within the segment.
template <class Pol, int NCH, int NT = MT>
__device__ __forceinline__ void seg_scan(typename Pol::V (&fe)[NCH], typename Pol::V (&be)[NCH],
                                         int ts, typename Pol::V* sh /* [2][NCH][NT/32] */) {
    typedef typename Pol::V V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = ts < 32 ? ts : 32;
    const int lw = lane & (w - 1);
    V fi[NCH], bi[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) { fi[c] = fe[c]; bi[c] = be[c]; }
    // inclusive scans within sub-warps of width w
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (o >= w) break;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            V yf = shfl_up_t(fi[c], o, w);
            V yb = shfl_down_t(bi[c], o, w);
            if (lw >= o) fi[c] = Pol::add(yf, fi[c]);
            if (lw + o < w) bi[c] = Pol::add(bi[c], yb);
        }
    }
    // exclusive versions within the sub-warp
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        V ef = shfl_up_t(fi[c], 1, w);
        V eb = shfl_down_t(bi[c], 1, w);
        fe[c] = (lw == 0) ? Pol::zero() : ef;
        be[c] = (lw == w - 1) ? Pol::zero() : eb;
    }
    if (ts <= 32) return;
    // segments spanning several warps: add the totals of earlier / later warps
    const int wps = ts >> 5;                 // warps per segment
    if (lane == 31) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) sh[(0 * NCH + c) * (NT / 32) + warp] = fi[c];
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) sh[(1 * NCH + c) * (NT / 32) + warp] = bi[c];
    }
    __syncthreads();
    const int seg0 = warp & ~(wps - 1);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        V accf = Pol::zero(), accb = Pol::zero();
        for (int q = seg0; q < warp; ++q) accf = Pol::add(accf, sh[(0 * NCH + c) * (NT / 32) + q]);
        for (int q = warp + 1; q < seg0 + wps; ++q) accb = Pol::add(accb, sh[(1 * NCH + c) * (NT / 32) + q]);
        fe[c] = Pol::add(accf, fe[c]);
        be[c] = Pol::add(be[c], accb);
    }
    __syncthreads();
}

// The merge kernel.  PH_PLAIN: merge only.  PH_TOTALS: per-CTA channel totals
// of the source weights (CTAs inside a merged block longer than a tile).
// PH_SWEEP: merge plus the Merge1D sweep contributions to the targets.
template <class Pol, int CLSB, int PHASE>
__global__ void __launch_bounds__(MT) k_merge(MergeArgs a, Pol pol, typename Pol::V* __restrict__ totals,
                                              const typename Pol::V* __restrict__ carries) {
    typedef typename Pol::V V;
    constexpr int NCH = 2 << CLSB;
    constexpr uint32_t CMASK = (1u << CLSB) - 1u;
    constexpr int MP = MTILE + MTILE / 32;   // padded tile (bank conflicts)
    __shared__ uint32_t s_key[MP];
    __shared__ uint32_t s_meta[MP];
    __shared__ int64_t s_co[6];
    __shared__ V s_scan[(PHASE == PH_PLAIN) ? 1 : 2 * NCH * (MT / 32)];

    const int64_t n = a.n;
    const int64_t R = (int64_t)1 << a.logR;
    const int64_t R2 = R << 1;
    const int64_t o0 = (int64_t)blockIdx.x * MTILE;
    if (o0 >= n) return;
    const int64_t o1 = min(o0 + (int64_t)MTILE, n);
    const int64_t ln = o1 - o0;                 // outputs of this CTA
    const bool big = R2 > MTILE;
    int64_t lc = 0;                              // big: local length of the C part
    if (big) {
        if (threadIdx.x < 64) {
            const int64_t bs = (o0 / R2) * R2;
            const int64_t cl = min(R, n - bs);
            const int64_t dl = max((int64_t)0, min(R2, n - bs) - cl);
            const int64_t q0 = o0 - bs, q1 = o1 - bs;
            const int64_t iq = merge_path_warp(a.key_in + bs, cl, a.key_in + bs + cl, dl,
                                               threadIdx.x < 32 ? q0 : q1);
            if (threadIdx.x == 0) { s_co[0] = bs + iq; s_co[2] = bs + cl + (q0 - iq); s_co[4] = iq; }
            if (threadIdx.x == 32) s_co[5] = iq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t i0 = s_co[4], i1 = s_co[5];
            const int64_t bs = (o0 / R2) * R2;
            const int64_t q0 = o0 - bs, q1 = o1 - bs;
            s_co[1] = i1 - i0;                 // C range [bs+i0, bs+i1)
            s_co[3] = (q1 - i1) - (q0 - i0);   // D range length
        }
        __syncthreads();
        lc = s_co[1];
        const int64_t cs = s_co[0], ds = s_co[2], ldd = s_co[3];
        for (int64_t i = threadIdx.x; i < lc; i += MT) { s_key[mpd(i)] = a.key_in[cs + i]; s_meta[mpd(i)] = a.meta_in[cs + i]; }
        for (int64_t i = threadIdx.x; i < ldd; i += MT) {
            s_key[mpd(lc + i)] = a.key_in[ds + i];
            s_meta[mpd(lc + i)] = a.meta_in[ds + i];
        }
    } else {
        for (int64_t i = threadIdx.x; i < ln; i += MT) { s_key[mpd(i)] = a.key_in[o0 + i]; s_meta[mpd(i)] = a.meta_in[o0 + i]; }
    }
    __syncthreads();

    if (PHASE == PH_TOTALS) {
        // channel totals of this CTA's inputs (order does not matter)
        V tf[NCH], tb[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) { tf[c] = Pol::zero(); tb[c] = Pol::zero(); }
        for (int64_t i = threadIdx.x; i < ln; i += MT) {
            const uint32_t m = s_meta[mpd(i)];
            const int half = (i >= lc) ? 1 : 0;
            const uint32_t item = m & kItemMask;
            if (pol.is_src(item)) {
                V wf, wb;
                pol.src_weights(item, half, wf, wb);
                const int ch = (half << CLSB) | (int)(m >> kItemBits);
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == ch) { tf[c] = Pol::add(tf[c], wf); tb[c] = Pol::add(tb[c], wb); }
            }
        }
        // CTA reduction through the scan helper: inclusive total = excl + own
        V fe[NCH], be[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) { fe[c] = tf[c]; be[c] = tb[c]; }
        seg_scan<Pol, NCH>(fe, be, MT, s_scan);
        if (threadIdx.x == MT - 1) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) totals[((int64_t)blockIdx.x * 2 + 0) * NCH + c] = Pol::add(fe[c], tf[c]);
        }
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) totals[((int64_t)blockIdx.x * 2 + 1) * NCH + c] = Pol::add(be[c], tb[c]);
        }
        return;
    }

    // ---------------------------------------------------------------- merge
    uint32_t ek[MI], em[MI];
    int eh[MI];
    int cnt = 0;
    {
        const int64_t p0 = (int64_t)threadIdx.x * MI;
        int64_t bsl = 0, cl = 0, dl = 0, i = 0, j = 0;
        for (int e = 0; e < MI; ++e) {
            const int64_t p = p0 + e;
            if (p >= ln) break;
            if (e == 0 || (!big && (p % R2) == 0)) {
                if (big) { bsl = 0; cl = lc; dl = ln - lc; }
                else { bsl = (p / R2) * R2; cl = min(R, ln - bsl); dl = min(R2, ln - bsl) - cl; }
                MAccP A{s_key, (int)bsl}, B{s_key, (int)(bsl + cl)};
                i = merge_path(A, cl, B, dl, p - bsl);
                j = (p - bsl) - i;
            }
            bool takeC = (i < cl) && (j >= dl || s_key[mpd(bsl + i)] <= s_key[mpd(bsl + cl + j)]);
            if (takeC) { ek[e] = s_key[mpd(bsl + i)]; em[e] = s_meta[mpd(bsl + i)]; eh[e] = 0; ++i; }
            else { ek[e] = s_key[mpd(bsl + cl + j)]; em[e] = s_meta[mpd(bsl + cl + j)]; eh[e] = 1; ++j; }
            cnt = e + 1;
        }
    }
    // write merged output (the class bits travel unchanged)
    {
        const int64_t p0 = o0 + (int64_t)threadIdx.x * MI;
        if (cnt == MI) {
            uint4* kk = reinterpret_cast<uint4*>(a.key_out + p0);
            uint4* mm = reinterpret_cast<uint4*>(a.meta_out + p0);
            kk[0] = make_uint4(ek[0], ek[1], ek[2], ek[3]);
            kk[1] = make_uint4(ek[4], ek[5], ek[6], ek[7]);
            mm[0] = make_uint4(em[0], em[1], em[2], em[3]);
            mm[1] = make_uint4(em[4], em[5], em[6], em[7]);
        } else {
            for (int e = 0; e < cnt; ++e) { a.key_out[p0 + e] = ek[e]; a.meta_out[p0 + e] = em[e]; }
        }
    }
    if (PHASE == PH_PLAIN) return;

    // ---------------------------------------------------------------- sweep
    // per-element source weights (zero for pure targets)
    V wf[MI], wb[MI];
#pragma unroll
    for (int e = 0; e < MI; ++e) {
        wf[e] = Pol::zero();
        wb[e] = Pol::zero();
        if (e < cnt) {
            const uint32_t item = em[e] & kItemMask;
            if (pol.is_src(item)) pol.src_weights(item, eh[e], wf[e], wb[e]);
        }
    }
    const int ts = big ? MT : (int)(R2 / MI);   // threads per merged block (0/1: thread-local)
    V fe[NCH], be[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) { fe[c] = Pol::zero(); be[c] = Pol::zero(); }
    if (ts > 1) {
        // thread totals -> exclusive segmented scans
#pragma unroll
        for (int e = 0; e < MI; ++e) {
            if (e < cnt) {
                const int ch = (eh[e] << CLSB) | (int)(em[e] >> kItemBits);
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == ch) { fe[c] = Pol::add(fe[c], wf[e]); be[c] = Pol::add(be[c], wb[e]); }
            }
        }
        seg_scan<Pol, NCH>(fe, be, ts, s_scan);
        if (big && carries) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                fe[c] = Pol::add(carries[((int64_t)blockIdx.x * 2 + 0) * NCH + c], fe[c]);
                be[c] = Pol::add(be[c], carries[((int64_t)blockIdx.x * 2 + 1) * NCH + c]);
            }
        }
    }
    // forward walk: value before each element of the complementary channel
    V fwd[MI];
    {
        V run[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) run[c] = fe[c];
        const int64_t p0 = (int64_t)threadIdx.x * MI;
#pragma unroll
        for (int e = 0; e < MI; ++e) {
            fwd[e] = Pol::zero();
            if (e < cnt) {
                if (ts <= 1 && e > 0 && ((p0 + e) % R2) == 0) {
#pragma unroll
                    for (int c = 0; c < NCH; ++c) run[c] = Pol::zero();
                }
                const int cls = (int)(em[e] >> kItemBits);
                const int own = (eh[e] << CLSB) | cls;
                const int opp = ((1 - eh[e]) << CLSB) | (int)(~(uint32_t)cls & CMASK);
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == opp) fwd[e] = run[c];
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == own) run[c] = Pol::add(run[c], wf[e]);
            }
        }
    }
    // backward walk and target update
    {
        V run[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) run[c] = be[c];
        const int64_t p0 = (int64_t)threadIdx.x * MI;
#pragma unroll
        for (int e = MI - 1; e >= 0; --e) {
            if (e < cnt) {
                if (ts <= 1 && e < cnt - 1 && ((p0 + e + 1) % R2) == 0) {
#pragma unroll
                    for (int c = 0; c < NCH; ++c) run[c] = Pol::zero();
                }
                const int cls = (int)(em[e] >> kItemBits);
                const int own = (eh[e] << CLSB) | cls;
                const int opp = ((1 - eh[e]) << CLSB) | (int)(~(uint32_t)cls & CMASK);
                V bwd = Pol::zero();
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == opp) bwd = run[c];
                const uint32_t item = em[e] & kItemMask;
                if (pol.is_tgt(item)) {
                    // position bits: bit 0 = half on axis 1, bit j = class bit of axis j+1
                    const uint32_t pb = (uint32_t)eh[e] | ((uint32_t)cls << 1);
                    pol.target(item, pb, fwd[e], bwd);
                }
#pragma unroll
                for (int c = 0; c < NCH; ++c)
                    if (c == own) run[c] = Pol::add(run[c], wb[e]);
            }
        }
    }
}


// ------------------------------------------------------------------ tile-local levels
// All merge levels whose merged runs fit in one tile of LT items run in shared
// memory in one launch.  The tile is gathered straight from the enclosing
// state (items sorted by P_1 inside their nodes): key = P_0[item], class bits,
// and the policy's per-item weights.  Targets accumulate their sums in shared
// memory, indexed by the item's slot in the tile and by (half, direction):
// inside one innermost sort the side bits of the enclosing axes are fixed, so
// those four sums are all a target receives; they are flushed to the global
// accumulators once (Pol::flush) after the last local level.
__device__ __forceinline__ int lpd(int p) { return p + (p >> 5); }
struct LAccP {
    const uint32_t* p;
    int base;
    __device__ uint32_t operator()(int64_t i) const { return p[lpd(base + (int)i)]; }
};

template <class Pol>
struct LocalCfg {
    static constexpr int T = Pol::kLocalT;     // items per tile
    static constexpr int NT = 512;             // threads
    static constexpr int IT = T / NT;          // items per thread
};

template <class Pol, int CLSB>
__global__ void __launch_bounds__(512) k_local_sweep(const uint32_t* __restrict__ seq, int64_t n,
                                                     const uint32_t* __restrict__ P0, ClassSpecK cs, int levels,
                                                     Pol pol, uint32_t* __restrict__ key_out,
                                                     uint32_t* __restrict__ meta_out, int write_out) {
    typedef typename Pol::V V;
    typedef typename Pol::LW LW;
    constexpr int T = LocalCfg<Pol>::T, NT = LocalCfg<Pol>::NT, IT = LocalCfg<Pol>::IT;
    constexpr int NCH = 2 << CLSB;
    constexpr uint32_t CMASK = (1u << CLSB) - 1u;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TP = T + T / 32;                                      // padded row (bank conflicts)
    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem_raw);             // [2][TP]
    uint32_t* s_meta = s_key + 2 * TP;                                  // [2][TP]
    uint16_t* s_home = reinterpret_cast<uint16_t*>(s_meta + 2 * TP);    // [2][TP]
    V* s_acc = reinterpret_cast<V*>(s_home + 2 * TP + (TP & 1) * 2);    // [T][4]
    LW* s_w = reinterpret_cast<LW*>(s_acc + 4 * T);                     // [T][4]
    V* s_scan = reinterpret_cast<V*>(s_w + (Pol::kUnitWeights ? 0 : 4 * T));   // [2][NCH][NT/32]

    const int64_t t0 = (int64_t)blockIdx.x * T;
    const int ln = (int)min((int64_t)T, n - t0);
    for (int i = threadIdx.x; i < T; i += NT) {
        if (i < ln) {
            const uint32_t item = seq[t0 + i];
            const uint32_t c = class_of_k(cs, item);
            s_key[lpd(i)] = P0[item];
            s_meta[lpd(i)] = item | (c << kItemBits);
            s_home[lpd(i)] = (uint16_t)i;
            pol.prep_item(item, c);
            if constexpr (!Pol::kUnitWeights) {
                if (pol.is_src(item)) pol.local_weights(item, c, &s_w[4 * i]);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) s_acc[4 * i + j] = Pol::zero();
    }
    __syncthreads();
    int buf = 0;
    for (int m = 0; m < levels; ++m) {
        const int R = 1 << m, R2 = 2 << m;
        const uint32_t* ik = s_key + buf * TP;
        const uint32_t* im = s_meta + buf * TP;
        const uint16_t* ih = s_home + buf * TP;
        uint32_t em[IT];
        uint16_t eh2[IT];
        uint32_t ek[IT];
        int eh[IT];
        int cnt = 0;
        {
            const int p0 = threadIdx.x * IT;
            int bsl = 0, cl = 0, dl = 0, i = 0, j = 0;
#pragma unroll
            for (int e = 0; e < IT; ++e) {
                const int p = p0 + e;
                if (p < ln) {
                    if (e == 0 || (p % R2) == 0) {
                        bsl = (p / R2) * R2;
                        cl = min(R, ln - bsl);
                        dl = min(R2, ln - bsl) - cl;
                        LAccP A{ik, bsl}, B{ik, bsl + cl};
                        i = (int)merge_path(A, cl, B, dl, p - bsl);
                        j = (p - bsl) - i;
                    }
                    const bool takeC = (i < cl) && (j >= dl || ik[lpd(bsl + i)] <= ik[lpd(bsl + cl + j)]);
                    const int src = takeC ? lpd(bsl + i) : lpd(bsl + cl + j);
                    ek[e] = ik[src];
                    em[e] = im[src];
                    eh2[e] = ih[src];
                    eh[e] = takeC ? 0 : 1;
                    if (takeC) ++i; else ++j;
                    cnt = e + 1;
                }
            }
        }
        // sweep over the merged blocks of length R2
        V wf[IT], wb[IT];
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            wf[e] = Pol::zero();
            wb[e] = Pol::zero();
            if (e < cnt) {
                const uint32_t item = em[e] & kItemMask;
                if (pol.is_src(item)) {
                    if constexpr (Pol::kUnitWeights) { wf[e] = Pol::one(); wb[e] = Pol::one(); }
                    else {
                        wf[e] = Pol::from_lw(s_w[4 * eh2[e] + eh[e] * 2 + 0]);
                        wb[e] = Pol::from_lw(s_w[4 * eh2[e] + eh[e] * 2 + 1]);
                    }
                }
            }
        }
        const int ts = R2 / IT;   // threads per merged block (0 or 1: thread-local)
        V fe[NCH], be[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) { fe[c] = Pol::zero(); be[c] = Pol::zero(); }
        if (ts > 1) {
#pragma unroll
            for (int e = 0; e < IT; ++e) {
                if (e < cnt) {
                    const int ch = (eh[e] << CLSB) | (int)(em[e] >> kItemBits);
#pragma unroll
                    for (int c = 0; c < NCH; ++c)
                        if (c == ch) { fe[c] = Pol::add(fe[c], wf[e]); be[c] = Pol::add(be[c], wb[e]); }
                }
            }
            seg_scan<Pol, NCH, NT>(fe, be, ts, s_scan);
        }
        V fwd[IT];
        {
            V run[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) run[c] = fe[c];
            const int p0 = threadIdx.x * IT;
#pragma unroll
            for (int e = 0; e < IT; ++e) {
                fwd[e] = Pol::zero();
                if (e < cnt) {
                    if (ts <= 1 && e > 0 && ((p0 + e) % R2) == 0) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) run[c] = Pol::zero();
                    }
                    const int cls = (int)(em[e] >> kItemBits);
                    const int own = (eh[e] << CLSB) | cls;
                    const int opp = ((1 - eh[e]) << CLSB) | (int)(~(uint32_t)cls & CMASK);
#pragma unroll
                    for (int c = 0; c < NCH; ++c)
                        if (c == opp) fwd[e] = run[c];
#pragma unroll
                    for (int c = 0; c < NCH; ++c)
                        if (c == own) run[c] = Pol::add(run[c], wf[e]);
                }
            }
        }
        {
            V run[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) run[c] = be[c];
            const int p0 = threadIdx.x * IT;
#pragma unroll
            for (int e = IT - 1; e >= 0; --e) {
                if (e < cnt) {
                    if (ts <= 1 && e < cnt - 1 && ((p0 + e + 1) % R2) == 0) {
#pragma unroll
                        for (int c = 0; c < NCH; ++c) run[c] = Pol::zero();
                    }
                    const int cls = (int)(em[e] >> kItemBits);
                    const int own = (eh[e] << CLSB) | cls;
                    const int opp = ((1 - eh[e]) << CLSB) | (int)(~(uint32_t)cls & CMASK);
                    V bwd = Pol::zero();
#pragma unroll
                    for (int c = 0; c < NCH; ++c)
                        if (c == opp) bwd = run[c];
                    const uint32_t item = em[e] & kItemMask;
                    if (pol.is_tgt(item)) {
                        V* a = s_acc + 4 * eh2[e] + 2 * eh[e];
                        a[0] = Pol::add(a[0], fwd[e]);
                        a[1] = Pol::add(a[1], bwd);
                    }
#pragma unroll
                    for (int c = 0; c < NCH; ++c)
                        if (c == own) run[c] = Pol::add(run[c], wb[e]);
                }
            }
        }
        // write the merged level into the other buffer
        uint32_t* ok = s_key + (buf ^ 1) * TP;
        uint32_t* om = s_meta + (buf ^ 1) * TP;
        uint16_t* oh = s_home + (buf ^ 1) * TP;
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            if (e < cnt) {
                const int p = lpd(threadIdx.x * IT + e);
                ok[p] = ek[e];
                om[p] = em[e];
                oh[p] = eh2[e];
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    // flush the per-target sums and write the tile out for the global levels
    for (int i = threadIdx.x; i < ln; i += NT) {
        const uint32_t m = s_meta[buf * TP + lpd(i)];
        const uint32_t item = m & kItemMask;
        if (write_out) {
            key_out[t0 + i] = s_key[buf * TP + lpd(i)];
            meta_out[t0 + i] = m;
        }
        if (pol.is_tgt(item)) {
            const int h = s_home[buf * TP + lpd(i)];
            pol.flush(item, m >> kItemBits, s_acc + 4 * h);
        }
    }
}

template <class Pol, int CLSB>
constexpr size_t local_smem_bytes() {
    constexpr int T = LocalCfg<Pol>::T, NT = LocalCfg<Pol>::NT;
    constexpr int NCH = 2 << CLSB;
    constexpr int TP = T + T / 32;
    return (size_t)TP * (2 * 4 + 2 * 4 + 2 * 2) + 16 + (size_t)T * 4 * sizeof(typename Pol::V) +
           (Pol::kUnitWeights ? 0 : (size_t)T * 4 * sizeof(typename Pol::LW)) +
           (size_t)2 * NCH * (NT / 32) * sizeof(typename Pol::V) + 64;
}

// Carries for merged blocks that span several CTAs: exclusive prefix of the
// forward totals and exclusive suffix of the backward totals over the CTAs of
// each merged block.  One thread per (block, channel, direction).
template <class Pol, int NCH>
__global__ void k_carries(const typename Pol::V* __restrict__ totals, typename Pol::V* __restrict__ carries,
                          int64_t n, int logR) {
    typedef typename Pol::V V;
    const int64_t R2 = (int64_t)2 << logR;
    const int64_t ctas = (n + MTILE - 1) / MTILE;
    const int64_t per = R2 / MTILE;            // CTAs per full merged block
    const int64_t nblocks = (ctas + per - 1) / per;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nblocks * NCH * 2) return;
    const int dir = (int)(t % 2);
    const int c = (int)((t / 2) % NCH);
    const int64_t b = t / (2 * NCH);
    const int64_t c0 = b * per, c1 = min(c0 + per, ctas);
    V run = Pol::zero();
    if (dir == 0) {
        for (int64_t q = c0; q < c1; ++q) {
            carries[(q * 2 + 0) * NCH + c] = run;
            run = Pol::add(run, totals[(q * 2 + 0) * NCH + c]);
        }
    } else {
        for (int64_t q = c1 - 1; q >= c0; --q) {
            carries[(q * 2 + 1) * NCH + c] = run;
            run = Pol::add(run, totals[(q * 2 + 1) * NCH + c]);
        }
    }
}

}  // namespace dc
}  // namespace fk
