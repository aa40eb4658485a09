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

#include <climits>
#include <type_traits>

#include "fk_internal.cuh"

namespace fk {
namespace dc {

constexpr int MT = 256;            // threads per CTA of a merge level
// Outputs per thread of a merge level (its tile: MT x that many items).  The
// folded kernel sums on records with at most 96 bytes of running sums per
// thread take four: their merge kernels are then held to two or three CTAs
// per SM (FoldOcc) and hide more latency.  Everything else takes eight: the
// wider sums need so many registers that the CTAs per SM do not change, and
// the plain, counting and weighted merges (no occupancy bound) gain nothing
// from smaller tiles but twice the co-rank searches per item.
template <class Pol, int CLSB>
struct MergeItems {
    static constexpr int value = (Pol::kRecords && sizeof(typename Pol::V) * (2 << CLSB) <= 96) ? 4 : 8;
};
constexpr int kMergeTileMin = MT * 4;   // the smallest merge tile (buffer sizing)
constexpr int kItemBits = 26;      // meta = item | cls << 26
constexpr uint32_t kItemMask = (1u << kItemBits) - 1u;

struct MergeArgs {
    const uint32_t* key_in;
    const uint32_t* meta_in;
    uint32_t* key_out;
    uint32_t* meta_out;
    int64_t n;
    int logR;     // input runs of length R = 2^logR, output runs 2R
    // Optional [2 x CTAs] merge-path co-ranks of each CTA's first and last
    // output in runs longer than a tile: the totals pass of a level finds and
    // writes them (co_read == 0), the sweep pass of the same level reads them.
    int64_t* co = nullptr;
    int co_read = 0;
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

// Word-wise select between two accumulator values (no branches).
template <class T>
__device__ __forceinline__ T sel_t(bool p, const T& a, const T& b) {
    T r;
    const uint32_t* x = reinterpret_cast<const uint32_t*>(&a);
    const uint32_t* y = reinterpret_cast<const uint32_t*>(&b);
    uint32_t* q = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) q[i] = p ? x[i] : y[i];
    return r;
}
// Channel c of a register array (selects instead of dynamic indexing).
// A multiplexer tree on the bits of c (N a power of two).
template <class T, int N>
__device__ __forceinline__ T pick(const T (&a)[N], int c) {
    static_assert((N & (N - 1)) == 0, "channel count must be a power of two");
    if constexpr (N == 1) {
        return a[0];
    } else {
        T h[N / 2];
        const bool b = (c & 1) != 0;
#pragma unroll
        for (int k = 0; k < N / 2; ++k) h[k] = sel_t(b, a[2 * k + 1], a[2 * k]);
        return pick(h, c >> 1);
    }
}
// a[c] += w with one addition whatever c is.
template <class Pol, int N>
__device__ __forceinline__ void add_at(typename Pol::V (&a)[N], int c, const typename Pol::V& w) {
    const typename Pol::V s = Pol::add(pick(a, c), w);
#pragma unroll
    for (int k = 0; k < N; ++k) a[k] = sel_t(c == k, s, a[k]);
}

// Asynchronous 8-byte global -> shared copies (cp.async): a thread waits only
// for its own copies, so no barrier is needed when it reads back only what it
// copied.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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
#pragma unroll
    for (int j = 0; j < 6; ++j)      // static indices keep cs out of local memory
        if (j < cs.nb) c |= ((cs.idx[j][item] >> cs.lvl[j]) & 1u) << j;
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
    // segments spanning several warps: exclusive scans of the warp totals
    // inside each segment, one (direction, channel) row per warp
    constexpr int NW = NT / 32;
    const int wps = ts >> 5;                 // warps per segment
    if (lane == 31) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) sh[(0 * NCH + c) * NW + warp] = fi[c];
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) sh[(1 * NCH + c) * NW + warp] = bi[c];
    }
    __syncthreads();
    for (int row = warp; row < 2 * NCH; row += NW) {
        const bool fw = row < NCH;
        V v = (lane < NW) ? sh[row * NW + lane] : Pol::zero();
        const int lq = lane & (wps - 1);
        for (int o = 1; o < wps; o <<= 1) {
            if (fw) {
                const V y = shfl_up_t(v, o, wps);
                if (lq >= o) v = Pol::add(y, v);
            } else {
                const V y = shfl_down_t(v, o, wps);
                if (lq + o < wps) v = Pol::add(v, y);
            }
        }
        V x = fw ? shfl_up_t(v, 1, wps) : shfl_down_t(v, 1, wps);
        if (fw ? (lq == 0) : (lq == wps - 1)) x = Pol::zero();
        if (lane < NW) sh[row * NW + lane] = x;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        fe[c] = Pol::add(sh[(0 * NCH + c) * NW + warp], fe[c]);
        be[c] = Pol::add(be[c], sh[(1 * NCH + c) * NW + warp]);
    }
    __syncthreads();
}

// Merge of a loaded tile (padded rows): every thread takes MI consecutive
// outputs from p0.  big: the tile is one merged block, C = [0, lc), D =
// [lc, ln); otherwise it holds whole merged blocks of R2 (> 1) items.  The
// keys at the heads of C and D stay in registers, so an output reads only
// its meta and the key of the head it advances.  eh: 0 from C, 1 from D; sl:
// the output's slot in the tile.  Returns the outputs made.
template <int MI>
__device__ __forceinline__ int tile_merge(const uint32_t* s_key, const uint32_t* s_meta, int ln, int lc, bool big,
                                          int64_t R2l, int p0, uint32_t (&ek)[MI], uint32_t (&em)[MI], int (&eh)[MI],
                                          int (&sl)[MI]) {
    const int R2 = big ? 1 : (int)R2l;      // runs of a tile-sized merge fit an int
    int bsl = 0, cl = 0, dl = 0, i = 0, j = 0, cnt = 0;
    uint32_t kc = 0, kd = 0;
#pragma unroll
    for (int e = 0; e < MI; ++e) {
        const int p = p0 + e;
        if (p < ln) {
            if (e == 0 || (!big && (p % R2) == 0)) {
                if (big) { bsl = 0; cl = lc; dl = ln - lc; }
                else { bsl = (p / R2) * R2; cl = min(R2 / 2, ln - bsl); dl = min(R2, ln - bsl) - cl; }
                MAccP A{s_key, bsl}, B{s_key, bsl + cl};
                i = (int)merge_path(A, cl, B, dl, p - bsl);
                j = (p - bsl) - i;
                kc = (i < cl) ? s_key[mpd(bsl + i)] : 0u;
                kd = (j < dl) ? s_key[mpd(bsl + cl + j)] : 0u;
            }
            const bool takeC = (i < cl) && (j >= dl || kc <= kd);
            const int slot = takeC ? bsl + i : bsl + cl + j;
            ek[e] = takeC ? kc : kd;
            em[e] = s_meta[mpd(slot)];
            eh[e] = takeC ? 0 : 1;
            sl[e] = slot;
            i += takeC ? 1 : 0;
            j += takeC ? 0 : 1;
            const bool v = takeC ? (i < cl) : (j < dl);
            const uint32_t nk = v ? s_key[mpd(takeC ? bsl + i : bsl + cl + j)] : 0u;
            kc = takeC ? nk : kc;
            kd = takeC ? kd : nk;
            cnt = e + 1;
        }
    }
    return cnt;
}

// The inputs of one CTA of a merge level in shared memory (padded rows).
// Runs of 2R longer than a tile (big): the CTA's co-ranks are found by a
// warp-cooperative merge-path search and its C part [cs, cs+lc) and D part
// [ds, ds+ldd) are loaded one after the other; otherwise the tile
// [o0, o0+ln) holds whole runs.
struct MergeTile {
    int64_t ln, lc, cs, ds, ldd;
    bool big;
};
template <int MI, bool KEYS = true>   // KEYS: also stage the keys (a totals pass reads only metas)
__device__ __forceinline__ MergeTile merge_tile_load(const MergeArgs& a, uint32_t* s_key, uint32_t* s_meta,
                                                     int64_t* s_co) {
    constexpr int MTILE = MT * MI;
    const int64_t n = a.n;
    const int64_t R = (int64_t)1 << a.logR;
    const int64_t R2 = R << 1;
    const int64_t o0 = (int64_t)blockIdx.x * MTILE;
    const int64_t o1 = min(o0 + (int64_t)MTILE, n);
    MergeTile t;
    t.ln = o1 - o0;
    t.big = R2 > MTILE;
    t.lc = t.cs = t.ds = t.ldd = 0;
    if (t.big) {
        if (a.co && a.co_read) {
            if (threadIdx.x == 0) {
                const int64_t bs = (o0 / R2) * R2;
                const int64_t cl = min(R, n - bs);
                const int64_t q0 = o0 - bs;
                const int64_t iq0 = a.co[2 * (int64_t)blockIdx.x], iq1 = a.co[2 * (int64_t)blockIdx.x + 1];
                s_co[0] = bs + iq0; s_co[2] = bs + cl + (q0 - iq0); s_co[4] = iq0; s_co[5] = iq1;
            }
        } else if (threadIdx.x < 64) {
            const int64_t bs = (o0 / R2) * R2;
            const int64_t cl = min(R, n - bs);
            const int64_t dl = max((int64_t)0, min(R2, n - bs) - cl);
            const int64_t q0 = o0 - bs, q1 = o1 - bs;
            const int64_t iq = merge_path_warp(a.key_in + bs, cl, a.key_in + bs + cl, dl,
                                               threadIdx.x < 32 ? q0 : q1);
            if (threadIdx.x == 0) {
                s_co[0] = bs + iq; s_co[2] = bs + cl + (q0 - iq); s_co[4] = iq;
                if (a.co) a.co[2 * (int64_t)blockIdx.x] = iq;
            }
            if (threadIdx.x == 32) {
                s_co[5] = iq;
                if (a.co) a.co[2 * (int64_t)blockIdx.x + 1] = iq;
            }
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
        t.lc = s_co[1];
        t.cs = s_co[0];
        t.ds = s_co[2];
        t.ldd = s_co[3];
    }
    // Tile slot i holds C element i (i < lc) or D element i - lc; a tile of
    // whole runs is the contiguous range from o0.  Asynchronous copies: every
    // thread has all its slots in flight at once, so the tile arrives in one
    // memory round trip without staging through registers.
#pragma unroll
    for (int j = 0; j < MI; ++j) {
        const int i = (int)threadIdx.x + j * MT;
        const int64_t g = !t.big ? o0 + i : (i < t.lc ? t.cs + i : t.ds + (i - t.lc));
        if (i < t.ln) {
            if constexpr (KEYS) cp_async4(&s_key[mpd(i)], &a.key_in[g]);
            cp_async4(&s_meta[mpd(i)], &a.meta_in[g]);
        }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    return t;
}

// The merge kernel.  PH_PLAIN: merge only.  PH_TOTALS: per-CTA channel totals
// of the source weights (CTAs inside a merged block longer than a tile).
// PH_SWEEP: merge plus the Merge1D sweep contributions to the targets.
template <class Pol, int CLSB, int PHASE>
__global__ void __launch_bounds__(MT) k_merge(MergeArgs a, Pol pol, typename Pol::V* __restrict__ totals,
                                              const typename Pol::V* __restrict__ carries) {
    typedef typename Pol::V V;
    constexpr int MI = MergeItems<Pol, CLSB>::value, MTILE = MT * MI;
    constexpr int NCH = 2 << CLSB;
    constexpr uint32_t CMASK = (1u << CLSB) - 1u;
    constexpr int MP = MTILE + MTILE / 32;   // padded tile (bank conflicts)
    __shared__ uint32_t s_key[MP];
    __shared__ uint32_t s_meta[MP];
    __shared__ int64_t s_co[6];
    __shared__ V s_scan[(PHASE == PH_PLAIN) ? 1 : 2 * NCH * (MT / 32)];

    const int64_t n = a.n;
    const int64_t R2 = (int64_t)2 << a.logR;
    const int64_t o0 = (int64_t)blockIdx.x * MTILE;
    if (o0 >= n) return;
    const MergeTile mt = merge_tile_load<MI, PHASE != PH_TOTALS>(a, s_key, s_meta, s_co);
    const int64_t ln = mt.ln, lc = mt.lc;
    const bool big = mt.big;
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
                add_at<Pol>(tf, ch, wf);
                add_at<Pol>(tb, ch, wb);
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
        int sl[MI];
        cnt = tile_merge(s_key, s_meta, (int)ln, (int)lc, big, R2, threadIdx.x * MI, ek, em, eh, sl);
    }
    // write merged output (the class bits travel unchanged)
    {
        const int64_t p0 = o0 + (int64_t)threadIdx.x * MI;
        if (cnt == MI) {
            uint4* kk = reinterpret_cast<uint4*>(a.key_out + p0);
            uint4* mm = reinterpret_cast<uint4*>(a.meta_out + p0);
#pragma unroll
            for (int v = 0; v < MI / 4; ++v) {
                kk[v] = make_uint4(ek[4 * v], ek[4 * v + 1], ek[4 * v + 2], ek[4 * v + 3]);
                mm[v] = make_uint4(em[4 * v], em[4 * v + 1], em[4 * v + 2], em[4 * v + 3]);
            }
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
                add_at<Pol>(fe, ch, wf[e]);
                add_at<Pol>(be, ch, wb[e]);
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
                fwd[e] = pick(run, opp);
                add_at<Pol>(run, own, wf[e]);
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
                const V bwd = pick(run, opp);
                const uint32_t item = em[e] & kItemMask;
                if (pol.is_tgt(item)) {
                    // position bits: bit 0 = half on axis 1, bit j = class bit of axis j+1
                    const uint32_t pb = (uint32_t)eh[e] | ((uint32_t)cls << 1);
                    pol.target(item, pb, fwd[e], bwd);
                }
                add_at<Pol>(run, own, wb[e]);
            }
        }
    }
}


// ------------------------------------------------------------------ folded records
// Records of the folded kernel sums for the merge levels longer than a tile
// (structure of arrays, ping-pong): the four factor products F(h, dir)
// (mantissa, shift; index 2h + dir), the source weight (0: no source role)
// and the target's sum so far travel with every element, so a level streams
// its payload instead of gathering it per item, and a target's sum is
// flushed once, after the last level.
template <class Pol>
struct FoldRecs {
    typename Pol::M* fm;    // [n][4]
    int* fs;                // [n][4]
    typename Pol::M* wt;    // [n]
    typename Pol::FA* fa;   // [n][NW]
};

// ------------------------------------------------------------------ tile-local levels
// All merge levels whose merged runs fit in one tile of T items run in shared
// memory in one launch.  The tile is gathered straight from the enclosing
// state (items sorted by P_1 inside their nodes): key = P_0[item], class bits,
// and the policy's per-item weights.  Inside one innermost sort the side bits
// of the enclosing axes are fixed, so what a target receives depends only on
// its half on axis 1 and the direction on axis 0 at each level:
//
//  * plain form: four sums per target, indexed by (half, direction), flushed
//    to the global accumulators once (Pol::flush) after the last level, which
//    keeps the orthants apart (orthant sums, per-orthant kernel terms);
//  * folded form (kernel sums without per-orthant terms): a source in half h
//    carries w F(h, dir), F(h, dir) = B E1^{h} E0^{dir} (the factor products
//    of eq. Laplacian decomposition nD, mantissa and power-of-two shift), and
//    a target in half h turns its forward and backward sums into kernel values
//    with F(h, -) and F(h, +): the same per-item products read with the other
//    direction.  The values are bounded by the sum of the weights, so one
//    compensated accumulator per target and weight channel holds them.
//
// The key, meta and home (slot of the item's per-item data) arrays are
// single-buffered: each level merges into registers, then writes back.
__device__ __forceinline__ int lpd(int p) { return p + (p >> 5); }
struct LAccP {
    const uint32_t* p;
    int base;
    __device__ uint32_t operator()(int64_t i) const { return p[lpd(base + (int)i)]; }
};

// HALF: the tile-size option of the batched autotuner (half the default tile).
template <class Pol, int CLSB, bool FOLD, bool HALF = false>
struct LocalCfg {
    // items per tile (the folded form halves it at d = 4 to keep its
    // per-thread state in registers)
    static constexpr int T = (FOLD ? (CLSB >= 2 ? Pol::kFoldT / 2 : Pol::kFoldT) : Pol::kLocalT) / (HALF ? 2 : 1);
    // threads: 512, or 256 when the per-thread channel sums alone would take
    // more than 32 registers (so that they stay in registers)
    static constexpr int NT = sizeof(typename Pol::V) * (2 << CLSB) > 128 ? 256 : 512;
    static constexpr int IT = T / NT;                              // items per thread
    static constexpr int TP = T + T / 32;                          // padded rows (bank conflicts)
    // resident CTAs per SM asked of the compiler: two for the half tile of the
    // one-channel mixed path (its shared memory allows two; registers decide)
    static constexpr int kMinBlocks = (FOLD && HALF && CLSB <= 1 && Pol::kNW == 1 && sizeof(typename Pol::M) == 4) ? 2 : 1;
    typedef typename Pol::V V;
    typedef typename Pol::LW LW;
    typedef typename Pol::M M;
    typedef typename Pol::FA FA;
    // shared memory layout (byte offsets)
    static constexpr size_t o_key = 0;
    static constexpr size_t o_meta = o_key + 4 * (size_t)TP;
    static constexpr size_t o_home = o_meta + 4 * (size_t)TP;
    static constexpr size_t o_data = (o_home + 2 * (size_t)TP + 15) / 16 * 16;
    // plain form: sums [T][4] and weights [T][4]
    static constexpr size_t o_acc = o_data;
    static constexpr size_t o_w = o_acc + (FOLD ? 0 : (size_t)T * 4 * sizeof(V));
    // folded form: factors [T][4] (mantissa, shift), weights [T], sums [T][NW]
    static constexpr size_t o_fm = o_data;
    static constexpr size_t o_fs = o_fm + (FOLD ? (size_t)T * 4 * sizeof(M) : 0);
    static constexpr size_t o_wt = o_fs + (FOLD ? (size_t)T * 4 * 4 : 0);
    static constexpr size_t o_fa = o_wt + (FOLD ? ((size_t)T * sizeof(M) + 15) / 16 * 16 : 0);
    static constexpr size_t o_end_data =
        FOLD ? o_fa + (size_t)T * Pol::kNW * sizeof(FA)
             : o_w + (Pol::kUnitWeights ? 0 : (size_t)T * 4 * sizeof(LW));
    static constexpr size_t o_scan = (o_end_data + 15) / 16 * 16;
    static constexpr size_t bytes = o_scan + (size_t)2 * (2 << CLSB) * (NT / 32) * sizeof(V);
};

// One tile-local merge level: each thread takes IT consecutive outputs of
// the merge of the runs of length R (read from the single-buffered arrays);
// eh packs the item's home slot (low 16 bits) and its half (bit 16).
// Returns the number of outputs taken.
template <int IT>
__device__ __forceinline__ int local_merge(const uint32_t* s_key, const uint32_t* s_meta, const uint16_t* s_home,
                                           int ln, int R, uint32_t (&ek)[IT], uint32_t (&em)[IT],
                                           uint32_t (&eh)[IT]) {
    const int R2 = 2 * R;
    const int p0 = threadIdx.x * IT;
    int bsl = 0, cl = 0, dl = 0, i = 0, j = 0, cnt = 0;
    uint32_t kc = 0, kd = 0;     // keys at the heads of C and D (kept in registers)
#pragma unroll
    for (int e = 0; e < IT; ++e) {
        const int p = p0 + e;
        if (p < ln) {
            if (e == 0 || (p % R2) == 0) {
                bsl = (p / R2) * R2;
                cl = min(R, ln - bsl);
                dl = min(R2, ln - bsl) - cl;
                LAccP A{s_key, bsl}, B{s_key, bsl + cl};
                i = (int)merge_path(A, cl, B, dl, p - bsl);
                j = (p - bsl) - i;
                kc = (i < cl) ? s_key[lpd(bsl + i)] : 0u;
                kd = (j < dl) ? s_key[lpd(bsl + cl + j)] : 0u;
            }
            const bool takeC = (i < cl) && (j >= dl || kc <= kd);
            const int src = takeC ? lpd(bsl + i) : lpd(bsl + cl + j);
            ek[e] = takeC ? kc : kd;
            em[e] = s_meta[src];
            eh[e] = (uint32_t)s_home[src] | (takeC ? 0u : 0x10000u);
            i += takeC ? 1 : 0;
            j += takeC ? 0 : 1;
            const bool v = takeC ? (i < cl) : (j < dl);
            const uint32_t nk = v ? s_key[takeC ? lpd(bsl + i) : lpd(bsl + cl + j)] : 0u;
            kc = takeC ? nk : kc;
            kd = takeC ? kd : nk;
            cnt = e + 1;
        }
    }
    return cnt;
}

// Writes a merged level back into the single-buffered arrays.
template <int IT>
__device__ __forceinline__ void local_store(uint32_t* s_key, uint32_t* s_meta, uint16_t* s_home, int cnt,
                                            const uint32_t (&ek)[IT], const uint32_t (&em)[IT],
                                            const uint32_t (&eh)[IT]) {
    __syncthreads();   // every read of this level is done
#pragma unroll
    for (int e = 0; e < IT; ++e) {
        if (e < cnt) {
            const int p = lpd(threadIdx.x * IT + e);
            s_key[p] = ek[e];
            s_meta[p] = em[e];
            s_home[p] = (uint16_t)(eh[e] & 0xffffu);
        }
    }
    __syncthreads();
}

// Plain form: four sums per target, flushed with the target factors.
template <class Pol, int CLSB>
__global__ void __launch_bounds__(LocalCfg<Pol, CLSB, false>::NT)
    k_local_sweep(const uint32_t* __restrict__ seq, int64_t n, const uint32_t* __restrict__ P0, ClassSpecK cs,
                  int levels, Pol pol, uint32_t* __restrict__ key_out, uint32_t* __restrict__ meta_out,
                  int write_out) {
    typedef LocalCfg<Pol, CLSB, false> Cfg;
    typedef typename Pol::V V;
    typedef typename Pol::LW LW;
    constexpr int T = Cfg::T, NT = Cfg::NT, IT = Cfg::IT;
    constexpr int NCH = 2 << CLSB;
    constexpr uint32_t CMASK = (1u << CLSB) - 1u;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_key);
    uint32_t* s_meta = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_meta);
    uint16_t* s_home = reinterpret_cast<uint16_t*>(smem_raw + Cfg::o_home);
    V* s_acc = reinterpret_cast<V*>(smem_raw + Cfg::o_acc);
    LW* s_w = reinterpret_cast<LW*>(smem_raw + Cfg::o_w);
    V* s_scan = reinterpret_cast<V*>(smem_raw + Cfg::o_scan);

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
    for (int m = 0; m < levels; ++m) {
        const int R2 = 2 << m;
        uint32_t ek[IT], em[IT], eh[IT];
        const int cnt = local_merge<IT>(s_key, s_meta, s_home, ln, 1 << m, ek, em, eh);
        V wf[IT], wb[IT];
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            wf[e] = Pol::zero();
            wb[e] = Pol::zero();
            if (e < cnt && pol.is_src(em[e] & kItemMask)) {
                if constexpr (Pol::kUnitWeights) { wf[e] = Pol::one(); wb[e] = Pol::one(); }
                else {
                    const LW* l = s_w + 4 * (eh[e] & 0xffffu) + 2 * (eh[e] >> 16);
                    wf[e] = Pol::from_lw(l[0]);
                    wb[e] = Pol::from_lw(l[1]);
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
                    const int ch = (int)((eh[e] >> 16) << CLSB) | (int)(em[e] >> kItemBits);
                    add_at<Pol>(fe, ch, wf[e]);
                    add_at<Pol>(be, ch, wb[e]);
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
                    const int half = (int)(eh[e] >> 16), cls = (int)(em[e] >> kItemBits);
                    const int own = (half << CLSB) | cls;
                    const int opp = ((1 - half) << CLSB) | (int)(~(uint32_t)cls & CMASK);
                    fwd[e] = pick(run, opp);
                    add_at<Pol>(run, own, wf[e]);
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
                    const int half = (int)(eh[e] >> 16), cls = (int)(em[e] >> kItemBits);
                    const int own = (half << CLSB) | cls;
                    const int opp = ((1 - half) << CLSB) | (int)(~(uint32_t)cls & CMASK);
                    const V bwd = pick(run, opp);
                    if (pol.is_tgt(em[e] & kItemMask)) {
                        V* a = s_acc + 4 * (eh[e] & 0xffffu) + 2 * half;
                        a[0] = Pol::add(a[0], fwd[e]);
                        a[1] = Pol::add(a[1], bwd);
                    }
                    add_at<Pol>(run, own, wb[e]);
                }
            }
        }
        local_store<IT>(s_key, s_meta, s_home, cnt, ek, em, eh);
    }
    // flush the per-target sums and write the tile out for the global levels
    for (int i = threadIdx.x; i < ln; i += NT) {
        const uint32_t m = s_meta[lpd(i)];
        const uint32_t item = m & kItemMask;
        if (write_out) {
            key_out[t0 + i] = s_key[lpd(i)];
            meta_out[t0 + i] = m;
        }
        if (pol.is_tgt(item)) pol.flush(item, m >> kItemBits, s_acc + 4 * s_home[lpd(i)]);
    }
}

// Folded form (kernel policies without per-orthant terms).  Source weights
// are rebuilt from the per-item factors when needed instead of being held.
// ------------------------------------------------------------------ scaled tiles
// The shifted values of the folded sweep (mantissa and power-of-two shift per
// value) keep e^{+-x/h} factors in range whatever their spread, at the price
// of exponent bookkeeping on every addition and product.  Within one tile the
// factors usually span far less than the FP32 exponent range, so a tile whose
// factors all lie within 2^{+-kFastL} of a per-tile reference can run the same
// sweep in plain FP32: each item's factor F(h, dir) of its class c is stored
// once, scaled by 2^{-R[dir][h][c]}.  A source adds w F(h, dir) 2^{-R} to the
// running sum of its channel (h, c); a target of the opposite channel
// (1 - h, ~c) reads that sum with its own factor F(1 - h, 1 - dir), which is
// stored scaled by 2^{-R[1-dir][1-h][~c]}.  Choosing R[1-dir][1-h][~c] =
// -R[dir][h][c] makes the two scalings cancel in the product, so the same
// scaled value serves an item as a source term and as a target factor and
// the product is the kernel value itself (bounded by the source weight).
// Bounds: scaled factors lie in [2^{-kFastL-2}, 2^{kFastL+2}] (mantissas of up
// to four factors carry up to 2^{+-2}); with nonzero weights in
// [2^{kFastWmin}, 2^{kFastWmax+1}) and at most 2^12 terms per sum, every term
// and partial sum stays a normal FP32 number.  A tile outside these bounds
// keeps the shifted arithmetic.
constexpr int kFastL = 96, kFastWmax = 14, kFastWmin = -26;

template <int NW>
struct FastLO {
    struct V { float v[NW]; };
    __device__ static V zero() {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = 0.f;
        return r;
    }
    __device__ static V add(V a, V b) {
        V r;
#pragma unroll
        for (int i = 0; i < NW; ++i) r.v[i] = a.v[i] + b.v[i];
        return r;
    }
};

// Per-tile references of the scaled form.  Returns (uniformly over the CTA)
// whether the tile qualifies; if so, s_fm[4 i + 2 h + dir] has been replaced
// by F(h, dir) 2^{-R[dir][h][c]} (c = cls_of(i), the class of home slot i)
// and s_ref[(2 h + dir) * NCLS + c] holds R.  s_fs (the shifts) is left as it
// was.
template <int CLSB, int NT, class ClsOf>
__device__ __forceinline__ bool fold_fast_setup(ClsOf cls_of, float* s_fm, const int* s_fs, const float* s_wt, int ln,
                                                int* s_ref) {
    constexpr int NCLS = 1 << CLSB, NS = 4 * NCLS;
    __shared__ int s_lo[NS], s_hi[NS], s_wr[2], s_ok;
    for (int i = threadIdx.x; i < NS; i += NT) { s_lo[i] = INT_MAX; s_hi[i] = INT_MIN; }
    if (threadIdx.x == 0) { s_wr[0] = INT_MAX; s_wr[1] = INT_MIN; }
    __syncthreads();
    int lo[NS], hi[NS], wlo = INT_MAX, whi = INT_MIN;
#pragma unroll
    for (int q = 0; q < NS; ++q) { lo[q] = INT_MAX; hi[q] = INT_MIN; }
    for (int i = threadIdx.x; i < ln; i += NT) {
        const int c = cls_of(i);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = s_fs[4 * i + j];
#pragma unroll
            for (int cc = 0; cc < NCLS; ++cc) {
                if (c == cc) { lo[j * NCLS + cc] = min(lo[j * NCLS + cc], e); hi[j * NCLS + cc] = max(hi[j * NCLS + cc], e); }
            }
        }
        const float w = s_wt[i];
        if (w != 0.f) {
            const int ew = (int)((__float_as_uint(w) >> 23) & 0xffu) - 127;   // -127: subnormal
            wlo = min(wlo, ew);
            whi = max(whi, ew);
        }
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        lo[q] = __reduce_min_sync(0xffffffffu, lo[q]);
        hi[q] = __reduce_max_sync(0xffffffffu, hi[q]);
    }
    wlo = __reduce_min_sync(0xffffffffu, wlo);
    whi = __reduce_max_sync(0xffffffffu, whi);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (lo[q] != INT_MAX) { atomicMin(&s_lo[q], lo[q]); atomicMax(&s_hi[q], hi[q]); }
        }
        if (wlo != INT_MAX) { atomicMin(&s_wr[0], wlo); atomicMax(&s_wr[1], whi); }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = (s_wr[0] == INT_MAX) || (s_wr[0] >= kFastWmin && s_wr[1] <= kFastWmax);
        // free references R[+][h][c]; R[-][1-h][~c] = -R[+][h][c]
        for (int h = 0; h < 2; ++h)
            for (int c = 0; c < NCLS; ++c) {
                const int q1 = (2 * h + 0) * NCLS + c;                        // slot (dir +, h, c)
                const int q2 = (2 * (1 - h) + 1) * NCLS + ((~c) & (NCLS - 1)); // slot (dir -, 1-h, ~c)
                long long a = -(1ll << 40), b = (1ll << 40);
                if (s_lo[q1] != INT_MAX) {
                    a = max(a, (long long)s_hi[q1] - kFastL);
                    b = min(b, (long long)s_lo[q1] + kFastL);
                }
                if (s_lo[q2] != INT_MAX) {
                    a = max(a, -(long long)s_lo[q2] - kFastL);
                    b = min(b, (long long)kFastL - (long long)s_hi[q2]);
                }
                long long r = 0;
                if (a > b) ok = false;
                else if (a > -(1ll << 40) && b < (1ll << 40)) r = (a + b) / 2;
                else if (a > -(1ll << 40)) r = a;
                else if (b < (1ll << 40)) r = b;
                s_ref[q1] = (int)r;
                s_ref[q2] = (int)(-r);
            }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return false;
    for (int i = threadIdx.x; i < ln; i += NT) {
        const int c = cls_of(i);
#pragma unroll
        for (int j = 0; j < 4; ++j) s_fm[4 * i + j] *= pow2f_any(s_fs[4 * i + j] - s_ref[j * NCLS + c]);
    }
    __syncthreads();
    return true;
}

// The tile-local merge levels of the folded kernel sums on a loaded tile
// (keys, metas and home slots in padded shared-memory rows; per-home factors,
// weights and target sums): `levels` merge levels with the forward and
// backward channel sweeps, each target adding its kernel values to s_fa.
// FAST: the scaled FP32 form (fold_fast_setup has scaled s_fm); else the
// shifted form.  Used by k_local_fold and k_nested_fold.
template <class Pol, int CLSB, int NT, int IT, bool FAST>
__device__ __forceinline__ void fold_tile_levels(uint32_t* s_key, uint32_t* s_meta, uint16_t* s_home,
                                                 const typename Pol::M* s_fm, const int* s_fs,
                                                 const typename Pol::M* s_wt, typename Pol::FA* s_fa, void* s_scan_v,
                                                 int ln, int levels, const Pol& pol) {
    typedef typename Pol::LOps LO;
    typedef typename Pol::M M;
    constexpr int NW = Pol::kNW;
    constexpr int NCH = 2 << CLSB;
    typedef typename std::conditional<FAST, FastLO<NW>, LO>::type LX;
    typedef typename LX::V VX;
    VX* s_scan = reinterpret_cast<VX*>(s_scan_v);
    // kernel value of a running sum v read with factor (m, s), per weight channel
    auto value = [&](const VX& v, M mm, int sh, M* c) {
        if constexpr (FAST) {
#pragma unroll
            for (int q = 0; q < NW; ++q) c[q] = v.v[q] * mm;
        } else {
            Pol::fold_value(v, mm, sh, c);
        }
    };
    // source term of an element (weight channel 1 of two-channel sums: 1 for sources)
    auto term = [&](M mm, int sh, M w, bool src) -> VX {
        if constexpr (FAST) {
            VX r;
#pragma unroll
            for (int q = 0; q < NW; ++q) r.v[q] = ((NW == 2 && q == 1) ? (src ? (M)1 : (M)0) : w) * mm;
            return r;
        } else {
            return Pol::fold_src(mm, sh, w, src);
        }
    };
    for (int m = 0; m < levels; ++m) {
        const int R2 = 2 << m;
        uint32_t ek[IT], em[IT], eh[IT];
        const int cnt = local_merge<IT>(s_key, s_meta, s_home, ln, 1 << m, ek, em, eh);
        // factors F(h, +) (index 0) and F(h, -) (index 1) of each element
        M f0[IT], f1[IT], wt[IT];
        int g0[IT], g1[IT];
#pragma unroll
        for (int e = 0; e < IT; ++e) {
            f0[e] = f1[e] = wt[e] = (M)0;
            g0[e] = g1[e] = 0;
            if (e < cnt) {
                const int b = 4 * (int)(eh[e] & 0xffffu) + 2 * (int)(eh[e] >> 16);
                f0[e] = s_fm[b];
                f1[e] = s_fm[b + 1];
                if constexpr (!FAST) {
                    g0[e] = s_fs[b];
                    g1[e] = s_fs[b + 1];
                }
                wt[e] = s_wt[eh[e] & 0xffffu];
            }
        }
        const int ts = R2 / IT;   // threads per merged block (0 or 1: thread-local)
        const int p0 = threadIdx.x * IT;
        // Walks from zero over the thread's elements (a thread's elements lie
        // in one merged block when ts > 1): kernel values of the thread-local
        // prefix (forward, with F(h, -) of the target) and suffix (backward,
        // F(h, +)); the walks end with the thread's channel totals.
        M cf[IT][NW], cb[IT][NW];
        VX fe[NCH], be[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) { fe[c] = LX::zero(); be[c] = LX::zero(); }
#pragma unroll
        for (int e = 0; e < IT; ++e) {
#pragma unroll
            for (int q = 0; q < NW; ++q) cf[e][q] = (M)0;
            if (e < cnt) {
                if (ts <= 1 && e > 0 && ((p0 + e) % R2) == 0) {
#pragma unroll
                    for (int c = 0; c < NCH; ++c) fe[c] = LX::zero();
                }
                const int own = (int)((eh[e] >> 16) << CLSB) | (int)(em[e] >> kItemBits);
                value(pick(fe, own ^ (NCH - 1)), f1[e], g1[e], cf[e]);
                add_at<LX>(fe, own, term(f0[e], g0[e], wt[e], pol.is_src(em[e] & kItemMask)));
            }
        }
#pragma unroll
        for (int e = IT - 1; e >= 0; --e) {
#pragma unroll
            for (int q = 0; q < NW; ++q) cb[e][q] = (M)0;
            if (e < cnt) {
                if (ts <= 1 && e < cnt - 1 && ((p0 + e + 1) % R2) == 0) {
#pragma unroll
                    for (int c = 0; c < NCH; ++c) be[c] = LX::zero();
                }
                const int own = (int)((eh[e] >> 16) << CLSB) | (int)(em[e] >> kItemBits);
                value(pick(be, own ^ (NCH - 1)), f0[e], g0[e], cb[e]);
                add_at<LX>(be, own, term(f1[e], g1[e], wt[e], pol.is_src(em[e] & kItemMask)));
            }
        }
        // blocks spanning several threads: the exclusive prefix / suffix of
        // the thread totals joins every element (the fold is linear)
        if (ts > 1) {
            seg_scan<LX, NCH, NT>(fe, be, ts, s_scan);
#pragma unroll
            for (int e = 0; e < IT; ++e) {
                if (e < cnt) {
                    const int opp = ((int)((eh[e] >> 16) << CLSB) | (int)(em[e] >> kItemBits)) ^ (NCH - 1);
                    M xf[NW], xb[NW];
                    value(pick(fe, opp), f1[e], g1[e], xf);
                    value(pick(be, opp), f0[e], g0[e], xb);
#pragma unroll
                    for (int q = 0; q < NW; ++q) { cf[e][q] += xf[q]; cb[e][q] += xb[q]; }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < IT; ++e)
            if (e < cnt && pol.is_tgt(em[e] & kItemMask)) {
                M sf, sb;
                pol.signs((int)(eh[e] >> 16), em[e] >> kItemBits, sf, sb);
                Pol::fold_add(s_fa + NW * (eh[e] & 0xffffu), cf[e], cb[e], sf, sb);
            }
        local_store<IT>(s_key, s_meta, s_home, cnt, ek, em, eh);
    }
}

template <class Pol, int CLSB, bool HALF>
__global__ void __launch_bounds__(LocalCfg<Pol, CLSB, true, HALF>::NT, (LocalCfg<Pol, CLSB, true, HALF>::kMinBlocks))
    k_local_fold(const uint32_t* __restrict__ seq, int64_t n, const uint32_t* __restrict__ P0, ClassSpecK cs,
                 int levels, Pol pol, uint32_t* __restrict__ key_out, uint32_t* __restrict__ meta_out,
                 int write_out, int rec_out, FoldRecs<Pol> rout) {
    typedef LocalCfg<Pol, CLSB, true, HALF> Cfg;
    typedef typename Pol::LOps LO;
    typedef typename LO::V V;          // tile-local sums
    typedef typename Pol::M M;
    typedef typename Pol::FA FA;
    constexpr int T = Cfg::T, NT = Cfg::NT, IT = Cfg::IT;
    constexpr int NW = Pol::kNW;
    constexpr int NCH = 2 << CLSB;
    constexpr uint32_t CMASK = (1u << CLSB) - 1u;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_key);
    uint32_t* s_meta = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_meta);
    uint16_t* s_home = reinterpret_cast<uint16_t*>(smem_raw + Cfg::o_home);
    M* s_fm = reinterpret_cast<M*>(smem_raw + Cfg::o_fm);
    int* s_fs = reinterpret_cast<int*>(smem_raw + Cfg::o_fs);
    M* s_wt = reinterpret_cast<M*>(smem_raw + Cfg::o_wt);
    FA* s_fa = reinterpret_cast<FA*>(smem_raw + Cfg::o_fa);
    V* s_scan = reinterpret_cast<V*>(smem_raw + Cfg::o_scan);

    const int64_t t0 = (int64_t)blockIdx.x * T;
    const int ln = (int)min((int64_t)T, n - t0);
    for (int i = threadIdx.x; i < T; i += NT) {
        if (i < ln) {
            const uint32_t item = seq[t0 + i];
            const uint32_t c = class_of_k(cs, item);
            s_key[lpd(i)] = P0[item];
            s_meta[lpd(i)] = item | (c << kItemBits);
            s_home[lpd(i)] = (uint16_t)i;
            // the longer levels read per-item bases only without records
            if constexpr (!Pol::kRecords) pol.prep_item(item, c);
            M wt;
            pol.fold_item(item, c, &s_fm[4 * i], &s_fs[4 * i], wt);
            s_wt[i] = pol.is_src(item) ? wt : (M)0;   // 0: no source role
        }
#pragma unroll
        for (int q = 0; q < NW; ++q) s_fa[NW * i + q] = Pol::fa_zero();
    }
    __syncthreads();
    // Scaled FP32 form when the tile's factors allow it (mixed path only).
    __shared__ int s_ref[4 << CLSB];
    bool fast = false;
    if constexpr (Pol::kFastLocal)   // home slot i sits at position i at this point
        fast = fold_fast_setup<CLSB, NT>([&](int i) { return (int)(s_meta[lpd(i)] >> kItemBits); }, s_fm, s_fs, s_wt,
                                         ln, s_ref);
    if constexpr (Pol::kFastLocal) {
        if (fast) fold_tile_levels<Pol, CLSB, NT, IT, true>(s_key, s_meta, s_home, s_fm, s_fs, s_wt, s_fa, s_scan, ln,
                                                            levels, pol);
        else fold_tile_levels<Pol, CLSB, NT, IT, false>(s_key, s_meta, s_home, s_fm, s_fs, s_wt, s_fa, s_scan, ln,
                                                        levels, pol);
    } else {
        fold_tile_levels<Pol, CLSB, NT, IT, false>(s_key, s_meta, s_home, s_fm, s_fs, s_wt, s_fa, s_scan, ln, levels,
                                                   pol);
    }
    // write the tile out for the longer merge levels (as records when they
    // run on records); targets not handed on as records are flushed
    for (int i = threadIdx.x; i < ln; i += NT) {
        const uint32_t m = s_meta[lpd(i)];
        const uint32_t item = m & kItemMask;
        const int h = s_home[lpd(i)];
        const int64_t d = t0 + i;
        if (write_out) {
            key_out[d] = s_key[lpd(i)];
            meta_out[d] = m;
        }
        if (rec_out) {
            const int c = (int)(m >> kItemBits);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                M fm = s_fm[4 * h + j];
                if constexpr (Pol::kFastLocal) {
                    if (fast) fm *= pow2f_any(s_ref[j * (1 << CLSB) + c] - s_fs[4 * h + j]);   // exact: a power of two
                }
                rout.fm[4 * d + j] = fm;
                rout.fs[4 * d + j] = s_fs[4 * h + j];
            }
            rout.wt[d] = s_wt[h];
#pragma unroll
            for (int q = 0; q < NW; ++q) rout.fa[d * NW + q] = s_fa[NW * h + q];
        } else if (pol.is_tgt(item)) {
            pol.fold_flush(item, s_fa + NW * h);
        }
    }
}

// ------------------------------------------------------------------ nested outer levels
// The outer levels of tree axis 2 whose nodes (2^{l+1} items) fit a tile of
// NFT items, nested in one launch (the kernel-sum counterpart of the
// counting engine's k_dom_nested).  A CTA loads its tile once; for each outer
// level l it merges the outer state by P_1 (the tree of Algorithms 3/4) in
// shared memory and runs that level's complete inner folded sweep (l + 1
// merge levels by P_0) on it; the targets' kernel values are summed in shared
// memory over all these levels and flushed once.  The side bit of axis 2 at
// level l is bit l of the item's slot in the tile (tiles start at multiples
// of NFT inside the enclosing nodes); the enclosing axes' bits (class bits
// 1 and up) are fixed per item.  The per-item factors depend on the class, so
// they are recomputed for every level.  The outer state itself is built by
// the regular merges (so the longer levels need not wait for this kernel).
constexpr int NFT = 1024;          // items per tile
constexpr int NFN = 256;           // threads
constexpr int NFI = NFT / NFN;     // items per thread

template <class Pol, int CLSB>
struct NestedCfg {
    typedef typename Pol::M M;
    typedef typename Pol::FA FA;
    typedef typename Pol::LOps::V V;
    static constexpr int TP = NFT + NFT / 32;
    static constexpr size_t a16(size_t x) { return (x + 15) / 16 * 16; }
    static constexpr size_t o_item = 0;                                   // [NFT] item of each slot
    static constexpr size_t o_p0 = o_item + 4 * NFT;                      // [NFT] P_0 of each slot
    static constexpr size_t o_cenc = o_p0 + 4 * NFT;                      // [NFT] enclosing class bits
    static constexpr size_t o_okey = o_cenc + 4 * NFT;                    // [2][TP] outer state: P_1
    static constexpr size_t o_oslot = o_okey + 8 * (size_t)TP;            // [2][TP] outer state: slot
    static constexpr size_t o_key = o_oslot + 8 * (size_t)TP;             // [TP] inner keys
    static constexpr size_t o_meta = o_key + 4 * (size_t)TP;              // [TP] inner metas
    static constexpr size_t o_home = o_meta + 4 * (size_t)TP;             // [TP] inner home slots (u16)
    static constexpr size_t o_fm = a16(o_home + 2 * (size_t)TP);          // [NFT][4] factor mantissas
    static constexpr size_t o_fs = o_fm + 4 * sizeof(M) * NFT;            // [NFT][4] factor shifts
    static constexpr size_t o_wt = o_fs + 16 * (size_t)NFT;               // [NFT] source weights
    static constexpr size_t o_fa = a16(o_wt + sizeof(M) * NFT);           // [NFT][NW] target sums
    static constexpr size_t o_scan = a16(o_fa + sizeof(FA) * Pol::kNW * NFT);
    static constexpr size_t bytes = o_scan + 2 * (2 << CLSB) * (NFN / 32) * sizeof(V);
};

// One plain merge level (runs 2^m -> 2^{m+1}) of (key, slot) pairs in padded
// shared-memory rows; every thread takes NFI consecutive outputs.
__device__ __forceinline__ void nested_outer_merge(const uint32_t* ik, const uint32_t* is, uint32_t* wk, uint32_t* ws,
                                                   int ln, int m) {
    const int R = 1 << m, R2 = 2 << m;
    const int p0 = threadIdx.x * NFI;
    uint32_t ok[NFI], os[NFI];
    int bsl = 0, cl = 0, dl = 0, i = 0, j = 0, cnt = 0;
#pragma unroll
    for (int e = 0; e < NFI; ++e) {
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
            ok[e] = ik[src];
            os[e] = is[src];
            i += takeC ? 1 : 0;
            j += takeC ? 0 : 1;
            cnt = e + 1;
        }
    }
#pragma unroll
    for (int e = 0; e < NFI; ++e)
        if (e < cnt) { wk[lpd(p0 + e)] = ok[e]; ws[lpd(p0 + e)] = os[e]; }
}

template <class Pol, int CLSB>
__global__ void __launch_bounds__(NFN) k_nested_fold(const uint32_t* __restrict__ seq, int64_t n,
                                                     const uint32_t* __restrict__ P0, const uint32_t* __restrict__ P1,
                                                     ClassSpecK cs, int levels, Pol pol) {
    typedef NestedCfg<Pol, CLSB> Cfg;
    typedef typename Pol::M M;
    typedef typename Pol::FA FA;
    constexpr int NW = Pol::kNW;
    constexpr int TP = Cfg::TP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* s_item = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_item);
    uint32_t* s_p0 = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_p0);
    uint32_t* s_cenc = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_cenc);
    uint32_t* s_okey = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_okey);
    uint32_t* s_oslot = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_oslot);
    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_key);
    uint32_t* s_meta = reinterpret_cast<uint32_t*>(smem_raw + Cfg::o_meta);
    uint16_t* s_home = reinterpret_cast<uint16_t*>(smem_raw + Cfg::o_home);
    M* s_fm = reinterpret_cast<M*>(smem_raw + Cfg::o_fm);
    int* s_fs = reinterpret_cast<int*>(smem_raw + Cfg::o_fs);
    M* s_wt = reinterpret_cast<M*>(smem_raw + Cfg::o_wt);
    FA* s_fa = reinterpret_cast<FA*>(smem_raw + Cfg::o_fa);
    void* s_scan = smem_raw + Cfg::o_scan;
    __shared__ int s_ref[4 << CLSB];

    const int64_t t0 = (int64_t)blockIdx.x * NFT;
    const int ln = (int)min((int64_t)NFT, n - t0);
    for (int i = threadIdx.x; i < ln; i += NFN) {
        const uint32_t item = seq[t0 + i];
        uint32_t c = 0;
        for (int q = 1; q < cs.nb; ++q) c |= ((cs.idx[q][item] >> cs.lvl[q]) & 1u) << q;
        s_item[i] = item;
        s_p0[i] = P0[item];
        s_cenc[i] = c;
        s_okey[lpd(i)] = P1[item];
        s_oslot[lpd(i)] = (uint32_t)i;
#pragma unroll
        for (int q = 0; q < NW; ++q) s_fa[NW * i + q] = Pol::fa_zero();
    }
    __syncthreads();
    int ob = 0;
    for (int l = 0; l < levels; ++l) {
        nested_outer_merge(s_okey + ob * TP, s_oslot + ob * TP, s_okey + (ob ^ 1) * TP, s_oslot + (ob ^ 1) * TP, ln,
                           l);
        __syncthreads();
        ob ^= 1;
        // this level's inner tile (outer order) and the factors of its classes
        for (int p = threadIdx.x; p < ln; p += NFN) {
            const uint32_t sl = s_oslot[ob * TP + lpd(p)];
            const uint32_t cls = ((sl >> l) & 1u) | s_cenc[sl];
            s_key[lpd(p)] = s_p0[sl];
            s_meta[lpd(p)] = s_item[sl] | (cls << kItemBits);
            s_home[lpd(p)] = (uint16_t)sl;
        }
        for (int i = threadIdx.x; i < ln; i += NFN) {
            const uint32_t item = s_item[i];
            const uint32_t cls = (((uint32_t)i >> l) & 1u) | s_cenc[i];
            M wt;
            pol.fold_item(item, cls, &s_fm[4 * i], &s_fs[4 * i], wt);
            s_wt[i] = pol.is_src(item) ? wt : (M)0;
        }
        __syncthreads();
        bool fast = false;
        if constexpr (Pol::kFastLocal)
            fast = fold_fast_setup<CLSB, NFN>([&](int i) { return (int)((((uint32_t)i >> l) & 1u) | s_cenc[i]); },
                                              s_fm, s_fs, s_wt, ln, s_ref);
        if (fast) fold_tile_levels<Pol, CLSB, NFN, NFI, Pol::kFastLocal>(s_key, s_meta, s_home, s_fm, s_fs, s_wt, s_fa,
                                                                        s_scan, ln, l + 1, pol);
        else fold_tile_levels<Pol, CLSB, NFN, NFI, false>(s_key, s_meta, s_home, s_fm, s_fs, s_wt, s_fa, s_scan, ln,
                                                          l + 1, pol);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ln; i += NFN) {
        const uint32_t item = s_item[i];
        if (pol.is_tgt(item)) pol.fold_flush(item, s_fa + NW * i);
    }
}

// Reads element s (factors of half h, weight) and, if d >= 0, copies its
// factors and weight to slot d of `out`.
template <class Pol>
__device__ __forceinline__ void rec_move(const FoldRecs<Pol>& in, int64_t s, const FoldRecs<Pol>& out, int64_t d,
                                         int h, typename Pol::M& f0, typename Pol::M& f1, int& g0, int& g1,
                                         typename Pol::M& wt) {
    if constexpr (sizeof(typename Pol::M) == 4) {
        const float4 f = reinterpret_cast<const float4*>(in.fm)[s];
        if (d >= 0) reinterpret_cast<float4*>(out.fm)[d] = f;
        f0 = h ? f.z : f.x;
        f1 = h ? f.w : f.y;
    } else {
        const double2 fa = reinterpret_cast<const double2*>(in.fm)[2 * s];
        const double2 fb = reinterpret_cast<const double2*>(in.fm)[2 * s + 1];
        if (d >= 0) {
            reinterpret_cast<double2*>(out.fm)[2 * d] = fa;
            reinterpret_cast<double2*>(out.fm)[2 * d + 1] = fb;
        }
        f0 = h ? fb.x : fa.x;
        f1 = h ? fb.y : fa.y;
    }
    const int4 g = reinterpret_cast<const int4*>(in.fs)[s];
    if (d >= 0) reinterpret_cast<int4*>(out.fs)[d] = g;
    g0 = h ? g.z : g.x;
    g1 = h ? g.w : g.y;
    wt = in.wt[s];
    if (d >= 0) out.wt[d] = wt;
}

// Merge level of the folded records.  PH_TOTALS: per-CTA channel totals of
// the source weights (runs longer than a tile).  PH_SWEEP: merge, payload
// move and the sweep; each thread walks its elements from zero, the
// segmented scan over threads and the inter-CTA carries give the prefix /
// suffix before them, and every target adds the kernel values of its
// forward and backward sums to its record (flushed on the last level).
// Resident CTAs per SM asked of the compiler, by the bytes of running sums a
// thread holds and its items per thread:
//   sums <= 48 B (one channel, d <= 3):   totals 3, sweep 3 on 4-item tiles (2 on 8-item tiles)
//   sums <= 96 B (d = 4, or two channels): 2 on 4-item tiles; on 8-item tiles totals 2 up to 64 B
//   wider sums:                            1
template <class Pol, int CLSB, int PHASE>
struct FoldOcc {
    static constexpr size_t bytes = sizeof(typename Pol::V) * (2 << CLSB);
    static constexpr bool small_tile = MergeItems<Pol, CLSB>::value <= 4;
    static constexpr int totals = bytes <= 48 ? 3 : bytes <= (small_tile ? 96 : 64) ? 2 : 1;
    static constexpr int sweep = bytes <= 48 ? (small_tile ? 3 : 2) : (small_tile && bytes <= 96) ? 2 : 1;
    static constexpr int value = PHASE == PH_TOTALS ? totals : sweep;
};

template <class Pol, int CLSB, int PHASE>
__global__ void __launch_bounds__(MT, (FoldOcc<Pol, CLSB, PHASE>::value)) k_merge_fold(MergeArgs a, FoldRecs<Pol> rin, FoldRecs<Pol> rout, Pol pol,
                                                   typename Pol::V* __restrict__ totals,
                                                   const typename Pol::V* __restrict__ carries, int last) {
    typedef typename Pol::V V;
    typedef typename Pol::M M;
    typedef typename Pol::FA FA;
    constexpr int MI = MergeItems<Pol, CLSB>::value, MTILE = MT * MI;
    constexpr int NW = Pol::kNW;
    constexpr int NCH = 2 << CLSB;
    constexpr int MP = MTILE + MTILE / 32;
    __shared__ uint32_t s_key[MP];
    __shared__ uint32_t s_meta[MP];
    __shared__ int64_t s_co[6];
    __shared__ V s_scan[2 * NCH * (MT / 32)];
    // the sweep's running target sums, copied in asynchronously while the
    // walks and the scan run (8-byte sums only; others are read at the end)
    constexpr bool kPreFA = PHASE == PH_SWEEP && sizeof(FA) * NW == 8;
    __shared__ __align__(8) FA s_fa[kPreFA ? MTILE * NW : 1];

    const int64_t n = a.n;
    const int64_t R2 = (int64_t)2 << a.logR;
    const int64_t o0 = (int64_t)blockIdx.x * MTILE;
    if (o0 >= n) return;
    const MergeTile mt = merge_tile_load<MI, PHASE != PH_TOTALS>(a, s_key, s_meta, s_co);
    const int64_t ln = mt.ln, lc = mt.lc;
    const bool big = mt.big;

    if (PHASE == PH_TOTALS) {
        V tf[NCH], tb[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) { tf[c] = Pol::zero(); tb[c] = Pol::zero(); }
        // the thread's slots in batches of TB: all record loads of a batch
        // are issued before its first sum
        constexpr int TB = MI / 2;
#pragma unroll
        for (int j0 = 0; j0 < MI; j0 += TB) {
            M f0[TB], f1[TB], wt[TB];
            int g0[TB], g1[TB], ch[TB];
            bool sv[TB];
#pragma unroll
            for (int j = 0; j < TB; ++j) {
                const int i = (int)threadIdx.x + (j0 + j) * MT;
                const uint32_t m = i < ln ? s_meta[mpd(i)] : 0u;
                const int half = (i >= lc) ? 1 : 0;
                sv[j] = i < ln && pol.is_src(m & kItemMask);
                ch[j] = (half << CLSB) | (int)(m >> kItemBits);
                f0[j] = f1[j] = wt[j] = (M)0;
                g0[j] = g1[j] = 0;
                if (sv[j]) rec_move<Pol>(rin, half ? mt.ds + (i - lc) : mt.cs + i, rin, -1, half, f0[j], f1[j],
                                         g0[j], g1[j], wt[j]);
            }
#pragma unroll
            for (int j = 0; j < TB; ++j) {
                if (sv[j]) {
                    add_at<Pol>(tf, ch[j], Pol::fold_src_g(f0[j], g0[j], wt[j], true));
                    add_at<Pol>(tb, ch[j], Pol::fold_src_g(f1[j], g1[j], wt[j], true));
                }
            }
        }
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
    int eh[MI], es[MI];      // half, and the shared-memory slot the element came from
    int cnt = 0;
    const int64_t p0 = (int64_t)threadIdx.x * MI;
    cnt = tile_merge(s_key, s_meta, (int)ln, (int)lc, big, R2, (int)p0, ek, em, eh, es);
    if (!last) {
        const int64_t q0 = o0 + p0;
        if (cnt == MI) {
            uint4* kk = reinterpret_cast<uint4*>(a.key_out + q0);
            uint4* mm = reinterpret_cast<uint4*>(a.meta_out + q0);
#pragma unroll
            for (int v = 0; v < MI / 4; ++v) {
                kk[v] = make_uint4(ek[4 * v], ek[4 * v + 1], ek[4 * v + 2], ek[4 * v + 3]);
                mm[v] = make_uint4(em[4 * v], em[4 * v + 1], em[4 * v + 2], em[4 * v + 3]);
            }
        } else {
            for (int e = 0; e < cnt; ++e) { a.key_out[q0 + e] = ek[e]; a.meta_out[q0 + e] = em[e]; }
        }
    }
    // global position of the element held in shared-memory slot q
    auto gpos = [&](int q) -> int64_t {
        return big ? (q < lc ? mt.cs + q : mt.ds + (q - lc)) : o0 + q;
    };
    // payload move; the factors of the element's half stay in registers
    M f0[MI], f1[MI], wt[MI];
    int g0[MI], g1[MI];
#pragma unroll
    for (int e = 0; e < MI; ++e) {
        f0[e] = f1[e] = wt[e] = (M)0;
        g0[e] = g1[e] = 0;
        if (e < cnt)
            rec_move<Pol>(rin, gpos(es[e]), rout, last ? -1 : o0 + p0 + e, eh[e], f0[e], f1[e], g0[e], g1[e], wt[e]);
    }
    if constexpr (kPreFA) {
        // slot e * MT + thread: each thread copies and later reads only its own
#pragma unroll
        for (int e = 0; e < MI; ++e)
            if (e < cnt) cp_async8(&s_fa[e * MT + threadIdx.x], &rin.fa[gpos(es[e]) * NW]);
        cp_async_commit();
    }
    // walks from zero over the thread's elements
    const int ts = big ? MT : (int)(R2 / MI);   // threads per merged block (0/1: thread-local)
    M cf[MI][NW], cb[MI][NW];
    V fe[NCH], be[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) { fe[c] = Pol::zero(); be[c] = Pol::zero(); }
#pragma unroll
    for (int e = 0; e < MI; ++e) {
#pragma unroll
        for (int q = 0; q < NW; ++q) cf[e][q] = (M)0;
        if (e < cnt) {
            if (ts <= 1 && e > 0 && ((p0 + e) % R2) == 0) {
#pragma unroll
                for (int c = 0; c < NCH; ++c) fe[c] = Pol::zero();
            }
            const int own = (eh[e] << CLSB) | (int)(em[e] >> kItemBits);
            Pol::fold_value_g(pick(fe, own ^ (NCH - 1)), f1[e], g1[e], cf[e]);
            add_at<Pol>(fe, own, Pol::fold_src_g(f0[e], g0[e], wt[e], pol.is_src(em[e] & kItemMask)));
        }
    }
#pragma unroll
    for (int e = MI - 1; e >= 0; --e) {
#pragma unroll
        for (int q = 0; q < NW; ++q) cb[e][q] = (M)0;
        if (e < cnt) {
            if (ts <= 1 && e < cnt - 1 && ((p0 + e + 1) % R2) == 0) {
#pragma unroll
                for (int c = 0; c < NCH; ++c) be[c] = Pol::zero();
            }
            const int own = (eh[e] << CLSB) | (int)(em[e] >> kItemBits);
            Pol::fold_value_g(pick(be, own ^ (NCH - 1)), f0[e], g0[e], cb[e]);
            add_at<Pol>(be, own, Pol::fold_src_g(f1[e], g1[e], wt[e], pol.is_src(em[e] & kItemMask)));
        }
    }
    if (ts > 1) {
        seg_scan<Pol, NCH>(fe, be, ts, s_scan);
        if (big && carries) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                fe[c] = Pol::add(carries[((int64_t)blockIdx.x * 2 + 0) * NCH + c], fe[c]);
                be[c] = Pol::add(be[c], carries[((int64_t)blockIdx.x * 2 + 1) * NCH + c]);
            }
        }
#pragma unroll
        for (int e = 0; e < MI; ++e) {
            if (e < cnt) {
                const int opp = ((eh[e] << CLSB) | (int)(em[e] >> kItemBits)) ^ (NCH - 1);
                M xf[NW], xb[NW];
                Pol::fold_value_g(pick(fe, opp), f1[e], g1[e], xf);
                Pol::fold_value_g(pick(be, opp), f0[e], g0[e], xb);
#pragma unroll
                for (int q = 0; q < NW; ++q) { cf[e][q] += xf[q]; cb[e][q] += xb[q]; }
            }
        }
    }
    // target sums: read, add this level's kernel values, write on (or flush)
    if constexpr (kPreFA) cp_async_wait_all();
#pragma unroll
    for (int e = 0; e < MI; ++e) {
        if (e < cnt) {
            const uint32_t item = em[e] & kItemMask;
            const int64_t src = gpos(es[e]);
            FA acc[NW];
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                if constexpr (kPreFA) acc[q] = s_fa[e * MT + threadIdx.x];
                else acc[q] = rin.fa[src * NW + q];
            }
            if (pol.is_tgt(item)) {
                M sf, sb;
                pol.signs(eh[e], em[e] >> kItemBits, sf, sb);
                Pol::fold_add(acc, cf[e], cb[e], sf, sb);
            }
            if (!last) {
#pragma unroll
                for (int q = 0; q < NW; ++q) rout.fa[(o0 + p0 + e) * NW + q] = acc[q];
            } else if (pol.is_tgt(item)) {
                pol.fold_flush(item, acc);
            }
        }
    }
}

// Carries for merged blocks that span several CTAs: exclusive prefix of the
// forward totals and exclusive suffix of the backward totals over the CTAs of
// each merged block.  One warp per (block, channel, direction): each lane
// sums a contiguous run of CTAs (in scan order), a warp scan combines the
// lanes, and each lane writes the carries of its run.
template <class Pol, int NCH, int MTILE>
__global__ void k_carries(const typename Pol::V* __restrict__ totals, typename Pol::V* __restrict__ carries,
                          int64_t n, int logR) {
    typedef typename Pol::V V;
    const int64_t R2 = (int64_t)2 << logR;
    const int64_t ctas = (n + MTILE - 1) / MTILE;
    const int64_t per = R2 / MTILE;            // CTAs per full merged block
    const int64_t nblocks = (ctas + per - 1) / per;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // uniform per warp
    const int lane = threadIdx.x & 31;
    if (wid >= nblocks * NCH * 2) return;
    const int dir = (int)(wid % 2);
    const int c = (int)((wid / 2) % NCH);
    const int64_t b = wid / (2 * NCH);
    const int64_t c0 = b * per, c1 = min(c0 + per, ctas);
    const int64_t len = c1 - c0, chunk = (len + 31) / 32;
    // position of the idx-th CTA in scan order (backward: from the block's end)
    auto at = [&](int64_t idx) -> int64_t { return ((dir ? c1 - 1 - idx : c0 + idx) * 2 + dir) * NCH + c; };
    V sum = Pol::zero();
    for (int64_t i = 0; i < chunk; ++i) {
        const int64_t idx = lane * chunk + i;
        if (idx < len) sum = Pol::add(sum, totals[at(idx)]);
    }
    V incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = shfl_up_t(incl, o, 32);
        if (lane >= o) incl = Pol::add(y, incl);
    }
    V run = shfl_up_t(incl, 1, 32);
    if (lane == 0) run = Pol::zero();
    for (int64_t i = 0; i < chunk; ++i) {
        const int64_t idx = lane * chunk + i;
        if (idx < len) {
            carries[at(idx)] = run;
            run = Pol::add(run, totals[at(idx)]);
        }
    }
}

}  // namespace dc
}  // namespace fk
