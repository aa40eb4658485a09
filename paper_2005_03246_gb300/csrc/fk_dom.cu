// fk_dom.cu -- exact orthant counts at the sample points by inclusion-exclusion
// over single-orthant dominance counts.
//
// With y == 1 every orthant sum is an integer count, so the 2^d orthants of
// eq. (ECDFdelta) follow exactly from the "<= on every axis of A" counts
//     C_A(t) = #{ sources s : x_k(s) <= z_k(t) for all k in A },  A subset of axes,
// by inclusion-exclusion: with pos(o) the axes tested with <= and neg(o) those
// tested with >,  S_o(t) = sum_{T subset neg(o)} (-1)^{|T|} C_{pos(o) u T}(t),
// and C_{} = N.  |A| = 1 is a rank count; |A| >= 2 is the dominance problem of
// Sec. 2.2 (Algorithms 2-5) in |A| dimensions, needing only the sources that
// lie below the target on every axis (a single channel, forward only).
//
// The dominance engine is the same nested merge-sort formulation as fk_dc.cuh
// but carries, with every item, the number of "active" sources before it in
// its current run (pref) and the count it has received so far (acc).  At a
// merge of runs C and D, an element at merged position p has i(p) elements of
// C and j(p) of D before it, so its new prefix is pref_C[i] + pref_D[j], and a
// target from D receives pref_C[i] -- both lookups, no scan.  Active sources
// are sources on the lower side of every enclosing axis (class 0); receiving
// targets are targets on the upper side of every enclosing axis (class all
// ones) and in D.
#include <algorithm>

#include "fk_dc_ops.cuh"

namespace fk {
namespace dom {

using dc::kItemBits;
using dc::kItemMask;
using dc::merge_path;
using dc::SAcc;
using dc::GAcc;
using dc::ClassSpecK;
using dc::class_of_k;

// Shared-memory index padding: one spare word per 32 makes the stride-8 access
// pattern of "each thread owns 8 consecutive outputs" free of bank conflicts.
__device__ __forceinline__ int pd(int p) { return p + (p >> 5); }
struct SAccP {
    const uint32_t* p;
    int base;
    __device__ uint32_t operator()(int64_t i) const { return p[pd(base + (int)i)]; }
};

// Item roles: flat (sources [0, n_src), targets [tgt_off, tgt_off + n_tgt)) or
// batched segments as in dc::ItemMap.
struct Items {
    int64_t n_src, tgt_off, n_tgt;
    uint32_t full;      // class value of a receiving target (all enclosing bits set)
    const int64_t* seg;
    int segE;
    __device__ __forceinline__ bool is_src(uint32_t it) const {
        if (!seg) return (int64_t)it < n_src;
        return (int64_t)(it & ((1u << segE) - 1u)) < seg[4 * (int64_t)(it >> segE)];
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
    __device__ __forceinline__ bool src_active(uint32_t meta) const {
        return (meta >> kItemBits) == 0u && is_src(meta & kItemMask);
    }
    __device__ __forceinline__ bool tgt_active(uint32_t meta) const {
        return (meta >> kItemBits) == full && is_tgt(meta & kItemMask);
    }
};

// One merge level of the propagated-prefix dominance merge on padded
// shared-memory arrays (key, meta, pref, acc): every thread produces NI
// consecutive outputs starting at p0.  The thread keeps the heads of both
// runs in registers -- key and prefix of C's next element (or C's total
// once C is exhausted) and the same for D -- so an output needs only its own
// meta and count from shared memory, plus the key and prefix of the head it
// advances.  An output's new prefix is always the sum of the two head
// prefixes; a receiving target from D adds C's head prefix (the active C
// sources merged before it, C first on equal keys).  Returns the outputs made.
// whole: the tile is one merged block whose C part is [0, wcl), D part
// [wcl, ln), and whose runs' totals (w_ct, w_dt) come from outside the tile
// (a global merge level with runs longer than a tile); otherwise the tile
// holds whole merged blocks of 2^(m+1).
template <int NI, class SrcF, class TgtF>
__device__ __forceinline__ int dom_merge_level(const uint32_t* ik, const uint32_t* imt, const uint32_t* ip,
                                               const uint32_t* ia, int ln, int m, int p0, uint32_t (&ok)[NI],
                                               uint32_t (&om)[NI], uint32_t (&op)[NI], uint32_t (&oa)[NI],
                                               SrcF src_active, TgtF tgt_active, bool whole = false, int wcl = 0,
                                               uint32_t w_ct = 0, uint32_t w_dt = 0) {
    const int R = whole ? 0 : 1 << m, R2 = whole ? 1 : 2 << m;
    int bsl = 0, cl = 0, dl = 0, i = 0, j = 0, cnt = 0;
    uint32_t ctot = 0, dtot = 0, kc = 0, kd = 0, pcv = 0, pdv = 0;
#pragma unroll
    for (int e = 0; e < NI; ++e) {
        const int p = p0 + e;
        if (p < ln) {
            if (e == 0 || (!whole && (p % R2) == 0)) {
                if (whole) {
                    bsl = 0; cl = wcl; dl = ln - wcl;
                    ctot = w_ct; dtot = w_dt;
                } else {
                    bsl = (p / R2) * R2;
                    cl = min(R, ln - bsl);
                    dl = min(R2, ln - bsl) - cl;
                    ctot = ip[pd(bsl + cl - 1)] + (src_active(imt[pd(bsl + cl - 1)]) ? 1u : 0u);
                    dtot = dl > 0 ? ip[pd(bsl + cl + dl - 1)] + (src_active(imt[pd(bsl + cl + dl - 1)]) ? 1u : 0u) : 0u;
                }
                SAccP A{ik, bsl}, B{ik, bsl + cl};
                i = (int)merge_path(A, cl, B, dl, p - bsl);
                j = (p - bsl) - i;
                kc = (i < cl) ? ik[pd(bsl + i)] : 0u;
                pcv = (i < cl) ? ip[pd(bsl + i)] : ctot;
                kd = (j < dl) ? ik[pd(bsl + cl + j)] : 0u;
                pdv = (j < dl) ? ip[pd(bsl + cl + j)] : dtot;
            }
            const bool tc = (i < cl) && (j >= dl || kc <= kd);
            const int s = tc ? pd(bsl + i) : pd(bsl + cl + j);
            const uint32_t mt = imt[s], ac = ia[s];
            ok[e] = tc ? kc : kd;
            om[e] = mt;
            op[e] = pcv + pdv;
            oa[e] = ac + ((!tc && tgt_active(mt)) ? pcv : 0u);
            // advance the head that was taken
            i += tc ? 1 : 0;
            j += tc ? 0 : 1;
            const bool v = tc ? (i < cl) : (j < dl);
            const int q = tc ? pd(bsl + i) : pd(bsl + cl + j);
            const uint32_t nk = v ? ik[q] : 0u;
            const uint32_t np = v ? ip[q] : (tc ? ctot : dtot);
            kc = tc ? nk : kc;
            pcv = tc ? np : pcv;
            kd = tc ? kd : nk;
            pdv = tc ? pdv : np;
            cnt = e + 1;
        }
    }
    return cnt;
}

constexpr int LNT = 256;          // threads of the tile-local kernel (tiles of 1024, 2048 or 4096 items)

// Tile-local merge levels.  Input: the enclosing state (items sorted by the
// tree axis inside their nodes); output (if more levels follow): key, meta,
// pref, acc in merged order; otherwise the received counts are flushed.
template <int LT>
__global__ void __launch_bounds__(LNT) k_dom_local(const uint32_t* __restrict__ seq, int64_t n,
                                                   const uint32_t* __restrict__ P0, ClassSpecK cs, int levels,
                                                   Items im, uint32_t* __restrict__ key_out,
                                                   uint32_t* __restrict__ meta_out, uint32_t* __restrict__ pref_out,
                                                   uint32_t* __restrict__ acc_out, int write_out,
                                                   uint32_t* __restrict__ C) {
    constexpr int LIT = LT / LNT;      // items per thread
    extern __shared__ __align__(16) uint32_t s_dyn[];
    constexpr int LP = LT + LT / 32;   // padded row
    uint32_t(*s_key)[LP] = reinterpret_cast<uint32_t(*)[LP]>(s_dyn);
    uint32_t(*s_meta)[LP] = reinterpret_cast<uint32_t(*)[LP]>(s_dyn + 2 * LP);
    uint32_t(*s_pref)[LP] = reinterpret_cast<uint32_t(*)[LP]>(s_dyn + 4 * LP);
    uint32_t(*s_acc)[LP] = reinterpret_cast<uint32_t(*)[LP]>(s_dyn + 6 * LP);
    const int64_t t0 = (int64_t)blockIdx.x * LT;
    const int ln = (int)min((int64_t)LT, n - t0);
    {
        uint32_t it[LIT];
#pragma unroll
        for (int e = 0; e < LIT; ++e) {
            const int i = threadIdx.x + e * LNT;
            it[e] = (i < ln) ? seq[t0 + i] : 0u;
        }
        uint32_t kk[LIT], cc[LIT];
#pragma unroll
        for (int e = 0; e < LIT; ++e) {
            const int i = threadIdx.x + e * LNT;
            if (i < ln) { kk[e] = P0[it[e]]; cc[e] = class_of_k(cs, it[e]); }
        }
#pragma unroll
        for (int e = 0; e < LIT; ++e) {
            const int i = threadIdx.x + e * LNT;
            if (i < ln) {
                s_key[0][pd(i)] = kk[e];
                s_meta[0][pd(i)] = it[e] | (cc[e] << kItemBits);
                s_pref[0][pd(i)] = 0u;
                s_acc[0][pd(i)] = 0u;
            }
        }
    }
    __syncthreads();
    int b = 0;
    for (int m = 0; m < levels; ++m) {
        uint32_t ok[LIT], om[LIT], op[LIT], oa[LIT];
        const int p0 = threadIdx.x * LIT;
        const int cnt = dom_merge_level<LIT>(s_key[b], s_meta[b], s_pref[b], s_acc[b], ln, m, p0, ok, om, op, oa,
                                            [&](uint32_t mt) { return im.src_active(mt); },
                                            [&](uint32_t mt) { return im.tgt_active(mt); });
        __syncthreads();
#pragma unroll
        for (int e = 0; e < LIT; ++e) {
            if (e < cnt) {
                const int p = pd(p0 + e);
                s_key[b ^ 1][p] = ok[e];
                s_meta[b ^ 1][p] = om[e];
                s_pref[b ^ 1][p] = op[e];
                s_acc[b ^ 1][p] = oa[e];
            }
        }
        __syncthreads();
        b ^= 1;
    }
    for (int i = threadIdx.x; i < ln; i += LNT) {
        const uint32_t m = s_meta[b][pd(i)];
        if (write_out) {
            key_out[t0 + i] = s_key[b][pd(i)];
            meta_out[t0 + i] = m;
            pref_out[t0 + i] = s_pref[b][pd(i)];
            acc_out[t0 + i] = s_acc[b][pd(i)];
        } else if (s_acc[b][pd(i)]) {
            atomicAdd(C + im.tgt_index(m & kItemMask), s_acc[b][pd(i)]);
        }
    }
}

// ------------------------------------------------------------------ nested tile levels
// For the outermost-but-one tree axis (axis index 2 of the subset): every
// outer level l whose nodes (2^{l+1} items) fit in a tile of NTT items is done
// inside one CTA -- the outer merge by P_1 (the tree of Algorithm 3/4) and,
// for each l, the complete inner dominance sort of that level -- with the
// received counts summed per item in shared memory and flushed once.  The
// side bit of axis 2 at level l is bit l of the item's slot in the tile
// (tiles start at multiples of NTT inside the enclosing nodes).
constexpr int NTT = 1024;          // items per tile
constexpr int NTN = 256;           // threads
constexpr int NTI = NTT / NTN;     // items per thread
constexpr int NTP = NTT + NTT / 32; // padded row

struct DomSmem {
    uint32_t* key;     // [2][NTT]
    uint32_t* meta;    // [2][NTT]  slot | class << 16
    uint32_t* pref;    // [2][NTT]
    uint32_t* acc;     // [2][NTT]
};

// One merge level (runs 2^m -> 2^{m+1}) of the propagated-prefix dominance
// merge on shared-memory state.  Activity of an element is decided from its
// slot and class bits through the two predicates.
template <class SrcF, class TgtF>
__device__ __forceinline__ void dom_level_smem(DomSmem S, int b, int ln, int m, SrcF src_active, TgtF tgt_active) {
    uint32_t ok[NTI], om[NTI], op[NTI], oa[NTI];
    const int p0 = threadIdx.x * NTI;
    const int cnt = dom_merge_level<NTI>(S.key + b * NTP, S.meta + b * NTP, S.pref + b * NTP, S.acc + b * NTP, ln, m,
                                         p0, ok, om, op, oa, src_active, tgt_active);
    uint32_t* wk = S.key + (b ^ 1) * NTP;
    uint32_t* wm = S.meta + (b ^ 1) * NTP;
    uint32_t* wp = S.pref + (b ^ 1) * NTP;
    uint32_t* wa = S.acc + (b ^ 1) * NTP;
#pragma unroll
    for (int e = 0; e < NTI; ++e) {
        if (e < cnt) {
            const int p = pd(p0 + e);
            wk[p] = ok[e]; wm[p] = om[e]; wp[p] = op[e]; wa[p] = oa[e];
        }
    }
}

// Plain merge level on (key, slot) pairs in shared memory.
__device__ __forceinline__ void plain_level_smem(const uint32_t* ik, const uint32_t* ih, uint32_t* wk, uint32_t* wh,
                                                 int ln, int m) {
    const int R = 1 << m, R2 = 2 << m;
    uint32_t ok[NTI], oh[NTI];
    int cnt = 0;
    const int p0 = threadIdx.x * NTI;
    int bsl = 0, cl = 0, dl = 0, i = 0, j = 0;
#pragma unroll
    for (int e = 0; e < NTI; ++e) {
        const int p = p0 + e;
        if (p < ln) {
            if (e == 0 || (p % R2) == 0) {
                bsl = (p / R2) * R2;
                cl = min(R, ln - bsl);
                dl = min(R2, ln - bsl) - cl;
                SAccP A{ik, bsl}, B{ik, bsl + cl};
                i = (int)merge_path(A, cl, B, dl, p - bsl);
                j = (p - bsl) - i;
            }
            const bool takeC = (i < cl) && (j >= dl || ik[pd(bsl + i)] <= ik[pd(bsl + cl + j)]);
            const int s = takeC ? pd(bsl + i) : pd(bsl + cl + j);
            ok[e] = ik[s];
            oh[e] = ih[s];
            if (takeC) ++i; else ++j;
            cnt = e + 1;
        }
    }
#pragma unroll
    for (int e = 0; e < NTI; ++e)
        if (e < cnt) { wk[pd(p0 + e)] = ok[e]; wh[pd(p0 + e)] = oh[e]; }
}

__global__ void __launch_bounds__(NTN) k_dom_nested(const uint32_t* __restrict__ seq, int64_t n,
                                                    const uint32_t* __restrict__ P0, const uint32_t* __restrict__ P1,
                                                    ClassSpecK cs, int levels, Items im,
                                                    uint32_t* __restrict__ okey_out, uint32_t* __restrict__ oitem_out,
                                                    uint32_t* __restrict__ C) {
    extern __shared__ __align__(16) uint32_t s_dyn[];
    uint32_t* s_item = s_dyn;                 // [NTT] items of the tile (slot -> item)
    uint32_t* s_p0 = s_item + NTT;            // [NTT] P_0 by slot
    uint32_t* s_cenc = s_p0 + NTT;            // [NTT] enclosing class bits by slot (bits >= 1)
    uint32_t* s_sum = s_cenc + NTT;           // [NTT] received counts by slot
    uint32_t* s_okey = s_sum + NTT;           // [2][NTP] outer state: P_1 (padded positions)
    uint32_t* s_oslot = s_okey + 2 * NTP;     // [2][NTP] outer state: slot
    DomSmem S{s_oslot + 2 * NTP, s_oslot + 4 * NTP, s_oslot + 6 * NTP, s_oslot + 8 * NTP};
    const int64_t t0 = (int64_t)blockIdx.x * NTT;
    const int ln = (int)min((int64_t)NTT, n - t0);
    {
        uint32_t it[NTI];
#pragma unroll
        for (int e = 0; e < NTI; ++e) {
            const int i = threadIdx.x + e * NTN;
            it[e] = (i < ln) ? seq[t0 + i] : 0u;
        }
        uint32_t a0[NTI], a1[NTI], ce[NTI];
#pragma unroll
        for (int e = 0; e < NTI; ++e) {
            const int i = threadIdx.x + e * NTN;
            if (i < ln) {
                a0[e] = P0[it[e]];
                a1[e] = P1[it[e]];
                uint32_t c = 0;
                for (int q = 1; q < cs.nb; ++q) c |= ((cs.idx[q][it[e]] >> cs.lvl[q]) & 1u) << q;
                ce[e] = c;
            }
        }
#pragma unroll
        for (int e = 0; e < NTI; ++e) {
            const int i = threadIdx.x + e * NTN;
            if (i < ln) {
                s_item[i] = it[e]; s_p0[i] = a0[e]; s_cenc[i] = ce[e]; s_sum[i] = 0u;
                s_okey[pd(i)] = a1[e]; s_oslot[pd(i)] = (uint32_t)i;
            }
        }
    }
    __syncthreads();
    const int nbt = cs.nb > 1 ? cs.nb : 1;
    const uint32_t full = (1u << nbt) - 1u;
    auto src_active = [&](uint32_t mt) { return (mt >> 16) == 0u && im.is_src(s_item[mt & 0xffffu]); };
    auto tgt_active = [&](uint32_t mt) { return (mt >> 16) == full && im.is_tgt(s_item[mt & 0xffffu]); };
    int ob = 0;
    for (int l = 0; l < levels; ++l) {
        plain_level_smem(s_okey + ob * NTP, s_oslot + ob * NTP, s_okey + (ob ^ 1) * NTP, s_oslot + (ob ^ 1) * NTP, ln, l);
        __syncthreads();
        ob ^= 1;
        // inner sort of level l: nodes of 2^{l+1} sorted by P_1, merged by P_0
        for (int p = threadIdx.x; p < ln; p += NTN) {
            const uint32_t sl = s_oslot[ob * NTP + pd(p)];
            const uint32_t cls = ((sl >> l) & 1u) | s_cenc[sl];
            S.key[pd(p)] = s_p0[sl];
            S.meta[pd(p)] = sl | (cls << 16);
            S.pref[pd(p)] = 0u;
            S.acc[pd(p)] = 0u;
        }
        __syncthreads();
        int b = 0;
        for (int m = 0; m <= l; ++m) {
            dom_level_smem(S, b, ln, m, src_active, tgt_active);
            __syncthreads();
            b ^= 1;
        }
        for (int p = threadIdx.x; p < ln; p += NTN) {
            const uint32_t a = S.acc[b * NTP + pd(p)];
            if (a) s_sum[S.meta[b * NTP + pd(p)] & 0xffffu] += a;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ln; i += NTN) {
        okey_out[t0 + i] = s_okey[ob * NTP + pd(i)];
        oitem_out[t0 + i] = s_item[s_oslot[ob * NTP + pd(i)]];
        const uint32_t a = s_sum[i];
        if (a) atomicAdd(C + im.tgt_index(s_item[i]), a);
    }
}

constexpr int GT = 256, GI = 4, GTILE = GT * GI;

// One global merge level with propagated prefixes.  The last level flushes
// the received counts instead of writing the state.
__global__ void __launch_bounds__(GT) k_dom_merge(const uint32_t* __restrict__ key_in, const uint32_t* __restrict__ meta_in,
                                                  const uint32_t* __restrict__ pref_in, const uint32_t* __restrict__ acc_in,
                                                  uint32_t* __restrict__ key_out, uint32_t* __restrict__ meta_out,
                                                  uint32_t* __restrict__ pref_out, uint32_t* __restrict__ acc_out,
                                                  int64_t n, int logR, Items im, int last, uint32_t* __restrict__ C) {
    constexpr int GP = GTILE + GTILE / 32 + 2;   // padded tile
    __shared__ uint32_t s_key[GP], s_meta[GP], s_pref[GP], s_acc[GP];
    __shared__ int64_t s_co[6];
    const int64_t R = (int64_t)1 << logR, R2 = R << 1;
    const int64_t o0 = (int64_t)blockIdx.x * GTILE;
    if (o0 >= n) return;
    const int64_t o1 = min(o0 + (int64_t)GTILE, n);
    const int ln = (int)(o1 - o0);
    // Runs are at least one tile long here (R2 > GTILE is not required: when a
    // tile holds several merged blocks each block is handled from smem).
    const bool big = R2 > GTILE;
    int lc = 0, ldd = 0;
    uint32_t cnext = 0, dnext = 0;
    if (big) {
        if (threadIdx.x < 64) {
            const int64_t bs = (o0 / R2) * R2;
            const int64_t cl = min(R, n - bs);
            const int64_t dl = max((int64_t)0, min(R2, n - bs) - cl);
            const int64_t q0 = o0 - bs, q1 = o1 - bs;
            const int64_t iq = dc::merge_path_warp(key_in + bs, cl, key_in + bs + cl, dl, threadIdx.x < 32 ? q0 : q1);
            if (threadIdx.x == 0) s_co[0] = iq;
            if (threadIdx.x == 32) s_co[1] = iq;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t bs = (o0 / R2) * R2;
            const int64_t cl = min(R, n - bs);
            const int64_t dl = max((int64_t)0, min(R2, n - bs) - cl);
            const int64_t q0 = o0 - bs, q1 = o1 - bs;
            const int64_t i0 = s_co[0], i1 = s_co[1];
            s_co[0] = bs + i0;
            s_co[1] = i1 - i0;
            s_co[2] = bs + cl + (q0 - i0);
            s_co[3] = (q1 - i1) - (q0 - i0);
            // prefix just past each loaded range (the next element's, or the run total)
            const int64_t cend = bs + i1, dend = bs + cl + (q1 - i1);
            const uint32_t ct = pref_in[bs + cl - 1] + (im.src_active(meta_in[bs + cl - 1]) ? 1u : 0u);
            const uint32_t dt = dl > 0 ? pref_in[bs + cl + dl - 1] + (im.src_active(meta_in[bs + cl + dl - 1]) ? 1u : 0u) : 0u;
            s_co[4] = (cend < bs + cl) ? pref_in[cend] : ct;
            s_co[5] = (dend < bs + cl + dl) ? pref_in[dend] : dt;
        }
        __syncthreads();
        lc = (int)s_co[1];
        ldd = (int)s_co[3];
        cnext = (uint32_t)s_co[4];
        dnext = (uint32_t)s_co[5];
    }
    {
        // Tile slot i holds C element i (i < lc) or D element i - lc of a long
        // run, else element o0 + i.  Asynchronous copies: every thread has all
        // its slots in flight at once (one memory round trip per tile).
        const int64_t cs = big ? s_co[0] : 0, ds = big ? s_co[2] : 0;
#pragma unroll
        for (int j = 0; j < GI; ++j) {
            const int i = (int)threadIdx.x + j * GT;
            const int64_t g = !big ? o0 + i : (i < lc ? cs + i : ds + (i - lc));
            if (i < ln) {
                const int q = pd(i);
                dc::cp_async4(&s_key[q], &key_in[g]);
                dc::cp_async4(&s_meta[q], &meta_in[g]);
                dc::cp_async4(&s_pref[q], &pref_in[g]);
                dc::cp_async4(&s_acc[q], &acc_in[g]);
            }
        }
        dc::cp_async_commit();
        dc::cp_async_wait_all();
    }
    __syncthreads();
    const int p0 = threadIdx.x * GI;
    uint32_t rk[GI], rm[GI], rp[GI], ra[GI];
    const int cnt = dom_merge_level<GI>(s_key, s_meta, s_pref, s_acc, ln, big ? 0 : logR, p0, rk, rm, rp, ra,
                                        [&](uint32_t mt) { return im.src_active(mt); },
                                        [&](uint32_t mt) { return im.tgt_active(mt); }, big, lc, cnext, dnext);
    if (last) {
#pragma unroll
        for (int e = 0; e < GI; ++e)
            if (e < cnt && ra[e]) atomicAdd(C + im.tgt_index(rm[e] & kItemMask), ra[e]);
    }
    if (last) return;
    const int64_t ob = o0 + p0;
    if (cnt == GI) {
        // GI consecutive outputs per thread: GI / 4 16-byte stores per array
        uint4* a = reinterpret_cast<uint4*>(key_out + ob);
        uint4* b = reinterpret_cast<uint4*>(meta_out + ob);
        uint4* c = reinterpret_cast<uint4*>(pref_out + ob);
        uint4* dd = reinterpret_cast<uint4*>(acc_out + ob);
#pragma unroll
        for (int v = 0; v < GI / 4; ++v) {
            a[v] = make_uint4(rk[4 * v], rk[4 * v + 1], rk[4 * v + 2], rk[4 * v + 3]);
            b[v] = make_uint4(rm[4 * v], rm[4 * v + 1], rm[4 * v + 2], rm[4 * v + 3]);
            c[v] = make_uint4(rp[4 * v], rp[4 * v + 1], rp[4 * v + 2], rp[4 * v + 3]);
            dd[v] = make_uint4(ra[4 * v], ra[4 * v + 1], ra[4 * v + 2], ra[4 * v + 3]);
        }
    } else {
        for (int e = 0; e < cnt; ++e) {
            key_out[ob + e] = rk[e]; meta_out[ob + e] = rm[e]; pref_out[ob + e] = rp[e]; acc_out[ob + e] = ra[e];
        }
    }
}

// rank counts: C_k(t) = number of sources before target t in the axis-k order
__global__ void k_src_flags(const uint32_t* __restrict__ P, int64_t n, Items im, uint32_t* __restrict__ f) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n) f[P[it]] = im.is_src((uint32_t)it) ? 1u : 0u;
}
// (the count restarts at every segment of 2^E positions in the batched layout)
__global__ void k_rank_counts(const uint32_t* __restrict__ P, const uint32_t* __restrict__ scanned, int64_t n,
                              Items im, int E, uint32_t* __restrict__ C) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n || !im.is_tgt((uint32_t)it)) return;
    const uint32_t p = P[it];
    const uint32_t s0 = (E >= 32) ? 0u : ((p >> E) << E);
    C[im.tgt_index((uint32_t)it)] = scanned[p] - scanned[s0];
}
__global__ void k_seq_from_pos(const uint32_t* __restrict__ P, int64_t n, uint32_t* __restrict__ seq) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n) seq[P[it]] = (uint32_t)it;
}

struct CTab { const uint32_t* c[256]; };   // C_A for every subset A of the d <= 8 axes (A as a bitmask)

// Orthant o: sum over subsets T of neg(o) of (-1)^|T| C_{pos(o) | T}.
// self_add: 1 when the targets are the sources themselves, held as one item
// each (the engine never pairs an item with itself), else 0.
__global__ void k_combine(CTab ct, int d, int64_t n_tgt, uint32_t n_src, uint32_t self_add, dc::SelMap sel,
                          int64_t* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    const uint32_t full = (1u << d) - 1u;
    for (int r = 0; r < sel.n; ++r) {
        const uint32_t o = (uint32_t)sel.o[r];
        const uint32_t pos = full & ~o, neg = o;
        int64_t s = 0;
        // enumerate the subsets T of neg
        uint32_t T = 0;
        while (true) {
            const uint32_t A = pos | T;
            const int64_t v = (A == 0) ? (int64_t)n_src : (int64_t)ct.c[A][t] + self_add;
            s += (__popc(T) & 1) ? -v : v;
            if (T == neg) break;
            T = (T - neg) & neg;
        }
        out[(int64_t)r * n_tgt + t] = s;
    }
}

// Batched combine: target t of dataset b (tbase[b] <= t < tbase[b+1]) writes
// orthant o to out[obase[b] + o * n_b + (t - tbase[b])].
__global__ void k_combine_seg(CTab ct, int d, int64_t n_tgt, const int64_t* __restrict__ seg, int segE,
                              BatchOut bo, int64_t* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    int lo = 0, hi = bo.nb;                 // dataset of t: last b with tbase[b] <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bo.tbase[mid] <= t) lo = mid; else hi = mid;
    }
    const int b = lo;
    const int64_t nb = bo.tbase[b + 1] - bo.tbase[b];
    const int64_t loc = t - bo.tbase[b];
    const int64_t nsrc = seg[4 * (int64_t)b];
    const uint32_t full = (1u << d) - 1u;
    for (uint32_t o = 0; o <= full; ++o) {
        const uint32_t pos = full & ~o, neg = o;
        int64_t s = 0;
        uint32_t T = 0;
        while (true) {
            const uint32_t A = pos | T;
            const int64_t v = (A == 0) ? nsrc : (int64_t)ct.c[A][t];
            s += (__popc(T) & 1) ? -v : v;
            if (T == neg) break;
            T = (T - neg) & neg;
        }
        out[bo.obase[b] + (int64_t)o * nb + loc] = s;
    }
}

}  // namespace dom

using namespace dom;

// Streams for the independent dominance problems of one orthant-count call,
// and for the concurrent levels of tree axis 2 inside one problem.
constexpr int kCountStreams = 4;
constexpr int kLevelStreams = 4;

// Dominance count C_A for the axes in `axes` (sorted, size k >= 2): the
// innermost merge sort over the second axis by the first, nested inside merge
// sorts of the outer axes, as in fk_dc_drv.cuh.
struct DomInner {          // state of one innermost sort (ping-pong)
    uint32_t* k[2];
    uint32_t* m[2];
    uint32_t* p[2];
    uint32_t* a[2];
};
struct DomBuf {
    DomInner in[kPoolStreams];               // one per stream of concurrent levels
    int S;                                   // streams for the levels of tree axis 2
    uint32_t* ok[8][kPoolStreams + 1];       // level states: ping-pong, or a ring of S + 1 at axis 2
    uint32_t* om[8][kPoolStreams + 1];
    uint32_t* idx[8];
};

template <int LT>
static fk_status dom_local_launch(const uint32_t* seq, int64_t n, int E, const uint32_t* P0, ClassSpecK cs, Items im,
                                  DomInner& B, uint32_t* C, int& L0, cudaStream_t st) {
    int lt = 0;
    while ((1 << (lt + 1)) <= LT) ++lt;
    L0 = E < lt ? E : lt;
    ProfScope ps(PF_LOCAL, 8.0 * n + 8.0 * n * (E > L0 ? 2 : 0) + 8.0 * im.n_tgt, st);
    constexpr int smem = 8 * (LT + LT / 32) * 4;
    static bool attr = false;
    if (!attr) {
        FK_CUDA(cudaFuncSetAttribute(k_dom_local<LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k_dom_local<LT><<<grid_for(n, LT), LNT, smem, st>>>(seq, n, P0, cs, L0, im, B.k[0], B.m[0], B.p[0], B.a[0],
                                                        E > L0 ? 1 : 0, C);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

static fk_status dom_inner(const uint32_t* seq, int64_t n, int E, const uint32_t* P0, ClassSpecK cs, Items im,
                           DomInner& B, uint32_t* C, int count_tile, cudaStream_t st) {
    int L0 = 0;
    if (count_tile == 1) FK_TRY(dom_local_launch<1024>(seq, n, E, P0, cs, im, B, C, L0, st));
    else if (count_tile == 2) FK_TRY(dom_local_launch<4096>(seq, n, E, P0, cs, im, B, C, L0, st));
    else FK_TRY(dom_local_launch<2048>(seq, n, E, P0, cs, im, B, C, L0, st));
    int cur = 0;
    for (int m = L0; m < E; ++m) {
        const int last = (m == E - 1);
        ProfScope ps(PF_MERGE_SWEEP, 16.0 * n + (last ? 8.0 * im.n_tgt : 16.0 * n), st);
        k_dom_merge<<<grid_for(n, GTILE), GT, 0, st>>>(B.k[cur], B.m[cur], B.p[cur], B.a[cur], B.k[cur ^ 1],
                                                       B.m[cur ^ 1], B.p[cur ^ 1], B.a[cur ^ 1], n, m, im, last, C);
        FK_LAUNCH_CHECK();
        cur ^= 1;
    }
    return FK_OK;
}

static fk_status dom_recurse(int k, const uint32_t* seq, int64_t n, int E, const uint32_t* const* P, ClassSpecK cs,
                             Items im, DomBuf& B, uint32_t* C, int count_tile, cudaStream_t st) {
    if (k == 1) {
        Items it = im;
        it.full = (1u << cs.nb) - 1u;
        return dom_inner(seq, n, E, P[0], cs, it, B.in[0], C, count_tile, st);
    }
    const uint32_t* idx = P[k];
    if (B.idx[k]) {
        FK_TRY(dc::record_index(seq, n, E, B.idx[k], st));
        idx = B.idx[k];
    }
    int l0 = 0;
    if (k == 2) {
        // outer levels whose nodes fit in a tile: one nested launch
        int lt = 0;
        while ((1 << (lt + 1)) <= NTT) ++lt;
        l0 = E < lt ? E : lt;
        constexpr int smem = 4 * NTT * 4 + 4 * NTP * 4 + 8 * NTP * 4;
        static bool attr = false;
        if (!attr) {
            FK_CUDA(cudaFuncSetAttribute(k_dom_nested, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            attr = true;
        }
        ProfScope ps(PF_LOCAL, 16.0 * n + 8.0 * im.n_tgt, st);
        k_dom_nested<<<grid_for(n, NTT), NTN, smem, st>>>(seq, n, P[0], P[1], cs, l0, im, B.ok[k][0], B.om[k][0], C);
        FK_LAUNCH_CHECK();
    } else {
        FK_TRY(dc::gather_outer(seq, n, P[k - 1], B.ok[k][0], B.om[k][0], st));
    }
    auto class_of_level = [&](int l) {
        ClassSpecK c2 = cs;
        c2.idx[k - 2] = idx;
        c2.lvl[k - 2] = l;
        if (c2.nb < k - 1) c2.nb = k - 1;
        return c2;
    };
    if (k == 2 && B.S > 1) {
        // merges on the caller's stream ahead of the inner sorts, which run on
        // S forked streams (state per stream); level states in a ring of S + 1
        const int S = B.S, R = S + 1;
        StreamFork fork;
        FK_TRY(fork.begin(2, st, S));
        cudaEvent_t ready = fork.ev[0];
        cudaEvent_t* done = fork.ev + 1;
        fk_status rc = FK_OK;
        for (int l = l0; l < E && rc == FK_OK; ++l) {
            const int j = l - l0;
            const int in = j % R, out = (j + 1) % R;
            if (j >= R) {
                const cudaError_t e = cudaStreamWaitEvent(st, done[(j - R) % R], 0);
                if (e != cudaSuccess) { rc = cuda_error(e, "level wait"); break; }
            }
            dc::MergeArgs a{B.ok[k][in], B.om[k][in], B.ok[k][out], B.om[k][out], n, l};
            rc = dc::plain_merge_level(a, st);
            if (rc != FK_OK) break;
            const int q = j % S;
            cudaError_t e = cudaEventRecord(ready, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(fork.s[q], ready, 0);
            if (e != cudaSuccess) { rc = cuda_error(e, "level fork"); break; }
            ClassSpecK c2 = class_of_level(l);
            Items it = im;
            it.full = (1u << c2.nb) - 1u;
            rc = dom_inner(B.om[k][out], n, l + 1, P[0], c2, it, B.in[q], C, count_tile, fork.s[q]);
            if (rc != FK_OK) break;
            e = cudaEventRecord(done[j % R], fork.s[q]);
            if (e != cudaSuccess) rc = cuda_error(e, "level done");
        }
        const fk_status rj = fork.end();
        return rc != FK_OK ? rc : rj;
    }
    int cur = 0;
    for (int l = l0; l < E; ++l) {
        dc::MergeArgs a{B.ok[k][cur], B.om[k][cur], B.ok[k][cur ^ 1], B.om[k][cur ^ 1], n, l};
        FK_TRY(dc::plain_merge_level(a, st));
        cur ^= 1;
        FK_TRY(dom_recurse(k - 1, B.om[k][cur], n, l + 1, P, class_of_level(l), im, B, C, count_tile, st));
    }
    return FK_OK;
}

// Orthant counts of N sources at the targets from the positions P[0..d-1]
// (sources before targets on ties), by inclusion-exclusion.
// C_A for every non-empty subset A of the d axes (rank counts for |A| = 1,
// nested dominance for |A| >= 2); E levels of the outermost merge sort.
// The dominance problems of the subsets with |A| >= 2 are independent: with
// streams > 1 they run concurrently on forked streams, each stream with its
// own engine buffers.
// Subsets A of the d axes (bitmasks) whose counts C_A an orthant selection
// needs: orthant o reads C_{pos(o) | T} for every subset T of neg(o).
struct SubsetSet {
    uint32_t w[8];
    bool has(int A) const { return (w[A >> 5] >> (A & 31)) & 1u; }
};
static SubsetSet subsets_for(int d, const uint32_t* mask) {
    SubsetSet ss = {};
    const uint32_t full = (1u << d) - 1u;
    for (int o = 0; o < (1 << d); ++o) {
        if (mask && !((mask[o >> 5] >> (o & 31)) & 1u)) continue;
        const uint32_t pos = full & ~(uint32_t)o, neg = (uint32_t)o;
        uint32_t T = 0;
        while (true) {
            const uint32_t A = pos | T;
            ss.w[A >> 5] |= 1u << (A & 31);
            if (T == neg) break;
            T = (T - neg) & neg;
        }
    }
    return ss;
}

static fk_status dom_counts_core(int d, int64_t n, Items im, int E, const uint32_t* const* P, uint32_t** Cs,
                                 Arena& ar, cudaStream_t st, int count_tile = 0, int streams = 1,
                                 const SubsetSet* need = nullptr) {
    const int nsub = 1 << d;
    const int64_t n_tgt = im.n_tgt;
    int nbig = 0;
    for (int A = 1; A < nsub; ++A) {
        Cs[A] = nullptr;
        if (need && !need->has(A)) continue;      // no selected orthant reads C_A
        Cs[A] = ar.take<uint32_t>((size_t)n_tgt);
        if (__builtin_popcount((unsigned)A) >= 2) ++nbig;
    }
    const int S = std::max(1, std::min(streams, std::min(nbig, kPoolStreams)));
    // levels of tree axis 2 sorted concurrently (subsets with |A| >= 3)
    const int SL = (streams > 1 && d >= 3) ? kLevelStreams : 1;
    DomBuf B[kPoolStreams] = {};
    uint32_t* seq[kPoolStreams] = {};
    for (int q = 0; q < S; ++q) {
        B[q].S = SL;
        for (int s2 = 0; s2 < SL; ++s2)
            for (int r = 0; r < 2; ++r) {
                B[q].in[s2].k[r] = ar.take<uint32_t>(n); B[q].in[s2].m[r] = ar.take<uint32_t>(n);
                B[q].in[s2].p[r] = ar.take<uint32_t>(n); B[q].in[s2].a[r] = ar.take<uint32_t>(n);
            }
        for (int k = 2; k < d; ++k) {
            const int nb = (k == 2 && SL > 1) ? SL + 1 : 2;
            for (int r = 0; r < nb; ++r) { B[q].ok[k][r] = ar.take<uint32_t>(n); B[q].om[k][r] = ar.take<uint32_t>(n); }
            B[q].idx[k] = ar.take<uint32_t>(n);
        }
        seq[q] = ar.take<uint32_t>(n);
    }
    uint32_t* flags = ar.take<uint32_t>(n);
    uint32_t* scanned = ar.take<uint32_t>(n);
    uint32_t* stmp = ar.take<uint32_t>(scan_u32_tmp_words(n));
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (orthant counts)");
    for (int A = 1; A < nsub; ++A)
        if (Cs[A]) FK_CUDA(cudaMemsetAsync(Cs[A], 0, (size_t)n_tgt * 4, st));
    const unsigned g = grid_for(n, 256);
    // rank counts (|A| = 1) on the caller's stream
    for (int A = 1; A < nsub; ++A) {
        if (__builtin_popcount((unsigned)A) != 1 || !Cs[A]) continue;
        const uint32_t* PA = P[__builtin_ctz((unsigned)A)];
        k_src_flags<<<g, 256, 0, st>>>(PA, n, im, flags);
        FK_LAUNCH_CHECK();
        FK_TRY(scan_u32_exclusive(flags, scanned, n, stmp, st));
        k_rank_counts<<<g, 256, 0, st>>>(PA, scanned, n, im, E, Cs[A]);
        FK_LAUNCH_CHECK();
    }
    StreamFork fork;
    FK_TRY(fork.begin(1, st, S));
    fk_status rc = FK_OK;
    int j = 0;
    for (int A = 1; A < nsub && rc == FK_OK; ++A) {
        const int k = __builtin_popcount((unsigned)A);
        if (k < 2 || !Cs[A]) continue;
        const int q = j++ % S;
        cudaStream_t ss = fork.s[q];
        const uint32_t* PA[8];
        int c = 0;
        for (int a = 0; a < d; ++a)
            if ((A >> a) & 1) PA[c++] = P[a];
        // items in the order of the outermost axis of A
        k_seq_from_pos<<<g, 256, 0, ss>>>(PA[k - 1], n, seq[q]);
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) { rc = cuda_error(le, "k_seq_from_pos"); break; }
        note_launch();
        DomBuf BB = B[q];
        for (int kk = 2; kk < 8; ++kk) BB.idx[kk] = (kk < k - 1) ? B[q].idx[kk] : nullptr;
        ClassSpecK cs = {};
        rc = dom_recurse(k - 1, seq[q], n, E, PA, cs, im, BB, Cs[A], count_tile, ss);
    }
    const fk_status rj = fork.end();
    return rc != FK_OK ? rc : rj;
}

fk_status dom_orthant_counts(int d, int64_t n, int64_t n_src, int64_t tgt_off, int64_t n_tgt,
                             const uint32_t* const* P, const uint32_t* mask, int64_t* out, Arena& ar,
                             cudaStream_t st) {
    const int nsub = 1 << d;
    uint32_t* Cs[256] = {};
    Items im{n_src, tgt_off, n_tgt, 0u, nullptr, 0};
    const SubsetSet need = subsets_for(d, mask);
    FK_TRY(dom_counts_core(d, n, im, dc::ceil_log2(n), P, Cs, ar, st, 0, kCountStreams, &need));
    if (ar.sizing) return FK_OK;
    dc::SelMap sel;
    sel.n = 0;
    for (int o = 0; o < nsub; ++o)
        if (!mask || ((mask[o >> 5] >> (o & 31)) & 1u)) sel.o[sel.n++] = o;
    if (sel.n == 0 || n_tgt == 0) return FK_OK;
    CTab ct = {};
    for (int A = 1; A < nsub; ++A) ct.c[A] = Cs[A];
    k_combine<<<grid_for(n_tgt, 256), 256, 0, st>>>(ct, d, n_tgt, (uint32_t)n_src, 0u, sel, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

fk_status dom_orthant_counts_seg(int d, int64_t n, const int64_t* seg, int segE, int64_t n_tgt,
                                 const uint32_t* const* P, BatchOut bo, int64_t* out, Arena& ar,
                                 cudaStream_t st, int count_tile) {
    const int nsub = 1 << d;
    uint32_t* Cs[256] = {};
    Items im{0, 0, n_tgt, 0u, seg, segE};
    FK_TRY(dom_counts_core(d, n, im, segE, P, Cs, ar, st, count_tile));
    if (ar.sizing || n_tgt == 0) return FK_OK;
    CTab ct = {};
    for (int A = 1; A < nsub; ++A) ct.c[A] = Cs[A];
    k_combine_seg<<<grid_for(n_tgt, 256), 256, 0, st>>>(ct, d, n_tgt, seg, segE, bo, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}


// ------------------------------------------------------------------ one item per sample point
// At the sample points every point can be a single item that is both a
// source and a target (half the items of the source/target-copy layout);
// the ties this misses are corrected by tie_fix_counts (fk_ties.cu).
fk_status dom_self_counts(int d, int64_t n, const uint32_t* const* P, const void* x, fk_dtype xd,
                          const uint32_t* mask, int64_t* out, Arena& ar, cudaStream_t st, bool* fallback) {
    const int nsub = 1 << d;
    uint32_t* sorted = ar.take<uint32_t>((size_t)n);
    unsigned long long* stats = ar.take<unsigned long long>(2);
    if (!ar.sizing) {
        if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (orthant counts)");
        FK_TRY(tie_check(x, xd, d, n, P, sorted, stats, st, fallback));
        if (*fallback) return FK_OK;
    }
    uint32_t* Cs[256] = {};
    Items im{n, 0, n, 0u, nullptr, 0};
    const SubsetSet need = subsets_for(d, mask);
    FK_TRY(dom_counts_core(d, n, im, dc::ceil_log2(n), P, Cs, ar, st, 0, kCountStreams, &need));
    if (ar.sizing) return FK_OK;
    FK_TRY(tie_fix_counts(x, xd, d, n, P, sorted, Cs, st));
    dc::SelMap sel;
    sel.n = 0;
    for (int o = 0; o < nsub; ++o)
        if (!mask || ((mask[o >> 5] >> (o & 31)) & 1u)) sel.o[sel.n++] = o;
    if (sel.n == 0) return FK_OK;
    CTab ct = {};
    for (int A = 1; A < nsub; ++A) ct.c[A] = Cs[A];
    k_combine<<<grid_for(n, 256), 256, 0, st>>>(ct, d, n, (uint32_t)n, 1u, sel, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

}  // namespace fk
