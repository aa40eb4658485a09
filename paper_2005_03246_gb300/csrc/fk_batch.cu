// fk_batch.cu -- many independent datasets of uneven N and d in one call.
//
// Datasets are grouped by (d, E) where 2^E is the smallest power of two
// holding a dataset's items (2N for orthant counts at the sample points, N for
// the kernel sums).  A group is laid out as consecutive segments of 2^E slots,
// one dataset per segment, with padding slots that are neither source nor
// target.  Each axis is sorted by (segment, coordinate), so every position
// lies inside its own segment; all merge blocks of the engine are aligned
// power-of-two blocks, so stopping its merge sorts at level E keeps every
// dataset separate while each kernel launch works on all datasets of the group
// at once.  The per-dataset descriptors are written to device memory by a
// kernel whose launch parameters carry them, so the whole call can be captured
// in a CUDA graph.
#include <algorithm>
#include <map>
#include <vector>

#include "fk_dc_ops.cuh"

namespace fk {
namespace {

constexpr int kChunk = 48;   // datasets per descriptor-fill launch (keeps parameters small)

struct DescChunk {
    const void* x[kChunk];
    const void* y[kChunk];
    int64_t n[kChunk];
    int64_t obase_e[kChunk];
    int64_t obase_k[kChunk];
    int count;
    int first;          // index of the first dataset of the chunk inside the group
};

// Group tables: seg[4s..4s+3] (see dc::ItemMap), tbase[s] (global target base),
// obase[s], x[s], y[s], n[s].
struct GroupTab {
    int64_t* seg;
    int64_t* tbase;     // [ns + 1]
    int64_t* obase_e;
    int64_t* obase_k;
    const void** x;
    const void** y;
    int64_t* n;
};

__global__ void k_fill_desc(DescChunk c, GroupTab t, int doubled) {
    const int i = threadIdx.x;
    if (i >= c.count) return;
    const int s = c.first + i;
    t.x[s] = c.x[i];
    t.y[s] = c.y[i];
    t.n[s] = c.n[i];
    t.obase_e[s] = c.obase_e[i];
    t.obase_k[s] = c.obase_k[i];
    t.seg[4 * s + 0] = c.n[i];                   // sources: slots [0, N)
    t.seg[4 * s + 1] = doubled ? c.n[i] : 0;     // targets start (copies, or the same slots)
    t.seg[4 * s + 2] = c.n[i];
}

// target bases: exclusive prefix of N over the segments (one thread; groups are small)
__global__ void k_tbase(GroupTab t, int ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int s = 0; s < ns; ++s) {
        t.tbase[s] = run;
        t.seg[4 * s + 3] = run;
        run += t.n[s];
    }
    t.tbase[ns] = run;
}

template <class T>
__global__ void k_batch_gather(GroupTab t, int64_t n, int E, int d, int doubled, T* __restrict__ xg, int* err) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    const int64_t s = it >> E, loc = it & (((int64_t)1 << E) - 1);
    const int64_t N = t.n[s];
    int64_t pt = -1;
    if (loc < N) pt = loc;
    else if (doubled && loc < 2 * N) pt = loc - N;
    const T* xb = (const T*)t.x[s];
    for (int k = 0; k < d; ++k) {
        // padding slots sort after every real point of their segment
        const T v = (pt >= 0) ? xb[pt * d + k] : (T)__int_as_float(0x7f800000);
        if (pt >= 0 && !isfinite(v)) note_nonfinite(err);
        xg[it * d + k] = v;
    }
}

__global__ void k_batch_keys32(const float* __restrict__ xg, int d, int k, int64_t n, int E,
                               uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    float v = xg[it * d + k];
    if (v == 0.0f) v = 0.0f;
    uint32_t u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    key[it] = ((uint64_t)(it >> E) << 32) | u;
    val[it] = (uint32_t)it;
}
__global__ void k_batch_keys64(const double* __restrict__ xg, int d, int k, int64_t n,
                               uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    double v = xg[it * d + k];
    if (v == 0.0) v = 0.0;
    uint64_t u = (uint64_t)__double_as_longlong(v);
    key[it] = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    val[it] = (uint32_t)it;
}
__global__ void k_seg_of_sorted(const uint32_t* __restrict__ sorted, int64_t n, int E, uint32_t* __restrict__ key) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) key[p] = sorted[p] >> E;
}
__global__ void k_scatter_pos(const uint32_t* __restrict__ sorted, int64_t n, uint32_t* __restrict__ P) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) P[sorted[p]] = (uint32_t)p;
}

template <class T, class F>
__global__ void k_batch_factors(const T* __restrict__ xg, int d, int d_eff, int64_t n, double h, F* __restrict__ fac) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    for (int k = 0; k < d_eff; ++k) {
        double t = 0.0;
        if (k < d) {
            const double v = (double)xg[it * d + k];
            t = (v == v && v < 1e300) ? v / (h * 0.69314718055994530942) : 0.0;   // padding: factor 1
            t = fmin(fmax(t, -1.0e7), 1.0e7);
        }
        const double r = rint(t), f = t - r;
        F o;
        if constexpr (sizeof(o.mp) == 4) {     // mixed path: FP32 exp2 of the FP64-split fraction
            o.mp = exp2f((float)f);
            o.mm = exp2f(-(float)f);
        } else {
            o.mp = exp2(f);
            o.mm = exp2(-f);
        }
        o.s = (int)r;
        fac[(int64_t)k * n + it] = o;
    }
}

template <class T, class W>
__global__ void k_batch_weights(GroupTab t, int64_t n, int E, W* __restrict__ w) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    const int64_t s = it >> E, loc = it & (((int64_t)1 << E) - 1);
    const T* yb = (const T*)t.y[s];
    w[it] = (loc < t.n[s]) ? (yb ? (W)yb[loc] : (W)1) : (W)0;
}

// f = C_b (acc + self) with C_b = 1 / (2^d N_b h^d); self = the point's own weight.
template <class A, class W>
__global__ void k_batch_fin_kde(const A* __restrict__ acc, GroupTab t, int ns, int E, int d, double h, const W* __restrict__ w,
                                int64_t n_tgt, double* __restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_tgt) return;
    int lo = 0, hi = ns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.tbase[mid] <= q) lo = mid; else hi = mid;
    }
    const int s = lo;
    const int64_t loc = q - t.tbase[s];
    const int64_t item = ((int64_t)s << E) + loc;
    double C = ldexp(1.0, -d) / (double)t.n[s];
    for (int k = 0; k < d; ++k) C /= h;
    out[t.obase_k[s] + loc] = C * (dc_as_f64(acc[q]) + (double)w[item]);
}

}  // namespace

struct Grp {
    int d;
    int E;
    bool doubled;
    std::vector<int> ids;
};

// Groups of one pass: datasets by (d, E) with E rounded up to a multiple of
// coarsen + 1 (coarser groups: fewer, larger launches, more padding); no
// group exceeds 2^25 slots.
static std::vector<Grp> make_groups(const fk_dataset* sets, int count, bool doubled, int coarsen) {
    const int w = coarsen + 1;
    std::map<std::pair<int, int>, Grp> m;
    for (int b = 0; b < count; ++b) {
        const int64_t items = doubled ? 2 * sets[b].N : sets[b].N;
        int E = dc::ceil_log2(items < 2 ? 2 : items);
        E = ((E + w - 1) / w) * w;
        Grp& g = m[{sets[b].d, E}];
        g.d = sets[b].d;
        g.E = E;
        g.doubled = doubled;
        g.ids.push_back(b);
    }
    std::vector<Grp> out;
    for (auto& kv : m) {
        const Grp& g = kv.second;
        const size_t per = std::max<size_t>(1, ((size_t)1 << 25) >> g.E);
        for (size_t i = 0; i < g.ids.size(); i += per) {
            Grp c;
            c.d = g.d;
            c.E = g.E;
            c.doubled = doubled;
            c.ids.assign(g.ids.begin() + i, g.ids.begin() + std::min(g.ids.size(), i + per));
            out.push_back(c);
        }
    }
    return out;
}

// One group: tables, layout, positions, then the orthant counts or the KDE.
static fk_status run_group(const fk_dataset* sets, const Grp& g, fk_dtype xd, double h,
                           const std::vector<int64_t>& obe, const std::vector<int64_t>& obk, int64_t* ecdf_out,
                           double* kde_out, fk_path path, const BatchCfg& cfg, Arena& ar, cudaStream_t st) {
    const bool doubled = g.doubled;
    // groups run concurrently on their own; their sweeps stay serial
    const int opts = (cfg.kernel_tile == 1 ? dc::OPT_HALF_TILE : 0) | dc::OPT_SERIAL;
    const int ns = (int)g.ids.size();
    const int E = g.E, d = g.d, d_eff = d < 2 ? 2 : d;
    const int64_t n = (int64_t)ns << E;
    int64_t n_tgt = 0;
    for (int b : g.ids) n_tgt += sets[b].N;
    const size_t es = xd == FK_F64 ? 8 : 4;
    GroupTab t;
    t.seg = ar.take<int64_t>(4 * (size_t)ns);
    t.tbase = ar.take<int64_t>((size_t)ns + 1);
    t.obase_e = ar.take<int64_t>(ns);
    t.obase_k = ar.take<int64_t>(ns);
    t.x = (const void**)ar.take<void*>(ns);
    t.y = (const void**)ar.take<void*>(ns);
    t.n = ar.take<int64_t>(ns);
    void* xg = ar.take<char>((size_t)n * d * es);
    uint32_t* P[8] = {};
    for (int k = 0; k < d_eff; ++k) P[k] = ar.take<uint32_t>(n);
    uint32_t* seq_top = ar.take<uint32_t>(n);
    uint64_t* k0 = ar.take<uint64_t>(n);
    uint64_t* k1 = ar.take<uint64_t>(n);
    uint32_t* v0 = ar.take<uint32_t>(n);
    uint32_t* v1 = ar.take<uint32_t>(n);
    const size_t tmpb = radix_sort_tmp_bytes(n, 64);
    void* tmp = ar.take<char>(tmpb);
    const bool fp64 = (path == FK_PATH_FP64);
    void *fac = nullptr, *base = nullptr, *wts = nullptr, *acc = nullptr;
    if (!doubled) {
        fac = ar.take<char>((size_t)d_eff * n * (fp64 ? sizeof(FacD) : sizeof(FacF)));
        base = ar.take<char>((size_t)n * (fp64 ? sizeof(dc::BaseD) : sizeof(dc::BaseF)));
        wts = ar.take<char>((size_t)n * (fp64 ? 8 : 4));
        acc = ar.take<char>((size_t)n_tgt * 8);
    }
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (batched)");
    const int64_t* seg = t.seg;
    // the engine plans its own buffers above this point
    if (ar.sizing) {
        if (doubled) {
            dom_orthant_counts_seg(d, n, seg, E, n_tgt, P, BatchOut{nullptr, nullptr, ns}, nullptr, ar, st,
                                   cfg.count_tile);
        } else {
            dc::ItemMap im{0, 0, n_tgt, seg, E};
            if (fp64) { dc::PolKD<1> p{}; static_cast<dc::ItemMap&>(p) = im; dc::sweep_kd1(d_eff, n, P, seq_top, p, ar, st, E, opts); }
            else { dc::PolKF<1> p{}; static_cast<dc::ItemMap&>(p) = im; dc::sweep_kf1(d_eff, n, P, seq_top, p, ar, st, E, opts); }
        }
        return FK_OK;
    }
    // descriptors
    for (int c0 = 0; c0 < ns; c0 += kChunk) {
        DescChunk c = {};
        c.count = std::min(kChunk, ns - c0);
        c.first = c0;
        for (int i = 0; i < c.count; ++i) {
            const int b = g.ids[c0 + i];
            c.x[i] = sets[b].x; c.y[i] = sets[b].y; c.n[i] = sets[b].N;
            c.obase_e[i] = obe[b]; c.obase_k[i] = obk[b];
        }
        k_fill_desc<<<1, kChunk, 0, st>>>(c, t, doubled ? 1 : 0);
        FK_LAUNCH_CHECK();
    }
    k_tbase<<<1, 1, 0, st>>>(t, ns);
    FK_LAUNCH_CHECK();
    const unsigned gg = grid_for(n, 256);
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    if (xd == FK_F32) k_batch_gather<float><<<gg, 256, 0, st>>>(t, n, E, d, doubled ? 1 : 0, (float*)xg, errw);
    else k_batch_gather<double><<<gg, 256, 0, st>>>(t, n, E, d, doubled ? 1 : 0, (double*)xg, errw);
    FK_LAUNCH_CHECK();
    // positions: sort every axis by (segment, coordinate), sources first on ties
    int segbits = 0;
    while ((1 << segbits) < ns) ++segbits;
    for (int k = 0; k < d; ++k) {
        bool alt = false;
        const uint32_t* sorted = nullptr;
        if (xd == FK_F32) {
            k_batch_keys32<<<gg, 256, 0, st>>>((const float*)xg, d, k, n, E, k0, v0);
            FK_LAUNCH_CHECK();
            FK_TRY(radix_sort_pairs_u64(k0, v0, k1, v1, n, 32 + segbits, tmp, tmpb, st, &alt));
            sorted = alt ? v1 : v0;
        } else {
            k_batch_keys64<<<gg, 256, 0, st>>>((const double*)xg, d, k, n, k0, v0);
            FK_LAUNCH_CHECK();
            FK_TRY(radix_sort_pairs_u64(k0, v0, k1, v1, n, 64, tmp, tmpb, st, &alt));
            uint32_t* sv = alt ? v1 : v0;
            uint32_t* ov = alt ? v0 : v1;
            uint32_t* kk = (uint32_t*)(alt ? k0 : k1);
            uint32_t* ko = (uint32_t*)(alt ? k1 : k0);
            k_seg_of_sorted<<<gg, 256, 0, st>>>(sv, n, E, kk);
            FK_LAUNCH_CHECK();
            bool alt2 = false;
            FK_TRY(radix_sort_pairs_u32(kk, sv, ko, ov, n, segbits > 0 ? segbits : 1, tmp, tmpb, st, &alt2));
            sorted = alt2 ? ov : sv;
        }
        k_scatter_pos<<<gg, 256, 0, st>>>(sorted, n, P[k]);
        FK_LAUNCH_CHECK();
        if (k == d_eff - 1) FK_CUDA(cudaMemcpyAsync(seq_top, sorted, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (d < d_eff) {
        // d == 1: a padding axis on which every slot ties keeps slot order
        dc::iota_u32(P[1], n, st);
        dc::iota_u32(seq_top, n, st);
    }
    if (doubled) {
        BatchOut bo{t.tbase, t.obase_e, ns};
        return dom_orthant_counts_seg(d, n, seg, E, n_tgt, P, bo, ecdf_out, ar, st, cfg.count_tile);
    }
    // kernel sums
    if (xd == FK_F32) {
        if (fp64) k_batch_factors<float, FacD><<<gg, 256, 0, st>>>((const float*)xg, d, d_eff, n, h, (FacD*)fac);
        else k_batch_factors<float, FacF><<<gg, 256, 0, st>>>((const float*)xg, d, d_eff, n, h, (FacF*)fac);
    } else {
        if (fp64) k_batch_factors<double, FacD><<<gg, 256, 0, st>>>((const double*)xg, d, d_eff, n, h, (FacD*)fac);
        else k_batch_factors<double, FacF><<<gg, 256, 0, st>>>((const double*)xg, d, d_eff, n, h, (FacF*)fac);
    }
    FK_LAUNCH_CHECK();
    if (xd == FK_F32) {
        if (fp64) k_batch_weights<float, double><<<gg, 256, 0, st>>>(t, n, E, (double*)wts);
        else k_batch_weights<float, float><<<gg, 256, 0, st>>>(t, n, E, (float*)wts);
    } else {
        if (fp64) k_batch_weights<double, double><<<gg, 256, 0, st>>>(t, n, E, (double*)wts);
        else k_batch_weights<double, float><<<gg, 256, 0, st>>>(t, n, E, (float*)wts);
    }
    FK_LAUNCH_CHECK();
    FK_CUDA(cudaMemsetAsync(acc, 0, (size_t)n_tgt * 8, st));
    dc::ItemMap im{0, 0, n_tgt, seg, E};
    const unsigned gt = grid_for(n_tgt, 256);
    if (fp64) {
        dc::PolKD<1> p{};
        static_cast<dc::ItemMap&>(p) = im;
        p.w = (const double*)wts; p.fac = (const FacD*)fac; p.n_items = n; p.nbase = d_eff - 2;
        p.base = (dc::BaseD*)base; p.acc = (double*)acc; p.terms = nullptr; p.pbmask = (1u << (d_eff - 1)) - 1u;
        FK_TRY(dc::sweep_kd1(d_eff, n, P, seq_top, p, ar, st, E, opts));
        k_batch_fin_kde<double, double><<<gt, 256, 0, st>>>((const double*)acc, t, ns, E, d, h, (const double*)wts, n_tgt, kde_out);
    } else {
        dc::PolKF<1> p{};
        static_cast<dc::ItemMap&>(p) = im;
        p.w = (const float*)wts; p.fac = (const FacF*)fac; p.n_items = n; p.nbase = d_eff - 2;
        p.base = (dc::BaseF*)base; p.acc = (double*)acc; p.terms = nullptr; p.pbmask = (1u << (d_eff - 1)) - 1u;
        FK_TRY(dc::sweep_kf1(d_eff, n, P, seq_top, p, ar, st, E, opts));
        k_batch_fin_kde<double, float><<<gt, 256, 0, st>>>((const double*)acc, t, ns, E, d, h, (const float*)wts, n_tgt, kde_out);
    }
    FK_LAUNCH_CHECK();
    return FK_OK;
}

// All groups of both passes; with cfg.streams > 1 they are spread over that
// many streams (the caller's and library-owned ones, forked from and joined
// back to the caller's stream by events, so the call stays capturable), each
// stream with its own workspace slot sized for its largest group.
fk_status batched_run(const fk_dataset* sets, int count, fk_dtype xd, unsigned what, double h, int64_t* ecdf_out,
                      double* kde_out, fk_path path, const BatchCfg& cfg, Arena& ar, cudaStream_t st) {
    std::vector<int64_t> obe(count), obk(count);
    int64_t re = 0, rk = 0;
    for (int b = 0; b < count; ++b) {
        obe[b] = re;
        obk[b] = rk;
        re += ((int64_t)1 << sets[b].d) * sets[b].N;
        rk += sets[b].N;
    }
    std::vector<Grp> groups;
    for (int pass = 0; pass < 2; ++pass) {
        const bool doubled = (pass == 0);
        if (doubled && !(what & FK_BATCH_ECDF)) continue;
        if (!doubled && !(what & FK_BATCH_KDE)) continue;
        for (Grp& g : make_groups(sets, count, doubled, cfg.coarsen)) groups.push_back(g);
    }
    if (groups.empty()) return FK_OK;
    // workspace of every group, largest first, dealt round-robin to the streams
    std::vector<size_t> need(groups.size());
    for (size_t i = 0; i < groups.size(); ++i) {
        Arena a;
        run_group(sets, groups[i], xd, h, obe, obk, nullptr, nullptr, path, cfg, a, st);
        need[i] = (a.used + 255) & ~(size_t)255;
    }
    std::vector<size_t> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return need[a] > need[b]; });
    const int S = std::max(1, std::min<int>(cfg.streams, std::min<int>(kPoolStreams, (int)groups.size())));
    std::vector<std::vector<size_t>> slot(S);
    std::vector<size_t> slot_need(S, 0);
    for (size_t q = 0; q < order.size(); ++q) {
        const int s = (int)(q % S);
        slot[s].push_back(order[q]);
        slot_need[s] = std::max(slot_need[s], need[order[q]]);
    }
    std::vector<size_t> off(S + 1, 0);
    for (int s = 0; s < S; ++s) off[s + 1] = off[s] + slot_need[s];
    const size_t base = (ar.used + 255) & ~(size_t)255;
    if (ar.sizing) {
        ar.used = base + off[S];
        return FK_OK;
    }
    if (base + off[S] > ar.cap) return set_error(FK_ERR_WORKSPACE, "workspace too small (batched)");
    StreamFork fork;
    FK_TRY(fork.begin(0, st, S));
    fk_status rc = FK_OK;
    for (int s = 0; s < S && rc == FK_OK; ++s) {
        for (size_t i : slot[s]) {
            Arena a;
            a.sizing = false;
            a.base = ar.base + base + off[s];
            a.cap = slot_need[s];
            a.used = 0;
            rc = run_group(sets, groups[i], xd, h, obe, obk, ecdf_out, kde_out, path, cfg, a, fork.s[s]);
            if (rc != FK_OK) break;
        }
    }
    // join every forked stream, also after an error, so no capture is left open
    const fk_status rj = fork.end();
    if (rc == FK_OK) rc = rj;
    ar.used = base + off[S];
    return rc;
}

}  // namespace fk
