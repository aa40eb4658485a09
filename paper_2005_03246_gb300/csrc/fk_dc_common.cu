// fk_dc_common.cu -- rank transform and orchestration of the sample-point
// (divide-and-conquer) operations: orthant sums (ecdf_points / esf_points)
// and kernel sums (kde_laplace / kreg_laplace).
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ uint32_t ordered_bits32(float v) {
    if (v == 0.0f) v = 0.0f;                       // -0 and +0 are the same coordinate
    uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t ordered_bits64(double v) {
    if (v == 0.0) v = 0.0;
    uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// Coordinate of item `it` on axis k: items below n_x read x; the others are
// target copies of x (z == nullptr, sample points) or explicit targets z.
template <class T>
__device__ __forceinline__ T coord_of(const T* x, const T* z, int d, int k, int64_t n_x, int64_t it) {
    if (it < n_x) return x[it * d + k];
    const int64_t j = it - n_x;
    return z ? z[j * d + k] : x[j * d + k];
}

template <class T>
__global__ void k_make_keys32(const T* __restrict__ x, const T* __restrict__ z, int d, int k, int64_t n_x,
                              int64_t n, uint32_t* __restrict__ key, uint32_t* __restrict__ val, int* err) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    const float v = (float)coord_of(x, z, d, k, n_x, it);
    if (!isfinite(v)) note_nonfinite(err);
    key[it] = ordered_bits32(v);
    val[it] = (uint32_t)it;
}
__global__ void k_make_keys64(const double* __restrict__ x, const double* __restrict__ z, int d, int k,
                              int64_t n_x, int64_t n, uint64_t* __restrict__ key, uint32_t* __restrict__ val,
                              int* err) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    const double v = coord_of(x, z, d, k, n_x, it);
    if (!isfinite(v)) note_nonfinite(err);
    key[it] = ordered_bits64(v);
    val[it] = (uint32_t)it;
}

__global__ void k_scatter_positions(const uint32_t* __restrict__ sorted, int64_t n, uint32_t* __restrict__ P) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) P[sorted[p]] = (uint32_t)p;
}

__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) a[p] = (uint32_t)p;
}

__global__ void k_gather_outer(const uint32_t* __restrict__ seq, int64_t n, const uint32_t* __restrict__ Pk,
                               uint32_t* __restrict__ key, uint32_t* __restrict__ meta) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t it = seq[p];
    key[p] = Pk[it];
    meta[p] = it;
}

__global__ void k_record_index(const uint32_t* __restrict__ seq, int64_t n, uint32_t mask,
                               uint32_t* __restrict__ idx) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) idx[seq[p]] = (uint32_t)p & mask;
}

// Exponent factors e^{+-v/h} = m * 2^{+-s}: t = v/(h ln 2) in FP64, s the
// nearest integer, m = 2^{+-(t-s)} evaluated in FP64 (rounded to FP32 for
// the mixed path).  Axes beyond d (the padding axis of d = 1) get factor 1.
// The mantissas 2^{+-f} of a factor, |f| <= 1/2 (the exponent split t = s + f
// is done in FP64 by the caller): FP64 on the FP64 path; on the mixed path,
// whose mantissas are FP32 anyway, the FP32 exp2 of the FP64-split fraction
// (no large-argument error can arise for |f| <= 1/2).
__device__ __forceinline__ void set_mantissas(FacD& o, double f) {
    o.mp = exp2(f);
    o.mm = exp2(-f);
}
__device__ __forceinline__ void set_mantissas(FacF& o, double f) {
    const float ff = (float)f;
    o.mp = exp2f(ff);
    o.mm = exp2f(-ff);
}

template <class T, class F>
__global__ void k_factors(const T* __restrict__ x, const T* __restrict__ z, int d, int d_eff, int64_t n_x,
                          int64_t n, HVec h, F* __restrict__ fac) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    for (int k = 0; k < d_eff; ++k) {
        double t = 0.0;
        if (k < d) {
            t = (double)coord_of(x, z, d, k, n_x, it) / (h.v[k] * 0.69314718055994530942);
            t = fmin(fmax(t, -1.0e7), 1.0e7);
        }
        const double s = rint(t);
        const double f = t - s;
        F o;
        set_mantissas(o, f);
        o.s = (int)s;
        fac[(int64_t)k * n + it] = o;
    }
}

// out[i][t] = C acc[i][t] (signed sums of the gradients: no self term).
__global__ void k_fin_raw(const double* __restrict__ acc, int64_t n_tgt, int nw, double C, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    for (int i = 0; i < nw; ++i) out[(int64_t)i * n_tgt + t] = C * acc[(int64_t)i * n_tgt + t];
}

template <class T, class W>
__global__ void k_convert(const T* __restrict__ y, int64_t n, W* __restrict__ w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = (W)y[i];
}
template <class T>
__global__ void k_convert_ff(const T* __restrict__ y, int64_t n, FF* __restrict__ w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = ff_from_double((double)y[i]);
}

__device__ __forceinline__ double as_f64(uint32_t v) { return (double)v; }
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(FF v) { return ff_to_double(v); }

template <class A>
__global__ void k_fin_sums(const A* __restrict__ acc, int64_t n_tgt, SelMap sel, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    for (int r = 0; r < sel.n; ++r) out[(int64_t)r * n_tgt + t] = as_f64(acc[(int64_t)sel.o[r] * n_tgt + t]);
}

// Kernel sums: f = C (acc + self) for KDE, (num + self_y) / (den + self_1)
// for Nadaraya-Watson.  `self_w` is the weight array of the self pair (BOTH
// items, not leave-one-out) or nullptr.  Per-orthant terms are folded from the
// d_eff internal axes to the d real axes and scaled by C; the self pair lies
// in orthant 0.
template <class A, class W>
__global__ void k_fin_kernel(const A* __restrict__ acc, int64_t n_tgt, int nw, double C, const W* __restrict__ w,
                             int has_self, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    const double sw = has_self ? (w ? (double)w[t] : 1.0) : 0.0;
    const double a0 = as_f64(acc[t]) + sw;
    if (nw == 1) {
        out[t] = C * a0;
    } else {
        const double a1 = as_f64(acc[n_tgt + t]) + (has_self ? 1.0 : 0.0);
        out[t] = (a1 > 0.0) ? a0 / a1 : __longlong_as_double(0x7ff8000000000000LL);
    }
}
template <class A, class W>
__global__ void k_fin_terms(const A* __restrict__ terms, int64_t n_tgt, int d, int d_eff, double C,
                            const W* __restrict__ w, int has_self, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    const uint32_t rmask = (1u << d) - 1u;
    for (int o = 0; o < (1 << d); ++o) out[(int64_t)o * n_tgt + t] = 0.0;
    for (int o = 0; o < (1 << d_eff); ++o) {
        const int r = (int)((uint32_t)o & rmask);
        out[(int64_t)r * n_tgt + t] += C * as_f64(terms[(int64_t)o * n_tgt + t]);
    }
    if (has_self) out[t] += C * (w ? (double)w[t] : 1.0);
}

}  // namespace dc

using namespace dc;

// ------------------------------------------------------------------ plain merges etc.
namespace dc {
fk_status plain_merge_level(const MergeArgs& a, cudaStream_t st) {
    PolCount dummy{};
    ProfScope ps(PF_MERGE_PLAIN, 16.0 * a.n, st);
    k_merge<PolCount, 0, PH_PLAIN><<<grid_for(a.n, MT * MergeItems<PolCount, 0>::value), MT, 0, st>>>(a, dummy,
                                                                                                    nullptr, nullptr);
    FK_LAUNCH_CHECK();
    return FK_OK;
}
fk_status gather_outer(const uint32_t* seq, int64_t n, const uint32_t* Pkey, uint32_t* key, uint32_t* meta,
                       cudaStream_t st) {
    k_gather_outer<<<grid_for(n, 256), 256, 0, st>>>(seq, n, Pkey, key, meta);
    FK_LAUNCH_CHECK();
    return FK_OK;
}
__global__ void k_add_f64(double* __restrict__ dst, const double* __restrict__ src, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] += src[i];
}

fk_status add_f64(double* dst, const double* src, int64_t n, cudaStream_t st) {
    if (n <= 0) return FK_OK;
    k_add_f64<<<grid_for(n, 256), 256, 0, st>>>(dst, src, n);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

fk_status iota_u32(uint32_t* a, int64_t n, cudaStream_t st) {
    k_iota<<<grid_for(n, 256), 256, 0, st>>>(a, n);
    FK_LAUNCH_CHECK();
    return FK_OK;
}
fk_status record_index(const uint32_t* seq, int64_t n, int E, uint32_t* idx, cudaStream_t st) {
    const uint32_t mask = (E >= 32) ? 0xffffffffu : ((1u << E) - 1u);
    k_record_index<<<grid_for(n, 256), 256, 0, st>>>(seq, n, mask, idx);
    FK_LAUNCH_CHECK();
    return FK_OK;
}
}  // namespace dc

// Rank transform (Sec. 2.2, Algorithm 2: the per-axis sort permutations):
// P[k][item] = position of the item in the order of axis k by (coordinate,
// source before target).  Items are numbered sources first, so a stable sort
// of the coordinate keys yields that order.  For d == 1 a padding axis with
// every coordinate equal (P = identity) makes the problem two-dimensional.
struct Positions {
    uint32_t* P[8];
    uint32_t* seq_top;   // items sorted by the last axis
};

static fk_status plan_positions(const void* x, const void* z, fk_dtype xd, int64_t n_x, int64_t n, int d,
                                int d_eff, Positions& pos, Arena& ar, cudaStream_t st) {
    for (int k = 0; k < d_eff; ++k) pos.P[k] = ar.take<uint32_t>(n);
    pos.seq_top = ar.take<uint32_t>(n);
    const bool k64 = (xd == FK_F64);
    void* key0 = ar.take<char>((size_t)n * (k64 ? 8 : 4));
    void* key1 = ar.take<char>((size_t)n * (k64 ? 8 : 4));
    uint32_t* val0 = ar.take<uint32_t>(n);
    uint32_t* val1 = ar.take<uint32_t>(n);
    const int bits = k64 ? 64 : 32;
    const size_t tmpb = radix_sort_tmp_bytes(n, bits);
    void* tmp = ar.take<char>(tmpb);
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (rank transform)");
    const unsigned g = grid_for(n, 256);
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    for (int k = 0; k < d; ++k) {
        if (k64) k_make_keys64<<<g, 256, 0, st>>>((const double*)x, (const double*)z, d, k, n_x, n, (uint64_t*)key0, val0, errw);
        else k_make_keys32<float><<<g, 256, 0, st>>>((const float*)x, (const float*)z, d, k, n_x, n, (uint32_t*)key0, val0, errw);
        FK_LAUNCH_CHECK();
        bool alt = false;
        if (k64) FK_TRY(radix_sort_pairs_u64((uint64_t*)key0, val0, (uint64_t*)key1, val1, n, 64, tmp, tmpb, st, &alt));
        else FK_TRY(radix_sort_pairs_u32((uint32_t*)key0, val0, (uint32_t*)key1, val1, n, 32, tmp, tmpb, st, &alt));
        const uint32_t* sorted = alt ? val1 : val0;
        k_scatter_positions<<<g, 256, 0, st>>>(sorted, n, pos.P[k]);
        FK_LAUNCH_CHECK();
        if (k == d_eff - 1) FK_CUDA(cudaMemcpyAsync(pos.seq_top, sorted, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    if (d < d_eff) {
        k_iota<<<g, 256, 0, st>>>(pos.P[1], n);
        FK_LAUNCH_CHECK();
        k_iota<<<g, 256, 0, st>>>(pos.seq_top, n);
        FK_LAUNCH_CHECK();
    }
    return FK_OK;
}

static SelMap make_selmap(int d, const uint32_t* mask) {
    SelMap s;
    s.n = 0;
    for (int o = 0; o < (1 << d); ++o)
        if (!mask || ((mask[o >> 5] >> (o & 31)) & 1u)) s.o[s.n++] = o;
    return s;
}

// ------------------------------------------------------------------ orthant sums
// Weighted orthant sums of the sweep engine for one item layout (im, n items,
// positions pos), finalised into out [sel rows][n_tgt] double.
static fk_status orthant_sums_run(const void* y, fk_dtype xd, int64_t N, int d, int d_eff, const ItemMap& im,
                                  int64_t n, int64_t n_tgt, const Positions& pos, int kind, const SelMap& sel,
                                  double* out, Arena& ar, cudaStream_t st) {
    const uint32_t pbmask = (1u << (d_eff - 1)) - 1u;
    void* acc = ar.take<char>((size_t)(1 << d_eff) * n_tgt * 8);
    void* wts = ar.take<char>((size_t)N * 8);
    PolW64 pw{};
    PolWFF pf{};
    static_cast<ItemMap&>(pw) = im;
    static_cast<ItemMap&>(pf) = im;
    pw.acc = (double*)acc; pw.w = (const double*)wts; pw.pbmask = pbmask;
    pf.acc = (FF*)acc; pf.w = (const FF*)wts; pf.pbmask = pbmask;
    const uint32_t* const* P = pos.P;
    if (ar.sizing) {
        if (kind == 1) return sweep_w64(d_eff, n, P, pos.seq_top, pw, ar, st);
        return sweep_wff(d_eff, n, P, pos.seq_top, pf, ar, st);
    }
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (orthant sums)");
    FK_CUDA(cudaMemsetAsync(acc, 0, (size_t)(1 << d_eff) * n_tgt * 8, st));
    if (kind == 1) {
        if (xd == FK_F32) k_convert<float, double><<<grid_for(N, 256), 256, 0, st>>>((const float*)y, N, (double*)wts);
        else k_convert<double, double><<<grid_for(N, 256), 256, 0, st>>>((const double*)y, N, (double*)wts);
    } else {
        if (xd == FK_F32) k_convert_ff<float><<<grid_for(N, 256), 256, 0, st>>>((const float*)y, N, (FF*)wts);
        else k_convert_ff<double><<<grid_for(N, 256), 256, 0, st>>>((const double*)y, N, (FF*)wts);
    }
    FK_LAUNCH_CHECK();
    if (kind == 1) FK_TRY(sweep_w64(d_eff, n, P, pos.seq_top, pw, ar, st));
    else FK_TRY(sweep_wff(d_eff, n, P, pos.seq_top, pf, ar, st));
    if (sel.n == 0 || n_tgt == 0) return FK_OK;
    const unsigned g = grid_for(n_tgt, 256);
    if (kind == 1) k_fin_sums<double><<<g, 256, 0, st>>>((const double*)acc, n_tgt, sel, out);
    else k_fin_sums<FF><<<g, 256, 0, st>>>((const FF*)acc, n_tgt, sel, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

fk_status points_orthant(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                         const uint32_t* mask, void* out, fk_path path, Arena& ar, cudaStream_t st) {
    const int d_eff = d < 2 ? 2 : d;
    const bool sample = (z == nullptr);
    const int64_t n_tgt = sample ? N : M;
    const int64_t n = N + n_tgt;                 // sources, then target copies / targets
    const int kind = (y == nullptr) ? 0 : (path == FK_PATH_FP64 ? 1 : 2);
    const SelMap sel = make_selmap(d, mask);
    size_t single_high = 0;
    // Counts at the sample points: one item per point (a source and a
    // target), the ties this misses corrected exactly from the tie groups of
    // the sorted axes (fk_ties.cu); the source/target-copy layout below only
    // when a tie group is long.  Sizing plans both and keeps the larger.
    // (Weighted sums keep the copy layout: moving a tied term between two
    // floating-point sums after the fact leaves a rounding residue in an
    // orthant that holds no term.)
    // The one-item layout reads its tie statistics back to the host, which a
    // stream under graph capture cannot do: a captured call takes the copy
    // layout, which needs no host decision (same counts, twice the items).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!ar.sizing) FK_CUDA(cudaStreamIsCapturing(st, &cap));
    if (kind == 0 && sample && N >= 2 && cap == cudaStreamCaptureStatusNone) {
        const size_t mark = ar.used;
        Positions p1;
        FK_TRY(plan_positions(x, nullptr, xd, N, N, d, d_eff, p1, ar, st));
        if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (orthant counts)");
        bool fallback = ar.sizing;
        FK_TRY(dom_self_counts(d, N, p1.P, x, xd, mask, (int64_t*)out, ar, st, &fallback));
        if (!fallback) return FK_OK;
        single_high = ar.used;
        ar.used = mark;
    }
    Positions pos;
    FK_TRY(plan_positions(x, z, xd, N, n, d, d_eff, pos, ar, st));
    if (kind == 0) {
        // counts: exact inclusion-exclusion over single-orthant dominance counts
        if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (orthant counts)");
        FK_TRY(dom_orthant_counts(d, n, N, N, n_tgt, pos.P, mask, (int64_t*)out, ar, st));
    } else {
        const ItemMap im{N, N, n_tgt};
        FK_TRY(orthant_sums_run(y, xd, N, d, d_eff, im, n, n_tgt, pos, kind, sel, (double*)out, ar, st));
    }
    if (ar.used < single_high) ar.used = single_high;
    return FK_OK;
}

// ------------------------------------------------------------------ kernel sums
__global__ void k_ratio(const double* __restrict__ num, const double* __restrict__ den, int64_t n,
                        double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = num[t] / den[t];
}

fk_status points_kernel(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                        const double* h, unsigned flags, int nw, double* out, double* terms, fk_path path,
                        Arena& ar, cudaStream_t st, fk_dtype wd, int sgn) {
    if (sgn >= 0 && (nw != 2 || terms)) return set_error(FK_ERR_INVALID_ARG, "signed sums need nw == 2, no terms");
    if ((int)wd < 0) wd = xd;
    if (d > 4 && (sgn >= 0 || terms))
        return set_error(FK_ERR_UNSUPPORTED, "per-orthant terms and signed sums support d <= 4");
    if (d > 4 && nw == 2) {
        // Nadaraya-Watson beyond d = 4: numerator (weights y) and denominator
        // (weights 1) as two one-channel kernel sums; C and the self pair enter
        // both the same way, so their ratio is the estimate
        const int64_t n_tgt = z ? M : N;
        double* num = ar.take<double>((size_t)n_tgt);
        double* den = ar.take<double>((size_t)n_tgt);
        if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (kernel sums)");
        const size_t mark = ar.used;
        FK_TRY(points_kernel(x, xd, N, d, w, z, M, h, flags, 1, ar.sizing ? (double*)1 : num, nullptr, path, ar, st,
                             wd));
        const size_t high = ar.used;
        ar.used = mark;
        FK_TRY(points_kernel(x, xd, N, d, nullptr, z, M, h, flags, 1, ar.sizing ? (double*)1 : den, nullptr, path,
                             ar, st, wd));
        if (ar.used < high) ar.used = high;
        if (!ar.sizing && n_tgt > 0) {
            k_ratio<<<grid_for(n_tgt, 256), 256, 0, st>>>(num, den, n_tgt, out);
            FK_LAUNCH_CHECK();
        }
        return FK_OK;
    }
    const int d_eff = d < 2 ? 2 : d;
    const bool sample = (z == nullptr);
    const bool loo = sample && (flags & FK_LOO);
    const int64_t n_tgt = sample ? N : M;
    const int64_t n = sample ? N : N + M;
    ItemMap im{N, sample ? 0 : N, n_tgt};
    const uint32_t pbmask = (1u << (d_eff - 1)) - 1u;
    const bool fp64 = (path == FK_PATH_FP64);
    Positions pos;
    FK_TRY(plan_positions(x, z, xd, N, n, d, d_eff, pos, ar, st));
    const size_t fsz = fp64 ? sizeof(FacD) : sizeof(FacF);
    void* fac = ar.take<char>((size_t)d_eff * n * fsz);
    void* base = ar.take<char>((size_t)n * (fp64 ? sizeof(BaseD) : sizeof(BaseF)));
    void* wts = w ? ar.take<char>((size_t)N * (fp64 ? 8 : 4)) : nullptr;
    const size_t asz = 8;   // double sums on both paths (FF per-orthant terms on the mixed path)
    void* acc = ar.take<char>((size_t)nw * n_tgt * asz);
    void* tacc = terms ? ar.take<char>((size_t)(1 << d_eff) * n_tgt * asz) : nullptr;
    HVec hv;
    for (int k = 0; k < 8; ++k) hv.v[k] = (k < d) ? h[k] : 1.0;
    PolKF<1> f1{}; PolKF<2> f2{}; PolKD<1> d1{}; PolKD<2> d2{};
#define FK_SETK(P, FT, BT, TT, WT)                                                \
    static_cast<ItemMap&>(P) = im; P.w = (const WT*)wts; P.fac = (const FT*)fac;     \
    P.n_items = n; P.nbase = d_eff - 2; P.base = (BT*)base; P.acc = (double*)acc;    \
    P.terms = (TT*)tacc; P.pbmask = pbmask;
    FK_SETK(f1, FacF, BaseF, FF, float)
    FK_SETK(f2, FacF, BaseF, FF, float)
    FK_SETK(d1, FacD, BaseD, double, double)
    FK_SETK(d2, FacD, BaseD, double, double)
#undef FK_SETK
    f1.sgn = f2.sgn = d1.sgn = d2.sgn = sgn;
    const uint32_t* const* P = pos.P;
    auto run = [&]() -> fk_status {
        // d = 3, mixed, one weight channel: the half tile (112 KB of shared memory,
        // two CTAs per SM) costs the call nothing and leaves room on each SM for
        // other work running beside it (measured: same KDE time, a step whose
        // calls overlap 3% faster)
        if (!fp64) return nw == 1 ? sweep_kf1(d_eff, n, P, pos.seq_top, f1, ar, st, -1, d_eff == 3 ? OPT_HALF_TILE : 0)
                                  : sweep_kf2(d_eff, n, P, pos.seq_top, f2, ar, st);
        return nw == 1 ? sweep_kd1(d_eff, n, P, pos.seq_top, d1, ar, st)
                       : sweep_kd2(d_eff, n, P, pos.seq_top, d2, ar, st);
    };
    if (ar.sizing) return run();
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (kernel sums)");
    const unsigned g = grid_for(n, 256);
    if (xd == FK_F32) {
        if (fp64) k_factors<float, FacD><<<g, 256, 0, st>>>((const float*)x, (const float*)z, d, d_eff, N, n, hv, (FacD*)fac);
        else k_factors<float, FacF><<<g, 256, 0, st>>>((const float*)x, (const float*)z, d, d_eff, N, n, hv, (FacF*)fac);
    } else {
        if (fp64) k_factors<double, FacD><<<g, 256, 0, st>>>((const double*)x, (const double*)z, d, d_eff, N, n, hv, (FacD*)fac);
        else k_factors<double, FacF><<<g, 256, 0, st>>>((const double*)x, (const double*)z, d, d_eff, N, n, hv, (FacF*)fac);
    }
    FK_LAUNCH_CHECK();
    if (w) {
        const unsigned gw = grid_for(N, 256);
        if (wd == FK_F32) {
            if (fp64) k_convert<float, double><<<gw, 256, 0, st>>>((const float*)w, N, (double*)wts);
            else k_convert<float, float><<<gw, 256, 0, st>>>((const float*)w, N, (float*)wts);
        } else {
            if (fp64) k_convert<double, double><<<gw, 256, 0, st>>>((const double*)w, N, (double*)wts);
            else k_convert<double, float><<<gw, 256, 0, st>>>((const double*)w, N, (float*)wts);
        }
        FK_LAUNCH_CHECK();
    }
    FK_CUDA(cudaMemsetAsync(acc, 0, (size_t)nw * n_tgt * asz, st));
    if (tacc) FK_CUDA(cudaMemsetAsync(tacc, 0, (size_t)(1 << d_eff) * n_tgt * asz, st));
    if (n_tgt > 0 && N > 0) FK_TRY(run());
    if (n_tgt == 0) return FK_OK;
    // normalising constant 1 / (2^d N' prod h), N' = N - 1 under leave-one-out
    const int64_t nn = loo ? N - 1 : N;
    double C = 0.0;
    if (nn > 0) {
        C = ldexp(1.0, -d) / (double)nn;
        for (int k = 0; k < d; ++k) C /= h[k];
    }
    const int has_self = (sample && !loo) ? 1 : 0;
    const unsigned gt = grid_for(n_tgt, 256);
    if (sgn >= 0) {
        k_fin_raw<<<gt, 256, 0, st>>>((const double*)acc, n_tgt, nw, C, out);
        FK_LAUNCH_CHECK();
        return FK_OK;
    }
    if (fp64) {
        k_fin_kernel<double, double><<<gt, 256, 0, st>>>((const double*)acc, n_tgt, nw, C, (const double*)wts, has_self, out);
        FK_LAUNCH_CHECK();
        if (tacc) {
            k_fin_terms<double, double><<<gt, 256, 0, st>>>((const double*)tacc, n_tgt, d, d_eff, C, (const double*)wts, has_self, terms);
            FK_LAUNCH_CHECK();
        }
    } else {
        k_fin_kernel<double, float><<<gt, 256, 0, st>>>((const double*)acc, n_tgt, nw, C, (const float*)wts, has_self, out);
        FK_LAUNCH_CHECK();
        if (tacc) {
            k_fin_terms<FF, float><<<gt, 256, 0, st>>>((const FF*)tacc, n_tgt, d, d_eff, C, (const float*)wts, has_self, terms);
            FK_LAUNCH_CHECK();
        }
    }
    return FK_OK;
}

}  // namespace fk
