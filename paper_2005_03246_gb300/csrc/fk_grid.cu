// fk_grid.cu -- orthant sums on a rectilinear grid.
//
// Sec. 2.1 of the paper: bin every point into the generalized histogram of
// eq. (partial sums) (Appendix A: Algorithm 6 by search, Algorithm 7 by mesh
// division on uniform axes), then obtain F_N at every grid point from the
// local sums by the lexicographic fast summation of Algorithm 1
// (eq. ECDF decomposition).  Algorithm 1 is the delta = (+,...,+) case; every
// other orthant replaces the inclusive prefix along axis k by the strict
// suffix over bins j+1 .. M_k+1 (delta_k = -1, eq. ECDFdelta reflected).
// Because the d-dimensional prefix is separable, the 2^d orthants are formed
// by one pass per axis, each pass doubling the number of channels.
#include "fk_gridgeom.cuh"

namespace fk {

struct SelTable { int s[256]; };   // orthant -> output row, or -1

namespace {

template <class T>
__device__ __forceinline__ double as_double(T v) { return (double)v; }

template <class T>
__global__ void k_grid_hist_count(const T* __restrict__ x, int64_t n, GridGeom g,
                                  uint32_t* __restrict__ hist, int* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t cell = 0;
    for (int k = 0; k < g.d; ++k) {
        const double v = as_double(x[i * g.d + k]);
        if (!isfinite(v)) note_nonfinite(err);     // binned in range all the same (bin_of never leaves [0, M])
        int64_t j = bin_of(v, g.z[k], g.M[k], g.info[k].uniform, g.info[k].z0, g.info[k].inv_dz);
        cell = cell * (g.M[k] + 1) + j;
    }
    atomicAdd(&hist[cell], 1u);
}

template <class T>
__global__ void k_grid_hist_weighted(const T* __restrict__ x, const T* __restrict__ y, int64_t n,
                                     GridGeom g, double* __restrict__ hist, int* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t cell = 0;
    for (int k = 0; k < g.d; ++k) {
        const double v = as_double(x[i * g.d + k]);
        if (!isfinite(v)) note_nonfinite(err);
        int64_t j = bin_of(v, g.z[k], g.M[k], g.info[k].uniform, g.info[k].z0, g.info[k].inv_dz);
        cell = cell * (g.M[k] + 1) + j;
    }
    atomicAdd(&hist[cell], as_double(y[i]));
}

// ---------------------------------------------------------------- accumulator ops
struct OpCount {
    typedef uint32_t A;
    typedef int64_t O;
    __device__ static A zero() { return 0u; }
    __device__ static A add(A a, A b) { return a + b; }
    __device__ static O out(A a) { return (int64_t)a; }
};
struct OpF64 {
    typedef double A;
    typedef double O;
    __device__ static A zero() { return 0.0; }
    __device__ static A add(A a, A b) { return a + b; }
    __device__ static O out(A a) { return a; }
};
struct OpFF {
    typedef FF A;
    typedef double O;
    __device__ static A zero() { return ff_zero(); }
    __device__ static A add(A a, A b) { return ff_add(a, b); }
    __device__ static O out(A a) { return ff_to_double(a); }
};

// Convert the FP64 histogram into the mixed path's compensated pairs.
__global__ void k_hist_to_ff(const double* __restrict__ h, FF* __restrict__ o, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = ff_from_double(h[i]);
}

// One pass along an outer axis k (inner stride > 1).  Input channel c holds
// [outer][E][inner]; it produces channels 2c (inclusive prefix over bins 0..j,
// delta_k = +1) and 2c+1 (strict suffix over bins j+1..E-1, delta_k = -1) of
// shape [outer][E-1][inner].  Threads walk columns, consecutive threads take
// consecutive inner indices so every step is a coalesced row access.
template <class Op, bool kFinal>
__global__ void k_axis_pass_cols(const typename Op::A* __restrict__ in, void* __restrict__ outp,
                                 int64_t cin, int64_t outer, int64_t E, int64_t inner,
                                 SelTable sel, int64_t out_row) {
    typedef typename Op::A A;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = cin * outer * inner;
    if (t >= total) return;
    int64_t ii = t % inner;
    int64_t rest = t / inner;
    int64_t oo = rest % outer;
    int64_t c = rest / outer;
    const A* src = in + ((c * outer + oo) * E) * inner + ii;
    const int64_t M = E - 1;
    // output row (final pass) or a needed flag (>= 0) of each output channel
    const int s_plus = sel.s[2 * c], s_minus = sel.s[2 * c + 1];
    // prefix (delta_k = +1)
    if (s_plus >= 0) {
        A run = Op::zero();
        for (int64_t e = 0; e < M; ++e) {
            run = Op::add(run, src[e * inner]);
            int64_t o = (oo * M + e) * inner + ii;
            if (kFinal) ((typename Op::O*)outp)[s_plus * out_row + o] = Op::out(run);
            else ((A*)outp)[((2 * c) * outer) * M * inner + o] = run;
        }
    }
    // strict suffix (delta_k = -1)
    if (s_minus >= 0) {
        A run = Op::zero();
        for (int64_t e = M; e >= 1; --e) {
            run = Op::add(run, src[e * inner]);
            int64_t o = (oo * M + (e - 1)) * inner + ii;
            if (kFinal) ((typename Op::O*)outp)[s_minus * out_row + o] = Op::out(run);
            else ((A*)outp)[((2 * c + 1) * outer) * M * inner + o] = run;
        }
    }
}

// Pass along the innermost (contiguous) axis: one warp per line of E values,
// processed in chunks of 32*kPer with a warp scan and a running carry.
template <class Op, bool kFinal>
__global__ void k_axis_pass_rows(const typename Op::A* __restrict__ in, void* __restrict__ outp,
                                 int64_t lines_per_ch, int64_t cin, int64_t E,
                                 SelTable sel, int64_t out_row) {
    typedef typename Op::A A;
    constexpr int kPer = 8;
    const int lane = threadIdx.x & 31;
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wid >= cin * lines_per_ch) return;
    int64_t c = wid / lines_per_ch;
    int64_t line = wid % lines_per_ch;
    const A* src = in + (c * lines_per_ch + line) * E;
    const int64_t M = E - 1;
    for (int dir = 0; dir < 2; ++dir) {
        const int srow = sel.s[2 * c + dir];   // output row, or a needed flag before the last pass
        if (srow < 0) continue;
        A carry = Op::zero();
        const int64_t chunk = 32 * kPer;
        int64_t nchunks = (E + chunk - 1) / chunk;
        for (int64_t q = 0; q < nchunks; ++q) {
            int64_t cb = dir == 0 ? q * chunk : (nchunks - 1 - q) * chunk;
            A v[kPer];
            A loc = Op::zero();
            // dir 0: lane owns elements cb + lane*kPer + j, scanned forward.
            // dir 1: the same elements, scanned backward (suffix).
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                int jj = dir == 0 ? j : kPer - 1 - j;
                int64_t e = cb + (int64_t)lane * kPer + jj;
                v[jj] = (e < E) ? src[e] : Op::zero();
            }
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                int jj = dir == 0 ? j : kPer - 1 - j;
                loc = Op::add(loc, v[jj]);
            }
            // exclusive warp scan of lane totals, forward (dir 0) or backward (dir 1)
            A incl = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                A y;
                if (dir == 0) {
                    y = shfl_up_any(incl, o);
                    if (lane >= o) incl = Op::add(y, incl);
                } else {
                    y = shfl_down_any(incl, o);
                    if (lane + o < 32) incl = Op::add(incl, y);
                }
            }
            A tot = shfl_idx_any(incl, dir == 0 ? 31 : 0);
            A excl = dir == 0 ? shfl_up_any(incl, 1) : shfl_down_any(incl, 1);
            bool first = dir == 0 ? lane == 0 : lane == 31;
            A run = first ? carry : Op::add(carry, excl);
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                int jj = dir == 0 ? j : kPer - 1 - j;
                int64_t e = cb + (int64_t)lane * kPer + jj;
                if (dir == 0) {
                    // inclusive prefix at bin e, output at grid index e (e < M)
                    run = Op::add(run, v[jj]);
                    if (e < M) {
                        int64_t o = line * M + e;
                        if (kFinal) ((typename Op::O*)outp)[srow * out_row + o] = Op::out(run);
                        else ((A*)outp)[(2 * c) * lines_per_ch * M + o] = run;
                    }
                } else {
                    // strict suffix: grid index e-1 receives bins e..M
                    run = Op::add(run, v[jj]);
                    if (e >= 1 && e <= M) {
                        int64_t o = line * M + (e - 1);
                        if (kFinal) ((typename Op::O*)outp)[srow * out_row + o] = Op::out(run);
                        else ((A*)outp)[(2 * c + 1) * lines_per_ch * M + o] = run;
                    }
                }
            }
            carry = Op::add(carry, tot);
        }
    }
}

template <class Op>
fk_status run_passes(typename Op::A* hist, typename Op::A* b1, typename Op::A* b2, int d,
                     const int64_t* M, const SelTable& sel, void* out, int64_t out_row,
                     cudaStream_t st) {
    typedef typename Op::A A;
    A* cur = hist;
    A* nxt = b1;
    int64_t cin = 1;
    for (int k = d - 1; k >= 0; --k) {
        bool fin = (k == 0);
        // Output channel ch of the pass on axis k holds the directions of axes
        // k..d-1 (bit i - k for axis i); before the last pass only the channels
        // that feed a selected orthant o (o >> k == ch) are computed.
        SelTable need;
        if (!fin) {
            for (int ch = 0; ch < 256; ++ch) need.s[ch] = -1;
            for (int o = 0; o < (1 << d); ++o)
                if (sel.s[o] >= 0) need.s[o >> k] = 0;
        }
        const SelTable& tab = fin ? sel : need;
        int64_t outer = 1, inner = 1;
        for (int a = 0; a < k; ++a) outer *= (M[a] + 1);
        for (int a = k + 1; a < d; ++a) inner *= M[a];
        int64_t E = M[k] + 1;
        // algorithmic bytes: every input cell read once, every output written once
        const double obytes = fin ? (double)sizeof(typename Op::O) : (double)sizeof(A);
        int64_t nin = 0, nout = 0;   // input channels read, output channels written
        for (int64_t c = 0; c < cin; ++c) {
            const int64_t o = (tab.s[2 * c] >= 0 ? 1 : 0) + (tab.s[2 * c + 1] >= 0 ? 1 : 0);
            nout += o;
            nin += o > 0 ? 1 : 0;
        }
        ProfScope ps(PF_GRID_PASS, (double)outer * inner * ((double)nin * E * sizeof(A) + (double)nout * (E - 1) * obytes),
                     st);
        if (inner == 1) {
            int64_t warps = cin * outer;
            unsigned blocks = grid_for(warps * 32, 256);
            if (fin) k_axis_pass_rows<Op, true><<<blocks, 256, 0, st>>>(cur, out, outer, cin, E, tab, out_row);
            else k_axis_pass_rows<Op, false><<<blocks, 256, 0, st>>>(cur, nxt, outer, cin, E, tab, 0);
        } else {
            int64_t threads = cin * outer * inner;
            unsigned blocks = grid_for(threads, 256);
            if (fin) k_axis_pass_cols<Op, true><<<blocks, 256, 0, st>>>(cur, out, cin, outer, E, inner, tab, out_row);
            else k_axis_pass_cols<Op, false><<<blocks, 256, 0, st>>>(cur, nxt, cin, outer, E, inner, tab, 0);
        }
        FK_LAUNCH_CHECK();
        cin *= 2;
        cur = nxt;
        nxt = (nxt == b1) ? b2 : b1;
    }
    return FK_OK;
}

}  // namespace

// ----------------------------------------------------------------- host driver
SelTable make_sel(int d, const uint32_t* mask, int* nsel) {
    SelTable t;
    int n = 0;
    for (int o = 0; o < 256; ++o) t.s[o] = -1;
    for (int o = 0; o < (1 << d); ++o)
        if (!mask || ((mask[o >> 5] >> (o & 31)) & 1u)) t.s[o] = n++;
    *nsel = n;
    return t;
}

fk_status grid_run(const void* x, fk_dtype xd, int64_t N, int d, const void* y,
                   const double* z_dev, const int64_t* M, const uint32_t* mask, void* out,
                   fk_path path, Arena& ar, cudaStream_t st, int* err_word) {
    const bool weighted = (y != nullptr);
    int64_t cells = 1, grid_pts = 1;
    for (int k = 0; k < d; ++k) { cells *= (M[k] + 1); grid_pts *= M[k]; }
    // largest intermediate channel array (after passes on axes d-1 .. 1)
    int64_t maxbuf = 1;
    for (int k = d - 1; k >= 1; --k) {
        int64_t sz = (int64_t)1 << (d - k);
        for (int a = 0; a < k; ++a) sz *= (M[a] + 1);
        for (int a = k; a < d; ++a) sz *= M[a];
        if (sz > maxbuf) maxbuf = sz;
    }
    AxisInfo* info = ar.take<AxisInfo>(8);
    const size_t esz = weighted ? 8 : 4;   // u32 counts, double or FF pairs
    char* hist = ar.take<char>((size_t)cells * (weighted ? 8 : 4));
    char* b1 = ar.take<char>((size_t)maxbuf * esz);
    char* b2 = ar.take<char>((size_t)maxbuf * esz);
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small for ecdf_grid");
    int nsel = 0;
    SelTable sel = make_sel(d, mask, &nsel);
    if (nsel == 0) return FK_OK;

    GridGeom g;
    g.d = d;
    int64_t off = 0;
    for (int k = 0; k < 8; ++k) { g.M[k] = 0; g.z[k] = nullptr; }
    for (int k = 0; k < d; ++k) { g.M[k] = M[k]; g.z[k] = z_dev + off; off += M[k]; }
    g.info = info;
    FK_CUDA(cudaMemsetAsync(hist, 0, (size_t)cells * (weighted ? 8 : 4), st));
    k_axis_setup<<<d, 256, 0, st>>>(g, info, err_word);
    FK_LAUNCH_CHECK();
    unsigned blocks = grid_for(N, 256);
    if (N > 0) {
        ProfScope ps(PF_GRID_HIST, (double)N * (d * (xd == FK_F64 ? 8 : 4) + (weighted ? 16 : 8)), st);
        if (!weighted) {
            if (xd == FK_F32) k_grid_hist_count<float><<<blocks, 256, 0, st>>>((const float*)x, N, g, (uint32_t*)hist, err_word);
            else k_grid_hist_count<double><<<blocks, 256, 0, st>>>((const double*)x, N, g, (uint32_t*)hist, err_word);
        } else {
            if (xd == FK_F32) k_grid_hist_weighted<float><<<blocks, 256, 0, st>>>((const float*)x, (const float*)y, N, g, (double*)hist, err_word);
            else k_grid_hist_weighted<double><<<blocks, 256, 0, st>>>((const double*)x, (const double*)y, N, g, (double*)hist, err_word);
        }
        FK_LAUNCH_CHECK();
    }
    if (!weighted)
        return run_passes<OpCount>((uint32_t*)hist, (uint32_t*)b1, (uint32_t*)b2, d, M, sel, out, grid_pts, st);
    if (path == FK_PATH_FP64)
        return run_passes<OpF64>((double*)hist, (double*)b1, (double*)b2, d, M, sel, out, grid_pts, st);
    k_hist_to_ff<<<grid_for(cells, 256), 256, 0, st>>>((const double*)hist, (FF*)hist, cells);
    FK_LAUNCH_CHECK();
    return run_passes<OpFF>((FF*)hist, (FF*)b1, (FF*)b2, d, M, sel, out, grid_pts, st);
}

}  // namespace fk
