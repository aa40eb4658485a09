// fk_kgrid.cu -- the Laplacian KDE on a rectilinear grid, and multilinear
// interpolation of a grid function at arbitrary points.
//
// The grid form of eq. (Laplacian decomposition nD), exact at the grid
// points and free of overflow.  A point x in cell b_k of axis k (z_{b-1} <
// x_k <= z_b, the binning of eq. partial sums) lies, for a grid target z_t,
// below it (x_k <= z_t, delta_k = +1) iff b <= t, else above.  Its factor
// e^{-|z_t - x_k| / h_k} splits at the cell's grid line nearest the target:
//   below: e^{-(z_t - z_b)/h} e^{-(z_b - x)/h}        (upper line of the cell)
//   above: e^{-(z_{b-1} - z_t)/h} e^{-(x - z_{b-1})/h} (lower line of the cell)
// The second factors (<= 1) go into one histogram channel per orthant; the
// first ones are products of the per-step decays D_s = e^{-(z_s - z_{s-1})/h}
// (<= 1), which a linear recurrence along the axis applies:
//   delta_k = +1: S_t = c_t + D_t S_{t-1}          (inclusive, cells 0..t)
//   delta_k = -1: S_t = c_{t+1} + D_{t+1} S_{t+1}  (strict, cells t+1..M)
// one pass per axis for every channel (the fast summation of Algorithm 1
// with a decay, Sec. 2.1 and 3.1), and f(z) = C sum_delta S_delta(z) with
// C = 1 / (2^d N prod h).  Every intermediate is a sum of terms <= w.
#include "fk_gridgeom.cuh"

namespace fk {
namespace {

struct HInv { double v[8]; };

// One channel-factor histogram for all 2^d orthants: hist[o][cell] +=
// w prod_k phi_k(o), phi = e^{-(z_b - x)/h} (bit k of o clear, needs b < M)
// or e^{-(x - z_{b-1})/h} (bit set, needs b >= 1).
template <class T, bool F32EXP>
__global__ void k_kgrid_hist(const T* __restrict__ x, const T* __restrict__ w, int64_t n, GridGeom g, HInv hinv,
                             int64_t cells, double* __restrict__ hist, int* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = g.d;
    int64_t cell = 0;
    double lo[8], hi[8];      // factors towards the lower / upper line (0 if that line does not exist)
    for (int k = 0; k < d; ++k) {
        const double v = (double)x[i * d + k];
        if (!isfinite(v)) note_nonfinite(err);
        const int64_t b = bin_of(v, g.z[k], g.M[k], g.info[k].uniform, g.info[k].z0, g.info[k].inv_dz);
        cell = cell * (g.M[k] + 1) + b;
        const double au = (b < g.M[k]) ? (g.z[k][b] - v) * hinv.v[k] : -1.0;        // >= 0 when it exists
        const double al = (b >= 1) ? (v - g.z[k][b - 1]) * hinv.v[k] : -1.0;
        if (F32EXP) {
            hi[k] = au >= 0.0 ? (double)__expf(-(float)au) : 0.0;
            lo[k] = al >= 0.0 ? (double)__expf(-(float)al) : 0.0;
        } else {
            hi[k] = au >= 0.0 ? exp(-au) : 0.0;
            lo[k] = al >= 0.0 ? exp(-al) : 0.0;
        }
    }
    const double wi = w ? (double)w[i] : 1.0;
    for (int o = 0; o < (1 << d); ++o) {
        double f = wi;
        for (int k = 0; k < d; ++k) f *= ((o >> k) & 1) ? lo[k] : hi[k];
        if (f != 0.0) atomicAdd(hist + (int64_t)o * cells + cell, f);
    }
}

// Per-step decays of every axis: dec[off_k + s] = e^{-(z_s - z_{s-1})/h_k}, s >= 1.
__global__ void k_kgrid_decay(GridGeom g, HInv hinv, const int64_t* __restrict__ off, double* __restrict__ dec) {
    const int k = blockIdx.y;
    if (k >= g.d) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.M[k]; s += (int64_t)gridDim.x * blockDim.x)
        dec[off[k] + s] = (s >= 1) ? exp(-(g.z[k][s] - g.z[k][s - 1]) * hinv.v[k]) : 0.0;
}

// One pass along axis k for all channels: input [ch][outer][E][inner] with
// E = M_k + 1 cells, output [ch][outer][M_k][inner] (the grid index t).
// Channel o runs the inclusive recurrence (bit k clear) or the strict suffix
// (bit set).  One thread per line; consecutive threads take consecutive
// inner indices (coalesced), or consecutive lines of the contiguous axis.
__global__ void k_kgrid_pass(const double* __restrict__ in, double* __restrict__ out, int nch, int k,
                             int64_t outer, int64_t E, int64_t inner, const double* __restrict__ dec) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nch * outer * inner;
    if (t >= total) return;
    const int64_t ii = t % inner;
    const int64_t rest = t / inner;
    const int64_t oo = rest % outer;
    const int64_t c = rest / outer;
    const int64_t M = E - 1;
    const double* src = in + ((c * outer + oo) * E) * inner + ii;
    double* dst = out + ((c * outer + oo) * M) * inner + ii;
    double run = 0.0;
    if (!((c >> k) & 1)) {
        for (int64_t s = 0; s < M; ++s) {
            run = src[s * inner] + (s >= 1 ? dec[s] * run : 0.0);
            dst[s * inner] = run;
        }
    } else {
        // S_{M-1} = c_M; S_t = c_{t+1} + D_{t+1} S_{t+1}
        for (int64_t s = M - 1; s >= 0; --s) {
            run = src[(s + 1) * inner] + (s + 1 <= M - 1 ? dec[s + 1] * run : 0.0);
            dst[s * inner] = run;
        }
    }
}

// f(z) = C sum_o S_o(z)
__global__ void k_kgrid_combine(const double* __restrict__ s, int nch, int64_t pts, double C, double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pts) return;
    double a = 0.0;
    for (int o = 0; o < nch; ++o) a += s[(int64_t)o * pts + t];
    out[t] = C * a;
}

// Multilinear interpolation of f [M_1..M_d] at points q; a coordinate outside
// [z_0, z_{M-1}] is clamped to the nearest grid line.
template <class T>
__global__ void k_grid_interp(const double* __restrict__ f, GridGeom g, const T* __restrict__ q, int64_t nq,
                              double* __restrict__ out, int* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const int d = g.d;
    int64_t j0[8];
    double u[8];
    int64_t stride[8];
    int64_t st = 1;
    for (int k = d - 1; k >= 0; --k) { stride[k] = st; st *= g.M[k]; }
    for (int k = 0; k < d; ++k) {
        const double* z = g.z[k];
        const int64_t M = g.M[k];
        double v = (double)q[i * d + k];
        if (!isfinite(v)) note_nonfinite(err);
        if (!(v >= z[0])) v = z[0];                 // also maps NaN to the first line
        if (v > z[M - 1]) v = z[M - 1];
        if (M == 1) { j0[k] = 0; u[k] = 0.0; continue; }
        int64_t b = bin_of(v, z, M, g.info[k].uniform, g.info[k].z0, g.info[k].inv_dz);   // z_{b-1} < v <= z_b
        int64_t a = b >= 1 ? b - 1 : 0;
        if (a > M - 2) a = M - 2;
        j0[k] = a;
        u[k] = (v - z[a]) / (z[a + 1] - z[a]);
    }
    double acc = 0.0;
    for (int c = 0; c < (1 << d); ++c) {
        double wgt = 1.0;
        int64_t idx = 0;
        for (int k = 0; k < d; ++k) {
            const int up = (c >> k) & 1;
            if (g.M[k] == 1 && up) { wgt = 0.0; break; }
            wgt *= up ? u[k] : 1.0 - u[k];
            idx += (j0[k] + up) * stride[k];
        }
        if (wgt != 0.0) acc += wgt * f[idx];
    }
    out[i] = acc;
}

}  // namespace

static fk_status make_geom(int d, const int64_t* M, const double* z_dev, AxisInfo* info, GridGeom& g) {
    g.d = d;
    int64_t off = 0;
    for (int k = 0; k < 8; ++k) { g.M[k] = 0; g.z[k] = nullptr; }
    for (int k = 0; k < d; ++k) { g.M[k] = M[k]; g.z[k] = z_dev + off; off += M[k]; }
    g.info = info;
    return FK_OK;
}

fk_status kde_grid_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* z_dev,
                       const int64_t* M, const double* h, double* out, fk_path path, Arena& ar, cudaStream_t st,
                       int* err_word) {
    const int nch = 1 << d;
    int64_t cells = 1, pts = 1, msum = 0;
    for (int k = 0; k < d; ++k) { cells *= (M[k] + 1); pts *= M[k]; msum += M[k]; }
    AxisInfo* info = ar.take<AxisInfo>(8);
    int64_t* offs = ar.take<int64_t>(8);
    double* dec = ar.take<double>((size_t)msum);
    double* b0 = ar.take<double>((size_t)nch * cells);
    double* b1 = ar.take<double>((size_t)nch * cells);
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small for kde_grid");
    GridGeom g;
    make_geom(d, M, z_dev, info, g);
    HInv hinv;
    for (int k = 0; k < 8; ++k) hinv.v[k] = (k < d) ? 1.0 / h[k] : 1.0;
    int64_t hoff[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 1; k < d; ++k) hoff[k] = hoff[k - 1] + M[k - 1];
    FK_CUDA(cudaMemcpyAsync(offs, hoff, sizeof(hoff), cudaMemcpyHostToDevice, st));
    FK_CUDA(cudaMemsetAsync(b0, 0, (size_t)nch * cells * sizeof(double), st));
    k_axis_setup<<<d, 256, 0, st>>>(g, info, err_word);
    FK_LAUNCH_CHECK();
    k_kgrid_decay<<<dim3(grid_for(msum, 256) > 64 ? 64 : grid_for(msum, 256), d), 256, 0, st>>>(g, hinv, offs, dec);
    FK_LAUNCH_CHECK();
    if (N > 0) {
        const unsigned blocks = grid_for(N, 256);
        const bool f32 = (path == FK_PATH_MIXED);
        ProfScope ps(PF_GRID_HIST, (double)N * (d * (xd == FK_F64 ? 8 : 4) + (w ? 8 : 0) + nch * 8.0), st);
        if (xd == FK_F32) {
            if (f32) k_kgrid_hist<float, true><<<blocks, 256, 0, st>>>((const float*)x, (const float*)w, N, g, hinv, cells, b0, err_word);
            else k_kgrid_hist<float, false><<<blocks, 256, 0, st>>>((const float*)x, (const float*)w, N, g, hinv, cells, b0, err_word);
        } else {
            if (f32) k_kgrid_hist<double, true><<<blocks, 256, 0, st>>>((const double*)x, (const double*)w, N, g, hinv, cells, b0, err_word);
            else k_kgrid_hist<double, false><<<blocks, 256, 0, st>>>((const double*)x, (const double*)w, N, g, hinv, cells, b0, err_word);
        }
        FK_LAUNCH_CHECK();
    }
    // axes from the last (contiguous) to the first; the shape shrinks by one per axis
    int64_t dims[8];
    for (int k = 0; k < d; ++k) dims[k] = M[k] + 1;
    double* cur = b0;
    double* nxt = b1;
    for (int k = d - 1; k >= 0; --k) {
        int64_t outer = 1, inner = 1;
        for (int a = 0; a < k; ++a) outer *= dims[a];
        for (int a = k + 1; a < d; ++a) inner *= dims[a];
        const int64_t E = dims[k];
        const int64_t lines = (int64_t)nch * outer * inner;
        ProfScope ps(PF_GRID_PASS, (double)lines * (E + (E - 1)) * 8.0, st);
        k_kgrid_pass<<<grid_for(lines, 256), 256, 0, st>>>(cur, nxt, nch, k, outer, E, inner, dec + hoff[k]);
        FK_LAUNCH_CHECK();
        dims[k] = M[k];
        double* t = cur;
        cur = nxt;
        nxt = t;
    }
    double C = ldexp(1.0, -d) / (double)(N > 0 ? N : 1);
    for (int k = 0; k < d; ++k) C /= h[k];
    if (N == 0) C = 0.0;
    k_kgrid_combine<<<grid_for(pts, 256), 256, 0, st>>>(cur, nch, pts, C, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

fk_status grid_interp_run(const double* f, int d, const double* z_dev, const int64_t* M, const void* q, fk_dtype qd,
                          int64_t nq, double* out, Arena& ar, cudaStream_t st, int* err_word) {
    AxisInfo* info = ar.take<AxisInfo>(8);
    if (ar.sizing) return FK_OK;
    if (ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small for grid_interp");
    GridGeom g;
    make_geom(d, M, z_dev, info, g);
    k_axis_setup<<<d, 256, 0, st>>>(g, info, err_word);
    FK_LAUNCH_CHECK();
    if (nq == 0) return FK_OK;
    if (qd == FK_F32) k_grid_interp<float><<<grid_for(nq, 256), 256, 0, st>>>(f, g, (const float*)q, nq, out, err_word);
    else k_grid_interp<double><<<grid_for(nq, 256), 256, 0, st>>>(f, g, (const double*)q, nq, out, err_word);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

}  // namespace fk
