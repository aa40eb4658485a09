// fk_grad.cu -- adjoint of the Laplacian KDE and the leave-one-out likelihood.
//
// Exact derivatives of eq. (Laplacian kde nD), f(z_j) = C sum_i w_i e^{-D_ij},
// D_ij = sum_k |x_ik - z_jk| / h_k, C = 1 / (2^d N prod h), assembled from the
// same orthant sums as the forward pass:
//
//  * d f / d w_i        : the transposed kernel sum, i.e. the same engine with
//                         sources and targets swapped and weights g_j;
//  * d f(z_j) / d z_jk  : in orthant delta, |x_k - z_k| = delta_k (z_k - x_k),
//                         so the derivative is (1/h_k) sum_delta (-delta_k) T_delta(j)
//                         with T_delta the per-orthant terms of the forward pass
//                         (at x_k == z_k the pair sits in the <= orthant);
//  * d f(z_j) / d h_k   : -f_j/h_k + (1/h_k^2) sum_i C w_i e^{-D_ij} |x_ik - z_jk|,
//                         where the distance-weighted sum is
//                         sum_delta delta_k (z_jk T_delta(j) - U^k_delta(j)) and U^k
//                         are the orthant terms with weights w_i x_ik (the
//                         |x - z|-weighted orthant sums; the structure of eq.
//                         Matern32 decomposition nD, Appendix C).
//
// The leave-one-out log-likelihood L(h) = (1/N) sum_j log f_{-j}(x_j) and its
// gradient are the forward pass with FK_LOO and the h-adjoint with
// g_j = 1 / (N f_{-j}).
//
// Without weights (w == 1) the z- and h-adjoints need per axis k only the two
// signed sums sum_delta delta_k T_delta and sum_delta delta_k U^k_delta, which
// a target forms inside the folded sweep by signing each contribution with
// its orthant's delta_k: one two-channel pass (weights x_k and 1) per axis,
// instead of the 2^d per-orthant terms (mixed path; with weights, and on the
// FP64 path, the terms are used).
#include "fk_dc_ops.cuh"

namespace fk {
namespace {

template <class T>
__global__ void k_weight_times_coord(const T* __restrict__ x, const T* __restrict__ w, int d, int k, int64_t n,
                                     double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (w ? (double)w[i] : 1.0) * (double)x[i * d + k];
}

__global__ void k_grad_z(const double* __restrict__ T, const double* __restrict__ g, dc::HVec h, int d, int64_t m,
                         double* __restrict__ gz) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int k = 0; k < d; ++k) {
        double s = 0.0;
        for (int o = 0; o < (1 << d); ++o) {
            const double t = T[(int64_t)o * m + j];
            s += ((o >> k) & 1) ? t : -t;     // -delta_k
        }
        gz[j * d + k] = g[j] * s / h.v[k];
    }
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// gh[k] += sum_j g_j ( -f_j/h_k + (1/h_k^2) sum_delta delta_k (z_jk T_delta(j) - U_delta(j)) )
template <class T>
__global__ void k_grad_h_axis(const double* __restrict__ Tt, const double* __restrict__ U, const double* __restrict__ f,
                              const double* __restrict__ g, const T* __restrict__ zc, int d, int k, int64_t m, double hk,
                              double* __restrict__ gh) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < m) {
        const double zk = (double)zc[j * d + k];
        double s = 0.0;
        for (int o = 0; o < (1 << d); ++o) {
            const double t = zk * Tt[(int64_t)o * m + j] - U[(int64_t)o * m + j];
            s += ((o >> k) & 1) ? -t : t;      // delta_k
        }
        v = g[j] * (-f[j] / hk + s / (hk * hk));
    }
    const double b = block_sum(v);
    if (threadIdx.x == 0) atomicAdd(gh + k, b);
}

// Signed sums of axis k: a[0][j] = C sum_delta delta_k U_delta (weights x_k),
// a[1][j] = C sum_delta delta_k T_delta (weights 1).  The distance-weighted
// sum is z_jk a1 - a0, so
//   gh[k] += sum_j g_j ( -f_j/h_k + (z_jk a1_j - a0_j) / h_k^2 ),
//   gz[j][k] = -g_j a1_j / h_k.
template <class T>
__global__ void k_grad_signed(const double* __restrict__ a, const double* __restrict__ f,
                              const double* __restrict__ g, const T* __restrict__ zc, int d, int k, int64_t m,
                              double hk, double* __restrict__ gz, double* __restrict__ gh) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < m) {
        const double a0 = a[j], a1 = a[m + j];
        if (gz) gz[j * d + k] = -g[j] * a1 / hk;
        if (gh) v = g[j] * (-f[j] / hk + ((double)zc[j * d + k] * a1 - a0) / (hk * hk));
    }
    if (gh) {
        const double b = block_sum(v);
        if (threadIdx.x == 0) atomicAdd(gh + k, b);
    }
}

// g_j = 1 / (N f_j); L += (1/N) sum_j log f_j
__global__ void k_loo_prep(const double* __restrict__ f, int64_t n, double* __restrict__ g, double* __restrict__ L) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < n) {
        g[j] = 1.0 / ((double)n * f[j]);
        v = log(f[j]) / (double)n;
    }
    const double b = block_sum(v);
    if (threadIdx.x == 0) atomicAdd(L, b);
}

__global__ void k_scale(double* __restrict__ a, int64_t n, double s) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] *= s;
}

}  // namespace

// Runs a nested operation on the arena above `mark`, keeping the high-water mark.
struct Nested {
    Arena& ar;
    size_t mark;
    size_t high;
    explicit Nested(Arena& a) : ar(a), mark(a.used), high(a.used) {}
    void done() {
        if (ar.used > high) high = ar.used;
        ar.used = mark;
    }
    void finish() { ar.used = high; }
};

// h-adjoint: gh[k] = sum_j g_j d f_j / d h_k, given f and the orthant terms T
// of the forward pass.  Adds into gh (zeroed by the caller).
static fk_status grad_h_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                            const double* h, unsigned flags, const double* g, const double* f, const double* T,
                            double* gh, fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const int64_t m = sample ? N : M;
    const int no = 1 << d;
    double* U = ar.take<double>((size_t)no * m);
    double* fu = ar.take<double>((size_t)m);
    double* wx = ar.take<double>((size_t)N);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (h adjoint)");
    Nested nest(ar);
    for (int k = 0; k < d; ++k) {
        if (!ar.sizing) {
            if (xd == FK_F32)
                k_weight_times_coord<float><<<grid_for(N, 256), 256, 0, st>>>((const float*)x, (const float*)w, d, k, N, wx);
            else
                k_weight_times_coord<double><<<grid_for(N, 256), 256, 0, st>>>((const double*)x, (const double*)w, d, k, N, wx);
            FK_LAUNCH_CHECK();
        }
        // while sizing, the takes above return NULL: pass placeholders so that the
        // nested plan reserves the weight and orthant-term buffers
        const double* wxp = ar.sizing ? (const double*)1 : wx;
        double* Up = ar.sizing ? (double*)1 : U;
        FK_TRY(points_kernel(x, xd, N, d, wxp, z, M, h, flags, 1, fu, Up, path, ar, st, FK_F64));
        nest.done();
        if (!ar.sizing && m > 0) {
            const void* zc = sample ? x : z;
            if (xd == FK_F32)
                k_grad_h_axis<float><<<grid_for(m, 256), 256, 0, st>>>(T, U, f, g, (const float*)zc, d, k, m, h[k], gh);
            else
                k_grad_h_axis<double><<<grid_for(m, 256), 256, 0, st>>>(T, U, f, g, (const double*)zc, d, k, m, h[k], gh);
            FK_LAUNCH_CHECK();
        }
    }
    nest.finish();
    return FK_OK;
}

// z- and h-adjoints of the unweighted KDE from signed sums (gz, gh optional;
// gh zeroed by the caller).
static fk_status grad_signed_run(const void* x, fk_dtype xd, int64_t N, int d, const void* z, int64_t M,
                                 const double* h, unsigned flags, const double* g, const double* f, double* gz,
                                 double* gh, fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const int64_t m = sample ? N : M;
    double* wx = ar.take<double>((size_t)N);
    double* a2 = ar.take<double>((size_t)2 * m);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (signed adjoint)");
    Nested nest(ar);
    for (int k = 0; k < d; ++k) {
        if (!ar.sizing) {
            if (xd == FK_F32)
                k_weight_times_coord<float><<<grid_for(N, 256), 256, 0, st>>>((const float*)x, nullptr, d, k, N, wx);
            else
                k_weight_times_coord<double><<<grid_for(N, 256), 256, 0, st>>>((const double*)x, nullptr, d, k, N, wx);
            FK_LAUNCH_CHECK();
        }
        FK_TRY(points_kernel(x, xd, N, d, ar.sizing ? (const double*)1 : wx, z, M, h, flags, 2,
                             ar.sizing ? (double*)1 : a2, nullptr, path, ar, st, FK_F64, k));
        nest.done();
        if (!ar.sizing && m > 0) {
            const void* zc = sample ? x : z;
            if (xd == FK_F32)
                k_grad_signed<float><<<grid_for(m, 256), 256, 0, st>>>(a2, f, g, (const float*)zc, d, k, m, h[k], gz, gh);
            else
                k_grad_signed<double><<<grid_for(m, 256), 256, 0, st>>>(a2, f, g, (const double*)zc, d, k, m, h[k], gz, gh);
            FK_LAUNCH_CHECK();
        }
    }
    nest.finish();
    return FK_OK;
}

fk_status kde_backward_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                           const double* h, unsigned flags, const double* g, double* gw, double* gz, double* gh,
                           fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const int64_t m = sample ? N : M;
    const int no = 1 << d;
    // signed sums instead of per-orthant terms: unweighted, mixed path (the
    // FP64 path's cost is FP64 arithmetic, which two channels double)
    const bool fast = (w == nullptr) && path == FK_PATH_MIXED;
    double* T = ((gz || gh) && !fast) ? ar.take<double>((size_t)no * m) : nullptr;
    double* f = (gz || gh) ? ar.take<double>((size_t)m) : nullptr;
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (kde backward)");
    Nested nest(ar);
    if ((gz || gh) && fast) {
        FK_TRY(points_kernel(x, xd, N, d, nullptr, z, M, h, flags, 1, ar.sizing ? (double*)1 : f, nullptr, path, ar, st));
        nest.done();
        if (gh && !ar.sizing) FK_CUDA(cudaMemsetAsync(gh, 0, (size_t)d * sizeof(double), st));
        FK_TRY(grad_signed_run(x, xd, N, d, z, M, h, flags, g, f, gz, gh, path, ar, st));
        nest.done();
    }
    if ((gz || gh) && !fast) {
        FK_TRY(points_kernel(x, xd, N, d, w, z, M, h, flags, 1, f, ar.sizing ? (double*)1 : T, path, ar, st));
        nest.done();
    }
    if (gz && !fast && !ar.sizing && m > 0) {
        dc::HVec hv;
        for (int k = 0; k < 8; ++k) hv.v[k] = (k < d) ? h[k] : 1.0;
        k_grad_z<<<grid_for(m, 256), 256, 0, st>>>(T, g, hv, d, m, gz);
        FK_LAUNCH_CHECK();
    }
    if (gh && !fast) {
        if (!ar.sizing) FK_CUDA(cudaMemsetAsync(gh, 0, (size_t)d * sizeof(double), st));
        FK_TRY(grad_h_run(x, xd, N, d, w, z, M, h, flags, g, f, T, gh, path, ar, st));
        nest.done();
    }
    if (gw) {
        if (sample) {
            // transposed sum at the sample points: same engine, weights g
            FK_TRY(points_kernel(x, xd, N, d, ar.sizing ? (const double*)1 : g, nullptr, 0, h, flags, 1, gw, nullptr,
                                 path, ar, st, FK_F64));
        } else {
            // sources <-> targets: the M targets carry the weights g, the N points receive
            FK_TRY(points_kernel(z, xd, M, d, ar.sizing ? (const double*)1 : g, x, N, h, 0, 1, gw, nullptr, path, ar,
                                 st, FK_F64));
            if (!ar.sizing && N > 0) {
                k_scale<<<grid_for(N, 256), 256, 0, st>>>(gw, N, (double)M / (double)N);
                FK_LAUNCH_CHECK();
            }
        }
        nest.done();
    }
    nest.finish();
    return FK_OK;
}

fk_status loo_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const double* h, double* L,
                  double* gh, fk_path path, Arena& ar, cudaStream_t st) {
    const int no = 1 << d;
    const bool fast = (w == nullptr) && path == FK_PATH_MIXED;   // as in kde_backward_run
    double* T = (gh && !fast) ? ar.take<double>((size_t)no * N) : nullptr;
    double* f = ar.take<double>((size_t)N);
    double* g = ar.take<double>((size_t)N);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (loo)");
    Nested nest(ar);
    FK_TRY(points_kernel(x, xd, N, d, w, nullptr, 0, h, FK_LOO, 1, f,
                         (gh && !fast) ? (ar.sizing ? (double*)1 : T) : nullptr, path, ar, st));
    nest.done();
    if (!ar.sizing) {
        FK_CUDA(cudaMemsetAsync(L, 0, sizeof(double), st));
        k_loo_prep<<<grid_for(N, 256), 256, 0, st>>>(f, N, g, L);
        FK_LAUNCH_CHECK();
    }
    if (gh) {
        if (!ar.sizing) FK_CUDA(cudaMemsetAsync(gh, 0, (size_t)d * sizeof(double), st));
        if (fast) FK_TRY(grad_signed_run(x, xd, N, d, nullptr, 0, h, FK_LOO, g, f, nullptr, gh, path, ar, st));
        else FK_TRY(grad_h_run(x, xd, N, d, w, nullptr, 0, h, FK_LOO, g, f, T, gh, path, ar, st));
        nest.done();
    }
    nest.finish();
    return FK_OK;
}

}  // namespace fk
