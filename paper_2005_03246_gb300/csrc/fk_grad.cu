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

// Leave-one-out densities too small for the sweep's accumulators.  A kernel
// sum C sum_i w_i e^{-D_ij} is accumulated from terms w_i e^{-D_ij} held in
// the path's floating-point type; terms below its smallest normal number
// (2^-126 on the mixed path, 2^-1022 on the FP64 path) are lost.  A density
// whose sum lies within 2^(mantissa bits + 1) N of that limit may have lost
// more than the path's tolerance, and its logarithm enters the likelihood:
// such a target (an isolated point at a small bandwidth) is listed here and
// evaluated exactly by k_loo_exact instead.
__global__ void k_loo_flag(const double* __restrict__ f, int64_t n, double thr, uint32_t* __restrict__ list,
                           uint32_t* __restrict__ count) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && !(f[j] >= thr)) list[atomicAdd(count, 1u)] = (uint32_t)j;   // at most n entries
}

// Exact leave-one-out log-density and its h-gradient of the listed targets,
// one CTA per target (grid-stride over the list): a single pass over the N
// sources keeps, per thread, the smallest distance m seen so far and the
// sums S0 = sum w e^{-(D - m)}, S1_k = sum w e^{-(D - m)} |x_ik - x_jk|
// (rescaled when m drops), then merges the threads' states the same way.
// Distances in FP64; the exponential in FP32 on the mixed path (arguments
// D - m >= 0, relative error ~1e-7 per term) and in FP64 on the FP64 path.
//   lf[j] = log C + log S0 - m,
//   gh[k] += (1/N) (-1/h_k + S1_k / (h_k^2 S0)).
template <class T, bool F64EXP>
__global__ void __launch_bounds__(256) k_loo_exact(const T* __restrict__ x, const T* __restrict__ w, int64_t n, int d,
                                                   dc::HVec hinv, double logC, const uint32_t* __restrict__ list,
                                                   const uint32_t* __restrict__ count, double* __restrict__ lf,
                                                   double* __restrict__ gh) {
    __shared__ double s_m[256], s_s[256][5];
    const uint32_t cnt = *count;
    for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
        const int64_t j = list[e];
        double xj[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xj[k] = (k < d) ? (double)x[j * d + k] : 0.0;
        double m = INFINITY, S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            if (i == j) continue;
            double a[4], D = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = (k < d) ? fabs((double)x[i * d + k] - xj[k]) : 0.0;
                D += a[k] * hinv.v[k];
            }
            if (D < m) {                                   // rescale the sums to the new minimum
                const double r = (m == INFINITY) ? 0.0 : (F64EXP ? exp(D - m) : (double)__expf((float)(D - m)));
#pragma unroll
                for (int q = 0; q < 5; ++q) S[q] *= r;
                m = D;
            }
            const double t = (w ? (double)w[i] : 1.0) * (F64EXP ? exp(m - D) : (double)__expf((float)(m - D)));
            S[0] += t;
#pragma unroll
            for (int k = 0; k < 4; ++k) S[1 + k] += t * a[k];
        }
        s_m[threadIdx.x] = m;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {     // block minimum of m
            if (threadIdx.x < o) s_m[threadIdx.x] = fmin(s_m[threadIdx.x], s_m[threadIdx.x + o]);
            __syncthreads();
        }
        const double mb = s_m[0];
        const double r = (m == INFINITY) ? 0.0 : exp(mb - m);   // once per thread: FP64 on both paths
#pragma unroll
        for (int q = 0; q < 5; ++q) s_s[threadIdx.x][q] = S[q] * r;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o)
#pragma unroll
                for (int q = 0; q < 5; ++q) s_s[threadIdx.x][q] += s_s[threadIdx.x + o][q];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double S0 = s_s[0][0];
            lf[j] = logC + log(S0) - mb;
            for (int k = 0; gh && k < d; ++k)
                atomicAdd(gh + k, (-hinv.v[k] + s_s[0][1 + k] * hinv.v[k] * hinv.v[k] / S0) / (double)n);
        }
        __syncthreads();
    }
}

// g_j = 1 / (N f_j); L += (1/N) sum_j log f_j.  Targets below `thr` (listed
// and evaluated by k_loo_exact) take their log-density from lf and get g_j = 0:
// they add nothing to the sweep's adjoint, their gradient came from k_loo_exact.
__global__ void k_loo_prep(const double* __restrict__ f, int64_t n, double thr, const double* __restrict__ lf,
                           double* __restrict__ g, double* __restrict__ L) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (j < n) {
        const bool exact = !(f[j] >= thr);
        g[j] = exact ? 0.0 : 1.0 / ((double)n * f[j]);
        v = (exact ? lf[j] : log(f[j])) / (double)n;
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
    double* lf = ar.take<double>((size_t)N);
    uint32_t* list = ar.take<uint32_t>((size_t)N);
    uint32_t* count = ar.take<uint32_t>(1);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (loo)");
    Nested nest(ar);
    FK_TRY(points_kernel(x, xd, N, d, w, nullptr, 0, h, FK_LOO, 1, f,
                         (gh && !fast) ? (ar.sizing ? (double*)1 : T) : nullptr, path, ar, st));
    nest.done();
    if (!ar.sizing) {
        // C of the leave-one-out density, and the level below which its sum
        // is recomputed exactly (see k_loo_flag)
        double C = ldexp(1.0, -d) / (double)(N - 1);
        dc::HVec hinv;
        for (int k = 0; k < 8; ++k) hinv.v[k] = (k < d) ? 1.0 / h[k] : 0.0;
        for (int k = 0; k < d; ++k) C /= h[k];
        const int lgN = (int)ceil(log2((double)N));
        const double thr = C * ldexp(1.0, (path == FK_PATH_FP64 ? -1022 + 54 : -126 + 25) + lgN);
        FK_CUDA(cudaMemsetAsync(L, 0, sizeof(double), st));
        FK_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t), st));
        if (gh) FK_CUDA(cudaMemsetAsync(gh, 0, (size_t)d * sizeof(double), st));
        k_loo_flag<<<grid_for(N, 256), 256, 0, st>>>(f, N, thr, list, count);
        FK_LAUNCH_CHECK();
        int dev = 0, sms = 0;
        FK_CUDA(cudaGetDevice(&dev));
        FK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const unsigned ge = (unsigned)(2 * sms);
        if (xd == FK_F32) {
            if (path == FK_PATH_FP64)
                k_loo_exact<float, true><<<ge, 256, 0, st>>>((const float*)x, (const float*)w, N, d, hinv, log(C), list,
                                                             count, lf, gh);
            else
                k_loo_exact<float, false><<<ge, 256, 0, st>>>((const float*)x, (const float*)w, N, d, hinv, log(C),
                                                              list, count, lf, gh);
        } else {
            if (path == FK_PATH_FP64)
                k_loo_exact<double, true><<<ge, 256, 0, st>>>((const double*)x, (const double*)w, N, d, hinv, log(C),
                                                              list, count, lf, gh);
            else
                k_loo_exact<double, false><<<ge, 256, 0, st>>>((const double*)x, (const double*)w, N, d, hinv, log(C),
                                                               list, count, lf, gh);
        }
        FK_LAUNCH_CHECK();
        k_loo_prep<<<grid_for(N, 256), 256, 0, st>>>(f, N, thr, lf, g, L);
        FK_LAUNCH_CHECK();
    }
    if (gh) {
        if (fast) FK_TRY(grad_signed_run(x, xd, N, d, nullptr, 0, h, FK_LOO, g, f, nullptr, gh, path, ar, st));
        else FK_TRY(grad_h_run(x, xd, N, d, w, nullptr, 0, h, FK_LOO, g, f, T, gh, path, ar, st));
        nest.done();
    }
    nest.finish();
    return FK_OK;
}

}  // namespace fk
