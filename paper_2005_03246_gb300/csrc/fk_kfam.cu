// fk_kfam.cu -- more estimators on the same orthant engine:
//
//  * the uniform kernel, eq. (uniform decomposition nD) of Sec. 3.2: a signed
//    combination of 2^d ECDFs taken at the box corners z + delta h, where
//    delta_k = -1 asks for the strict x_k < z_k - h_k (eq. ECDFdelta);
//  * the additive multivariate Matern-3/2 kernel, eq. (Matern32 decomposition
//    nD) of Appendix C: the Laplacian orthant sums with weights w and
//    w x_l (2^d (d+1) CDFs);
//  * a full bandwidth matrix H = R diag(h)^2 R^T, Appendix B: both point sets
//    rotated by R^T, then the diagonal-bandwidth Laplacian KDE;
//  * locally linear regression with the Laplacian kernel: the weighted
//    least-squares fit of an affine function around each target, from the
//    kernel sums of the weights 1, u_k, u_k u_l, y, y u_k.
//
// Everything here orchestrates the existing engines (points_orthant,
// points_kernel); the new kernels only build corner targets, weights and
// rotated coordinates, and combine per-target results.
#include <math.h>

#include "fk_dc_ops.cuh"

namespace fk {
namespace {

// ------------------------------------------------------------------ uniform kernel
// Thresholds in the data's own type: x <= c  <=>  x <= le(c), and
// x < c  <=>  x <= lt(c), exactly, for every value x of that type.
template <class T>
struct Thr;
template <>
struct Thr<float> {
    static __device__ __forceinline__ float le(double c) { return __double2float_rd(c); }
    static __device__ __forceinline__ float lt(double c) {
        float f = __double2float_rd(c);
        if ((double)f == c) f = nextafterf(f, -INFINITY);
        return f;
    }
};
template <>
struct Thr<double> {
    static __device__ __forceinline__ double le(double c) { return c; }
    static __device__ __forceinline__ double lt(double c) { return nextafter(c, -INFINITY); }
};

// Corner c of target j is item c * m + j; bit k of c set means the lower
// corner z_k - h_k (strict), clear the upper corner z_k + h_k (inclusive).
// Both corners are rounded once in FP64, as the oracle does.
template <class T>
__global__ void k_uniform_corners(const T* __restrict__ zs, int d, int64_t m, int nc, dc::HVec h,
                                  T* __restrict__ zc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nc * m) return;
    const int c = (int)(t / m);
    const int64_t j = t - (int64_t)c * m;
    for (int k = 0; k < d; ++k) {
        const double zk = (double)zs[j * d + k];
        zc[t * d + k] = ((c >> k) & 1) ? Thr<T>::lt(zk - h.v[k]) : Thr<T>::le(zk + h.v[k]);
    }
}

// out[j] = C (sum_c (-1)^{|c|} S[c][j] - self_j); exact integer combination for counts.
template <class W>
__global__ void k_uniform_combine_counts(const int64_t* __restrict__ S, int nc, int64_t m, double C, int loo,
                                         double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int64_t s = 0;
    for (int c = 0; c < nc; ++c) {
        const int64_t v = S[(int64_t)c * m + j];
        s += (__popc(c) & 1) ? -v : v;
    }
    out[j] = C * (double)(s - (loo ? 1 : 0));
}
template <class W>
__global__ void k_uniform_combine_sums(const double* __restrict__ S, int nc, int64_t m, double C,
                                       const W* __restrict__ w, int loo, double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int c = 0; c < nc; ++c) {
        const double v = S[(int64_t)c * m + j];
        s += (__popc(c) & 1) ? -v : v;
    }
    if (loo) s -= (double)w[j];
    out[j] = C * s;
}

// ------------------------------------------------------------------ Matern-3/2 and local linear weights
// wt[i] = (y_i or 1) * (u_ik or 1) * (u_il or 1), u_i = x_i - x_0 (coordinates
// centred on the first point, which keeps the expanded moments small).
template <class T>
__global__ void k_poly_weight(const T* __restrict__ x, const T* __restrict__ y, int d, int k, int l, int64_t n,
                              double* __restrict__ wt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = y ? (double)y[i] : 1.0;
    if (k >= 0) v *= (double)x[i * d + k] - (double)x[k];
    if (l >= 0) v *= (double)x[i * d + l] - (double)x[l];
    wt[i] = v;
}

// Matern: acc[j] += (1/h_k) sum_i C w_i e^{-D_ij} |x_ik - z_jk| from the signed
// sums a[0] = C sum_delta delta_k U_delta (weights u_k), a[1] = C sum_delta delta_k T_delta.
template <class T>
__global__ void k_matern_acc_signed(const double* __restrict__ a, const T* __restrict__ zc, const T* __restrict__ x,
                                    int d, int k, int64_t m, double hk, double* __restrict__ acc) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double v = (double)zc[j * d + k] - (double)x[k];
    acc[j] += (v * a[m + j] - a[j]) / hk;
}
// ... and from the per-orthant terms T (weights w) and U (weights w u_k).
template <class T>
__global__ void k_matern_acc_terms(const double* __restrict__ Tt, const double* __restrict__ U,
                                   const T* __restrict__ zc, const T* __restrict__ x, int d, int k, int64_t m,
                                   double hk, double* __restrict__ acc) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double v = (double)zc[j * d + k] - (double)x[k];
    double s = 0.0;
    for (int o = 0; o < (1 << d); ++o) {
        const double t = v * Tt[(int64_t)o * m + j] - U[(int64_t)o * m + j];
        s += ((o >> k) & 1) ? -t : t;     // delta_k
    }
    acc[j] += s / hk;
}
__global__ void k_matern_fin(const double* __restrict__ f, const double* __restrict__ acc, int64_t m, double s,
                             double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) out[j] = (f[j] + acc[j]) * s;
}

// ------------------------------------------------------------------ matrix bandwidth
// xr[i][k] = sum_l R[l][k] x[i][l]  (R^T x), in FP64.
template <class T>
__global__ void k_rotate(const T* __restrict__ x, int d, int64_t n, dc::HVec r0, dc::HVec r1, double* __restrict__ xr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // R (d <= 4) packed row-major in r0 (rows 0, 1) and r1 (rows 2, 3)
    double xi[4];
    for (int l = 0; l < d; ++l) xi[l] = (double)x[i * d + l];
    for (int k = 0; k < d; ++k) {
        double s = 0.0;
        for (int l = 0; l < d; ++l) {
            const int e = l * d + k;
            const double rlk = e < 8 ? r0.v[e] : r1.v[e - 8];
            s = fma(rlk, xi[l], s);
        }
        xr[i * d + k] = s;
    }
}

// ------------------------------------------------------------------ locally linear fit
// Moments (all carrying the same constant C, which cancels): row 0 S0 = sum K,
// rows 1..d P_k = sum K u_k, then Q_kl (k <= l) = sum K u_k u_l, then T0 =
// sum K y, then R_k = sum K y u_k.  At target v = z - x_0:
//   S1_k = P_k - v_k S0,  S2_kl = Q_kl - v_k P_l - v_l P_k + v_k v_l S0,
//   T1_k = R_k - v_k T0,
// and [S0 S1^T; S1 S2] [a; b] = [T0; T1] gives m(z) = a (partial pivoting; NaN
// when a pivot vanishes).
template <class T>
__global__ void k_loclin_solve(const double* __restrict__ mom, const T* __restrict__ zc, const T* __restrict__ x,
                               int d, int64_t m, double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int np = d * (d + 1) / 2;
    double v[4];
    for (int k = 0; k < d; ++k) v[k] = (double)zc[j * d + k] - (double)x[k];
    const double S0 = mom[j];
    double P[4], R[4];
    for (int k = 0; k < d; ++k) P[k] = mom[(int64_t)(1 + k) * m + j];
    const double T0 = mom[(int64_t)(1 + d + np) * m + j];
    for (int k = 0; k < d; ++k) R[k] = mom[(int64_t)(2 + d + np + k) * m + j];
    const int n = d + 1;
    double A[5][6];
    A[0][0] = S0;
    A[0][n] = T0;
    for (int k = 0; k < d; ++k) {
        const double s1 = P[k] - v[k] * S0;
        A[0][1 + k] = s1;
        A[1 + k][0] = s1;
        A[1 + k][n] = R[k] - v[k] * T0;
    }
    int q = 0;
    for (int k = 0; k < d; ++k)
        for (int l = k; l < d; ++l, ++q) {
            const double Q = mom[(int64_t)(1 + d + q) * m + j];
            const double s2 = Q - v[k] * P[l] - v[l] * P[k] + v[k] * v[l] * S0;
            A[1 + k][1 + l] = s2;
            A[1 + l][1 + k] = s2;
        }
    // Gaussian elimination with partial pivoting on the augmented matrix
    bool ok = true;
    for (int c = 0; c < n && ok; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (!(A[p][c] != 0.0)) { ok = false; break; }
        if (p != c)
            for (int e = 0; e <= n; ++e) { const double t = A[c][e]; A[c][e] = A[p][e]; A[p][e] = t; }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int e = c; e <= n; ++e) A[r][e] -= f * A[c][e];
        }
    }
    double sol[5];
    if (ok) {
        for (int r = n - 1; r >= 0; --r) {
            double s = A[r][n];
            for (int e = r + 1; e < n; ++e) s -= A[r][e] * sol[e];
            sol[r] = s / A[r][r];
        }
    }
    out[j] = ok ? sol[0] : __longlong_as_double(0x7ff8000000000000LL);
}

template <class F>
void launch_typed(fk_dtype xd, F&& f) {
    if (xd == FK_F32) f((float)0);
    else f((double)0);
}

}  // namespace

// Runs a nested operation on the arena above `mark`, keeping the high-water mark.
struct NestedK {
    Arena& ar;
    size_t mark;
    size_t high;
    explicit NestedK(Arena& a) : ar(a), mark(a.used), high(a.used) {}
    void done() {
        if (ar.used > high) high = ar.used;
        ar.used = mark;
    }
    void finish() { ar.used = high; }
};

// ------------------------------------------------------------------ uniform kernel
fk_status uniform_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                      const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const bool loo = sample && (flags & FK_LOO);
    const int64_t m = sample ? N : M;
    const int nc = 1 << d;
    const size_t ds = (xd == FK_F64) ? 8 : 4;
    void* zc = ar.take<char>((size_t)nc * m * d * ds);
    void* S = ar.take<char>((size_t)nc * m * 8);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (uniform kernel)");
    dc::HVec hv;
    for (int k = 0; k < 8; ++k) hv.v[k] = (k < d) ? h[k] : 1.0;
    if (!ar.sizing && m > 0) {
        const void* zs = sample ? x : z;
        launch_typed(xd, [&](auto t) {
            using T = decltype(t);
            k_uniform_corners<T><<<grid_for((int64_t)nc * m, 256), 256, 0, st>>>((const T*)zs, d, m, nc, hv, (T*)zc);
        });
        FK_LAUNCH_CHECK();
    }
    uint32_t mask[8] = {1u, 0, 0, 0, 0, 0, 0, 0};     // orthant 0: x <= threshold on every axis
    NestedK nest(ar);
    FK_TRY(points_orthant(x, xd, N, d, w, ar.sizing ? (const void*)1 : zc, (int64_t)nc * m, mask,
                          ar.sizing ? nullptr : S, path, ar, st));
    nest.done();
    nest.finish();
    if (ar.sizing || m == 0) return FK_OK;
    const int64_t nn = loo ? N - 1 : N;
    double C = 0.0;
    if (nn > 0) {
        C = ldexp(1.0, -d) / (double)nn;
        for (int k = 0; k < d; ++k) C /= h[k];
    }
    const unsigned g = grid_for(m, 256);
    if (!w) {
        k_uniform_combine_counts<float><<<g, 256, 0, st>>>((const int64_t*)S, nc, m, C, loo ? 1 : 0, out);
    } else {
        launch_typed(xd, [&](auto t) {
            using T = decltype(t);
            k_uniform_combine_sums<T><<<g, 256, 0, st>>>((const double*)S, nc, m, C, (const T*)w, loo ? 1 : 0, out);
        });
    }
    FK_LAUNCH_CHECK();
    return FK_OK;
}

// ------------------------------------------------------------------ Matern-3/2 (additive)
fk_status matern32_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                       const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const int64_t m = sample ? N : M;
    const int no = 1 << d;
    // unweighted mixed path: signed sums formed inside the folded sweep (one
    // two-channel pass per axis); otherwise the per-orthant terms
    const bool fast = (w == nullptr) && path == FK_PATH_MIXED;
    double* f = ar.take<double>((size_t)m);
    double* acc = ar.take<double>((size_t)m);
    double* wt = ar.take<double>((size_t)N);
    double* a2 = fast ? ar.take<double>((size_t)2 * m) : nullptr;
    double* Tt = fast ? nullptr : ar.take<double>((size_t)no * m);
    double* U = fast ? nullptr : ar.take<double>((size_t)no * m);
    double* fu = fast ? nullptr : ar.take<double>((size_t)m);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (Matern kernel)");
    NestedK nest(ar);
    FK_TRY(points_kernel(x, xd, N, d, w, z, M, h, flags, 1, ar.sizing ? (double*)1 : f,
                         fast ? nullptr : (ar.sizing ? (double*)1 : Tt), path, ar, st));
    nest.done();
    if (!ar.sizing && m > 0) FK_CUDA(cudaMemsetAsync(acc, 0, (size_t)m * sizeof(double), st));
    const void* zc = sample ? x : z;
    for (int k = 0; k < d; ++k) {
        if (!ar.sizing && N > 0) {
            launch_typed(xd, [&](auto t) {
                using T = decltype(t);
                k_poly_weight<T><<<grid_for(N, 256), 256, 0, st>>>((const T*)x, fast ? nullptr : (const T*)w, d, k,
                                                                   -1, N, wt);
            });
            FK_LAUNCH_CHECK();
        }
        const double* wtp = ar.sizing ? (const double*)1 : wt;
        if (fast) {
            FK_TRY(points_kernel(x, xd, N, d, wtp, z, M, h, flags, 2, ar.sizing ? (double*)1 : a2, nullptr, path,
                                 ar, st, FK_F64, k));
        } else {
            FK_TRY(points_kernel(x, xd, N, d, wtp, z, M, h, flags, 1, ar.sizing ? (double*)1 : fu,
                                 ar.sizing ? (double*)1 : U, path, ar, st, FK_F64));
        }
        nest.done();
        if (!ar.sizing && m > 0) {
            launch_typed(xd, [&](auto t) {
                using T = decltype(t);
                if (fast)
                    k_matern_acc_signed<T><<<grid_for(m, 256), 256, 0, st>>>(a2, (const T*)zc, (const T*)x, d, k, m,
                                                                            h[k], acc);
                else
                    k_matern_acc_terms<T><<<grid_for(m, 256), 256, 0, st>>>(Tt, U, (const T*)zc, (const T*)x, d, k,
                                                                           m, h[k], acc);
            });
            FK_LAUNCH_CHECK();
        }
    }
    nest.finish();
    if (!ar.sizing && m > 0) {
        k_matern_fin<<<grid_for(m, 256), 256, 0, st>>>(f, acc, m, 1.0 / (double)(1 + d), out);
        FK_LAUNCH_CHECK();
    }
    return FK_OK;
}

// ------------------------------------------------------------------ matrix bandwidth
// R: row-major d x d (columns are the eigenvectors), hd: [d] > 0.
fk_status hmatrix_run(const void* x, fk_dtype xd, int64_t N, int d, const void* w, const void* z, int64_t M,
                      const double* R, const double* hd, unsigned flags, double* out, fk_path path, Arena& ar,
                      cudaStream_t st) {
    const bool sample = (z == nullptr);
    double* xr = ar.take<double>((size_t)N * d);
    double* zr = sample ? nullptr : ar.take<double>((size_t)M * d);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (matrix bandwidth)");
    if (!ar.sizing) {
        dc::HVec r0, r1;
        for (int e = 0; e < 8; ++e) {
            r0.v[e] = e < d * d ? R[e] : 0.0;
            r1.v[e] = e + 8 < d * d ? R[e + 8] : 0.0;
        }
        launch_typed(xd, [&](auto t) {
            using T = decltype(t);
            if (N > 0) k_rotate<T><<<grid_for(N, 256), 256, 0, st>>>((const T*)x, d, N, r0, r1, xr);
            if (!sample && M > 0) k_rotate<T><<<grid_for(M, 256), 256, 0, st>>>((const T*)z, d, M, r0, r1, zr);
        });
        FK_LAUNCH_CHECK();
    }
    NestedK nest(ar);
    FK_TRY(points_kernel(ar.sizing ? (const void*)1 : xr, FK_F64, N, d, w, sample ? nullptr : (ar.sizing ? (const void*)1 : zr),
                         M, hd, flags, 1, out, nullptr, path, ar, st, xd));
    nest.done();
    nest.finish();
    return FK_OK;
}

// ------------------------------------------------------------------ locally linear regression
fk_status loclin_run(const void* x, fk_dtype xd, int64_t N, int d, const void* y, const void* z, int64_t M,
                     const double* h, unsigned flags, double* out, fk_path path, Arena& ar, cudaStream_t st) {
    const bool sample = (z == nullptr);
    const int64_t m = sample ? N : M;
    const int np = d * (d + 1) / 2;
    const int nm = 2 + 2 * d + np;
    double* mom = ar.take<double>((size_t)nm * m);
    double* wt = ar.take<double>((size_t)N);
    if (!ar.sizing && ar.overflow()) return set_error(FK_ERR_WORKSPACE, "workspace too small (local linear)");
    NestedK nest(ar);
    // rows: 1, u_k, u_k u_l (k <= l), y, y u_k
    int row = 0;
    auto pass = [&](bool with_y, int k, int l) -> fk_status {
        const void* wp = nullptr;
        fk_dtype wd = FK_F64;
        if (with_y && k < 0) {
            wp = y;
            wd = xd;
        } else if (with_y || k >= 0) {
            if (!ar.sizing && N > 0) {
                launch_typed(xd, [&](auto t) {
                    using T = decltype(t);
                    k_poly_weight<T><<<grid_for(N, 256), 256, 0, st>>>((const T*)x, with_y ? (const T*)y : nullptr, d,
                                                                       k, l, N, wt);
                });
                FK_LAUNCH_CHECK();
            }
            wp = ar.sizing ? (const void*)1 : wt;
        }
        FK_TRY(points_kernel(x, xd, N, d, wp, z, M, h, flags, 1, ar.sizing ? (double*)1 : mom + (size_t)row * m,
                             nullptr, path, ar, st, wd));
        nest.done();
        ++row;
        return FK_OK;
    };
    FK_TRY(pass(false, -1, -1));
    for (int k = 0; k < d; ++k) FK_TRY(pass(false, k, -1));
    for (int k = 0; k < d; ++k)
        for (int l = k; l < d; ++l) FK_TRY(pass(false, k, l));
    FK_TRY(pass(true, -1, -1));
    for (int k = 0; k < d; ++k) FK_TRY(pass(true, k, -1));
    nest.finish();
    if (!ar.sizing && m > 0) {
        const void* zc = sample ? x : z;
        launch_typed(xd, [&](auto t) {
            using T = decltype(t);
            k_loclin_solve<T><<<grid_for(m, 128), 128, 0, st>>>(mom, (const T*)zc, (const T*)x, d, m, out);
        });
        FK_LAUNCH_CHECK();
    }
    return FK_OK;
}

}  // namespace fk
