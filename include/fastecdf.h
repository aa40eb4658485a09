/*
 * fastecdf.h -- C ABI of the GB300 (sm_103a) implementation of the fast exact
 * multivariate ECDF / ESF and Laplacian-kernel KDE / kernel regression of
 * Langrene & Warin, "Fast multivariate empirical cumulative distribution
 * function with connection to kernel density estimation" (arXiv 2005.03246).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Points.  x is [N][d] row-major (point i occupies x[i*d .. i*d+d-1]) in the
 *   dtype given by `xdtype` (FK_F32 or FK_F64).  Weights y / w, when given, are
 *   [N] in the same dtype.  Explicit targets z are [M][d] in the same dtype.
 * Orthants.  The problem statement (Sec. 1, eqs. ECDF, ESF, ECDFdelta) is read
 *   in the reflected form used by eq. (Laplacian decomposition nD), Sec. 3.1:
 *   orthant o in [0, 2^d) tests, on every axis k, x_k <= z_k when bit k of o is
 *   clear (delta_k = +1) and x_k > z_k when bit k is set (delta_k = -1).
 *   o = 0 is the ECDF (eq. ECDF), o = 2^d - 1 the ESF (eq. ESF); the 2^d
 *   orthants partition the sources.  A source equal to its target is counted
 *   once, in orthant 0.
 * Targets.  z == NULL always means the sample points; an empty explicit
 *   target set (M = 0) is passed with any non-NULL z and writes nothing.
 * Orthant selection.  `orthant_mask` is a HOST bitset of ceil(2^d/32) uint32
 *   words (bit o of word o/32 selects orthant o); NULL selects all orthants.
 *   Outputs hold the selected orthants in increasing index, one row each.
 *   A mask that selects no orthant writes nothing and returns FK_OK.
 * Normalisation.  Orthant outputs are UNNORMALISED sums (Remark 1, Sec. 2.1):
 *   divide by N for F_N.  Counts (y == NULL) are exact int64.
 * Precision.  FK_PATH_MIXED accumulates bulk sums in FP32 with compensated
 *   (two-sum) arithmetic and keeps exponent arithmetic and the final
 *   combination in FP64; FK_PATH_FP64 does everything in FP64.  Counts are
 *   exact on both paths.
 * Memory.  Every array argument may be a device pointer (the normal case) or
 *   a host pointer; host arrays are staged through device buffers that the
 *   library allocates and frees in stream order.  With device pointers the
 *   call is asynchronous on `stream`.  If every host array of the call is
 *   page-locked (cudaHostAlloc / cudaHostRegister) the call is asynchronous
 *   too: host outputs are written when `stream` reaches the copies, and host
 *   inputs must not change before then.  With any pageable host array the
 *   call returns only after the host outputs are written.  The caller owns
 *   every buffer; the library never frees caller memory and keeps no state
 *   between calls other than the per-device error word (fk_device_status),
 *   its own streams, and the memory its pool caches (fk_release_cached_memory).
 * Workspace.  `ws`/`ws_bytes` is caller-owned device scratch of at least the
 *   size returned by the matching *_workspace function (256-byte aligned).
 *   If ws == NULL the library allocates and frees its scratch itself
 *   (stream-ordered).  A non-NULL ws that is too small returns FK_ERR_WORKSPACE.
 *   The library's own allocations (scratch and host-array staging) come from
 *   a stream-ordered memory pool per device that keeps freed memory for later
 *   calls; fk_release_cached_memory() returns it to the driver.
 * Limits.  1 <= d <= 8 for the grid call and for orthant counts at the
 *   sample points (fk_ecdf_points / fk_esf_points with y == NULL; the work
 *   grows as N log^(d-1) N); 1 <= d <= 6 for the weighted orthant sums,
 *   fk_kde_laplace without orthant_terms and fk_kreg_laplace; 1 <= d <= 4 for
 *   per-orthant terms, the adjoint (fk_kde_laplace_backward), the
 *   leave-one-out likelihood (fk_loo_laplace) and the other kernels (uniform
 *   kernel with weights, Matern-3/2, full bandwidth matrix, locally linear);
 *   N + M must be below 2^26 items on the
 *   sample-point path (2N + ... when orthant sums are taken at the sample
 *   points, which doubles each point into a source and a target copy).
 *   Other values return FK_ERR_UNSUPPORTED.
 * Errors.  Each call returns an fk_status; fk_last_error() gives a thread-local
 *   message.  Nothing is thrown across the ABI.  Argument errors the host can
 *   see are returned at once.  Errors found on the device are recorded in the
 *   device's error word instead (the call itself stays asynchronous and
 *   returns FK_OK); fk_device_status() returns and clears the first one.
 *   Non-finite coordinates: a NaN or +-inf in x, in explicit targets z, or
 *   in the interpolation points q is detected by the kernel that first reads
 *   that coordinate (no extra pass over the data) and recorded as
 *   FK_ERR_NONFINITE; the outputs of that call are undefined, and no memory
 *   outside the call's buffers is touched.
 */
#ifndef FASTECDF_H
#define FASTECDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fk_stream_t;   /* same type as cudaStream_t */

typedef enum {
    FK_OK = 0,
    FK_ERR_INVALID_ARG = -1,
    FK_ERR_UNSUPPORTED = -2,
    FK_ERR_WORKSPACE = -3,
    FK_ERR_NONFINITE = -4,
    FK_ERR_CUDA = -5,
    FK_ERR_TIMEOUT = -6
} fk_status;

typedef enum { FK_F32 = 0, FK_F64 = 1 } fk_dtype;

typedef enum { FK_PATH_MIXED = 0, FK_PATH_FP64 = 1 } fk_path;

/* flags for the kernel-density calls */
#define FK_LOO 1u   /* leave one out: at the sample points, drop exactly the i == j term
                       and normalise by N - 1 */

/* Thread-local description of the last error returned on this thread. */
const char* fk_last_error(void);

/* Library version string. */
const char* fk_version(void);

/*
 * ---------------------------------------------------------------- grid path
 * fk_ecdf_grid -- orthant sums on a rectilinear grid (Sec. 2.1, Algorithm 1,
 * with the local sums of Appendix A, Algorithms 6-7).
 *   z_axes : concatenation of the d grid axes, axis k holding M[k] strictly
 *            increasing FP64 values (as eq. partial sums requires); host or
 *            device.  Not strictly increasing -> FK_ERR_INVALID_ARG.
 *   M      : HOST array of d axis lengths, each >= 1.
 *   y      : [N] weights or NULL (exact int64 counts).
 *   out    : [n_sel][M[0]]...[M[d-1]] (last axis fastest), int64 when y == NULL,
 *            else double.  n_sel = number of selected orthants.
 * Each point is binned with exact comparisons (mesh division plus an exact
 * fix-up on uniform axes, binary search otherwise), the generalized histogram
 * of eq. (partial sums) is formed without the 1/N factor (Remark 1), and the
 * orthant sums are obtained by per-axis inclusive prefix sums (delta_k = +1)
 * and strict suffix sums (delta_k = -1).
 */
size_t fk_ecdf_grid_workspace(int64_t N, int d, const int64_t* M, int weighted, fk_path path);
fk_status fk_ecdf_grid(const void* x, fk_dtype xdtype, int64_t N, int d, const void* y,
                       const double* z_axes, const int64_t* M,
                       const uint32_t* orthant_mask, void* out, fk_path path,
                       void* ws, size_t ws_bytes, fk_stream_t stream);

/*
 * fk_kde_grid -- the Laplacian KDE of eq. (Laplacian kde nD) at every point
 * of a rectilinear grid (x, w, z_axes, M as fk_ecdf_grid; h [d] > 0):
 *   out[M[0]]...[M[d-1]] (double) = 1/(2^d N prod h) sum_i w_i e^{-sum_k |x_ik - z_k| / h_k}.
 * The grid form of eq. (Laplacian decomposition nD): each point enters one
 * histogram channel per orthant with its factors relative to its own cell's
 * grid lines (all <= 1), and per-axis linear recurrences with the decays
 * e^{-(z_{k,s} - z_{k,s-1}) / h_k} (<= 1) carry them to every grid point --
 * the fast summation of Sec. 2.1 with a decay.  Exact at the grid points, no
 * exponent can overflow, any strictly increasing axes.  FK_PATH_MIXED takes
 * the point factors with an FP32 exponential (the recurrences stay FP64).
 * Workspace: 2 x 2^d x prod(M_k + 1) doubles.
 */
size_t fk_kde_grid_workspace(int64_t N, int d, const int64_t* M, fk_path path);
fk_status fk_kde_grid(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w,
                      const double* z_axes, const int64_t* M, const double* h, double* out,
                      fk_path path, void* ws, size_t ws_bytes, fk_stream_t stream);

/*
 * fk_grid_interp -- multilinear interpolation of a grid function
 * f [M[0]]...[M[d-1]] (double, device or host; e.g. the output of
 * fk_kde_grid) at Q points q [Q][d] (qdtype): out [Q] double.  Coordinates
 * outside [z_{k,0}, z_{k,M_k - 1}] are clamped to the nearest grid line.
 * Workspace: fk_grid_interp_workspace() bytes (or NULL: allocated).
 */
size_t fk_grid_interp_workspace(void);
fk_status fk_grid_interp(const double* f, int d, const double* z_axes, const int64_t* M, const void* q,
                         fk_dtype qdtype, int64_t Q, double* out, void* ws, size_t ws_bytes,
                         fk_stream_t stream);

/*
 * -------------------------------------------------------- sample-point path
 * fk_ecdf_points -- orthant sums at the sample points (z == NULL, M ignored)
 * or at M explicit targets z [M][d], by rank transform and divide-and-conquer
 * dominance sums (Sec. 2.2, Algorithms 2-5; all orthants in one recursion as
 * in Appendix D, Algorithms 8-12).
 *   out : [n_sel][M'] with M' = N (sample points) or M; int64 when y == NULL,
 *         else double.
 * Counts at the sample points (y == NULL, z == NULL, N >= 2) hold each point
 * as one item that is both a source and a target: equal coordinates are
 * ordered by point index, and the pairs this order misses (tied on an axis,
 * later index as the source) are added from the tie groups of the sorted
 * axes.  The call reads the tie statistics back once (it synchronises
 * `stream` after the rank transform); if some axis has a tie group longer
 * than 64 points it uses a source copy and a target copy of every point
 * instead.  Either way the counts are exact.  On a stream that is being
 * captured into a CUDA graph the call takes the copy layout directly (no
 * read-back, so it can be captured; with device arrays and ws given or the
 * library's stream-ordered pool); the captured graph gives the same counts.
 */
size_t fk_ecdf_points_workspace(int64_t N, int d, int64_t M, int sample_points,
                                int weighted, fk_path path);
fk_status fk_ecdf_points(const void* x, fk_dtype xdtype, int64_t N, int d, const void* y,
                         const void* z, int64_t M, const uint32_t* orthant_mask,
                         void* out, fk_path path, void* ws, size_t ws_bytes,
                         fk_stream_t stream);

/*
 * fk_esf_points -- the empirical survival function of eq. (ESF), Sec. 1:
 * sum_i y_i 1{x_i1 > z_1, ..., x_id > z_d}, i.e. orthant 2^d - 1 of
 * fk_ecdf_points.  out : [M'] int64 (y == NULL) or double.
 * Workspace: fk_ecdf_points_workspace with the same arguments.
 */
fk_status fk_esf_points(const void* x, fk_dtype xdtype, int64_t N, int d, const void* y,
                        const void* z, int64_t M, void* out, fk_path path,
                        void* ws, size_t ws_bytes, fk_stream_t stream);

/*
 * fk_kde_laplace -- Laplacian kernel density estimate, eq. (Laplacian kde nD):
 *   f(z_j) = 1/(2^d N prod_k h_k) sum_i w_i exp(-sum_k |x_ik - z_jk| / h_k),
 * assembled from the 2^d exponentially weighted orthant sums of eq.
 * (Laplacian decomposition nD) with source weights w_i e^{delta.x_i/h}, the
 * exponent factors carried as an FP64-computed mantissa with a separate
 * power-of-two shift so that no factor overflows.
 *   w      : [N] weights or NULL (w == 1).
 *   z      : [M][d] targets or NULL (the sample points; M ignored).
 *   h      : HOST [d] bandwidths, each finite and > 0.
 *   flags  : FK_LOO (only with z == NULL).
 *   out    : [M'] double.
 *   orthant_terms : optional [2^d][M'] double; receives the per-orthant terms
 *            C e^{-delta.z/h} S_delta (their sum is out); d <= 4.
 * 1 <= d <= 6 (d = 5, 6 run the same sweep with 16 and 32 channels).
 */
size_t fk_kde_laplace_workspace(int64_t N, int d, int64_t M, int sample_points,
                                int want_terms, fk_path path);
fk_status fk_kde_laplace(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w,
                         const void* z, int64_t M, const double* h, unsigned flags,
                         double* out, double* orthant_terms, fk_path path,
                         void* ws, size_t ws_bytes, fk_stream_t stream);

/*
 * fk_kreg_laplace -- Nadaraya-Watson kernel regression with the Laplacian
 * kernel (the weights of eq. localdens carrying the response, Sec. 3.1 and
 * Sec. 4): m(z_j) = sum_i y_i K_ij / sum_i K_ij, both sums taken by the same
 * orthant decomposition as fk_kde_laplace (for d = 5, 6 as two one-channel
 * sums, numerator and denominator).  out : [M'] double; NaN where the
 * denominator underflows to zero.  1 <= d <= 6.
 * Workspace: fk_kde_laplace_workspace(N, d, M, sample_points, 0, path) * 2.
 */
size_t fk_kreg_laplace_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path);
fk_status fk_kreg_laplace(const void* x, fk_dtype xdtype, int64_t N, int d, const void* y,
                          const void* z, int64_t M, const double* h, unsigned flags,
                          double* out, fk_path path, void* ws, size_t ws_bytes,
                          fk_stream_t stream);

/*
 * ---------------------------------------------------------------- adjoints
 * fk_kde_laplace_backward -- exact adjoint of fk_kde_laplace (derivatives of
 * eq. Laplacian kde nD), for the upstream gradient grad_out [M'] (double):
 *   grad_w [N]    sum_j g_j C e^{-D_ij}: the transposed kernel sum, computed by
 *                 the same engine with sources and targets swapped;
 *   grad_z [M][d] (explicit targets only) g_j (1/h_k) sum_delta (-delta_k) T_delta(j)
 *                 from the per-orthant terms T of eq. (Laplacian decomposition
 *                 nD); where x_ik == z_jk the pair counts in the <= orthant;
 *   grad_h [d]    sum_j g_j (-f_j/h_k + (1/h_k^2) sum_i C w_i e^{-D_ij}|x_ik - z_jk|),
 *                 the distance sums taken from d extra orthant-term passes with
 *                 weights w_i x_ik (|x - z|-weighted orthant sums).
 * Any of the three outputs may be NULL.  Same flags (FK_LOO), precision paths
 * and conventions as fk_kde_laplace; 1 <= d <= 4.
 */
size_t fk_kde_laplace_backward_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path);
fk_status fk_kde_laplace_backward(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w,
                                  const void* z, int64_t M, const double* h, unsigned flags,
                                  const double* grad_out, double* grad_w, double* grad_z, double* grad_h,
                                  fk_path path, void* ws, size_t ws_bytes, fk_stream_t stream);

/*
 * fk_loo_laplace -- leave-one-out log-likelihood of the Laplacian KDE at the
 * sample points, L(h) = (1/N) sum_j log f_{-j}(x_j) with f_{-j} the density of
 * the other N-1 points (normalised by N-1), and its gradient dL/dh [d]
 * (grad_h may be NULL): the forward pass with FK_LOO followed by the h-adjoint
 * with g_j = 1/(N f_{-j}).  loglik: [1] double.  N >= 2, 1 <= d <= 4.
 * Densities too small for the path's accumulators (within 2^25 N of FP32's
 * smallest normal number on the mixed path, 2^54 N of FP64's on the FP64
 * path: isolated points at a small h) are evaluated exactly by a separate
 * kernel (FP64 distances, one-pass log-sum-exp over all sources), which also
 * gives their part of the gradient, so the likelihood stays finite.
 */
size_t fk_loo_laplace_workspace(int64_t N, int d, fk_path path);
fk_status fk_loo_laplace(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w, const double* h,
                         double* loglik, double* grad_h, fk_path path, void* ws, size_t ws_bytes,
                         fk_stream_t stream);

/*
 * ------------------------------------------------ other kernels, full H, local linear
 * fk_kde_uniform -- uniform-kernel KDE, eq. (uniform kde nD), Sec. 3.2:
 *   f(z_j) = 1/(2^d N' prod h) sum_i w_i prod_k 1{z_jk - h_k <= x_ik <= z_jk + h_k},
 * computed as eq. (uniform decomposition nD): the signed sum over delta of
 * the ECDFs at the 2^d box corners z + delta h, the corner z_k - h_k taken
 * strict (x_k < z_k - h_k, eq. ECDFdelta).  Each corner is rounded once in
 * FP64 and turned into an exact threshold of the data's type, so the box test
 * is exact: without weights the result is the exact box count times the
 * constant.  The corners are 2^d M' explicit targets of one orthant-0 call of
 * the sample-point engine (N + 2^d M' < 2^26; d <= 8 without weights, d <= 4
 * with).  A weighted result is a signed difference of ECDFs: its error is
 * relative to the weight magnitude of the enclosing corner ECDFs.
 *   w : [N] or NULL;  z : [M][d] or NULL (the sample points);  h : HOST [d] > 0;
 *   flags : FK_LOO (z == NULL only: drops exactly i == j, N' = N - 1);
 *   out : [M'] double.
 */
size_t fk_kde_uniform_workspace(int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path);
fk_status fk_kde_uniform(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w, const void* z,
                         int64_t M, const double* h, unsigned flags, double* out, fk_path path, void* ws,
                         size_t ws_bytes, fk_stream_t stream);

/*
 * fk_kde_matern32 -- KDE with the additive multivariate Matern-3/2 kernel,
 * eq. (Matern32 average) of Appendix C with u = (x - z)/h:
 *   f(z_j) = 1/(2^d (1+d) N' prod h) sum_i w_i (1 + D_ij) e^{-D_ij},
 *   D_ij = sum_k |x_ik - z_jk| / h_k
 * (for d = 1, eq. Matern32 with bandwidth sqrt(3) h), assembled as eq.
 * (Matern32 decomposition nD): the Laplacian orthant sums with weights w
 * (giving sum w e^{-D}) plus, per axis, the orthant sums with weights w x_k,
 * which give sum w e^{-D} |x_k - z_k| (2^d (d+1) CDFs).  Coordinates are
 * centred on the first point before they become weights.  Arguments, flags,
 * limits (1 <= d <= 4) and precision paths as fk_kde_laplace.
 */
size_t fk_kde_matern32_workspace(int64_t N, int d, int64_t M, int sample_points, int weighted, fk_path path);
fk_status fk_kde_matern32(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w, const void* z,
                          int64_t M, const double* h, unsigned flags, double* out, fk_path path, void* ws,
                          size_t ws_bytes, fk_stream_t stream);

/*
 * fk_kde_laplace_hmatrix -- Laplacian KDE with a full bandwidth matrix,
 * eq. (kde nD H) of Appendix B:
 *   f(z) = 1/(|H|^{1/2} N') sum_i w_i 2^{-d} e^{-|H^{-1/2}(x_i - z)|_1},
 * with H = R diag(h)^2 R^T (symmetric eigendecomposition, cyclic Jacobi on
 * the host) and H^{-1/2} = diag(1/h) R^T, so that both point sets are rotated
 * by R^T (in FP64, on the device) and the diagonal-bandwidth KDE of
 * fk_kde_laplace runs on the rotated coordinates.  The L1 norm is not
 * rotation invariant: where H has a repeated eigenvalue the estimator
 * depends on the eigenbasis within that eigenspace (Appendix B fixes none;
 * this call uses the one its Jacobi iteration converges to).
 *   H : HOST [d][d] row-major, symmetric (to 1e-12 relative) positive
 *       definite, else FK_ERR_INVALID_ARG.  Other arguments as fk_kde_laplace
 *       (1 <= d <= 4).
 */
size_t fk_kde_laplace_hmatrix_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path);
fk_status fk_kde_laplace_hmatrix(const void* x, fk_dtype xdtype, int64_t N, int d, const void* w, const void* z,
                                 int64_t M, const double* H, unsigned flags, double* out, fk_path path, void* ws,
                                 size_t ws_bytes, fk_stream_t stream);
/*
 * fk_hmatrix_factor -- the host-side factorisation used by
 * fk_kde_laplace_hmatrix: H = R diag(h)^2 R^T with R [d][d] row-major
 * (orthonormal columns = eigenvectors) and h [d] > 0.  Host pointers only;
 * no device work.  1 <= d <= 8.
 */
fk_status fk_hmatrix_factor(const double* H, int d, double* R, double* h);

/*
 * fk_kreg_loclin_laplace -- locally linear kernel regression with the
 * Laplacian kernel K_ij = e^{-D_ij} (Sec. 4 names it beside Nadaraya-Watson):
 * m(z) = a, where (a, b) minimises sum_i K_i (y_i - a - b.(x_i - z))^2.  The
 * normal equations need the kernel sums of the weights 1, u_k, u_k u_l, y and
 * y u_k (u = x - x_0, the coordinates centred on the first point): 2 + 2d +
 * d(d+1)/2 Laplacian kernel sums, each by the engine of fk_kde_laplace; a
 * (d+1) x (d+1) solve with partial pivoting per target; NaN where a pivot
 * vanishes.  The expanded moments cancel by up to (|z - x_0| / h)^2, so only
 * FK_PATH_FP64 is accepted (FK_ERR_UNSUPPORTED otherwise).
 *   y : [N] responses (required);  other arguments as fk_kreg_laplace
 *   (FK_LOO drops i == j from every sum; 1 <= d <= 4).
 */
size_t fk_kreg_loclin_laplace_workspace(int64_t N, int d, int64_t M, int sample_points, fk_path path);
fk_status fk_kreg_loclin_laplace(const void* x, fk_dtype xdtype, int64_t N, int d, const void* y, const void* z,
                                 int64_t M, const double* h, unsigned flags, double* out, fk_path path, void* ws,
                                 size_t ws_bytes, fk_stream_t stream);

/*
 * ---------------------------------------------------------------- batching
 * fk_batched -- many independent datasets of uneven size and dimension in one
 * call (not in the paper, which treats one dataset).  Dataset b has N_b points
 * x_b [N_b][d_b] (1 <= d_b <= 4) and optional weights y_b [N_b], all DEVICE
 * pointers in the dtype `xdtype`.
 *   what & FK_BATCH_ECDF : all 2^d_b orthant counts of every dataset at its own
 *                          sample points (as fk_ecdf_points with y == NULL);
 *                          ecdf_out = concatenation over b of [2^d_b][N_b] int64.
 *   what & FK_BATCH_KDE  : the Laplacian KDE of every dataset at its own sample
 *                          points with bandwidth h on every axis and weights y_b
 *                          (1 if NULL), as fk_kde_laplace; kde_out =
 *                          concatenation over b of [N_b] double.
 * Datasets are grouped by dimension and padded size; each group runs as one
 * set of kernel launches covering all its datasets.  No host synchronisation;
 * with a caller workspace the call can be captured in a CUDA graph.
 */
typedef struct {
    const void* x;   /* [N][d] device */
    const void* y;   /* [N] device or NULL */
    int64_t N;
    int d;
    int reserved;
} fk_dataset;

#define FK_BATCH_ECDF 1u
#define FK_BATCH_KDE 2u

size_t fk_batched_workspace(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what, fk_path path);
fk_status fk_batched(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what, double h,
                     int64_t* ecdf_out, double* kde_out, fk_path path, void* ws, size_t ws_bytes,
                     fk_stream_t stream);

/*
 * Launch configuration of fk_batched (a tuning knob, not part of the paper's
 * problem; results agree across configurations within the stated tolerances,
 * counts exactly):
 *   streams     groups run concurrently on this many streams (1..8): the
 *               caller's stream and library-owned streams forked from it and
 *               joined back to it with events (so the call stays capturable in
 *               a CUDA graph); each stream gets its own workspace slot.
 *               Overlapping calls from several host threads are serialised
 *               while they enqueue.
 *   coarsen     datasets are grouped by dimension and padded size 2^E with E
 *               rounded up to a multiple of coarsen + 1 (0..2): fewer, larger
 *               launches against more padding.
 *   kernel_tile 0: default tile of the tile-local kernel-sum levels (4096
 *               items mixed, 2048 FP64), 1: half of it.
 *   count_tile  tile of the tile-local counting levels: 0: 2048, 1: 1024,
 *               2: 4096 items.
 * fk_batched uses fk_batched_config_default (1, 0, 0, 0).
 */
typedef struct {
    int streams;
    int coarsen;
    int kernel_tile;
    int count_tile;
} fk_batch_config;

void fk_batched_config_default(fk_batch_config* cfg);
size_t fk_batched_workspace_ex(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what, fk_path path,
                               const fk_batch_config* cfg);
fk_status fk_batched_ex(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what, double h,
                        int64_t* ecdf_out, double* kde_out, fk_path path, const fk_batch_config* cfg, void* ws,
                        size_t ws_bytes, fk_stream_t stream);

/*
 * fk_batched_autotune -- picks the configuration by measurement on the
 * caller's own datasets: coordinate descent over streams {1, 2, 4, 8},
 * coarsen {0, 1, 2}, count_tile {0, 1, 2} (with FK_BATCH_ECDF) and
 * kernel_tile {0, 1} (with FK_BATCH_KDE), each candidate run once to warm up
 * and timed as the best of two runs with CUDA events on `stream`.  The call
 * synchronises the stream (it cannot be captured) and leaves the outputs of
 * the last run in ecdf_out / kde_out.  ws: NULL (allocated per trial) or at
 * least fk_batched_autotune_workspace bytes (the largest candidate's need).
 * best receives the fastest configuration, best_ms (optional) its time.
 */
size_t fk_batched_autotune_workspace(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what,
                                     fk_path path);
fk_status fk_batched_autotune(const fk_dataset* sets, int count, fk_dtype xdtype, unsigned what, double h,
                              int64_t* ecdf_out, double* kde_out, fk_path path, void* ws, size_t ws_bytes,
                              fk_stream_t stream, fk_batch_config* best, double* best_ms);

/*
 * fk_ecdf_grid_counts_noalloc -- the paper has no counterpart to this call; it
 * exists for callers that may not allocate device memory while they run: loops
 * that forbid allocation after start-up (cudaMalloc can synchronise the device
 * and take unbounded time) and host applications that own the whole device
 * memory budget.  It computes the same int64 orthant counts as fk_ecdf_grid
 * with y == NULL, but never allocates: its scratch is a fixed 16 MiB array in
 * the library image, reserved on every GPU that loads the library until the
 * process exits.  A grid whose scratch (histogram and per-axis pass buffers,
 * about 4 bytes per cell of the (M_1+1)...(M_d+1) histogram plus two pass
 * buffers of up to 2^(d-1) (M_1+1)...(M_d+1) 4-byte entries) would exceed it
 * returns FK_ERR_UNSUPPORTED.  x, z_axes and out must be device pointers
 * (host arrays would need staging buffers); M and orthant_mask are host
 * arrays as for fk_ecdf_grid.  The first call on a device does a one-time
 * set-up: it looks up the scratch's device address on that device (make it
 * the current device), so make that first call before any stream capture.
 * That address is kept for the rest of the process: it does not survive a
 * reset of the device's primary context (cudaDeviceReset or a release of the
 * context by another owner), after which this call must not be used.
 * An orthant selection with no orthant returns FK_OK and writes nothing.
 * Every call uses the same scratch and zeroes the part it accumulates into;
 * calls whose work overlaps on the GPU (concurrent streams, or several host
 * threads on one device) race on it and must be serialised by the caller.
 */
fk_status fk_ecdf_grid_counts_noalloc(const void* x, fk_dtype xdtype, int64_t N, int d, const double* z_axes,
                                      const int64_t* M, const uint32_t* orthant_mask, int64_t* out,
                                      fk_stream_t stream);

/*
 * fk_release_cached_memory -- returns the memory the library's pool of the
 * current device keeps between calls (scratch and staging buffers freed by
 * earlier calls) to the driver.  Call it when no library call is in flight on
 * the device.
 */
fk_status fk_release_cached_memory(void);

/*
 * fk_device_status -- synchronises `stream` and returns (and clears) the
 * device-side error word of the current device: FK_OK, or the first error a
 * kernel recorded since the last call (e.g. FK_ERR_TIMEOUT from a bounded
 * wait).  Kernels never trap.
 */
fk_status fk_device_status(fk_stream_t stream);

/*
 * fk_debug_lookback_timeout -- a test hook for the bounded device waits (not
 * part of the paper's problem).  The rank transform's radix sort (Sec. 2.2)
 * runs one launch per digit pass in which each tile of 4096 keys waits, in a
 * decoupled look-back, for the per-digit counts the tiles before it publish;
 * every such wait gives up after a fixed number of polls (a fraction of a
 * second), records FK_ERR_TIMEOUT in the device error word and lets the
 * kernel finish.  This call runs one digit pass over n zero keys (n in
 * [8192, 2^24]) in which the first tile is never processed, so the waits run
 * out, then returns fk_device_status(stream): FK_ERR_TIMEOUT when the bound
 * works.  It allocates and frees its own device buffers and synchronises
 * `stream`; the device stays usable afterwards.  Other n: FK_ERR_INVALID_ARG.
 */
fk_status fk_debug_lookback_timeout(int64_t n, fk_stream_t stream);

/*
 * ---------------------------------------------------------------- diagnostics
 * Not part of the paper's problem statement: counters used to report
 * performance.  fk_kernel_launches returns the number of CUDA kernels this
 * library has launched in the calling process.  When profiling is enabled,
 * the main kernel families are bracketed by CUDA events recorded on the
 * stream each kernel is launched on, together with the launch's algorithmic
 * work; fk_profile_read synchronises on those events and sums them for one
 * family:
 *   0 divide-and-conquer merge with sweep, 1 its per-tile totals pass,
 *   2 plain merge (tree construction), 3 grid orthant pass, 4 grid histogram,
 *   5 radix-sort pass, 6 gathers, 7 tile-local merge levels (counts and
 *   orthant sums), 8 tile-local merge levels of the kernel sums.
 * The work (alg_bytes) is the bytes the launch must move (inputs read once,
 * outputs written once) for families 0-7, and for family 8 the arithmetic
 * operations of the sweep: 44 floating-point operations per item and merge
 * level (two compensated additions into the running sums, two scaled
 * compensated additions into the target's sum).
 */
uint64_t fk_kernel_launches(void);
void fk_profile_enable(int on);
void fk_profile_reset(void);
fk_status fk_profile_read(int family, double* total_ms, uint64_t* launches, double* alg_bytes);
/* The time the family kept the GPU busy: the union of its launches' intervals
 * (operations run independent parts on several streams, whose launches
 * overlap; total_ms above sums them). */
fk_status fk_profile_busy(int family, double* busy_ms);
/* The algorithmic bytes of the family's recorded launches (inputs read once,
 * outputs written once).  For families 0-7 this equals fk_profile_read's
 * alg_bytes; for family 8 it is the bytes its launches gather and write,
 * beside the arithmetic fk_profile_read reports.  Summed over every family it
 * gives the minimal traffic of the passes a call made. */
fk_status fk_profile_read_bytes(int family, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* FASTECDF_H */
