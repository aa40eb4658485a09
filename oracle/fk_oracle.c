/*
 * fk_oracle.c -- plain, slow, obviously-correct CPU oracle for the fast
 * multivariate ECDF / Laplacian KDE of Langrene & Warin (arXiv 2005.03246).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product (GPU) path links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Every routine is the definition written out by brute force, O(N*M*d):
 *   - orthant sums           : eq. (ECDF), (ESF), (ECDFdelta) of Sec. 1, in the
 *                              reflected reading used by eq. (Laplacian
 *                              decomposition nD) of Sec. 3.1: for orthant bit k
 *                              clear the test is x_k <= z_k, for bit k set it is
 *                              x_k > z_k.  Counts are exact int64; weighted sums
 *                              are FP64 with Neumaier compensation.
 *   - Laplacian KDE          : eq. (Laplacian kde nD), Sec. 3.1, each term
 *                              exp(-sum_k |x_k - z_k| / h_k) evaluated directly
 *                              (never through the 2^d decomposition, which can
 *                              overflow).
 *   - Nadaraya-Watson        : ratio of two kernel sums (Sec. 4 text on kernel
 *                              regression), with the kernel exponent shifted by
 *                              its minimum so the ratio is always defined.
 *   - uniform / Matern-3/2   : eq. (uniform kde nD) of Sec. 3.2 and the additive
 *                              Matern-3/2 kernel, eq. (Matern32 average) of
 *                              Appendix C, term by term.
 *   - gradients / LOO        : exact derivatives of eq. (Laplacian kde nD).
 *   - 2D Fenwick sweep       : an independent textbook sort + binary-indexed
 *                              tree count of 2D dominance (used as a second
 *                              full-output check at large N).
 *
 * Inputs are FP64; FP32 data is widened losslessly by the caller, so the oracle
 * sees exactly the bits the GPU sees.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FKO_OK 0
#define FKO_EINVAL (-1)
#define FKO_ENOMEM (-2)

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int fko_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Neumaier (improved Kahan-Babuska) compensated accumulator. */
typedef struct { double s, c; } neum_t;
static inline void neum_add(neum_t* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static inline double neum_get(const neum_t* a) { return a->s + a->c; }

/* Orthant index of source x relative to target z: bit k set <=> x_k > z_k. */
static inline uint32_t orthant_of(const double* xi, const double* zj, int d) {
    uint32_t o = 0;
    for (int k = 0; k < d; ++k)
        if (xi[k] > zj[k]) o |= (1u << k);
    return o;
}

/*
 * Generalized orthant sums S_delta(z_j) = sum_i y_i * prod_k 1{x_ik <=_delta z_jk}
 * (Sec. 1, eq. ECDFdelta, reflected reading).  `mask` is a bitset over the 2^d
 * orthant indices (bit o of word o/32), NULL selecting all of them.  Output
 * layout: the selected orthants in increasing index, each a row of length m.
 * If y == NULL the counts go to cnt_out (int64), else the sums to sum_out.
 */
int fko_orthant_sums(const double* x, int64_t n, int d, const double* y,
                     const double* z, int64_t m, const uint32_t* mask,
                     int64_t* cnt_out, double* sum_out, int nthreads) {
    if (d < 1 || d > 12 || n < 0 || m < 0) return FKO_EINVAL;
    uint32_t full = (1u << d) - 1u;
    int32_t slot[1 << 12];
    int no = 0;
    for (uint32_t o = 0; o <= full; ++o)
        slot[o] = (!mask || (mask[o >> 5] >> (o & 31u) & 1u)) ? no++ : -1;
    if (no == 0) return FKO_OK;
    set_threads(nthreads);
    const int64_t nstates = (int64_t)1 << d;
    int err = 0;
#pragma omp parallel
    {
        int64_t* cnt = NULL;
        neum_t* acc = NULL;
        if (y) acc = (neum_t*)malloc(sizeof(neum_t) * (size_t)nstates);
        else cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)nstates);
        if (!acc && !cnt) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t j = 0; j < m; ++j) {
                const double* zj = z + j * d;
                if (y) memset(acc, 0, sizeof(neum_t) * (size_t)nstates);
                else memset(cnt, 0, sizeof(int64_t) * (size_t)nstates);
                for (int64_t i = 0; i < n; ++i) {
                    uint32_t o = orthant_of(x + i * d, zj, d);
                    if (y) neum_add(&acc[o], y[i]);
                    else cnt[o] += 1;
                }
                for (uint32_t o = 0; o <= full; ++o) {
                    if (slot[o] < 0) continue;
                    if (y) sum_out[(int64_t)slot[o] * m + j] = neum_get(&acc[o]);
                    else cnt_out[(int64_t)slot[o] * m + j] = cnt[o];
                }
            }
        }
        free(acc);
        free(cnt);
    }
    return err ? FKO_ENOMEM : FKO_OK;
}

/* Normalising constant 1 / (2^d * N * prod h_k) of eq. (Laplacian kde nD). */
static double kde_const(int64_t n, int d, const double* h) {
    double c = ldexp(1.0, -d) / (double)n;
    for (int k = 0; k < d; ++k) c /= h[k];
    return c;
}

/* Scaled L1 distance sum_k |x_k - z_k| / h_k. */
static inline double l1h(const double* xi, const double* zj, const double* h, int d) {
    double a = 0.0;
    for (int k = 0; k < d; ++k) a += fabs(xi[k] - zj[k]) / h[k];
    return a;
}

/*
 * Laplacian KDE, eq. (Laplacian kde nD):
 *   f(z_j) = 1/(2^d N prod h) * sum_i w_i exp(-sum_k |x_ik - z_jk| / h_k).
 * If z == NULL the targets are the sources.  loo != 0 (only with z == NULL)
 * drops exactly the i == j term and normalises by N-1.
 * terms (optional, [2^d][m]) receives the per-orthant pieces
 * sum_{i in orthant} w_i exp(-...), already multiplied by the constant, so
 * that f = sum over orthants of terms (the decomposition of Sec. 3.1 evaluated
 * without its overflowing factorisation).
 */
int fko_kde(const double* x, int64_t n, int d, const double* w, const double* z,
            int64_t m, const double* h, int loo, double* out, double* terms,
            int nthreads) {
    if (d < 1 || d > 12 || n < 0) return FKO_EINVAL;
    if (loo && z) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    int64_t nn = loo ? n - 1 : n;
    if (nn <= 0) { for (int64_t j = 0; j < mm; ++j) out[j] = 0.0; return FKO_OK; }
    const double cst = kde_const(nn, d, h);
    const int64_t nstates = (int64_t)1 << d;
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        neum_t* acc = (neum_t*)malloc(sizeof(neum_t) * (size_t)nstates);
        if (!acc) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t j = 0; j < mm; ++j) {
                const double* zj = zz + j * d;
                memset(acc, 0, sizeof(neum_t) * (size_t)nstates);
                for (int64_t i = 0; i < n; ++i) {
                    if (loo && i == j) continue;
                    const double* xi = x + i * d;
                    double t = (w ? w[i] : 1.0) * exp(-l1h(xi, zj, h, d));
                    neum_add(&acc[terms ? orthant_of(xi, zj, d) : 0], t);
                }
                neum_t tot = {0.0, 0.0};
                for (int64_t o = 0; o < (terms ? nstates : 1); ++o) {
                    double v = neum_get(&acc[o]);
                    if (terms) terms[o * mm + j] = cst * v;
                    neum_add(&tot, v);
                }
                out[j] = cst * neum_get(&tot);
            }
        }
        free(acc);
    }
    return err ? FKO_ENOMEM : FKO_OK;
}

/*
 * The same KDE at a subset of the sample points: target j is x[idx[j]]; with
 * loo != 0 exactly the source i == idx[j] is dropped and the normalisation is
 * N-1 (the leave-one-out density f_{-j} of the bandwidth likelihood), so that
 * large-N checks can sample targets instead of evaluating all N.
 */
int fko_kde_at(const double* x, int64_t n, int d, const double* w, const int64_t* idx,
               int64_t m, const double* h, int loo, double* out, int nthreads) {
    if (d < 1 || d > 12 || n < 0 || m < 0) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    for (int64_t j = 0; j < m; ++j) if (idx[j] < 0 || idx[j] >= n) return FKO_EINVAL;
    int64_t nn = loo ? n - 1 : n;
    if (nn <= 0) { for (int64_t j = 0; j < m; ++j) out[j] = 0.0; return FKO_OK; }
    const double cst = kde_const(nn, d, h);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        const double* zj = x + idx[j] * d;
        neum_t acc = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            if (loo && i == idx[j]) continue;
            neum_add(&acc, (w ? w[i] : 1.0) * exp(-l1h(x + i * d, zj, h, d)));
        }
        out[j] = cst * neum_get(&acc);
    }
    return FKO_OK;
}

/*
 * Nadaraya-Watson regression with the Laplacian kernel:
 *   m(z_j) = sum_i y_i K_ij / sum_i K_ij,  K_ij = exp(-(a_ij - min_i a_ij)),
 *   a_ij = sum_k |x_ik - z_jk| / h_k.
 * The shift by min_i a_ij cancels in the ratio and keeps the denominator >= 1.
 */
int fko_kreg(const double* x, int64_t n, int d, const double* y, const double* z,
             int64_t m, const double* h, int loo, double* out, int nthreads) {
    if (d < 1 || d > 12 || n < 0) return FKO_EINVAL;
    if (loo && z) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < mm; ++j) {
        const double* zj = zz + j * d;
        double amin = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            if (loo && i == j) continue;
            double a = l1h(x + i * d, zj, h, d);
            if (a < amin) amin = a;
        }
        neum_t num = {0.0, 0.0}, den = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            if (loo && i == j) continue;
            double k = exp(-(l1h(x + i * d, zj, h, d) - amin));
            neum_add(&num, y[i] * k);
            neum_add(&den, k);
        }
        out[j] = (den.s + den.c) > 0.0 ? neum_get(&num) / neum_get(&den) : NAN;
    }
    return FKO_OK;
}

/*
 * Adjoint of the Laplacian KDE (exact derivatives of eq. Laplacian kde nD).
 * g[j] is the upstream gradient of f(z_j).  Outputs (each optional):
 *   grad_w[i] = sum_j g_j C exp(-a_ij)
 *   grad_z[j*d+k] = g_j C sum_i w_i exp(-a_ij) s_ijk / h_k,
 *        s_ijk = +1 if x_ik > z_jk else -1 (at x_ik == z_jk the pair belongs to
 *        the x <= z orthant, i.e. the one-sided derivative of that orthant)
 *   grad_h[k] = sum_j g_j ( -f_j / h_k + C/h_k^2 sum_i w_i exp(-a_ij) |x_ik-z_jk| )
 * grad_z is only defined for explicit targets (z != NULL).
 */
int fko_kde_grad(const double* x, int64_t n, int d, const double* w,
                 const double* z, int64_t m, const double* h, int loo,
                 const double* g, double* grad_w, double* grad_z, double* grad_h,
                 int nthreads) {
    if (d < 1 || d > 12 || n < 0) return FKO_EINVAL;
    if (loo && z) return FKO_EINVAL;
    if (grad_z && !z) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    int64_t nn = loo ? n - 1 : n;
    if (grad_w) for (int64_t i = 0; i < n; ++i) grad_w[i] = 0.0;
    if (grad_h) for (int k = 0; k < d; ++k) grad_h[k] = 0.0;
    if (nn <= 0) {
        if (grad_z) for (int64_t j = 0; j < mm * d; ++j) grad_z[j] = 0.0;
        return FKO_OK;
    }
    const double cst = kde_const(nn, d, h);
    set_threads(nthreads);
    int err = 0;
    /* grad_z and grad_h: loop over targets. */
#pragma omp parallel
    {
        neum_t* dist = (neum_t*)malloc(sizeof(neum_t) * (size_t)d);
        neum_t* sgn = (neum_t*)malloc(sizeof(neum_t) * (size_t)d);
        neum_t* gh = (neum_t*)calloc((size_t)d, sizeof(neum_t));
        if (!dist || !sgn || !gh) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t j = 0; j < mm; ++j) {
                const double* zj = zz + j * d;
                neum_t f = {0.0, 0.0};
                memset(dist, 0, sizeof(neum_t) * (size_t)d);
                memset(sgn, 0, sizeof(neum_t) * (size_t)d);
                for (int64_t i = 0; i < n; ++i) {
                    if (loo && i == j) continue;
                    const double* xi = x + i * d;
                    double t = (w ? w[i] : 1.0) * exp(-l1h(xi, zj, h, d));
                    neum_add(&f, t);
                    for (int k = 0; k < d; ++k) {
                        neum_add(&dist[k], t * fabs(xi[k] - zj[k]));
                        neum_add(&sgn[k], xi[k] > zj[k] ? t : -t);
                    }
                }
                double fj = cst * neum_get(&f);
                for (int k = 0; k < d; ++k) {
                    if (grad_z) grad_z[j * d + k] = g[j] * cst * neum_get(&sgn[k]) / h[k];
                    neum_add(&gh[k], g[j] * (-fj / h[k] + cst / (h[k] * h[k]) * neum_get(&dist[k])));
                }
            }
            if (grad_h) {
#pragma omp critical
                for (int k = 0; k < d; ++k) grad_h[k] += neum_get(&gh[k]);
            }
        }
        free(dist);
        free(sgn);
        free(gh);
    }
    if (err) return FKO_ENOMEM;
    /* grad_w: loop over sources (the transposed kernel sum). */
    if (grad_w) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            const double* xi = x + i * d;
            neum_t a = {0.0, 0.0};
            for (int64_t j = 0; j < mm; ++j) {
                if (loo && i == j) continue;
                neum_add(&a, g[j] * exp(-l1h(xi, zz + j * d, h, d)));
            }
            grad_w[i] = cst * neum_get(&a);
        }
    }
    return FKO_OK;
}

/*
 * Uniform-kernel KDE, eq. (uniform kde nD) of Sec. 3.2:
 *   f(z_j) = 1/(2^d N' prod h) sum_i w_i prod_k 1{lo_jk <= x_ik <= hi_jk},
 * with the box corners lo = z - h and hi = z + h each rounded once in FP64:
 * eq. (uniform decomposition nD) evaluates its ECDFs at exactly these corner
 * points z + delta h.  loo != 0 (z == NULL only) drops the i == j term and
 * uses N' = N - 1.  Weighted sums are Neumaier sums; without weights the box
 * count is exact before the final scaling.
 */
int fko_kde_uniform(const double* x, int64_t n, int d, const double* w, const double* z,
                    int64_t m, const double* h, int loo, double* out, int nthreads) {
    if (d < 1 || d > 12 || n < 0) return FKO_EINVAL;
    if (loo && z) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    int64_t nn = loo ? n - 1 : n;
    if (nn <= 0) { for (int64_t j = 0; j < mm; ++j) out[j] = 0.0; return FKO_OK; }
    const double cst = kde_const(nn, d, h);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < mm; ++j) {
        const double* zj = zz + j * d;
        double lo[12], hi[12];
        for (int k = 0; k < d; ++k) { lo[k] = zj[k] - h[k]; hi[k] = zj[k] + h[k]; }
        neum_t acc = {0.0, 0.0};
        int64_t cnt = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (loo && i == j) continue;
            const double* xi = x + i * d;
            int in = 1;
            for (int k = 0; k < d; ++k) in &= (lo[k] <= xi[k]) & (xi[k] <= hi[k]);
            if (!in) continue;
            if (w) neum_add(&acc, w[i]);
            else ++cnt;
        }
        out[j] = cst * (w ? neum_get(&acc) : (double)cnt);
    }
    return FKO_OK;
}

/*
 * Additive multivariate Matern-3/2 KDE, eq. (Matern32 average) of Appendix C
 * with u = (x - z)/h:
 *   f(z_j) = 1/(2^d (1+d) N' prod h) sum_i w_i (1 + D_ij) exp(-D_ij),
 *   D_ij = sum_k |x_ik - z_jk| / h_k,
 * each term evaluated directly (never through eq. Matern32 decomposition nD).
 * For d = 1 this is eq. (Matern32) with bandwidth sqrt(3) h.
 */
int fko_kde_matern32(const double* x, int64_t n, int d, const double* w, const double* z,
                     int64_t m, const double* h, int loo, double* out, int nthreads) {
    if (d < 1 || d > 12 || n < 0) return FKO_EINVAL;
    if (loo && z) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    int64_t nn = loo ? n - 1 : n;
    if (nn <= 0) { for (int64_t j = 0; j < mm; ++j) out[j] = 0.0; return FKO_OK; }
    const double cst = kde_const(nn, d, h) / (double)(1 + d);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < mm; ++j) {
        const double* zj = zz + j * d;
        neum_t acc = {0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            if (loo && i == j) continue;
            const double a = l1h(x + i * d, zj, h, d);
            neum_add(&acc, (w ? w[i] : 1.0) * (1.0 + a) * exp(-a));
        }
        out[j] = cst * neum_get(&acc);
    }
    return FKO_OK;
}

/*
 * Leave-one-out log-likelihood of the Laplacian KDE at the sample points,
 *   L(h) = (1/N) sum_j log f_{-j}(x_j),
 *   f_{-j} = 1/((N-1) 2^d prod h) sum_{i != j} w_i exp(-a_ij),
 * and its gradient dL/dh_k = (1/N) sum_j (d f_{-j}/d h_k) / f_{-j},
 *   d f_{-j}/d h_k = -f_{-j}/h_k + C/h_k^2 sum_{i!=j} w_i exp(-a_ij)|x_ik-x_jk|.
 * If f_{-j} underflows to 0 the log is -inf (reported as such).
 */
int fko_loo_loglik(const double* x, int64_t n, int d, const double* w,
                   const double* h, double* L, double* dL, int nthreads) {
    if (d < 1 || d > 12 || n < 2) return FKO_EINVAL;
    for (int k = 0; k < d; ++k) if (!(h[k] > 0.0)) return FKO_EINVAL;
    const double cst = kde_const(n - 1, d, h);
    set_threads(nthreads);
    neum_t Lacc = {0.0, 0.0};
    neum_t* dacc = (neum_t*)calloc((size_t)d, sizeof(neum_t));
    if (!dacc) return FKO_ENOMEM;
    int err = 0;
#pragma omp parallel
    {
        neum_t* dist = (neum_t*)malloc(sizeof(neum_t) * (size_t)d);
        neum_t* dl = (neum_t*)calloc((size_t)d, sizeof(neum_t));
        neum_t ll = {0.0, 0.0};
        if (!dist || !dl) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t j = 0; j < n; ++j) {
                const double* xj = x + j * d;
                neum_t f = {0.0, 0.0};
                memset(dist, 0, sizeof(neum_t) * (size_t)d);
                for (int64_t i = 0; i < n; ++i) {
                    if (i == j) continue;
                    const double* xi = x + i * d;
                    double t = (w ? w[i] : 1.0) * exp(-l1h(xi, xj, h, d));
                    neum_add(&f, t);
                    for (int k = 0; k < d; ++k) neum_add(&dist[k], t * fabs(xi[k] - xj[k]));
                }
                double s = neum_get(&f);
                neum_add(&ll, log(cst * s));
                for (int k = 0; k < d; ++k)
                    neum_add(&dl[k], -1.0 / h[k] + neum_get(&dist[k]) / (h[k] * h[k] * s));
            }
#pragma omp critical
            {
                neum_add(&Lacc, neum_get(&ll));
                for (int k = 0; k < d; ++k) neum_add(&dacc[k], neum_get(&dl[k]));
            }
        }
        free(dist);
        free(dl);
    }
    if (!err) {
        *L = neum_get(&Lacc) / (double)n;
        if (dL) for (int k = 0; k < d; ++k) dL[k] = neum_get(&dacc[k]) / (double)n;
    }
    free(dacc);
    return err ? FKO_ENOMEM : FKO_OK;
}

/* ---------------- independent 2D check: sort + Fenwick tree ---------------- */

typedef struct { double v0; int type; int64_t idx; } ev_t;   /* type 0 source, 1 target */

static int ev_cmp(const void* a, const void* b) {
    const ev_t* p = (const ev_t*)a;
    const ev_t* q = (const ev_t*)b;
    if (p->v0 < q->v0) return -1;
    if (p->v0 > q->v0) return 1;
    if (p->type != q->type) return p->type - q->type;   /* sources first on ties */
    return (p->idx < q->idx) ? -1 : (p->idx > q->idx);
}
static int dbl_cmp(const void* a, const void* b) {
    double p = *(const double*)a, q = *(const double*)b;
    return (p < q) ? -1 : (p > q);
}
/* number of entries of sorted s[0..n) that are <= v */
static int64_t upper_count(const double* s, int64_t n, double v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t mid = lo + (hi - lo) / 2; if (s[mid] <= v) lo = mid + 1; else hi = mid; }
    return lo;
}

/*
 * All four 2D orthant counts of N sources x[N,2] at M targets z[M,2] (z == NULL:
 * the sources), by a sweep on axis 0 (sources before targets on ties) with a
 * binary-indexed tree over axis 1, plus 1D counts and inclusion-exclusion
 * (exact in integers).  Output [4][m], orthant order 0..3 as above.
 */
int fko_fenwick2d(const double* x, int64_t n, const double* z, int64_t m, int64_t* out) {
    const double* zz = z ? z : x;
    int64_t mm = z ? m : n;
    ev_t* ev = (ev_t*)malloc(sizeof(ev_t) * (size_t)(n + mm));
    double* s0 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* s1 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t* bit = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* cpp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(mm > 0 ? mm : 1));
    if (!ev || !s0 || !s1 || !bit || !cpp) {
        free(ev); free(s0); free(s1); free(bit); free(cpp);
        return FKO_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        ev[i].v0 = x[2 * i]; ev[i].type = 0; ev[i].idx = i;
        s0[i] = x[2 * i]; s1[i] = x[2 * i + 1];
    }
    for (int64_t j = 0; j < mm; ++j) { ev[n + j].v0 = zz[2 * j]; ev[n + j].type = 1; ev[n + j].idx = j; }
    qsort(ev, (size_t)(n + mm), sizeof(ev_t), ev_cmp);
    qsort(s0, (size_t)n, sizeof(double), dbl_cmp);
    qsort(s1, (size_t)n, sizeof(double), dbl_cmp);
    for (int64_t e = 0; e < n + mm; ++e) {
        if (ev[e].type == 0) {
            /* position of this source's axis-1 value among sorted source values (1-based) */
            int64_t p = upper_count(s1, n, x[2 * ev[e].idx + 1]);
            for (; p <= n; p += p & (-p)) bit[p] += 1;
        } else {
            int64_t q = upper_count(s1, n, zz[2 * ev[e].idx + 1]);
            int64_t c = 0;
            for (; q > 0; q -= q & (-q)) c += bit[q];
            cpp[ev[e].idx] = c;
        }
    }
    for (int64_t j = 0; j < mm; ++j) {
        int64_t c0 = upper_count(s0, n, zz[2 * j]);       /* #{x0 <= z0} */
        int64_t c1 = upper_count(s1, n, zz[2 * j + 1]);   /* #{x1 <= z1} */
        out[0 * mm + j] = cpp[j];                          /* (<=, <=) */
        out[1 * mm + j] = c1 - cpp[j];                     /* (> , <=) */
        out[2 * mm + j] = c0 - cpp[j];                     /* (<=, > ) */
        out[3 * mm + j] = n - c0 - c1 + cpp[j];            /* (> , > ) */
    }
    free(ev); free(s0); free(s1); free(bit); free(cpp);
    return FKO_OK;
}
