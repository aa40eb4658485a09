"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and shapes them into point sets; it holds
none of the method's arithmetic, imports neither the CUDA binding nor the
oracle, and is the one module shared by the tests, the benchmark and the smoke
check.  The paper's own experiments use synthetic data only (X ~ N(0, I_d),
h = 0.1; Sec. 4), so no dataset is being stood in for.

Workloads (all seeds fixed):

* ``ecdf_small``   -- d=2, N=1e4, U[0,1]^2 in FP64, 10% of the coordinates
  replaced by rint(100 x)/100 to force ties; y == 1 and y ~ N(0,1) (seed 11);
  grid linspace(0,1,128) per axis, plus a tie grid k/100, k=0..100.
* ``ecdf_gauss3``  -- d=3, N=1e6, N(0, S) with S_ij = 0.5 off the diagonal
  (Cholesky in FP64, stored FP32, seed 2); y ~ U[0,1] FP32 (seed 12); grid of
  256 points per axis spanning [min x_k, max x_k].
* ``copula_t4``    -- d=2, N=1e6 Gaussian-copula sample, rho = 0.7, Student-t
  nu=4 marginals scaled to unit variance (FP32, seed 3); regression target
  y = sin(x1 + x2) + 0.1 N(0,1) (seed 13).
* ``batched``      -- 512 datasets, N_b = round(10^U(3,5)), d_b alternating
  2/3, x ~ U[0,1]^d FP32, y ~ N(0,1), seeds 4000+b.
* ``copula_exp4``  -- d=4, N=4e6, Gaussian copula with equicorrelation 0.3 and
  exponential(1) marginals standardised to mean 0 (x - 1), FP32 (seed 5).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _norm_cdf(g):
    # Phi(g) = (1 + erf(g / sqrt 2)) / 2, vectorised through the scipy/numpy erf.
    try:
        from scipy.special import ndtr
        return ndtr(g)
    except Exception:  # pragma: no cover - scipy is present on every machine used
        v = np.vectorize(lambda t: 0.5 * (1.0 + math.erf(t / math.sqrt(2.0))))
        return v(g)


def t4_quantile(u):
    """Closed-form quantile of Student's t with 4 degrees of freedom (Shaw 2006):
    sign(u-1/2) * 2 sqrt(q-1), q = cos(arccos(sqrt a)/3)/sqrt a, a = 4u(1-u)."""
    u = np.asarray(u, dtype=np.float64)
    a = 4.0 * u * (1.0 - u)
    a = np.clip(a, 1e-300, 1.0)
    sa = np.sqrt(a)
    q = np.cos(np.arccos(sa) / 3.0) / sa
    return np.sign(u - 0.5) * 2.0 * np.sqrt(np.maximum(q - 1.0, 0.0))


def ecdf_small(n=10_000, seed=1, tie_frac=0.10):
    """d=2 uniform points in FP64 with rounded (tied) coordinates."""
    r = _rng(seed)
    x = r.random((n, 2))
    mask = r.random((n, 2)) < tie_frac
    x[mask] = np.rint(100.0 * x[mask]) / 100.0
    y = _rng(seed + 10).standard_normal(n)
    grid = [np.linspace(0.0, 1.0, 128), np.linspace(0.0, 1.0, 128)]
    tie_grid = [np.arange(101) / 100.0, np.arange(101) / 100.0]
    return dict(x=x, y=y, grid=grid, tie_grid=tie_grid)


def ecdf_gauss3(n=1_000_000, seed=2, m_axis=256):
    """d=3 correlated Gaussian points (S_ij = 0.5 off the diagonal), FP32."""
    r = _rng(seed)
    cov = np.full((3, 3), 0.5)
    np.fill_diagonal(cov, 1.0)
    chol = np.linalg.cholesky(cov)
    x = (r.standard_normal((n, 3)) @ chol.T).astype(np.float32)
    y = _rng(seed + 10).random(n).astype(np.float32)
    x64 = x.astype(np.float64)
    grid = [np.linspace(x64[:, k].min(), x64[:, k].max(), m_axis) for k in range(3)]
    return dict(x=x, y=y, grid=grid)


def gauss_copula(n, d, corr, seed):
    """Uniforms u = Phi(g) of a Gaussian copula with the given correlation matrix."""
    r = _rng(seed)
    chol = np.linalg.cholesky(np.asarray(corr, dtype=np.float64))
    g = r.standard_normal((n, d)) @ chol.T
    u = _norm_cdf(g)
    return np.clip(u, 1e-16, 1.0 - 1e-16)


def copula_t4(n=1_000_000, seed=3, rho=0.7):
    """d=2 Gaussian copula with unit-variance Student-t(4) marginals, FP32."""
    u = gauss_copula(n, 2, [[1.0, rho], [rho, 1.0]], seed)
    x = (t4_quantile(u) / math.sqrt(2.0)).astype(np.float32)
    x64 = x.astype(np.float64)
    y = (np.sin(x64[:, 0] + x64[:, 1]) + 0.1 * _rng(seed + 10).standard_normal(n))
    return dict(x=x, y=y.astype(np.float32))


def copula_exp4(n=4_000_000, seed=5, rho=0.3):
    """d=4 Gaussian copula, equicorrelation rho, exponential(1) marginals - 1, FP32."""
    corr = np.full((4, 4), rho)
    np.fill_diagonal(corr, 1.0)
    u = gauss_copula(n, 4, corr, seed)
    x = (-np.log1p(-u) - 1.0).astype(np.float32)
    return dict(x=x)


def batched(count=512, seed0=4000, lo=3.0, hi=5.0):
    """List of independent datasets of uneven size and dimension."""
    out = []
    for b in range(count):
        r = _rng(seed0 + b)
        n = int(round(10.0 ** r.uniform(lo, hi)))
        d = 2 if (b % 2 == 0) else 3
        x = r.random((n, d)).astype(np.float32)
        y = r.standard_normal(n).astype(np.float32)
        out.append(dict(x=x, y=y, d=d, n=n))
    return out


def gaussian(n, d, seed, dtype=np.float32):
    """X ~ N(0, I_d), the paper's own test distribution (Sec. 4)."""
    return _rng(seed).standard_normal((n, d)).astype(dtype)


def sample_targets(n, k, seed, include=()):
    """k distinct seeded indices out of n, always containing ``include``."""
    r = _rng(seed)
    k = min(k, n)
    idx = set(int(i) for i in include if 0 <= int(i) < n)
    extra = r.choice(n, size=min(n, k + len(idx)), replace=False)
    for i in extra:
        if len(idx) >= k:
            break
        idx.add(int(i))
    return np.array(sorted(idx), dtype=np.int64)
