"""The seeded input recipes (no GPU): shapes, dtypes, reproducibility and the
distributional properties each workload is defined by (tie fraction, Gaussian
correlation, copula dependence via Kendall's tau, marginals)."""
import math

import numpy as np
import pytest

from paper_2005_03246_gb300 import datagen


def test_t4_quantile_closed_form_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    u = np.concatenate([np.logspace(-12, -1, 40), np.linspace(0.1, 0.9, 81), 1 - np.logspace(-12, -1, 40)])
    np.testing.assert_allclose(datagen.t4_quantile(u), stats.t.ppf(u, 4), rtol=1e-9, atol=1e-12)


def test_small_workload_ties_and_reproducibility():
    a = datagen.ecdf_small(n=20000)
    b = datagen.ecdf_small(n=20000)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])
    x = a["x"]
    assert x.dtype == np.float64 and x.shape == (20000, 2)
    assert x.min() >= 0.0 and x.max() <= 1.0
    on_lattice = np.rint(100.0 * x) / 100.0 == x
    assert abs(on_lattice.mean() - 0.10) < 0.01           # ~10% of the coordinates rounded
    assert len(a["grid"][0]) == 128 and np.array_equal(a["tie_grid"][0], np.arange(101) / 100.0)


def test_gauss3_workload_correlation_and_grid():
    d = datagen.ecdf_gauss3(n=200_000)
    x = d["x"]
    assert x.dtype == np.float32 and x.shape == (200_000, 3)
    c = np.corrcoef(x.astype(np.float64).T)
    np.testing.assert_allclose(c[np.triu_indices(3, 1)], 0.5, atol=0.01)
    np.testing.assert_allclose(x.astype(np.float64).std(axis=0), 1.0, atol=0.01)
    for k in range(3):
        g = d["grid"][k]
        assert len(g) == 256 and g[0] == x[:, k].astype(np.float64).min() and g[-1] == x[:, k].astype(np.float64).max()
    assert d["y"].dtype == np.float32 and 0.0 <= d["y"].min() and d["y"].max() < 1.0


def _kendall(x):
    stats = pytest.importorskip("scipy.stats")
    return stats.kendalltau(x[:, 0], x[:, 1])[0]


def test_copula_t4_dependence_and_marginal():
    stats = pytest.importorskip("scipy.stats")
    d = datagen.copula_t4(n=20000)
    x = d["x"].astype(np.float64)
    # Gaussian copula: Kendall's tau = (2/pi) arcsin(rho)
    assert abs(_kendall(x) - 2 / math.pi * math.asin(0.7)) < 0.02
    # marginal: Student-t(4) scaled by 1/sqrt(2); Kolmogorov-Smirnov distance
    ks = stats.kstest(x[:, 0] * math.sqrt(2.0), stats.t(4).cdf).statistic
    assert ks < 0.015
    assert d["y"].dtype == np.float32


def test_copula_exp4_dependence_and_marginal():
    d = datagen.copula_exp4(n=40000)
    x = d["x"].astype(np.float64)
    assert x.shape == (40000, 4) and d["x"].dtype == np.float32
    assert abs(_kendall(x[:, :2]) - 2 / math.pi * math.asin(0.3)) < 0.02
    assert abs(x.mean()) < 0.02                            # exponential(1) - 1 has mean 0
    assert x.min() >= -1.0


def test_batched_workload_shapes():
    sets = datagen.batched()
    assert len(sets) == 512
    ns = np.array([s["n"] for s in sets])
    assert ns.min() >= 1000 and ns.max() <= 100000
    assert [s["d"] for s in sets[:4]] == [2, 3, 2, 3]
    assert all(s["x"].shape == (s["n"], s["d"]) and s["x"].dtype == np.float32 for s in sets)
    assert 8e6 < ns.sum() < 1.4e7


def test_sample_targets_includes_and_is_reproducible():
    a = datagen.sample_targets(1000, 50, seed=3, include=(0, 999))
    b = datagen.sample_targets(1000, 50, seed=3, include=(0, 999))
    assert np.array_equal(a, b) and len(a) == 50 and 0 in a and 999 in a
    assert len(np.unique(a)) == 50
