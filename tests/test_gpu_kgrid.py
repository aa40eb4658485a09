"""GPU parity of the grid Laplacian KDE (the grid form of eq. Laplacian
decomposition nD with decaying per-axis recurrences) against the oracle's
brute-force KDE at the grid points, and of the multilinear grid interpolation
against scipy's on oracle values.

KDE values: relative error on values >= 1e-6 max, 1e-5 (mixed) / 1e-12 (FP64).
"""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu
TOL = {"mixed": 1e-5, "fp64": 1e-12}


def _fk():
    import paper_2005_03246_gb300 as fk
    return fk


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _rel(got, ref):
    big = np.abs(ref) >= 1e-6 * np.abs(ref).max()
    return np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big]))


def _grid_points(axes):
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def _axes(d, seed):
    r = np.random.default_rng(seed)
    out = []
    for k in range(d):
        m = [23, 14, 9][k]
        if k % 2 == 0:
            out.append(np.linspace(-1.5, 1.7, m))                          # uniform
        else:
            out.append(np.sort(r.uniform(-2.0, 2.0, m)) + np.arange(m) * 1e-3)   # non-uniform
    return out


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_kde_grid_matches_oracle_at_every_grid_point(path, d):
    r = np.random.default_rng(90 + d)
    axes = _axes(d, 91 + d)
    x = r.standard_normal((4000, d)) * 1.3                      # many points outside the grid box
    x[:200] = _grid_points(axes)[r.choice(int(np.prod([len(a) for a in axes])), 200)]   # on grid lines
    x = x.astype(np.float32)
    w = (r.random(4000) + 0.1).astype(np.float32)
    h = np.linspace(0.2, 0.45, d)
    got = _fk().kde_grid(_t(x), h, axes, w=_t(w), path=path).cpu().numpy()
    assert got.shape == tuple(len(a) for a in axes)
    ref = oracle.kde_laplace(x, h, w=w, z=_grid_points(axes)).reshape(got.shape)
    assert _rel(got.reshape(-1), ref.reshape(-1)) <= TOL[path]


def test_kde_grid_small_bandwidth_and_unweighted():
    """h far below the grid spacing: the decays underflow gracefully (no NaN,
    no overflow) and the values at the grid points stay exact."""
    r = np.random.default_rng(95)
    axes = [np.linspace(0.0, 10.0, 41), np.linspace(-3.0, 3.0, 13)]
    x = np.stack([r.uniform(-1, 11, 3000), r.normal(0, 1, 3000)], axis=1).astype(np.float32)
    for h in ([0.02, 0.05], [0.5, 0.5]):
        got = _fk().kde_grid(_t(x), h, axes, path="fp64").cpu().numpy()
        ref = oracle.kde_laplace(x, h, z=_grid_points(axes)).reshape(got.shape)
        assert np.all(np.isfinite(got))
        assert _rel(got.reshape(-1), ref.reshape(-1)) <= 1e-12


def test_kde_grid_full_size_d3_sampled():
    """d=3, N=1e6, h=0.1 on a 64^3 grid over the data range: sampled grid
    points against the oracle."""
    x = datagen.ecdf_gauss3()["x"]
    axes = [np.linspace(float(x[:, k].min()), float(x[:, k].max()), 64) for k in range(3)]
    pts = _grid_points(axes)
    idx = datagen.sample_targets(pts.shape[0], 512, seed=97)
    ref = oracle.kde_laplace(x, 0.1, z=pts[idx])
    for path in ("mixed", "fp64"):
        got = _fk().kde_grid(_t(x), 0.1, axes, path=path).cpu().numpy().reshape(-1)
        assert _rel(got[idx], ref) <= TOL[path], path


def test_grid_interp_reproduces_multilinear_functions():
    r = np.random.default_rng(98)
    axes = [np.sort(r.uniform(-1, 1, 7)), np.linspace(0, 2, 5), np.sort(r.uniform(0, 3, 6))]
    g = _grid_points(axes)
    f = (1.0 + 2.0 * g[:, 0] - 0.5 * g[:, 1] + 0.25 * g[:, 2] + 0.7 * g[:, 0] * g[:, 1]
         - 0.3 * g[:, 0] * g[:, 1] * g[:, 2]).reshape(7, 5, 6)
    q = np.stack([r.uniform(a[0], a[-1], 500) for a in axes], axis=1)
    expect = (1.0 + 2.0 * q[:, 0] - 0.5 * q[:, 1] + 0.25 * q[:, 2] + 0.7 * q[:, 0] * q[:, 1]
              - 0.3 * q[:, 0] * q[:, 1] * q[:, 2])
    got = _fk().grid_interp(_t(f), axes, _t(q)).cpu().numpy()
    assert np.max(np.abs(got - expect)) <= 1e-12 * np.abs(expect).max()
    # outside the box the coordinates are clamped to it
    qo = q.copy()
    qo[:, 0] = axes[0][-1] + 5.0
    qc = q.copy()
    qc[:, 0] = axes[0][-1]
    np.testing.assert_allclose(_fk().grid_interp(_t(f), axes, _t(qo)).cpu().numpy(),
                               _fk().grid_interp(_t(f), axes, _t(qc)).cpu().numpy(), rtol=0, atol=0)


def test_grid_interp_of_oracle_kde_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    r = np.random.default_rng(99)
    axes = [np.linspace(-2, 2, 17), np.sort(r.uniform(-2, 2, 11))]
    x = r.standard_normal((2000, 2))
    f = oracle.kde_laplace(x, [0.3, 0.4], z=_grid_points(axes)).reshape(17, 11)
    q = np.stack([r.uniform(-2, 2, 400), r.uniform(axes[1][0], axes[1][-1], 400)], axis=1)
    expect = interp.RegularGridInterpolator(axes, f, method="linear")(q)
    got = _fk().grid_interp(_t(f), axes, _t(q)).cpu().numpy()
    assert np.max(np.abs(got - expect)) <= 1e-13 * np.abs(f).max()
