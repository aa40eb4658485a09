"""GPU parity at the full sizes of the d=2 copula workload (N=1e6, Student-t4
marginals, h in {0.05, 0.1, 0.3}; KDE, Nadaraya-Watson and the adjoint) and of
the d=4 copula workload (N=4e6, exponential marginals: all 16 orthant counts,
leave-one-out KDE and likelihood gradient), in the launch configuration the
library uses at those sizes.

The oracle evaluates sampled targets one by one against all N sources (always
including the extreme points of every axis); what it cannot sample (the
likelihood's h-gradient, a sum over all N targets) is checked by properties
that hold at any size: central differences of the GPU's own FP64 likelihood,
and agreement of the mixed and FP64 paths.  Tolerances as in the other GPU
tests: counts bit-exact, KDE relative 1e-5 (mixed) / 1e-12 (FP64) on values
>= 1e-6 max, signed sums relative to their magnitude.
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


def _rel_kde(got, ref):
    big = np.abs(ref) >= 1e-6 * np.abs(ref).max()
    return np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big]))


def _extremes(x):
    return tuple(int(i) for k in range(x.shape[1]) for i in (np.argmin(x[:, k]), np.argmax(x[:, k])))


@pytest.fixture(scope="module")
def c3():
    d = datagen.copula_t4()
    x, y = d["x"], d["y"]
    idx = datagen.sample_targets(x.shape[0], 384, seed=31, include=_extremes(x))
    return x, y, idx


@pytest.fixture(scope="module")
def c5():
    x = datagen.copula_exp4()["x"]
    idx = datagen.sample_targets(x.shape[0], 192, seed=51, include=_extremes(x))
    return x, idx


# ------------------------------------------------------------------ d=2, N=1e6


@pytest.mark.parametrize("h", [0.05, 0.1, 0.3])
def test_c3_kde_and_regression_at_sampled_points(c3, h):
    x, y, idx = c3
    fk = _fk()
    ref_f = oracle.kde_laplace(x, h, z=x[idx])
    ref_m = oracle.kreg_laplace(x, y, h, z=x[idx])
    cond_m = oracle.kreg_laplace(x, np.abs(y), h, z=x[idx])
    for path in ("mixed", "fp64"):
        f = fk.kde_laplace(_t(x), h, path=path).cpu().numpy()
        assert _rel_kde(f[idx], ref_f) <= TOL[path], (path, h)
        m = fk.kreg_laplace(_t(x), _t(y), h, path=path).cpu().numpy()
        # a ratio of signed kernel sums: error relative to the regression of |y|
        err = np.abs(m[idx] - ref_m) / np.maximum(cond_m, 1e-6 * np.abs(ref_m).max())
        assert np.max(err) <= TOL[path], (path, h)


def test_c3_adjoint_at_explicit_targets(c3):
    """grad_z (every target) and grad_h against the oracle's brute-force
    gradient, grad_w at sampled sources against the transposed kernel sum,
    and grad_h against central differences of the GPU's FP64 forward."""
    x, _, _ = c3
    fk = _fk()
    r = np.random.default_rng(33)
    m = 768
    z = (x[r.choice(x.shape[0], m, replace=False)] + r.normal(0.0, 0.05, (m, 2))).astype(np.float32)
    g = r.standard_normal(m)
    h = np.array([0.1, 0.12])
    rw, rz, rh = oracle.kde_grad(x, h, g, z=z)
    sidx = datagen.sample_targets(x.shape[0], 256, seed=34, include=_extremes(x))
    for path, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        gw, gz, gh = fk.kde_laplace_backward(_t(x), h, _t(g), z=_t(z), path=path)
        gw, gz, gh = gw.cpu().numpy(), gz.cpu().numpy(), gh.cpu().numpy()
        assert np.max(np.abs(gz - rz)) <= tol * np.abs(rz).max(), path
        assert np.max(np.abs(gh - rh)) <= tol * np.abs(rh).max(), path
        assert np.max(np.abs(gw[sidx] - rw[sidx])) <= tol * np.abs(rw).max(), path
    # central differences of L(h) = <g, f(z; h)> along h -> h (1 + s)
    hp, hm = h * (1 + 1e-6), h * (1 - 1e-6)
    Lp = float(np.dot(g, fk.kde_laplace(_t(x), hp, z=_t(z), path="fp64").cpu().numpy()))
    Lm = float(np.dot(g, fk.kde_laplace(_t(x), hm, z=_t(z), path="fp64").cpu().numpy()))
    _, _, gh = fk.kde_laplace_backward(_t(x), h, _t(g), z=_t(z), need_w=False, need_z=False, path="fp64")
    fd = (Lp - Lm) / 2e-6
    assert abs(fd - float(np.dot(gh.cpu().numpy(), h))) <= 1e-4 * abs(fd)


# ------------------------------------------------------------------ d=3, N=1e6


def test_c2_weighted_orthant_sums_at_sampled_points():
    """The d=3 correlated-Gaussian workload with weights y ~ U[0,1]: all 8
    weighted orthant sums on both paths, at sampled targets against the
    oracle (y >= 0, so every sum is its own magnitude: relative error, and an
    empty orthant must be exactly 0), and the orthants' partition of sum(y)
    at every target."""
    d = datagen.ecdf_gauss3()
    x, y = d["x"], d["y"]
    idx = datagen.sample_targets(x.shape[0], 256, seed=21, include=_extremes(x))
    ref = oracle.orthant_sums(x, y=y, z=x[idx])
    ysum = float(np.sum(y.astype(np.float64)))
    for path in ("mixed", "fp64"):
        got = _fk().ecdf_points(_t(x), y=_t(y), path=path).cpu().numpy()
        assert got.shape == (8, x.shape[0])
        g = got[:, idx]
        assert np.all(g[ref == 0] == 0), path
        nz = ref > 0
        assert np.max(np.abs(g[nz] - ref[nz]) / ref[nz]) <= TOL[path], path
        assert np.max(np.abs(got.sum(axis=0) - ysum)) <= TOL[path] * ysum * 8, path


# ------------------------------------------------------------------ d=4, N=4e6


def test_c5_all_16_orthant_counts_at_sampled_points(c5):
    x, idx = c5
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert got.shape == (16, x.shape[0])
    ref = oracle.orthant_sums(x, z=x[idx])
    assert np.array_equal(got[:, idx], ref)
    # the 16 orthants partition the sources at every target (full output)
    assert np.all(got.sum(axis=0) == x.shape[0])


def test_c5_leave_one_out_kde_at_sampled_points(c5):
    x, idx = c5
    ref = oracle.kde_at_points(x, 0.5, idx, loo=True)
    for path in ("mixed", "fp64"):
        f = _fk().kde_laplace(_t(x), 0.5, loo=True, path=path).cpu().numpy()
        assert _rel_kde(f[idx], ref) <= TOL[path], path


def test_c5_likelihood_gradient_full_size(c5):
    """dL/dh at N=4e6, pinned through a chain that ends at the oracle: the
    leave-one-out densities f_{-j} at sampled targets equal the oracle's (the
    test above and below), L equals mean_j log f_{-j} over the full output of
    the leave-one-out KDE call, and dL/dh equals central differences of that
    L (along h -> h (1 + s)); the mixed path follows the FP64 path."""
    import torch
    x, idx = c5
    fk = _fk()
    h = np.array([0.5, 0.45, 0.55, 0.5])
    f = fk.kde_laplace(_t(x), h, loo=True, path="fp64")
    fs = f.cpu().numpy()
    assert _rel_kde(fs[idx[:48]], oracle.kde_at_points(x, h, idx[:48], loo=True)) <= TOL["fp64"]
    Lf = float(torch.log(f).mean().item())
    L64, g64 = fk.loo_laplace(_t(x), h, path="fp64")
    assert abs(float(L64.item()) - Lf) <= 1e-12 * max(1.0, abs(Lf))
    Lmx, gmx = fk.loo_laplace(_t(x), h, path="mixed")
    L64, g64, Lmx, gmx = float(L64.item()), g64.cpu().numpy(), float(Lmx.item()), gmx.cpu().numpy()
    assert abs(Lmx - L64) <= 1e-6 * max(1.0, abs(L64))
    assert np.max(np.abs(gmx - g64)) <= 1e-5 * np.abs(g64).max()
    Lp, _ = fk.loo_laplace(_t(x), h * (1 + 1e-5), path="fp64", grad=False)
    Lm, _ = fk.loo_laplace(_t(x), h * (1 - 1e-5), path="fp64", grad=False)
    fd = (float(Lp.item()) - float(Lm.item())) / 2e-5
    assert abs(fd - float(np.dot(g64, h))) <= 1e-4 * abs(fd)


def test_c5_bandwidth_steps_mixed_follow_fp64(c5):
    """Two ascent steps on log h at full size: the mixed path follows the FP64
    path (h, L and dL/dh per step)."""
    x, idx = c5
    fk = _fk()
    hm = fk.select_bandwidth_loo(_t(x), h0=0.5, steps=2, lr=0.5, path="mixed")
    hd = fk.select_bandwidth_loo(_t(x), h0=0.5, steps=2, lr=0.5, path="fp64")
    for (h1, L1, g1), (h2, L2, g2) in zip(hm, hd):
        assert np.max(np.abs(h1 - h2)) <= 1e-6 * np.max(h2)
        assert abs(L1 - L2) <= 1e-6 * max(1.0, abs(L2))
        assert np.max(np.abs(g1 - g2)) <= 1e-5 * np.abs(g2).max()
    # the densities the second FP64 step's likelihood is made of, at sampled
    # targets, against the oracle
    h2 = hd[1][0]
    f = fk.kde_laplace(_t(x), h2, loo=True, path="fp64").cpu().numpy()
    assert _rel_kde(f[idx[:48]], oracle.kde_at_points(x, h2, idx[:48], loo=True)) <= TOL["fp64"]
