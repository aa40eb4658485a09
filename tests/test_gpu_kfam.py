"""GPU parity of the other compatible kernels (uniform, eq. uniform
decomposition nD, Sec. 3.2; additive Matern-3/2, eq. Matern32 decomposition
nD, Appendix C), the full bandwidth matrix (eq. kde nD H, Appendix B) and
locally linear regression against the CPU oracle, through the C ABI.

Box counts of the uniform kernel are exact (compared as integers); weighted
uniform sums are signed differences of ECDFs and are held to their magnitude
scale C sum|w|; kernel values use the relative error on entries >= 1e-6 max,
within 1e-5 (mixed path) and 1e-12 (FP64 path).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
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


def _golden():
    sec, data = None, {}
    for line in open(os.path.join(GOLDEN, "compatible_kernels_1d.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        toks = line.split()
        if toks[0] in ("points", "h", "uniform", "matern32"):
            sec = toks[0]
            data[sec] = []
            continue
        data[sec].append([float(t) for t in toks])
    return data


def _lattice(n, d, seed, dtype):
    r = np.random.default_rng(seed)
    return (np.round(r.standard_normal((n, d)) * 8) / 8).astype(dtype)


def _const(n, d, h):
    return 1.0 / (2.0 ** d * n * np.prod(h))


# ------------------------------------------------------------------ uniform kernel


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_uniform_golden_1d(path):
    g = _golden()
    x = np.array(g["points"][0])[:, None]
    h = g["h"][0][0]
    z = np.array([[v[0]] for v in g["uniform"]])
    got = _fk().kde_uniform(_t(x), h, z=_t(z), path=path).cpu().numpy()
    np.testing.assert_allclose(got, [v[1] for v in g["uniform"]], rtol=1e-15, atol=0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_uniform_counts_exact(d, dtype):
    """Points and targets on a 1/8 lattice with h = 1/4: box corners land on
    data values, so both the inclusive upper and the strict lower end matter.
    Box counts (f / C) equal the oracle's exactly, at the sample points, with
    leave-one-out, and at explicit off-lattice targets."""
    n = 3000 if d <= 4 else 1500
    x = _lattice(n, d, 100 + d, dtype)
    h = np.full(d, 0.25)
    r = np.random.default_rng(200 + d)
    z = np.concatenate([x[:200], r.standard_normal((150, d)).astype(dtype)])
    C = _const(n, d, h)
    fk = _fk()
    got = fk.kde_uniform(_t(x), h).cpu().numpy()
    ref = oracle.kde_uniform(x, h)
    np.testing.assert_array_equal(np.rint(got / C), np.rint(ref / C))
    np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)
    gl = fk.kde_uniform(_t(x), h, loo=True).cpu().numpy()
    rl = oracle.kde_uniform(x, h, loo=True)
    Cl = _const(n - 1, d, h)
    np.testing.assert_array_equal(np.rint(gl / Cl), np.rint(rl / Cl))
    gz = fk.kde_uniform(_t(x), h, z=_t(z)).cpu().numpy()
    rz = oracle.kde_uniform(x, h, z=z)
    np.testing.assert_array_equal(np.rint(gz / C), np.rint(rz / C))


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [2, 3])
def test_uniform_weighted(d, path):
    """Signed weights: error relative to C sum|w| (the corner ECDFs' scale)."""
    n = 4000
    x = _lattice(n, d, 300 + d, np.float32)
    w = np.random.default_rng(400 + d).standard_normal(n).astype(np.float32)
    h = np.array([0.25, 0.5, 0.375][:d])
    scale = _const(n, d, h) * np.abs(w.astype(np.float64)).sum()
    got = _fk().kde_uniform(_t(x), h, w=_t(w), path=path).cpu().numpy()
    ref = oracle.kde_uniform(x, h, w=w)
    assert np.max(np.abs(got - ref)) <= TOL[path] * scale
    gl = _fk().kde_uniform(_t(x), h, w=_t(w), loo=True, path=path).cpu().numpy()
    rl = oracle.kde_uniform(x, h, w=w, loo=True)
    assert np.max(np.abs(gl - rl)) <= TOL[path] * scale * n / (n - 1)


def test_uniform_full_size_d3_sampled_targets():
    """d=3, N=1e6 correlated Gaussian (FP32), h = 0.1, at the sample points:
    8e6 corner targets in one call; 2048 sampled targets (extremes included)
    against the oracle's exact box counts."""
    data = datagen.ecdf_gauss3()
    x = data["x"]
    n = x.shape[0]
    h = np.full(3, 0.1)
    got = _fk().kde_uniform(_t(x), h).cpu().numpy()
    ext = [int(i) for k in range(3) for i in (x[:, k].argmin(), x[:, k].argmax())]
    idx = datagen.sample_targets(n, 2048, seed=5, include=ext)
    ref = oracle.kde_uniform(x, h, z=x[idx])
    C = _const(n, 3, h)
    np.testing.assert_array_equal(np.rint(got[idx] / C), np.rint(ref / C))
    assert got.min() >= C     # every point lies in its own box


# ------------------------------------------------------------------ Matern-3/2


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_matern32_golden_1d(path):
    g = _golden()
    x = np.array(g["points"][0])[:, None]
    h = g["h"][0][0]
    z = np.array([[v[0]] for v in g["matern32"]])
    got = _fk().kde_matern32(_t(x), h, z=_t(z), path=path).cpu().numpy()
    np.testing.assert_allclose(got, [v[1] for v in g["matern32"]], rtol=TOL[path])


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_matern32_small(d, path):
    """Sample points (plain and leave-one-out), explicit targets, weights, ties."""
    n = 3000
    r = np.random.default_rng(500 + d)
    x = r.standard_normal((n, d)).astype(np.float32)
    m = r.random((n, d)) < 0.3
    x[m] = np.round(x[m] * 8) / 8
    w = (r.random(n) + 0.5).astype(np.float32)
    z = r.standard_normal((400, d)).astype(np.float32) * 1.3
    h = np.linspace(0.2, 0.5, d)
    fk = _fk()
    tol = TOL[path]
    assert _rel_kde(fk.kde_matern32(_t(x), h, path=path).cpu().numpy(), oracle.kde_matern32(x, h)) <= tol
    assert _rel_kde(fk.kde_matern32(_t(x), h, loo=True, path=path).cpu().numpy(),
                    oracle.kde_matern32(x, h, loo=True)) <= tol
    assert _rel_kde(fk.kde_matern32(_t(x), h, z=_t(z), path=path).cpu().numpy(),
                    oracle.kde_matern32(x, h, z=z)) <= tol
    assert _rel_kde(fk.kde_matern32(_t(x), h, w=_t(w), path=path).cpu().numpy(),
                    oracle.kde_matern32(x, h, w=w)) <= tol
    assert _rel_kde(fk.kde_matern32(_t(x), h, w=_t(w), z=_t(z), path=path).cpu().numpy(),
                    oracle.kde_matern32(x, h, w=w, z=z)) <= tol


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_matern32_full_size_d3_sampled(path):
    data = datagen.ecdf_gauss3()
    x = data["x"]
    n = x.shape[0]
    got = _fk().kde_matern32(_t(x), 0.1, path=path).cpu().numpy()
    idx = datagen.sample_targets(n, 1024, seed=6)
    ref = oracle.kde_matern32(x, 0.1, z=x[idx])
    assert np.max(np.abs(got[idx] - ref) / ref) <= TOL[path]


# ------------------------------------------------------------------ matrix bandwidth


def _spd(d, seed):
    r = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(r.standard_normal((d, d)))
    ev = np.linspace(0.04, 0.25, d) ** 2 * np.linspace(1.0, 3.0, d)
    return Q @ np.diag(ev) @ Q.T


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_hmatrix_parity(d, path):
    n = 2500
    r = np.random.default_rng(600 + d)
    x = r.standard_normal((n, d)).astype(np.float32)
    w = (r.random(n) + 0.5).astype(np.float32)
    z = r.standard_normal((300, d)).astype(np.float32)
    H = _spd(d, 700 + d)
    fk = _fk()
    tol = TOL[path]
    assert _rel_kde(fk.kde_laplace_hmatrix(_t(x), H, path=path).cpu().numpy(),
                    oracle.kde_laplace_hmatrix(x, H)) <= tol
    assert _rel_kde(fk.kde_laplace_hmatrix(_t(x), H, w=_t(w), z=_t(z), path=path).cpu().numpy(),
                    oracle.kde_laplace_hmatrix(x, H, w=w, z=z)) <= tol


def test_hmatrix_diagonal_equals_laplacian_kde():
    r = np.random.default_rng(800)
    x = r.standard_normal((5000, 3))
    h = np.array([0.1, 0.2, 0.3])
    fk = _fk()
    a = fk.kde_laplace_hmatrix(_t(x), np.diag(h ** 2), path="fp64").cpu().numpy()
    b = fk.kde_laplace(_t(x), h, path="fp64").cpu().numpy()
    assert _rel_kde(a, b) <= 1e-13


# ------------------------------------------------------------------ locally linear regression


@pytest.mark.parametrize("d", [1, 2, 3])
def test_loclin_parity(d):
    """Targets where the local design is well conditioned (condition number of
    the normalised normal matrix < 1e6) are compared at 1e-8 of the response
    scale; every target must be finite or NaN exactly where the oracle's is."""
    n = 2000
    r = np.random.default_rng(900 + d)
    x = r.standard_normal((n, d)).astype(np.float32)
    y = (np.sin(x.astype(np.float64).sum(axis=1)) + 0.1 * r.standard_normal(n)).astype(np.float32)
    z = (r.standard_normal((300, d)) * 1.2).astype(np.float32)
    h = np.linspace(0.3, 0.5, d)
    fk = _fk()
    for zz, loo in ((None, False), (None, True), (z, False)):
        got = fk.kreg_loclin(_t(x), _t(y), h, z=None if zz is None else _t(zz), loo=loo).cpu().numpy()
        ref = oracle.kreg_loclin(x, y, h, z=zz, loo=loo)
        tz = (x if zz is None else zz).astype(np.float64)
        cond = np.empty(tz.shape[0])
        for j in range(tz.shape[0]):
            diff = x.astype(np.float64) - tz[j]
            K = np.exp(-(np.abs(diff) / h).sum(axis=1))
            if loo:
                K[j] = 0.0
            X = np.concatenate([np.ones((n, 1)), diff / h], axis=1)
            A = X.T @ (K[:, None] * X)
            cond[j] = np.linalg.cond(A)
        ok = cond < 1e6
        assert ok.mean() > 0.8
        assert np.max(np.abs(got[ok] - ref[ok])) <= 1e-8 * np.abs(y).max()


def test_loclin_exact_on_affine_responses():
    r = np.random.default_rng(950)
    x = r.standard_normal((3000, 2))
    y = 0.3 - 1.2 * x[:, 0] + 0.7 * x[:, 1]
    z = r.standard_normal((200, 2))
    got = _fk().kreg_loclin(_t(x), _t(y), 0.3, z=_t(z)).cpu().numpy()
    np.testing.assert_allclose(got, 0.3 - 1.2 * z[:, 0] + 0.7 * z[:, 1], rtol=0, atol=1e-9)


def test_loclin_refuses_mixed_path():
    fk = _fk()
    x = np.random.default_rng(1).standard_normal((100, 2))
    with pytest.raises(fk.FastEcdfError):
        fk.kreg_loclin(_t(x), _t(x[:, 0]), 0.3, path="mixed")


# ------------------------------------------------------------------ edge cases


def test_edge_cases_single_point_empty_targets_and_two_point_loo():
    """N = 1 (one source: the kernel itself), M = 0 explicit targets (an empty
    result), N = 2 with leave-one-out (each point sees only the other)."""
    import torch
    fk = _fk()
    x1 = np.array([[0.25, -0.5]])
    z = np.array([[0.25, -0.5], [0.3, -0.45], [1.0, 1.0], [0.5, -0.25]])
    h = np.array([0.25, 0.25])
    np.testing.assert_allclose(fk.kde_uniform(_t(x1), h, z=_t(z)).cpu().numpy(),
                               oracle.kde_uniform(x1, h, z=z), rtol=1e-15, atol=0)
    for path in ("mixed", "fp64"):
        np.testing.assert_allclose(fk.kde_matern32(_t(x1), h, z=_t(z), path=path).cpu().numpy(),
                                   oracle.kde_matern32(x1, h, z=z), rtol=TOL[path], atol=1e-300)
    H = np.array([[0.05, 0.01], [0.01, 0.04]])
    np.testing.assert_allclose(fk.kde_laplace_hmatrix(_t(x1), H, z=_t(z), path="fp64").cpu().numpy(),
                               oracle.kde_laplace_hmatrix(x1, H, z=z), rtol=1e-12, atol=1e-300)
    empty = torch.empty((0, 2), dtype=torch.float64, device="cuda:0")
    assert fk.kde_uniform(_t(x1), h, z=empty).shape == (0,)
    assert fk.kde_matern32(_t(x1), h, z=empty).shape == (0,)
    x2 = np.array([[0.0, 0.0], [0.1, 0.2]])
    np.testing.assert_allclose(fk.kde_uniform(_t(x2), h, loo=True).cpu().numpy(),
                               oracle.kde_uniform(x2, h, loo=True), rtol=1e-15, atol=0)
    for path in ("mixed", "fp64"):
        np.testing.assert_allclose(fk.kde_matern32(_t(x2), h, loo=True, path=path).cpu().numpy(),
                                   oracle.kde_matern32(x2, h, loo=True), rtol=TOL[path])


def test_invalid_arguments_are_refused():
    fk = _fk()
    x = np.random.default_rng(2).standard_normal((50, 2))
    with pytest.raises(fk.FastEcdfError):
        fk.kde_uniform(_t(x), [0.1, -0.1])                       # h <= 0
    with pytest.raises(fk.FastEcdfError):
        fk.kde_laplace_hmatrix(_t(x), np.array([[1.0, 2.0], [2.0, 1.0]]))   # indefinite
    with pytest.raises(fk.FastEcdfError):
        fk.kde_laplace_hmatrix(_t(x), np.array([[1.0, 0.2], [0.1, 1.0]]))   # not symmetric
    with pytest.raises(fk.FastEcdfError):
        fk.kde_matern32(_t(np.random.default_rng(3).standard_normal((50, 5))), 0.1)   # d > 4
