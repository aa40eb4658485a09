"""Pins for the oracle's other compatible kernels, matrix bandwidth and locally
linear regression (no GPU).

Each oracle routine is tied to something other than itself: hand-worked
values (tests/golden/compatible_kernels_1d.txt), the paper's own CDF
decompositions evaluated through the separately pinned ``orthant_sums``
(eq. uniform decomposition nD, Sec. 3.2; eq. Matern32 decomposition nD,
Appendix C), the univariate Matern family of eqs. (Matern kernel),
(Matern constant) with p = 1, numerical quadrature (unit mass), rotation
covariance and diagonal reduction (Appendix B), and textbook properties of the
local linear fit (exact on affine data, the d = 1 closed form, the global
least-squares limit).
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden():
    sec, data = None, {}
    with open(os.path.join(GOLDEN, "compatible_kernels_1d.txt")) as f:
        for line in f:
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


# ----------------------------------------------------------------------------- uniform kernel


def test_uniform_hand_worked():
    g = _read_golden()
    x = np.array(g["points"][0])[:, None]
    h = g["h"][0][0]
    for z, v in g["uniform"]:
        assert oracle.kde_uniform(x, h, z=np.array([[z]]))[0] == v


def _corner_threshold(c, strict):
    """x <= c, or x < c written as x <= (the largest double below c)."""
    return np.nextafter(c, -np.inf) if strict else c


@pytest.mark.parametrize("d", [1, 2, 3])
def test_uniform_matches_paper_decomposition(d):
    """eq. (uniform decomposition nD): f(z) = 1/(2^d N prod h) sum_delta
    (prod delta) F_N(z + delta h, delta; x, w), where F_N(c, delta) tests
    x_k <= c_k for delta_k = +1 and x_k < c_k for delta_k = -1 (eq. ECDFdelta),
    evaluated with ``orthant_sums`` (orthant 0 at the corner thresholds).
    Data and targets on a 1/8 lattice with h = 1/4 put corners exactly on
    data values, so both the inclusive and the strict ends are exercised."""
    r = np.random.default_rng(30 + d)
    n = 150
    x = np.round(r.standard_normal((n, d)) * 8) / 8
    w = r.standard_normal(n)
    z = np.concatenate([x[:25], np.round(r.standard_normal((15, d)) * 8) / 8])
    h = np.full(d, 0.25)
    for ww in (None, w):
        total = np.zeros(z.shape[0])
        for c in range(1 << d):
            delta = np.array([-1.0 if (c >> k & 1) else 1.0 for k in range(d)])
            corner = z + delta * h
            thr = np.stack([_corner_threshold(corner[:, k], delta[k] < 0) for k in range(d)], axis=1)
            S = oracle.orthant_sums(x, y=ww, z=thr, mask=1)[0]
            total += np.prod(delta) * S
        ref = total / (2 ** d * n * np.prod(h))
        got = oracle.kde_uniform(x, h, w=ww, z=z)
        if ww is None:
            np.testing.assert_array_equal(np.rint(got * (2 ** d * n * np.prod(h))), total)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_uniform_integer_lattice_brute_force():
    """Integer points, integer h: the box count by explicit enumeration."""
    r = np.random.default_rng(5)
    x = r.integers(-3, 4, size=(40, 2)).astype(float)
    z = r.integers(-3, 4, size=(12, 2)).astype(float)
    h = np.array([1.0, 2.0])
    got = oracle.kde_uniform(x, h, z=z)
    for j in range(z.shape[0]):
        cnt = 0
        for i in range(x.shape[0]):
            if abs(x[i, 0] - z[j, 0]) <= 1 and abs(x[i, 1] - z[j, 1]) <= 2:
                cnt += 1
        assert got[j] == pytest.approx(cnt / (4 * 40 * 2.0), rel=1e-15)


def test_uniform_large_h_and_loo():
    """All points in the box: f = sum w / (2^d N prod h); LOO drops w_j only."""
    r = np.random.default_rng(6)
    x = r.standard_normal((30, 2))
    w = r.random(30)
    h = [50.0, 60.0]
    f = oracle.kde_uniform(x, h, w=w)
    np.testing.assert_allclose(f, w.sum() / (4 * 30 * 3000.0), rtol=1e-14)
    fl = oracle.kde_uniform(x, h, w=w, loo=True)
    np.testing.assert_allclose(fl, (w.sum() - w) / (4 * 29 * 3000.0), rtol=1e-13)


# ----------------------------------------------------------------------------- Matern-3/2


def test_matern32_hand_worked():
    g = _read_golden()
    x = np.array(g["points"][0])[:, None]
    h = g["h"][0][0]
    for z, v in g["matern32"]:
        assert oracle.kde_matern32(x, h, z=np.array([[z]]))[0] == pytest.approx(v, rel=1e-15)


def test_matern32_1d_is_the_univariate_family_p1():
    """d = 1: the additive kernel is eq. (Matern kernel) with p = 1, constant
    gamma_1 from eq. (Matern constant), bandwidth b = sqrt(3) h."""
    p = 1
    gam = math.sqrt(2 * p + 1) / (2 * sum(math.factorial(p) / math.factorial(p - k)
                                          * math.factorial(2 * p - k) / math.factorial(2 * p) * 2 ** k
                                          for k in range(p + 1)))
    assert gam == pytest.approx(math.sqrt(3) / 4, rel=1e-15)
    h = 0.4
    b = math.sqrt(3) * h
    x = np.array([[0.7]])
    zs = np.linspace(-2, 3, 41)
    got = oracle.kde_matern32(x, h, z=zs[:, None])
    for z, v in zip(zs, got):
        u = abs(0.7 - z)
        poly = sum(math.factorial(p) / (math.factorial(k) * math.factorial(p - k))
                   * math.factorial(2 * p - k) / math.factorial(2 * p)
                   * (2 * math.sqrt(2 * p + 1)) ** k * (u / b) ** k for k in range(p + 1))
        ref = gam / b * poly * math.exp(-math.sqrt(2 * p + 1) * u / b)
        assert v == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_matern32_matches_paper_decomposition(d):
    """eq. (Matern32 decomposition nD): f(z) = 1/(2^d (1+d) prod h) sum_delta
    e^{-delta.z/h} [(1 + sum_l delta_l z_l/h_l) F(y0) - sum_l (delta_l/h_l) F(y_l)] / N,
    y0 = w e^{delta.x/h}, y_l = w x_l e^{delta.x/h}, with F the reflected
    orthant sums of ``orthant_sums``."""
    r = np.random.default_rng(40 + d)
    n = 120
    x = np.round(r.standard_normal((n, d)) * 4) / 4
    w = r.random(n)
    z = np.concatenate([x[:30], r.standard_normal((20, d))])
    h = np.linspace(0.7, 1.2, d)
    total = np.zeros(z.shape[0])
    for o in range(1 << d):
        delta = np.array([-1.0 if (o >> k & 1) else 1.0 for k in range(d)])
        e = np.exp((x * delta / h).sum(axis=1))
        F0 = oracle.orthant_sums(x, y=w * e, z=z, mask=1 << o)[0]
        part = (1 + (delta * z / h).sum(axis=1)) * F0
        for l in range(d):
            Fl = oracle.orthant_sums(x, y=w * x[:, l] * e, z=z, mask=1 << o)[0]
            part -= delta[l] / h[l] * Fl
        total += np.exp(-(z * delta / h).sum(axis=1)) * part
    ref = total / (2 ** d * (1 + d) * np.prod(h) * n)
    np.testing.assert_allclose(oracle.kde_matern32(x, h, w=w, z=z), ref, rtol=1e-11)


def _trapezoid_mass(fn, lo, hi, step):
    """2D trapezoid rule of fn on the lattice lo + step * Z^2 (one call of fn)."""
    a = np.arange(lo[0], hi[0] + step / 2, step)
    b = np.arange(lo[1], hi[1] + step / 2, step)
    A, B = np.meshgrid(a, b, indexing="ij")
    v = fn(np.stack([A.ravel(), B.ravel()], axis=1)).reshape(A.shape)
    wa = np.full(a.size, step)
    wa[[0, -1]] = step / 2
    wb = np.full(b.size, step)
    wb[[0, -1]] = step / 2
    return float(wa @ v @ wb)


def test_matern32_integrates_to_mean_weight():
    """int f = sum w / N (2D trapezoid rule with the kinks of the kernel on
    lattice lines, Richardson-extrapolated from steps 0.02 and 0.01)."""
    x = np.array([[0.1, -0.3], [0.9, 0.4], [-0.5, 0.2]])
    w = np.array([1.0, 0.5, 2.0])
    h = [0.3, 0.5]
    fn = lambda z: oracle.kde_matern32(x, h, w=w, z=z)
    m1 = _trapezoid_mass(fn, (-8, -10), (8, 10), 0.02)
    m2 = _trapezoid_mass(fn, (-8, -10), (8, 10), 0.01)
    assert (4 * m2 - m1) / 3 == pytest.approx(w.sum() / 3, rel=1e-6)


def test_matern32_loo():
    x = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 2.0]])
    f = oracle.kde_matern32(x, [1.0, 1.0], loo=True)
    e = math.exp
    c = 1.0 / (4 * 3 * 2)
    np.testing.assert_allclose(f, [c * (1 + 4 * e(-3)), c * (1 + 4 * e(-3)), c * 2 * 4 * e(-3)], rtol=1e-15)


# ----------------------------------------------------------------------------- matrix bandwidth


def test_hmatrix_diagonal_is_the_laplacian_kde():
    r = np.random.default_rng(11)
    x = r.standard_normal((80, 3))
    w = r.random(80)
    z = r.standard_normal((20, 3))
    h = np.array([0.3, 0.6, 0.9])
    f = oracle.kde_laplace_hmatrix(x, np.diag(h ** 2), w=w, z=z)
    np.testing.assert_allclose(f, oracle.kde_laplace(x, h, w=w, z=z), rtol=1e-13)


def test_hmatrix_rotation_covariance():
    """f_H(z; x) = f_{Q H Q^T}(Q z; Q x) for an orthogonal Q (eq. kde nD H)."""
    r = np.random.default_rng(12)
    x = r.standard_normal((60, 2))
    z = r.standard_normal((15, 2))
    H = np.array([[0.3, 0.1], [0.1, 0.2]])
    t = 0.7
    Q = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    f1 = oracle.kde_laplace_hmatrix(x, H, z=z)
    f2 = oracle.kde_laplace_hmatrix(x @ Q.T, Q @ H @ Q.T, z=z @ Q.T)
    np.testing.assert_allclose(f1, f2, rtol=1e-12)


def test_hmatrix_single_source_closed_form():
    """H = [[a, b], [b, a]]: eigenvalues a +- b on (1, 1)/sqrt2, (1, -1)/sqrt2, so
    f(z) = exp(-|u1|/sqrt(a+b) - |u2|/sqrt(a-b)) / (4 sqrt((a+b)(a-b)))."""
    a, b = 0.5, 0.2
    x = np.array([[0.2, -0.1]])
    z = np.array([[0.0, 0.0], [1.0, -0.5], [-0.3, 0.8]])
    f = oracle.kde_laplace_hmatrix(x, np.array([[a, b], [b, a]]), z=z)
    s = 1 / math.sqrt(2)
    for j in range(3):
        dx = x[0] - z[j]
        u1, u2 = s * (dx[0] + dx[1]), s * (dx[0] - dx[1])
        ref = math.exp(-abs(u1) / math.sqrt(a + b) - abs(u2) / math.sqrt(a - b)) / (4 * math.sqrt((a + b) * (a - b)))
        assert f[j] == pytest.approx(ref, rel=1e-13)


# ----------------------------------------------------------------------------- locally linear regression


@pytest.mark.parametrize("d", [1, 2, 3])
def test_loclin_exact_on_affine_data(d):
    """A local linear fit reproduces an affine function exactly (any kernel)."""
    r = np.random.default_rng(50 + d)
    x = r.standard_normal((200, d))
    a, b = 0.7, r.standard_normal(d)
    y = a + x @ b
    z = r.standard_normal((30, d)) * 1.5
    m = oracle.kreg_loclin(x, y, 0.4, z=z)
    np.testing.assert_allclose(m, a + z @ b, rtol=1e-9, atol=1e-9)


def test_loclin_1d_closed_form():
    """d = 1: m = (S2 T0 - S1 T1) / (S0 S2 - S1^2) with S_r = sum K (x - z)^r,
    T_r = sum K y (x - z)^r (the textbook local linear estimator)."""
    r = np.random.default_rng(60)
    x = r.standard_normal(150)
    y = np.sin(2 * x) + 0.1 * r.standard_normal(150)
    z = np.linspace(-2, 2, 17)
    h = 0.3
    got = oracle.kreg_loclin(x[:, None], y, h, z=z[:, None])
    for j, zj in enumerate(z):
        K = np.exp(-np.abs(x - zj) / h)
        u = x - zj
        S0, S1, S2 = K.sum(), (K * u).sum(), (K * u * u).sum()
        T0, T1 = (K * y).sum(), (K * y * u).sum()
        assert got[j] == pytest.approx((S2 * T0 - S1 * T1) / (S0 * S2 - S1 * S1), rel=1e-10)


def test_loclin_wide_bandwidth_is_global_least_squares():
    r = np.random.default_rng(61)
    x = r.random((100, 2))
    y = np.cos(3 * x[:, 0]) + x[:, 1] ** 2
    z = r.random((10, 2))
    X = np.concatenate([np.ones((100, 1)), x], axis=1)
    beta = np.linalg.lstsq(X, y, rcond=None)[0]
    got = oracle.kreg_loclin(x, y, 1e9, z=z)
    np.testing.assert_allclose(got, beta[0] + z @ beta[1:], rtol=1e-6)


def test_loclin_loo_drops_self():
    x = np.array([[0.0], [1.0], [2.0], [4.0]])
    y = np.array([0.0, 1.0, 5.0, 4.0])
    m = oracle.kreg_loclin(x, y, 1.0, loo=True)
    # at x = 4 without itself: fit through (0,0), (1,1), (2,5) weighted e^-4, e^-3, e^-2
    K = np.exp(-np.abs(np.array([0.0, 1.0, 2.0]) - 4.0))
    X = np.stack([np.ones(3), np.array([0.0, 1.0, 2.0]) - 4.0], axis=1)
    beta = np.linalg.solve(X.T @ (K[:, None] * X), X.T @ (K * y[:3]))
    assert m[3] == pytest.approx(beta[0], rel=1e-12)
