"""Pins for the CPU oracle (no GPU).

The oracle is the brute-force definition; these tests tie it to things other
than itself: the paper's printed identities (the 1D and nD Laplacian
decompositions of Sec. 3.1), a hand-worked example, closed forms, library
routines (sorted cumulative sums, scipy's Laplace density, numerical
quadrature), exact invariants (orthant partition, inclusion-exclusion,
reflection of integer lattices) and an independent Fenwick-tree count.  Each
test is chosen so that a plausible slip in the oracle (a wrong strictness, a
dropped orthant, a swapped sign, a missing 1/h) fails it.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_tie_golden():
    sec, data = None, {}
    with open(os.path.join(GOLDEN, "tie2d_orthants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            toks = line.split()
            if toks[0] in ("points", "orthant", "strict", "grid"):
                sec = " ".join(toks)
                data[sec] = []
                continue
            data[sec].append([float(t) for t in toks])
    return data


# ----------------------------------------------------------------------------- ECDF


def test_tie_example_hand_worked():
    """Hand-worked counts (eq. ECDFdelta).  For instance orthant 3 (x0>z0, x1>z1)
    at z=(0,0) counts the two copies of (1,1); at z=(0,1) orthant 1 (x0>z0,
    x1<=z1) counts (1,0),(1,1),(1,1)."""
    g = _read_tie_golden()
    x = np.array(g["points"])
    got = oracle.orthant_sums(x)
    for o in range(4):
        assert got[o].tolist() == [int(v) for v in g["orthant %d" % o][0]]
    # grid version, orthant 0 only
    F = oracle.ecdf_grid(x, [np.array([0.0, 1.0]), np.array([0.0, 1.0])], mask=1)
    assert F[0].tolist() == [[int(v) for v in row] for row in g["grid"]]


def test_strict_variant_via_shifted_lattice():
    """eq. (ECDFdelta) with delta=(-1,-1) means x0<z0 and x1<z1; on the integer
    lattice that is x <= z - 1, i.e. orthant 0 at shifted targets."""
    g = _read_tie_golden()
    x = np.array(g["points"])
    got = oracle.orthant_sums(x, z=x - 1.0, mask=1)[0]
    assert got.tolist() == [int(v) for v in g["strict"][0]]


def test_1d_equals_sorted_cumsum():
    """d=1: the <= orthant is the cumulative count in sorted order with tie groups
    taking their last value (numpy searchsorted), the > orthant its complement."""
    r = np.random.default_rng(7)
    x = np.round(r.random(500) * 50) / 50.0          # many ties
    z = np.concatenate([x, r.random(100)])
    got = oracle.orthant_sums(x[:, None], z=z[:, None])
    srt = np.sort(x)
    le = np.searchsorted(srt, z, side="right")
    assert np.array_equal(got[0], le)
    assert np.array_equal(got[1], x.size - le)
    y = r.standard_normal(500)
    gw = oracle.orthant_sums(x[:, None], y=y, z=z[:, None])
    order = np.argsort(x, kind="stable")
    cs = np.concatenate([[0.0], np.cumsum(y[order])])
    np.testing.assert_allclose(gw[0], cs[le], rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_partition_and_inclusion_exclusion(d):
    """The 2^d orthants partition the sources (sum = N exactly); dropping axis k
    from the test equals the sum of the two orthants that differ only in bit k."""
    r = np.random.default_rng(100 + d)
    x = r.integers(0, 4, size=(200, d)).astype(np.float64)   # heavy ties
    z = r.integers(-1, 5, size=(60, d)).astype(np.float64)
    S = oracle.orthant_sums(x, z=z)
    assert np.all(S.sum(axis=0) == x.shape[0])
    if d >= 2:
        for k in range(d):
            keep = [a for a in range(d) if a != k]
            Sk = oracle.orthant_sums(x[:, keep], z=z[:, keep])
            for o in range(1 << d):
                if o >> k & 1:
                    continue
                lo = o & ((1 << k) - 1)
                hi = o >> (k + 1)
                o_red = lo | (hi << k)
                assert np.array_equal(S[o] + S[o | (1 << k)], Sk[o_red])


@pytest.mark.parametrize("d", [1, 2, 3])
def test_reflection_on_integer_lattice(d):
    """On integers, x_k > z_k <=> -x_k <= -z_k - 1: reflecting a set A of axes
    (x -> -x, z -> -z-1 on A) maps orthant o onto orthant o XOR A."""
    r = np.random.default_rng(200 + d)
    x = r.integers(0, 3, size=(150, d)).astype(np.float64)
    z = r.integers(0, 3, size=(40, d)).astype(np.float64)
    S = oracle.orthant_sums(x, z=z)
    y = r.standard_normal(150)
    Sy = oracle.orthant_sums(x, y=y, z=z)
    for A in range(1 << d):
        xr, zr = x.copy(), z.copy()
        for k in range(d):
            if A >> k & 1:
                xr[:, k] = -x[:, k]
                zr[:, k] = -z[:, k] - 1.0
        R = oracle.orthant_sums(xr, z=zr)
        Ry = oracle.orthant_sums(xr, y=y, z=zr)
        for o in range(1 << d):
            assert np.array_equal(S[o], R[o ^ A])
            np.testing.assert_allclose(Sy[o], Ry[o ^ A], rtol=0, atol=1e-12)


def test_exhaustive_small_lattice_d2():
    """Every multiset of up to 3 points from {0,1,2}^2, targets = all 9 lattice
    points: partition, self-count and agreement with the Fenwick sweep."""
    pts = [(a, b) for a in range(3) for b in range(3)]
    lattice = np.array(pts, dtype=np.float64)
    for size in (1, 2, 3):
        for combo in itertools.combinations_with_replacement(range(9), size):
            x = lattice[list(combo)]
            S = oracle.orthant_sums(x, z=lattice)
            assert np.all(S.sum(axis=0) == size)
            assert np.array_equal(S, oracle.fenwick2d(x, z=lattice))
            Sp = oracle.orthant_sums(x)
            assert np.all(Sp[0] >= 1)            # each point dominates itself


def test_fenwick_matches_brute_force_with_ties():
    r = np.random.default_rng(11)
    x = np.round(r.random((3000, 2)) * 40) / 40.0
    z = np.round(r.random((500, 2)) * 40) / 40.0
    assert np.array_equal(oracle.orthant_sums(x), oracle.fenwick2d(x))
    assert np.array_equal(oracle.orthant_sums(x, z=z), oracle.fenwick2d(x, z=z))


def test_grid_corner_and_monotone():
    """F at a grid corner >= max x equals sum y (Sec. 2.1); the <= orthant is
    non-decreasing along every axis for y >= 0."""
    r = np.random.default_rng(5)
    x = r.random((400, 3))
    y = r.random(400)
    axes = [np.linspace(-0.1, 1.1, 9), np.linspace(0, 1, 7), np.linspace(-0.2, 1.0, 5)]
    F = oracle.ecdf_grid(x, axes, y=y, mask=1)[0]
    assert F[-1, -1, -1] == pytest.approx(y.sum(), rel=1e-14)
    for ax in range(3):
        assert np.all(np.diff(F, axis=ax) >= -1e-15)
    C = oracle.ecdf_grid(x, axes, mask=1)[0]
    assert C[-1, -1, -1] == 400


# ----------------------------------------------------------------------------- KDE


def test_kde_closed_form_two_points_1d():
    """d=1, x={0,1}, w=1, h=1: f(0) = (1+e^-1)/4, f(1/2) = e^-1/2 / 2."""
    x = np.array([[0.0], [1.0]])
    f = oracle.kde_laplace(x, 1.0, z=np.array([[0.0], [0.5]]))
    assert f[0] == pytest.approx((1.0 + math.exp(-1.0)) / 4.0, rel=1e-15)
    assert f[1] == pytest.approx(math.exp(-0.5) / 2.0, rel=1e-15)


def test_kde_closed_form_tie_example_2d():
    """The five tie points, h=(0.5, 1): C = 1/(4*5*0.5*1) = 1/10 and
    f(p) = (1/10) sum_i exp(-2|dx0| - |dx1|), expanded by hand per target."""
    g = _read_tie_golden()
    x = np.array(g["points"])
    e = math.exp
    expect = [
        (1 + e(-2) + e(-1) + 2 * e(-3)) / 10,          # z=(0,0)
        (e(-2) + 1 + e(-3) + 2 * e(-1)) / 10,          # z=(1,0)
        (e(-1) + e(-3) + 1 + 2 * e(-2)) / 10,          # z=(0,1)
        (e(-3) + e(-1) + e(-2) + 2) / 10,              # z=(1,1)
        (e(-3) + e(-1) + e(-2) + 2) / 10,
    ]
    f = oracle.kde_laplace(x, [0.5, 1.0])
    np.testing.assert_allclose(f, expect, rtol=1e-15)


def test_kde_single_source_is_product_laplace_density():
    """One source: the KDE is the product of scipy's Laplace densities."""
    stats = pytest.importorskip("scipy.stats")
    r = np.random.default_rng(3)
    x = np.array([[0.3, -1.2, 2.0]])
    h = np.array([0.2, 0.7, 1.5])
    z = r.standard_normal((50, 3))
    f = oracle.kde_laplace(x, h, z=z)
    ref = np.prod([stats.laplace.pdf(z[:, k], loc=x[0, k], scale=h[k]) for k in range(3)], axis=0)
    np.testing.assert_allclose(f, ref, rtol=1e-13)


def test_kde_integrates_to_mean_weight():
    """int f dz = sum(w)/N (1D quadrature, Sec. 3.1 normalisation)."""
    integrate = pytest.importorskip("scipy.integrate")
    r = np.random.default_rng(4)
    x = r.standard_normal((7, 1))
    w = r.random(7) + 0.5
    h = 0.3
    val, _ = integrate.quad(lambda t: oracle.kde_laplace(x, h, w=w, z=np.array([[t]]))[0],
                            -15, 15, points=sorted(x[:, 0]), limit=400)
    assert val == pytest.approx(w.sum() / 7, rel=1e-8)


def test_kde_matches_1d_decomposition():
    """eq. (Laplacian decomposition 1d): f(z) = 1/(2h) [e^{-z/h} F_N(z; x, w e^{x/h})
    + e^{z/h} Fbar_N(z; x, w e^{-x/h})], evaluated with sorted cumulative sums."""
    r = np.random.default_rng(8)
    x = r.standard_normal(300)
    w = r.random(300)
    z = np.concatenate([x[:50], r.standard_normal(80)])
    h = 0.7
    order = np.argsort(x)
    xs, ws = x[order], w[order]
    cp = np.concatenate([[0.0], np.cumsum(ws * np.exp(xs / h))])
    cm = np.concatenate([np.cumsum((ws * np.exp(-xs / h))[::-1])[::-1], [0.0]])
    k = np.searchsorted(xs, z, side="right")      # F: x <= z ; Fbar: x > z
    dec = (np.exp(-z / h) * cp[k] / 300 + np.exp(z / h) * cm[k] / 300) / (2 * h)
    f = oracle.kde_laplace(x[:, None], h, w=w, z=z[:, None])
    np.testing.assert_allclose(f, dec, rtol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_kde_matches_nd_decomposition(d):
    """eq. (Laplacian decomposition nD): f(z) = 1/(2^d prod h) sum_delta
    e^{-delta.z/h} (1/N) S_delta(z; y(delta)), y_i(delta) = w_i e^{delta.x_i/h},
    with the orthant sums taken from ``orthant_sums`` (a different routine).
    Also checks the per-orthant terms returned by ``kde_laplace``."""
    r = np.random.default_rng(20 + d)
    n = 120
    x = np.round(r.standard_normal((n, d)) * 4) / 4     # ties on purpose
    w = r.random(n)
    z = np.concatenate([x[:30], r.standard_normal((20, d))])
    h = np.linspace(0.6, 1.1, d)
    f, terms = oracle.kde_laplace(x, h, w=w, z=z, terms=True)
    total = np.zeros(z.shape[0])
    for o in range(1 << d):
        delta = np.array([-1.0 if (o >> k & 1) else 1.0 for k in range(d)])
        yd = w * np.exp((x * delta / h).sum(axis=1))
        S = oracle.orthant_sums(x, y=yd, z=z, mask=1 << o)[0]
        term = np.exp(-(z * delta / h).sum(axis=1)) * S / n / (2 ** d * np.prod(h))
        np.testing.assert_allclose(terms[o], term, rtol=1e-12, atol=1e-300)
        total += term
    np.testing.assert_allclose(f, total, rtol=1e-12)
    np.testing.assert_allclose(terms.sum(axis=0), f, rtol=1e-13)


def test_kde_loo_drops_exactly_self():
    """LOO removes the i == j term only (duplicates stay) and renormalises by N-1."""
    x = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 2.0]])
    h = [1.0, 1.0]
    f = oracle.kde_laplace(x, h, loo=True)
    e = math.exp
    c = 1.0 / (4 * 2)
    np.testing.assert_allclose(f, [c * (1 + e(-3)), c * (1 + e(-3)), c * 2 * e(-3)], rtol=1e-15)


def test_kde_at_sampled_points_closed_form():
    """KDE at a subset of the sample points, with and without leave-one-out,
    on the five tie points (h = (0.5, 1)), expanded by hand: the LOO constant
    is 1/(4*(5-1)*0.5*1) = 1/8 and only index idx[j] itself is dropped (the
    duplicate (1,1) stays); weights w = 1..5 scale each term."""
    g = _read_tie_golden()
    x = np.array(g["points"])
    e = math.exp
    h = [0.5, 1.0]
    idx = [3, 0, 3, 4]
    loo = oracle.kde_at_points(x, h, idx, loo=True)
    np.testing.assert_allclose(loo, [(e(-3) + e(-1) + e(-2) + 1) / 8, (e(-2) + e(-1) + 2 * e(-3)) / 8,
                                     (e(-3) + e(-1) + e(-2) + 1) / 8, (e(-3) + e(-1) + e(-2) + 1) / 8],
                               rtol=1e-15)
    full = oracle.kde_at_points(x, h, [0, 2])
    np.testing.assert_allclose(full, [(1 + e(-2) + e(-1) + 2 * e(-3)) / 10, (e(-1) + e(-3) + 1 + 2 * e(-2)) / 10],
                               rtol=1e-15)
    w = np.arange(1.0, 6.0)
    lw = oracle.kde_at_points(x, h, [3], w=w, loo=True)
    assert lw[0] == pytest.approx((1 * e(-3) + 2 * e(-1) + 3 * e(-2) + 5 * 1) / 8, rel=1e-15)


def test_kreg_constant_and_ratio():
    """NW: constant y gives that constant; in general m = kde(w=y) / kde(w=1)."""
    r = np.random.default_rng(9)
    x = r.standard_normal((200, 2))
    z = r.standard_normal((40, 2))
    h = [0.3, 0.5]
    assert np.allclose(oracle.kreg_laplace(x, np.full(200, 2.5), h, z=z), 2.5, rtol=1e-14)
    y = r.standard_normal(200)
    m = oracle.kreg_laplace(x, y, h, z=z)
    ratio = oracle.kde_laplace(x, h, w=y, z=z) / oracle.kde_laplace(x, h, z=z)
    np.testing.assert_allclose(m, ratio, rtol=1e-11, atol=1e-13)
    # far target: defined through the min-shift even where the plain kernel underflows
    far = oracle.kreg_laplace(x, y, [1e-3, 1e-3], z=np.array([[50.0, 50.0]]))
    assert np.isfinite(far[0])


def test_kreg_leave_one_out_hand_worked():
    """Leave-one-out NW, d=1, x={0,1,3}, y={1,2,4}, h=1, expanded by hand:
    target j averages y over the two other points with weights e^{-|x_i - x_j|}.
      j=0: (2 e^-1 + 4 e^-3) / (e^-1 + e^-3) = (2 + 4 e^-2) / (1 + e^-2)
      j=1: (1 e^-1 + 4 e^-2) / (e^-1 + e^-2) = (1 + 4 e^-1) / (1 + e^-1)
      j=2: (1 e^-3 + 2 e^-2) / (e^-3 + e^-2) = (e^-1 + 2) / (e^-1 + 1)
    and, with the self term kept, j=0: (1 + 2 e^-1 + 4 e^-3) / (1 + e^-1 + e^-3)."""
    e = math.exp
    x = np.array([[0.0], [1.0], [3.0]])
    y = np.array([1.0, 2.0, 4.0])
    loo = oracle.kreg_laplace(x, y, 1.0, loo=True)
    np.testing.assert_allclose(loo, [(2 + 4 * e(-2)) / (1 + e(-2)), (1 + 4 * e(-1)) / (1 + e(-1)),
                                     (e(-1) + 2) / (e(-1) + 1)], rtol=1e-15)
    full = oracle.kreg_laplace(x, y, 1.0)
    assert full[0] == pytest.approx((1 + 2 * e(-1) + 4 * e(-3)) / (1 + e(-1) + e(-3)), rel=1e-15)
    # the five tie points of the 2D example, h=(0.5, 1), y = point index:
    # leave-one-out drops index j only, so the duplicate (1,1) of point 3 stays
    g = _read_tie_golden()
    x2 = np.array(g["points"])
    y2 = np.arange(5.0)
    w3 = [e(-3), e(-1), e(-2), 1.0]          # weights of points 0, 1, 2, 4 seen from (1,1)
    m3 = (0 * w3[0] + 1 * w3[1] + 2 * w3[2] + 4 * w3[3]) / sum(w3)
    assert oracle.kreg_laplace(x2, y2, [0.5, 1.0], loo=True)[3] == pytest.approx(m3, rel=1e-15)
    # one point: nothing left to average
    assert np.isnan(oracle.kreg_laplace(np.array([[0.5]]), np.array([3.0]), 1.0, loo=True)[0])


# ----------------------------------------------------------------------------- gradients


def _fd(fun, v, eps):
    g = np.zeros_like(v)
    for idx in np.ndindex(v.shape):
        vp, vm = v.copy(), v.copy()
        vp[idx] += eps
        vm[idx] -= eps
        g[idx] = (fun(vp) - fun(vm)) / (2 * eps)
    return g


def test_kde_grad_matches_finite_differences():
    """grad_w (linear), grad_z (off kinks) and grad_h by central differences."""
    r = np.random.default_rng(12)
    n, m, d = 60, 25, 2
    x = r.standard_normal((n, d))
    w = r.random(n)
    z = r.standard_normal((m, d))
    h = np.array([0.4, 0.8])
    g = r.standard_normal(m)
    gw, gz, gh = oracle.kde_grad(x, h, g, w=w, z=z)
    L = lambda ww=w, zz=z, hh=h: float(g @ oracle.kde_laplace(x, hh, w=ww, z=zz))
    np.testing.assert_allclose(gw, _fd(lambda v: L(ww=v), w, 1e-3), rtol=1e-7)
    np.testing.assert_allclose(gz, _fd(lambda v: L(zz=v), z, 1e-6), rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(gh, _fd(lambda v: L(hh=v), h, 1e-6), rtol=1e-6)


def test_kde_grad_w_dot_product_adjoint():
    """The KDE is linear in w, f = A w, and grad_w is the transposed sum A^T g:
    <g, A w> = <A^T g, w> for any g and w, and A^T g is the same whatever w
    it was computed at."""
    r = np.random.default_rng(21)
    n, m, d = 80, 30, 3
    x = r.standard_normal((n, d))
    z = r.standard_normal((m, d))
    h = np.array([0.3, 0.6, 0.9])
    g = r.standard_normal(m)
    w1, w2 = r.standard_normal(n), r.random(n)
    gw1 = oracle.kde_grad(x, h, g, w=w1, z=z)[0]
    gw2 = oracle.kde_grad(x, h, g, w=w2, z=z)[0]
    np.testing.assert_allclose(gw1, gw2, rtol=1e-13, atol=0)
    for w in (w1, w2):
        lhs = float(g @ oracle.kde_laplace(x, h, w=w, z=z))
        bound = float(np.abs(g) @ oracle.kde_laplace(x, h, w=np.abs(w), z=z))
        assert abs(lhs - float(gw1 @ w)) <= 1e-12 * bound


def test_kde_grad_loo_sample_points():
    r = np.random.default_rng(13)
    x = r.standard_normal((40, 3))
    h = np.array([0.5, 0.9, 1.3])
    g = r.standard_normal(40)
    gw, gz, gh = oracle.kde_grad(x, h, g, loo=True)
    assert gz is None
    L = lambda ww=None, hh=h: float(g @ oracle.kde_laplace(x, hh, w=ww, loo=True))
    np.testing.assert_allclose(gw, _fd(lambda v: L(ww=v), np.ones(40), 1e-3), rtol=1e-7)
    np.testing.assert_allclose(gh, _fd(lambda v: L(hh=v), h, 1e-6), rtol=1e-6)


def test_loo_loglik_gradient():
    r = np.random.default_rng(14)
    x = r.standard_normal((80, 2))
    h = np.array([0.35, 0.6])
    L, dL = oracle.loo_loglik(x, h)
    f = oracle.kde_laplace(x, h, loo=True)
    assert L == pytest.approx(np.mean(np.log(f)), rel=1e-13)
    np.testing.assert_allclose(dL, _fd(lambda v: oracle.loo_loglik(x, v)[0], h, 1e-6), rtol=1e-6)
