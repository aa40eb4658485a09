"""GPU parity of the sample-point path (Sec. 2.2 and Appendix D: rank transform
+ divide-and-conquer) and of the Laplacian kernel sums (Sec. 3.1) against the
CPU oracle, through the C ABI.

Counts must be bit-exact.  Weighted sums of signed terms are compared against
the orthant sums of |y| (the condition of a sum); kernel values use the
relative error on entries >= 1e-6 max, within 1e-5 (mixed path) and 1e-12
(FP64 path).
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


def _rel_signed(got, ref, absref):
    return np.max(np.abs(got - ref) / np.maximum(absref, 1e-300))


def _rel_nw(got, ref, cond):
    """Nadaraya-Watson error per target, relative to the regression of |y| at
    that target (the sum of magnitudes of its numerator over its denominator):
    a ratio of signed kernel sums is only accurate relative to that condition.
    As in the signed-output metric, the scale never drops below 1e-6 of the
    largest reference value (targets whose whole numerator lies far below it,
    e.g. isolated points with y = 0, carry kernel values near the bottom of
    the FP32 range on the mixed path)."""
    return np.max(np.abs(got - ref) / np.maximum(cond, 1e-6 * np.abs(ref).max()))


def _c9(got, ref):
    """|g - o| / max(|o|, 1e-6 max|o|): the signed-output metric applied to
    every entry, including those near zero."""
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max()))


def _points(n, d, seed, ties=True, dtype=np.float32):
    r = np.random.default_rng(seed)
    x = r.standard_normal((n, d))
    if ties:
        m = r.random((n, d)) < 0.3
        x[m] = np.round(x[m] * 8) / 8
    return x.astype(dtype)


# ------------------------------------------------------------------ orthant sums


def test_tie_example_golden():
    """The hand-worked 5-point example with ties (eq. ECDFdelta)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tie2d_orthants.txt"))
            if l.strip() and not l.startswith("#")]
    pts = np.array([[float(v) for v in r] for r in rows[1:6]])
    expect = np.array([[int(v) for v in rows[7 + 2 * o]] for o in range(4)])
    got = _fk().ecdf_points(_t(pts)).cpu().numpy()
    assert np.array_equal(got, expect)


def test_small_config_counts_and_weights():
    """d=2, N=1e4, FP64, 10% rounded coordinates: all orthants at the sample points."""
    data = datagen.ecdf_small()
    x, y = data["x"], data["y"]
    ref = oracle.orthant_sums(x)
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert np.array_equal(got, ref)
    refw = oracle.orthant_sums(x, y=y)
    absw = oracle.orthant_sums(x, y=np.abs(y))
    for path in ("fp64", "mixed"):
        gw = _fk().ecdf_points(_t(x), y=_t(y), path=path).cpu().numpy()
        assert _rel_signed(gw, refw, absw) <= TOL[path], path


def test_small_config_explicit_grid_targets_match_grid_path():
    """The same counts at the 128x128 grid points as explicit targets equal the
    grid path and the oracle."""
    data = datagen.ecdf_small()
    x = data["x"]
    z = oracle.grid_points(data["grid"])
    got = _fk().ecdf_points(_t(x), z=_t(z)).cpu().numpy()
    ref = oracle.orthant_sums(x, z=z)
    assert np.array_equal(got, ref)
    grid = _fk().ecdf_grid(_t(x), data["grid"]).cpu().numpy().reshape(4, -1)
    assert np.array_equal(got, grid)


@pytest.mark.parametrize("d,n", [(1, 3000), (2, 2500), (3, 3100), (4, 1500), (3, 70000)])
def test_orthant_counts_dims(d, n):
    """All orthants, ties on every axis, sizes spanning several CTA tiles and a
    ragged tail; n=70000 exercises merged blocks larger than one tile."""
    x = _points(n, d, seed=100 + d)
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    if n <= 5000:
        ref = oracle.orthant_sums(x)
        assert np.array_equal(got, ref)
    else:
        idx = datagen.sample_targets(n, 512, seed=7, include=(0, n - 1))
        ref = oracle.orthant_sums(x, z=x[idx])
        assert np.array_equal(got[:, idx], ref)
    assert np.all(got.sum(axis=0) == n)          # the orthants partition the sources


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_esf_and_mask(d):
    x = _points(1200, d, seed=300 + d)
    y = np.random.default_rng(1).random(1200).astype(np.float32)
    full = (1 << d) - 1
    got = _fk().esf_points(_t(x)).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(x, mask=[full])[0])
    sel = [full, 0] if d > 0 else [0]
    g2 = _fk().ecdf_points(_t(x), y=_t(y), orthants=sel, path="fp64").cpu().numpy()
    r2 = oracle.orthant_sums(x, y=y, mask=sorted(sel))
    assert np.max(np.abs(g2 - r2) / np.maximum(r2, 1e-300)) <= 1e-12


def test_explicit_targets_with_ties_between_sources_and_targets():
    r = np.random.default_rng(9)
    x = np.round(r.random((4000, 3)) * 20) / 20
    z = np.round(r.random((900, 3)) * 20) / 20
    got = _fk().ecdf_points(_t(x), z=_t(z)).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(x, z=z))


def test_empty_and_single_point():
    fk = _fk()
    x0 = np.zeros((0, 2), dtype=np.float32)
    assert fk.ecdf_points(_t(x0)).shape == (4, 0)
    x1 = np.array([[0.5, -1.0]], dtype=np.float32)
    got = fk.ecdf_points(_t(x1)).cpu().numpy()
    assert got.tolist() == [[1], [0], [0], [0]]
    z = np.array([[0.0, 0.0], [1.0, -2.0]], dtype=np.float32)
    got = fk.ecdf_points(_t(x1), z=_t(z)).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(x1, z=z))


def test_full_size_d3_sampled_targets():
    """d=3, N=1e6 correlated Gaussian (FP32): 2048 sampled targets against the
    oracle, plus the exact partition invariant on every target."""
    data = datagen.ecdf_gauss3()
    x = data["x"]
    n = x.shape[0]
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert np.all(got.sum(axis=0) == n)
    idx = datagen.sample_targets(n, 2048, seed=5, include=(0, n - 1, int(np.argmax(x[:, 0]))))
    ref = oracle.orthant_sums(x, z=x[idx])
    assert np.array_equal(got[:, idx], ref)


def test_full_size_d2_fenwick_every_target():
    """d=2, N=1e6 (copula, FP32): every output checked by the Fenwick sweep."""
    x = datagen.copula_t4()["x"]
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert np.array_equal(got, oracle.fenwick2d(x))


# ------------------------------------------------------------------ kernel sums


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d,n", [(1, 2000), (2, 3000), (3, 2500), (4, 1200)])
def test_kde_sample_points(path, d, n):
    x = _points(n, d, seed=500 + d)
    h = np.linspace(0.15, 0.4, d)
    w = np.random.default_rng(d).random(n).astype(np.float32)
    got = _fk().kde_laplace(_t(x), h, w=_t(w), path=path).cpu().numpy()
    ref = oracle.kde_laplace(x, h, w=w)
    assert _rel_kde(got, ref) <= TOL[path]


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_kde_explicit_targets_terms_and_loo(path):
    x = _points(3000, 3, seed=11)
    z = _points(700, 3, seed=12)
    h = [0.2, 0.3, 0.25]
    got, terms = _fk().kde_laplace(_t(x), h, z=_t(z), terms=True, path=path)
    ref, rterms = oracle.kde_laplace(x, h, z=z, terms=True)
    assert _rel_kde(got.cpu().numpy(), ref) <= TOL[path]
    tt = terms.cpu().numpy()
    assert np.max(np.abs(tt - rterms)) <= TOL[path] * ref.max() * 8
    gl = _fk().kde_laplace(_t(x), h, loo=True, path=path).cpu().numpy()
    assert _rel_kde(gl, oracle.kde_laplace(x, h, loo=True)) <= TOL[path]


@pytest.mark.parametrize("h", [0.05, 0.1, 0.3])
def test_kde_copula_heavy_tails_no_overflow(h):
    """Student-t tails with small h: e^{|x|/h} overflows FP64 without the shifts."""
    x = datagen.copula_t4(n=20000)["x"]
    for path in ("mixed", "fp64"):
        got = _fk().kde_laplace(_t(x), h, path=path).cpu().numpy()
        idx = datagen.sample_targets(x.shape[0], 800, seed=3, include=(int(np.argmax(x[:, 0])),))
        ref = oracle.kde_laplace(x, h, z=x[idx])
        assert np.all(np.isfinite(got))
        assert _rel_kde(got[idx], ref) <= TOL[path], path


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("h", [0.05, 0.1, 0.3])
def test_kreg(path, h):
    d = datagen.copula_t4(n=6000)
    x, y = d["x"], d["y"]
    got = _fk().kreg_laplace(_t(x), _t(y), h, path=path).cpu().numpy()
    ref = oracle.kreg_laplace(x, y, h)
    cond = oracle.kreg_laplace(x, np.abs(y), h)
    assert _rel_nw(got, ref, cond) <= TOL[path]
    if path == "fp64":
        assert _c9(got, ref) <= TOL[path]


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_kreg_leave_one_out(path, d):
    """Leave-one-out NW at the sample points: each target averages y over the
    other points only (index j dropped, equal-valued duplicates kept)."""
    r = np.random.default_rng(90 + d)
    x = r.standard_normal((4000, d))
    tie = r.random((4000, d)) < 0.2
    x[tie] = np.round(x[tie] * 4) / 4
    x = x.astype(np.float32)
    x[7] = x[11]                                    # an exact duplicate pair
    y = (np.cos(x.sum(axis=1)) + 0.2 * r.standard_normal(4000)).astype(np.float32)
    h = np.linspace(0.15, 0.3, d)
    got = _fk().kreg_laplace(_t(x), _t(y), h, loo=True, path=path).cpu().numpy()
    ref = oracle.kreg_laplace(x, y, h, loo=True)
    cond = oracle.kreg_laplace(x, np.abs(y), h, loo=True)
    assert _rel_nw(got, ref, cond) <= TOL[path]
    # leave-one-out differs from the estimate that keeps the self pair
    full = oracle.kreg_laplace(x, y, h)
    assert np.max(np.abs(ref - full)) > 1e-3


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_kreg_explicit_targets(path, d):
    """Nadaraya-Watson at explicit targets: the target items carry no weight
    in either channel (numerator y, denominator 1)."""
    r = np.random.default_rng(60 + d)
    x = r.standard_normal((5000, d)).astype(np.float32)
    y = (np.sin(x.sum(axis=1)) + 0.1 * r.standard_normal(5000)).astype(np.float32)
    z = (r.standard_normal((700, d)) * 1.1).astype(np.float32)
    h = np.linspace(0.2, 0.35, d)
    got = _fk().kreg_laplace(_t(x), _t(y), h, z=_t(z), path=path).cpu().numpy()
    ref = oracle.kreg_laplace(x, y, h, z=z)
    cond = oracle.kreg_laplace(x, np.abs(y), h, z=z)
    assert _rel_nw(got, ref, cond) <= TOL[path]


def test_kde_full_size_d3_sampled():
    """d=3, N=1e6, h=0.1 (the paper's bandwidth): 1024 sampled targets."""
    x = datagen.ecdf_gauss3()["x"]
    n = x.shape[0]
    idx = datagen.sample_targets(n, 1024, seed=8, include=(0, n - 1))
    ref = oracle.kde_laplace(x, 0.1, z=x[idx])
    for path in ("mixed", "fp64"):
        got = _fk().kde_laplace(_t(x), 0.1, path=path).cpu().numpy()
        assert _rel_kde(got[idx], ref) <= TOL[path], path


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_kernel_sums_with_zero_weights_and_wide_spread(path):
    """Weights and responses with many exact zeros, points spread over 30
    bandwidth-scaled units per axis (shifts of the factors differ by far more
    than the FP32 exponent range): a zero term must not disturb the sums."""
    r = np.random.default_rng(41)
    n = 4000
    x = (r.random((n, 3)) * 30.0).astype(np.float32)
    x[: n // 2] = (r.standard_normal((n // 2, 3)) * 0.3 + 15.0).astype(np.float32)
    h = [0.05, 0.08, 0.06]
    w = r.random(n).astype(np.float32)
    w[r.random(n) < 0.4] = 0.0
    got = _fk().kde_laplace(_t(x), h, w=_t(w), path=path).cpu().numpy()
    ref = oracle.kde_laplace(x, h, w=w)
    assert _rel_kde(got, ref) <= TOL[path]
    y = r.standard_normal(n).astype(np.float32)
    y[r.random(n) < 0.4] = 0.0
    gk = _fk().kreg_laplace(_t(x), _t(y), h, path=path).cpu().numpy()
    rk = oracle.kreg_laplace(x, y, h)
    ck = oracle.kreg_laplace(x, np.abs(y), h)
    ok = np.isfinite(rk)
    assert _rel_nw(gk[ok], rk[ok], ck[ok]) <= TOL[path]


@pytest.mark.parametrize("d,n", [(5, 1500), (6, 900), (8, 300)])
def test_orthant_counts_high_dimension(d, n):
    """Exact counts at the sample points for d = 5..8 (inclusion-exclusion
    over dominance counts of up to 8 axes), with ties; explicit targets with
    an orthant mask; the ESF."""
    x = _points(n, d, seed=700 + d)
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert got.shape == (1 << d, n)
    assert np.array_equal(got, oracle.orthant_sums(x))
    z = _points(120, d, seed=800 + d)
    sel = [0, 1, (1 << d) - 1, 5, (1 << (d - 1))]
    got_z = _fk().ecdf_points(_t(x), z=_t(z), orthants=sel).cpu().numpy()
    assert np.array_equal(got_z, oracle.orthant_sums(x, z=z, mask=sel))
    esf = _fk().esf_points(_t(x)).cpu().numpy()
    assert np.array_equal(esf.reshape(-1), oracle.orthant_sums(x, mask=[(1 << d) - 1])[0])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_counts_single_item_tie_correction(d, dtype):
    """Counts at the sample points with one item per point: ties in short
    groups (half the coordinates on a 1/256 lattice, and 5% of the points
    exact duplicates of others, tied on every axis) are corrected exactly."""
    r = np.random.default_rng(900 + d)
    n = 4000 if d <= 4 else 1500
    x = r.standard_normal((n, d))
    m = r.random((n, d)) < 0.5
    x[m] = np.round(x[m] * 256) / 256
    dup = r.choice(n, size=n // 20, replace=False)
    x[dup] = x[r.integers(0, n, size=dup.size)]
    x = x.astype(dtype)
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(x))
    esf = _fk().esf_points(_t(x)).cpu().numpy()
    assert np.array_equal(esf.reshape(-1), oracle.orthant_sums(x, mask=[(1 << d) - 1])[0])


@pytest.mark.parametrize("d", [2, 3])
def test_counts_long_tie_groups_fall_back(d):
    """Integer points in {0..3}^d: tie groups of hundreds of points on every
    axis (the copy layout is used); counts still exact."""
    r = np.random.default_rng(950 + d)
    x = r.integers(0, 4, size=(3000, d)).astype(np.float32)
    got = _fk().ecdf_points(_t(x)).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(x))


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_weighted_sums_with_short_ties_and_duplicates(d, dtype, path):
    """Weighted orthant sums at the sample points with short tie groups and
    exact duplicates (tied on every axis); error against the oracle relative
    to the orthant sums of |y| (exact zeros where an orthant holds no point);
    an orthant mask selects a subset of rows; the ESF."""
    r = np.random.default_rng(1000 + d)
    n = 3000
    x = r.standard_normal((n, d))
    m = r.random((n, d)) < 0.5
    x[m] = np.round(x[m] * 256) / 256
    dup = r.choice(n, size=n // 20, replace=False)
    x[dup] = x[r.integers(0, n, size=dup.size)]
    x = x.astype(dtype)
    y = r.standard_normal(n).astype(dtype)
    got = _fk().ecdf_points(_t(x), y=_t(y), path=path).cpu().numpy()
    ref = oracle.orthant_sums(x, y=y)
    absw = oracle.orthant_sums(x, y=np.abs(y))
    assert _rel_signed(got, ref, absw) <= TOL[path]
    sel = [0, (1 << d) - 1, 1]
    g2 = _fk().ecdf_points(_t(x), y=_t(y), orthants=sel, path=path).cpu().numpy()
    assert _rel_signed(g2, ref[sorted(sel)], absw[sorted(sel)]) <= TOL[path]
    esf = _fk().esf_points(_t(x), y=_t(y), path=path).cpu().numpy()
    assert _rel_signed(esf.reshape(-1), ref[-1], absw[-1]) <= TOL[path]


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_weighted_sums_integer_lattice(path):
    r = np.random.default_rng(1100)
    x = r.integers(0, 5, size=(2500, 3)).astype(np.float64)
    y = r.standard_normal(2500)
    got = _fk().ecdf_points(_t(x), y=_t(y), path=path).cpu().numpy()
    ref = oracle.orthant_sums(x, y=y)
    absw = oracle.orthant_sums(x, y=np.abs(y))
    assert _rel_signed(got, ref, absw) <= TOL[path]


@pytest.mark.parametrize("d", [2, 3, 5])
def test_orthant_subsets_only_what_the_selection_needs(d):
    """A selection of orthants computes only the dominance counts it reads: the
    plain ECDF (orthant 0, one d-axis dominance count), the ESF (all subsets)
    and a mixed selection agree with the oracle, at the sample points (with
    ties) and at explicit targets."""
    x = _points(2500, d, seed=1200 + d)
    z = _points(300, d, seed=1300 + d)
    full = (1 << d) - 1
    for sel in ([0], [full], [1, (1 << d) - 2], [0, 3, full]):
        got = _fk().ecdf_points(_t(x), orthants=sel).cpu().numpy()
        assert np.array_equal(got, oracle.orthant_sums(x, mask=sorted(sel))), sel
        gz = _fk().ecdf_points(_t(x), z=_t(z), orthants=sel).cpu().numpy()
        assert np.array_equal(gz, oracle.orthant_sums(x, z=z, mask=sorted(sel))), sel


# ------------------------------------------------------------------ d = 5, 6


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d,n", [(5, 1200), (6, 700)])
def test_high_dimension_kernel_and_weighted_sums(path, d, n):
    """d = 5, 6 at the sample points (16 and 32 sweep channels): the Laplacian
    KDE, its leave-one-out form, explicit targets, Nadaraya-Watson (two
    one-channel sums) and the weighted orthant sums, against the oracle."""
    r = np.random.default_rng(900 + d)
    x = _points(n, d, seed=910 + d)
    h = np.linspace(0.4, 0.7, d)
    got = _fk().kde_laplace(_t(x), h, path=path).cpu().numpy()
    assert _rel_kde(got, oracle.kde_laplace(x, h)) <= TOL[path]
    gl = _fk().kde_laplace(_t(x), h, loo=True, path=path).cpu().numpy()
    assert _rel_kde(gl, oracle.kde_laplace(x, h, loo=True)) <= TOL[path]
    z = (r.standard_normal((150, d)) * 0.9).astype(np.float32)
    gz = _fk().kde_laplace(_t(x), h, z=_t(z), path=path).cpu().numpy()
    assert _rel_kde(gz, oracle.kde_laplace(x, h, z=z)) <= TOL[path]
    y = (np.sin(x.sum(axis=1)) + 0.1 * r.standard_normal(n)).astype(np.float32)
    gk = _fk().kreg_laplace(_t(x), _t(y), h, path=path).cpu().numpy()
    assert _rel_nw(gk, oracle.kreg_laplace(x, y, h), oracle.kreg_laplace(x, np.abs(y), h)) <= TOL[path]
    w = r.random(n).astype(np.float32)
    gw = _fk().ecdf_points(_t(x), y=_t(w), path=path).cpu().numpy()
    ref = oracle.orthant_sums(x, y=w)
    absref = oracle.orthant_sums(x, y=np.abs(w))
    assert gw.shape == (1 << d, n)
    assert _rel_signed(gw, ref, absref) <= TOL[path]


def test_high_dimension_refusals():
    """What needs per-orthant terms or two weight channels in one sweep stays
    at d <= 4: refused with FK_ERR_UNSUPPORTED."""
    import torch
    fk = _fk()
    x = _t(_points(300, 5, seed=5))
    with pytest.raises(fk.FastEcdfError, match="d <= 4"):
        fk.kde_laplace_backward(x, 0.5, torch.ones(300, dtype=torch.float64, device="cuda:0"))
    with pytest.raises(fk.FastEcdfError, match="d <= 4"):
        fk.loo_laplace(x, 0.5)
    with pytest.raises(fk.FastEcdfError, match="d <= 4"):
        fk.kde_laplace(x, 0.5, terms=True)
