"""GPU parity of the grid path (Sec. 2.1, Algorithms 1, 6, 7) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu


def _fk():
    import paper_2005_03246_gb300 as fk
    return fk


def _dev():
    import torch
    return torch.device("cuda:0")


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def test_grid_small_config_counts_bit_exact():
    """d=2, N=1e4, 128x128 grid, all 4 orthants, y == 1: bit-exact counts."""
    import torch
    data = datagen.ecdf_small()
    x = torch.as_tensor(data["x"], device=_dev())
    got = _fk().ecdf_grid(x, data["grid"]).cpu().numpy()
    ref = oracle.ecdf_grid(data["x"], data["grid"])
    assert got.dtype == np.int64
    assert np.array_equal(got, ref)


def test_grid_tie_grid_points_on_grid_lines():
    """Rounded coordinates land exactly on the k/100 grid lines: x == z must bin
    into the <= side (eq. partial sums), which mesh division alone can miss."""
    import torch
    data = datagen.ecdf_small()
    x = torch.as_tensor(data["x"], device=_dev())
    got = _fk().ecdf_grid(x, data["tie_grid"]).cpu().numpy()
    ref = oracle.ecdf_grid(data["x"], data["tie_grid"])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("path,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_grid_weighted_signed(path, tol):
    """y ~ N(0,1).  A sum of signed terms is only accurate relative to the sum of
    their magnitudes, so the error is measured against the orthant sums of |y|."""
    import torch
    data = datagen.ecdf_small()
    x = torch.as_tensor(data["x"], device=_dev())
    y = torch.as_tensor(data["y"], device=_dev())
    got = _fk().ecdf_grid(x, data["grid"], y=y, path=path).cpu().numpy()
    ref = oracle.ecdf_grid(data["x"], data["grid"], y=data["y"])
    den = oracle.ecdf_grid(data["x"], data["grid"], y=np.abs(data["y"]))
    assert np.max(np.abs(got - ref) / np.maximum(den, 1e-300)) <= tol


@pytest.mark.parametrize("d,M", [(1, (37,)), (3, (5, 9, 7)), (4, (3, 4, 5, 2))])
def test_grid_other_dims_and_nonuniform_axes(d, M):
    import torch
    r = np.random.default_rng(40 + d)
    xn = np.round(r.standard_normal((2500, d)) * 3) / 3
    axes = [np.sort(r.choice(np.linspace(-3, 3, 61), size=m, replace=False)) for m in M]
    x = torch.as_tensor(xn.astype(np.float32), device=_dev())
    got = _fk().ecdf_grid(x, axes).cpu().numpy()
    ref = oracle.ecdf_grid(xn.astype(np.float32), axes)
    assert np.array_equal(got, ref)
    # a subset of orthants, in increasing index
    sel = [0, (1 << d) - 1]
    got2 = _fk().ecdf_grid(x, axes, orthants=sel).cpu().numpy()
    assert np.array_equal(got2, ref[sel])


def test_grid_empty_input_and_single_cell():
    import torch
    x = torch.zeros((0, 2), dtype=torch.float64, device=_dev())
    got = _fk().ecdf_grid(x, [np.array([0.0]), np.array([0.0, 1.0])]).cpu().numpy()
    assert got.shape == (4, 1, 2) and not got.any()


def test_grid_host_buffers_match_device():
    """The ABI also accepts host pointers and stages them itself."""
    import ctypes
    import torch
    from paper_2005_03246_gb300 import _lib, mask_words
    lib = _lib.load()
    data = datagen.ecdf_small(n=2000)
    axes = data["grid"]
    M = np.array([len(a) for a in axes], dtype=np.int64)
    z = np.concatenate(axes)
    out = np.zeros((4, len(axes[0]), len(axes[1])), dtype=np.int64)
    x = np.ascontiguousarray(data["x"])
    rc = lib.fk_ecdf_grid(x.ctypes.data_as(ctypes.c_void_p), _lib.FK_F64, x.shape[0], 2, None,
                          z.ctypes.data_as(ctypes.c_void_p), M.ctypes.data_as(ctypes.c_void_p),
                          None, out.ctypes.data_as(ctypes.c_void_p), 0, None, 0, None)
    _lib.check(rc, "fk_ecdf_grid(host)")
    assert np.array_equal(out, oracle.ecdf_grid(data["x"], axes))


def test_pinned_host_buffers_are_asynchronous_and_correct():
    """With page-locked host arrays the calls stay asynchronous: three calls on
    three streams, outputs checked after the streams finish (sample-point
    counts, grid counts and the KDE, against the oracle)."""
    import ctypes
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    P = ctypes.c_void_p
    data = datagen.ecdf_small(n=3000)
    axes = data["grid"]
    M = np.array([len(a) for a in axes], dtype=np.int64)
    xh = torch.as_tensor(np.ascontiguousarray(data["x"])).pin_memory()
    zh = torch.as_tensor(np.concatenate(axes)).pin_memory()
    og = torch.full((4, len(axes[0]) * len(axes[1])), -1, dtype=torch.int64).pin_memory()
    op = torch.full((4, 3000), -1, dtype=torch.int64).pin_memory()
    of = torch.full((3000,), -1.0, dtype=torch.float64).pin_memory()
    h = np.array([0.05, 0.05])
    ss = [torch.cuda.Stream() for _ in range(3)]
    _lib.check(lib.fk_ecdf_grid(P(xh.data_ptr()), _lib.FK_F64, 3000, 2, None, P(zh.data_ptr()),
                                M.ctypes.data_as(P), None, P(og.data_ptr()), 0, None, 0, P(ss[0].cuda_stream)),
               "fk_ecdf_grid(pinned)")
    _lib.check(lib.fk_ecdf_points(P(xh.data_ptr()), _lib.FK_F64, 3000, 2, None, None, 0, None, P(op.data_ptr()),
                                  0, None, 0, P(ss[1].cuda_stream)), "fk_ecdf_points(pinned)")
    _lib.check(lib.fk_kde_laplace(P(xh.data_ptr()), _lib.FK_F64, 3000, 2, None, None, 0, h.ctypes.data_as(P), 0,
                                  P(of.data_ptr()), None, 1, None, 0, P(ss[2].cuda_stream)), "fk_kde_laplace(pinned)")
    for s in ss:
        s.synchronize()
    assert np.array_equal(og.numpy().reshape(4, len(axes[0]), len(axes[1])), oracle.ecdf_grid(data["x"], axes))
    assert np.array_equal(op.numpy(), oracle.orthant_sums(data["x"]))
    ref = oracle.kde_laplace(data["x"], h)
    assert np.max(np.abs(of.numpy() - ref) / ref) <= 1e-12


def test_pool_memory_reuse_and_release():
    """Calls without a workspace allocate from the library's pool; the cached
    memory can be released between calls and later calls still work."""
    import ctypes
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    data = datagen.ecdf_small(n=2000)
    x = np.ascontiguousarray(data["x"])
    ref = oracle.orthant_sums(x)
    for k in range(3):
        out = np.zeros((4, 2000), dtype=np.int64)
        rc = lib.fk_ecdf_points(x.ctypes.data_as(ctypes.c_void_p), _lib.FK_F64, 2000, 2, None, None, 0, None,
                                out.ctypes.data_as(ctypes.c_void_p), 0, None, 0, None)
        _lib.check(rc, "fk_ecdf_points(host)")
        assert np.array_equal(out, ref)
        if k == 1:
            _lib.check(lib.fk_release_cached_memory(), "fk_release_cached_memory")


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_grid_orthant_selection(d):
    """Orthant selections on the grid (only the channels that feed a selected
    orthant are scanned): the plain ECDF, the ESF, and mixed selections, counts
    and weighted sums, against the oracle."""
    r = np.random.default_rng(1400 + d)
    n = 3000
    x = np.round(r.standard_normal((n, d)) * 4) / 4
    y = r.standard_normal(n)
    axes = [np.sort(np.unique(np.round(r.standard_normal(9 - d) * 4) / 4)) for _ in range(d)]
    full = (1 << d) - 1
    sels = [[0], [full], sorted({0, full}), sorted({1 % (1 << d), full - 1 if full > 1 else 0})]
    for sel in sels:
        got = _fk().ecdf_grid(_t(x), axes, orthants=sel).cpu().numpy()
        assert np.array_equal(got, oracle.ecdf_grid(x, axes, mask=sel)), sel
        gw = _fk().ecdf_grid(_t(x), axes, y=_t(y), orthants=sel, path="fp64").cpu().numpy()
        rw = oracle.ecdf_grid(x, axes, y=y, mask=sel)
        aw = oracle.ecdf_grid(x, axes, y=np.abs(y), mask=sel)
        assert np.max(np.abs(gw - rw) / np.maximum(aw, 1e-300)) <= 1e-12, sel
