"""Non-finite coordinates through the C ABI: a NaN or an infinity in x (or in
explicit targets z, or interpolation points q) is found by the kernel that
first reads the coordinate and recorded in the device error word; the call
stays asynchronous, and fk_device_status returns FK_ERR_NONFINITE once and
clears it.  A following call on finite data is unaffected."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
P = ctypes.c_void_p
FK_ERR_NONFINITE = -4


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _st():
    import torch
    return P(torch.cuda.current_stream().cuda_stream)


def _status():
    from paper_2005_03246_gb300 import _lib
    return _lib.load().fk_device_status(_st())


def _pts(bad, dtype, seed=0, n=3000, d=3):
    x = np.random.default_rng(seed).standard_normal((n, d)).astype(dtype)
    if bad is not None:
        x[n // 3, d - 1] = bad
    return x


BAD = [np.nan, np.inf, -np.inf]


@pytest.mark.parametrize("bad", BAD)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_points_and_kde_record_nonfinite(bad, dtype):
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    code = _lib.FK_F64 if dtype == np.float64 else _lib.FK_F32
    assert _status() == 0
    x = _t(_pts(bad, dtype))
    n, d = x.shape
    out = torch.empty((1 << d, n), dtype=torch.int64, device="cuda:0")
    rc = lib.fk_ecdf_points(P(x.data_ptr()), code, n, d, None, None, 0, None, P(out.data_ptr()), 0, None, 0, _st())
    assert rc == 0
    assert _status() == FK_ERR_NONFINITE
    assert b"non-finite" in lib.fk_last_error()
    assert _status() == 0                                    # cleared
    f = torch.empty((n,), dtype=torch.float64, device="cuda:0")
    h = np.full(d, 0.2)
    rc = lib.fk_kde_laplace(P(x.data_ptr()), code, n, d, None, None, 0, h.ctypes.data_as(P), 0,
                            P(f.data_ptr()), None, 0, None, 0, _st())
    assert rc == 0
    assert _status() == FK_ERR_NONFINITE
    # finite data afterwards: no error, and the counts are right
    xg = _pts(None, dtype, seed=1, n=500)
    og = torch.empty((1 << d, 500), dtype=torch.int64, device="cuda:0")
    rc = lib.fk_ecdf_points(P(_t(xg).data_ptr()), code, 500, d, None, None, 0, None, P(og.data_ptr()), 0, None, 0,
                            _st())
    assert rc == 0
    assert _status() == 0
    assert np.array_equal(og.cpu().numpy(), oracle.orthant_sums(xg))


@pytest.mark.parametrize("bad", BAD)
def test_explicit_targets_record_nonfinite(bad):
    import torch
    import paper_2005_03246_gb300 as fk
    assert _status() == 0
    x = _t(_pts(None, np.float32))
    z = _pts(bad, np.float32, seed=2, n=100)
    fk.kde_laplace(x, 0.2, z=_t(z))
    assert _status() == FK_ERR_NONFINITE
    with pytest.raises(fk.FastEcdfError):
        fk.kde_laplace(x, 0.2, z=_t(z))
        fk.device_status()
    torch.cuda.synchronize()


@pytest.mark.parametrize("bad", BAD)
def test_grid_paths_record_nonfinite(bad):
    import torch
    import paper_2005_03246_gb300 as fk
    assert _status() == 0
    x = _pts(bad, np.float64, n=2000, d=2)
    axes = [np.linspace(-2, 2, 33), np.linspace(-2, 2, 17)]
    fk.ecdf_grid(_t(x), axes)
    assert _status() == FK_ERR_NONFINITE
    fk.kde_grid(_t(x), 0.3, axes)
    assert _status() == FK_ERR_NONFINITE
    f = fk.kde_grid(_t(_pts(None, np.float64, n=2000, d=2)), 0.3, axes)
    assert _status() == 0
    fk.grid_interp(f, axes, _t(_pts(bad, np.float64, n=50, d=2)))
    assert _status() == FK_ERR_NONFINITE
    torch.cuda.synchronize()


def test_batched_records_nonfinite():
    import paper_2005_03246_gb300 as fk
    assert _status() == 0
    xs = [_t(_pts(None, np.float32, seed=s, n=700, d=2)) for s in range(3)]
    xs.append(_t(_pts(np.nan, np.float32, seed=9, n=900, d=2)))
    fk.Batched(xs, h=0.1, graph=False).run()
    assert _status() == FK_ERR_NONFINITE
    fk.Batched(xs[:3], h=0.1, graph=False).run()
    assert _status() == 0
