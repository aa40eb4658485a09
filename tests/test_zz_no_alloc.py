"""fk_ecdf_grid_counts_noalloc: grid orthant counts with no device allocation.

Callers that may not allocate device memory while they run (allocation-free
real-time loops, or applications that own the whole device memory budget) use
this entry point; it keeps its scratch in a fixed array inside the library.
These checks call it through the C ABI with device buffers.  The same case
runs twice in a row, and both results must equal the oracle's counts and the
allocating fk_ecdf_grid (the second call must not see the first call's
histogram).  A partial orthant selection and an empty one go through the same
entry, and an oversized grid is refused.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu

P = ctypes.c_void_p


def _code(x):
    from paper_2005_03246_gb300 import _lib
    return _lib.FK_F64 if x.element_size() == 8 else _lib.FK_F32


def _alloc_call(lib, x, z, M, mask, out, st):
    from paper_2005_03246_gb300 import _lib
    rc = lib.fk_ecdf_grid(P(x.data_ptr()), _code(x), x.shape[0], x.shape[1], None, P(z.data_ptr()),
                          M.ctypes.data_as(P), None if mask is None else mask.ctypes.data_as(P),
                          P(out.data_ptr()), 0, None, 0, st)
    _lib.check(rc, "fk_ecdf_grid")


def _noalloc_call(lib, x, z, M, mask, out, st):
    return lib.fk_ecdf_grid_counts_noalloc(P(x.data_ptr()), _code(x), x.shape[0], x.shape[1], P(z.data_ptr()),
                                           M.ctypes.data_as(P), None if mask is None else mask.ctypes.data_as(P),
                                           P(out.data_ptr()), st)


def _case(seed, n, axes, dtype):
    import torch
    r = np.random.default_rng(seed)
    d = len(axes)
    xn = (np.round(r.standard_normal((n, d)) * 4) / 4).astype(dtype)   # many points on grid lines
    x = torch.as_tensor(xn, device="cuda:0")
    z = torch.as_tensor(np.concatenate(axes).astype(np.float64), device="cuda:0")
    M = np.array([len(a) for a in axes], dtype=np.int64)
    return xn, x, z, M


def _run_twice(lib, x, z, M, mask, nsel, st):
    import torch
    from paper_2005_03246_gb300 import _lib
    shape = (nsel, int(np.prod(M)))
    outs = []
    for _ in range(2):
        got = torch.full(shape, -1, dtype=torch.int64, device="cuda:0")
        _lib.check(_noalloc_call(lib, x, z, M, mask, got, st), "fk_ecdf_grid_counts_noalloc")
        outs.append(got)
    ref = torch.empty(shape, dtype=torch.int64, device="cuda:0")
    _alloc_call(lib, x, z, M, mask, ref, st)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], ref.cpu().numpy()


def test_noalloc_same_case_twice_matches_oracle():
    """d = 3, all 8 orthants, twice in a row: oracle counts bit-exact both times."""
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    axes = [np.linspace(-2, 2, 17), np.linspace(-3, 1, 13), np.linspace(-1, 2, 11)]
    xn, x, z, M = _case(7, 5000, axes, np.float32)
    want = oracle.ecdf_grid(xn, axes).reshape(8, -1)
    outs, ref = _run_twice(lib, x, z, M, None, 8, st)
    for got in outs:
        assert np.array_equal(got, want)
    assert np.array_equal(ref, want)


def test_noalloc_small_workload_twice_matches_oracle():
    """The d = 2, N = 1e4 FP64 tie workload on its 128 x 128 grid, twice in a row."""
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    small = datagen.ecdf_small()
    x = torch.as_tensor(small["x"], device="cuda:0")
    z = torch.as_tensor(np.concatenate(small["grid"]), device="cuda:0")
    M = np.array([len(a) for a in small["grid"]], dtype=np.int64)
    want = oracle.ecdf_grid(small["x"], small["grid"]).reshape(4, -1)
    outs, ref = _run_twice(lib, x, z, M, None, 4, st)
    for got in outs:
        assert np.array_equal(got, want)
    assert np.array_equal(ref, want)


def test_noalloc_partial_orthant_selection_matches_oracle():
    """A selection of orthants {1, 4, 6} at d = 3: rows in increasing orthant index."""
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    axes = [np.linspace(-2, 2, 9), np.linspace(-1.5, 1.5, 15), np.linspace(-1, 2, 12)]
    xn, x, z, M = _case(11, 3000, axes, np.float64)
    sel = [1, 4, 6]
    mask = oracle.mask_bits(3, sel)
    want = oracle.ecdf_grid(xn, axes, mask=sel).reshape(len(sel), -1)
    outs, ref = _run_twice(lib, x, z, M, mask, len(sel), st)
    for got in outs:
        assert np.array_equal(got, want)
    assert np.array_equal(ref, want)


def test_noalloc_empty_selection_writes_nothing():
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    axes = [np.linspace(-1, 1, 5)] * 2
    _, x, z, M = _case(5, 100, axes, np.float32)
    out = torch.full((1, 25), -7, dtype=torch.int64, device="cuda:0")
    rc = _noalloc_call(lib, x, z, M, np.zeros(1, dtype=np.uint32), out, st)
    _lib.check(rc, "fk_ecdf_grid_counts_noalloc")
    torch.cuda.synchronize()
    assert bool((out == -7).all())


def test_noalloc_refuses_grid_beyond_its_scratch():
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    axes = [np.linspace(0, 1, 256)] * 3            # needs far more than 16 MiB of scratch
    _, x, z, M = _case(3, 100, axes, np.float32)
    out = torch.empty((8, 1), dtype=torch.int64, device="cuda:0")   # never written
    rc = _noalloc_call(lib, x, z, M, None, out, st)
    assert rc == -2                                  # FK_ERR_UNSUPPORTED
    assert b"static scratch" in lib.fk_last_error()
