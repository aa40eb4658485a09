"""fk_ecdf_grid_counts_noalloc: grid orthant counts with no device allocation.

Callers that may not allocate device memory while they run (allocation-free
real-time loops, or applications that own the whole device memory budget) use
this entry point; it keeps its scratch in a fixed array inside the library.
These checks call it through the C ABI with device buffers and compare it with
the allocating fk_ecdf_grid on two calls in a row (the second call must not see
the first call's histogram), and check that an oversized grid is refused.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu

P = ctypes.c_void_p


def _alloc_call(lib, x, z, M, out, st):
    from paper_2005_03246_gb300 import _lib
    code = _lib.FK_F64 if x.dtype.is_floating_point and x.element_size() == 8 else _lib.FK_F32
    rc = lib.fk_ecdf_grid(P(x.data_ptr()), code, x.shape[0], x.shape[1], None, P(z.data_ptr()),
                          M.ctypes.data_as(P), None, P(out.data_ptr()), 0, None, 0, st)
    _lib.check(rc, "fk_ecdf_grid")


def _noalloc_call(lib, x, z, M, out, st):
    from paper_2005_03246_gb300 import _lib
    code = _lib.FK_F64 if x.element_size() == 8 else _lib.FK_F32
    return lib.fk_ecdf_grid_counts_noalloc(P(x.data_ptr()), code, x.shape[0], x.shape[1], P(z.data_ptr()),
                                           M.ctypes.data_as(P), None, P(out.data_ptr()), st)


def _case(seed, n, axes, dtype):
    import torch
    r = np.random.default_rng(seed)
    d = len(axes)
    xn = np.round(r.standard_normal((n, d)) * 4) / 4
    x = torch.as_tensor(xn.astype(dtype), device="cuda:0")
    z = torch.as_tensor(np.concatenate(axes).astype(np.float64), device="cuda:0")
    M = np.array([len(a) for a in axes], dtype=np.int64)
    shape = (1 << d, int(np.prod(M)))
    return x, z, M, shape


def test_noalloc_matches_allocating_call_two_calls_in_a_row():
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    small = datagen.ecdf_small()
    cases = [
        (torch.as_tensor(small["x"], device="cuda:0"),
         torch.as_tensor(np.concatenate(small["grid"]), device="cuda:0"),
         np.array([len(a) for a in small["grid"]], dtype=np.int64), (4, 128 * 128)),
        _case(7, 20000, [np.linspace(-2, 2, 40), np.linspace(-3, 1, 33), np.linspace(-1, 2, 27)], np.float32),
    ]
    for x, z, M, shape in cases:
        ref = torch.empty(shape, dtype=torch.int64, device="cuda:0")
        _alloc_call(lib, x, z, M, ref, st)
        got = torch.full(shape, -1, dtype=torch.int64, device="cuda:0")
        rc = _noalloc_call(lib, x, z, M, got, st)
        _lib.check(rc, "fk_ecdf_grid_counts_noalloc")
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_refuses_grid_beyond_its_scratch():
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    st = P(torch.cuda.current_stream().cuda_stream)
    axes = [np.linspace(0, 1, 256)] * 3            # needs far more than 16 MiB of scratch
    x, z, M, shape = _case(3, 100, axes, np.float32)
    out = torch.empty((8, 1), dtype=torch.int64, device="cuda:0")   # never written
    rc = _noalloc_call(lib, x, z, M, out, st)
    assert rc == -2                                  # FK_ERR_UNSUPPORTED
    assert b"static scratch" in lib.fk_last_error()
