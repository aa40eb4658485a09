"""Bounded device waits through the C ABI.  The rank transform's radix sort
(Sec. 2.2) finds the start of each tile's digit runs by a decoupled look-back
in which a tile waits for counts published by the tiles before it; each wait
gives up after a fixed number of polls and records FK_ERR_TIMEOUT in the
device error word instead of spinning on.  fk_debug_lookback_timeout runs one
digit pass whose first tile never publishes, so the waits must run out; the
call returns the timeout, clears it, and the device stays usable: a following
sort-based call on fresh data gives exact counts and no error."""
import ctypes
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
P = ctypes.c_void_p
FK_ERR_TIMEOUT = -6


def _st():
    import torch
    return P(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("n", [2 * 4096, 3 * 4096 + 17, 64 * 4096])
def test_lookback_wait_runs_out_and_reports_timeout(n):
    import torch
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    torch.zeros(1, device="cuda:0")
    assert lib.fk_device_status(_st()) == 0
    t0 = time.perf_counter()
    rc = lib.fk_debug_lookback_timeout(n, _st())
    dt = time.perf_counter() - t0
    assert rc == FK_ERR_TIMEOUT, (_lib.STATUS.get(rc, rc), lib.fk_last_error())
    assert b"bounded device wait" in lib.fk_last_error()
    assert dt < 30.0                                  # the bound is a fraction of a second per wait
    assert lib.fk_device_status(_st()) == 0          # read once, then cleared
    # the context is intact: the rank transform (the same sort, waits satisfied) gives exact counts
    x = np.random.default_rng(n).standard_normal((20000, 3)).astype(np.float32)
    xt = torch.as_tensor(x, device="cuda:0")
    out = torch.empty((8, x.shape[0]), dtype=torch.int64, device="cuda:0")
    rc = lib.fk_ecdf_points(P(xt.data_ptr()), _lib.FK_F32, x.shape[0], 3, None, None, 0, None, P(out.data_ptr()), 0,
                            None, 0, _st())
    assert rc == 0
    assert lib.fk_device_status(_st()) == 0
    idx = np.random.default_rng(1).choice(x.shape[0], 64, replace=False)
    ref = oracle.orthant_sums(x, z=x[idx])
    assert np.array_equal(out.cpu().numpy()[:, idx], ref)
