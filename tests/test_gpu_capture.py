"""CUDA-graph capture of the sample-point counts (Sec. 2.2): a call made on a
capturing stream takes the source/target-copy layout, which needs no host
read-back, so the whole call is captured; replays give the oracle's exact
counts, also with ties and an orthant selection, and with new values written
into the captured input between replays."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _pts(n, d, seed):
    r = np.random.default_rng(seed)
    x = r.standard_normal((n, d))
    m = r.random((n, d)) < 0.3
    x[m] = np.round(x[m] * 4) / 4                 # long tie groups on every axis
    return x.astype(np.float32)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_ecdf_points_counts_captured_and_replayed(d):
    import torch
    import paper_2005_03246_gb300 as fk
    xn = _pts(3000, d, 40 + d)
    x = torch.as_tensor(xn, device="cuda:0")
    fk.ecdf_points(x)                             # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = fk.ecdf_points(x)
        sel = fk.ecdf_points(x, orthants=[0, (1 << d) - 1])
    g.replay()
    torch.cuda.synchronize()
    ref = oracle.orthant_sums(xn)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(sel.cpu().numpy(), ref[[0, (1 << d) - 1]])
    # new data in the same storage, replayed again
    xn2 = _pts(3000, d, 90 + d)
    x.copy_(torch.as_tensor(xn2, device="cuda:0"))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.orthant_sums(xn2))


def test_uncaptured_call_unchanged():
    """Outside capture the one-item layout still runs (same counts)."""
    import torch
    import paper_2005_03246_gb300 as fk
    xn = _pts(2000, 3, 7)
    got = fk.ecdf_points(torch.as_tensor(xn, device="cuda:0")).cpu().numpy()
    assert np.array_equal(got, oracle.orthant_sums(xn))
