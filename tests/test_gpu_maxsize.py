"""The largest inputs the sample-point path accepts (its item index has 26
bits): orthant counts at the sample points for N = 2^25 - 1 points (2^26 - 2
items in the source/target-copy layout, the one the fallback may need), and
the refusal one point later.  Sampled targets are checked against the oracle
(extreme points included); every target's counts must add up to N."""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu

N_MAX = (1 << 25) - 1


def test_counts_at_the_item_limit():
    import torch
    import paper_2005_03246_gb300 as fk
    r = np.random.default_rng(77)
    # FP32 uniform coordinates: ~2^24 distinct values per axis, so ties are everywhere
    x = r.random((N_MAX, 2), dtype=np.float32)
    xt = torch.as_tensor(x, device="cuda:0")
    got = fk.ecdf_points(xt)
    assert bool((got.sum(dim=0) == N_MAX).all())
    ext = [int(i) for k in range(2) for i in (x[:, k].argmin(), x[:, k].argmax())]
    idx = datagen.sample_targets(N_MAX, 96, seed=3, include=ext)
    ref = oracle.orthant_sums(x, z=x[idx])
    assert np.array_equal(got[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy(), ref)
    del got, xt
    torch.cuda.empty_cache()


def test_one_point_beyond_the_item_limit_is_refused():
    import torch
    import paper_2005_03246_gb300 as fk
    x = torch.zeros((N_MAX + 1, 2), dtype=torch.float32, device="cuda:0")
    with pytest.raises(fk.FastEcdfError):
        fk.ecdf_points(x)
