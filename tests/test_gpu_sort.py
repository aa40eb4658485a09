"""The rank transform (the per-axis sort permutations of Sec. 2.2, Algorithm 2)
under key patterns that stress its one-sweep radix sort: every key in one
digit bin (a constant axis), keys already in order and in reverse order,
signed zeros and negative values, FP64 keys (eight digit passes), and sizes
at and around multiples of the 4096-key sort tile, so that the decoupled
look-back runs over one, two and several tiles.  The counts at the sample
points are exact integers, so every case is compared bit for bit with the
oracle at sampled targets (the first and last points included), and the
orthants must partition the sources."""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu

TILE = 4096


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _points(pattern, n, dtype, seed):
    r = np.random.default_rng(seed)
    x = r.standard_normal((n, 2))
    if pattern == "constant":
        x[:, 0] = 0.5
    elif pattern == "sorted":
        x[:, 0] = np.sort(x[:, 0])
    elif pattern == "reversed":
        x[:, 0] = np.sort(x[:, 0])[::-1]
    elif pattern == "signed_zeros":
        z = r.random(n) < 0.3
        x[z, 0] = np.where(r.random(int(z.sum())) < 0.5, -0.0, 0.0)
        x[:, 1] = -np.abs(x[:, 1])
    return x.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [TILE, TILE + 1, 3 * TILE - 1, 3 * TILE, 5 * TILE + 123])
@pytest.mark.parametrize("pattern", ["constant", "sorted", "reversed", "signed_zeros"])
def test_rank_transform_key_patterns(pattern, n, dtype):
    from paper_2005_03246_gb300 import ecdf_points
    x = _points(pattern, n, dtype, seed=n + len(pattern))
    got = ecdf_points(_t(x)).cpu().numpy()
    idx = datagen.sample_targets(n, 200, seed=11, include=(0, 1, n - 2, n - 1))
    assert np.array_equal(got[:, idx], oracle.orthant_sums(x, z=x[idx]))
    assert np.all(got.sum(axis=0) == n)
