"""The bench's sampled accuracy report (host logic, no GPU): the step's outputs
are gathered at the oracle's sample and compared with it.  Here the "GPU
outputs" are the oracle's own full outputs as CPU tensors, in the layouts the
library returns, so the gather must line up with the sample exactly; a planted
layout mistake (transposed grid axes, a perturbed count or density) must show."""
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2005_03246_gb300 import datagen  # noqa: E402


@pytest.fixture(scope="module")
def case():
    oracle.build()
    x = datagen.ecdf_gauss3(n=3000)["x"]
    grid = [np.linspace(-2.5, 2.5, 7), np.linspace(-2.0, 2.0, 9), np.linspace(-3.0, 3.0, 11)]
    _, ref = bench._oracle_sample(x, grid, 40, seed=1, keep=True)
    g = torch.as_tensor(oracle.ecdf_grid(x, grid))            # [8, 7, 9, 11]
    p = torch.as_tensor(oracle.orthant_sums(x))               # [8, N]
    f = torch.as_tensor(oracle.kde_laplace(x, bench.H))       # [N]
    return x, grid, ref, g, p, f


def test_sample_shapes(case):
    x, grid, ref, g, p, f = case
    assert ref["points"].shape == (8, 40) and ref["kde"].shape == (40,)
    gcount = max(1, round(40 * 7 * 9 * 11 / 3000))
    assert ref["gi"].shape == (gcount, 3) and ref["grid"].shape == (8, gcount)
    assert all(ref["gi"][:, k].max() < len(grid[k]) for k in range(3))


def test_exact_outputs_agree(case):
    _, _, ref, g, p, f = case
    acc = bench._accuracy(ref, bench._gather(g, p, f, ref))
    assert acc["points_count_mismatches"] == 0 and acc["grid_count_mismatches"] == 0
    assert acc["kde_mixed_max_rel_err"] < 1e-13
    assert acc["sample_points"] == 40


def test_planted_mistakes_show(case):
    _, _, ref, g, p, f = case
    # grid axes in the wrong order (a transposed output layout)
    gt = g.permute(0, 1, 3, 2).contiguous().reshape(8, 7, 9, 11)
    assert bench._accuracy(ref, bench._gather(gt, p, f, ref))["grid_count_mismatches"] > 0
    # orthant rows swapped
    assert bench._accuracy(ref, bench._gather(g, p.flip(0), f, ref))["points_count_mismatches"] > 0
    # one density off by 1e-4 relative
    f2 = f.clone()
    f2[int(ref["idx"][3])] *= 1 + 1e-4
    assert bench._accuracy(ref, bench._gather(g, p, f2, ref))["kde_mixed_max_rel_err"] == pytest.approx(1e-4, rel=1e-6)


def test_check_failure_is_reported_not_raised(case):
    x, grid, _, g, p, f = case
    out = bench._cpu_baseline(x, grid, target_s=0.05, gpu_out=(g, p[:, :5], f))
    assert out["accuracy"]["error"].startswith("ValueError") and out["value"] > 0
    out = bench._cpu_baseline(x, grid, target_s=0.05, gpu_out=(g[:, :, :, :3], p, f))
    assert out["accuracy"]["error"].startswith("ValueError")
