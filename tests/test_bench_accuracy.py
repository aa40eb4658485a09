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


def _extra_samples(x, err=0.0, count_err=False):
    """Samples of the other workloads in the layout bench._extras builds, with
    "GPU values" taken from the oracle (optionally perturbed)."""
    r = np.random.default_rng(3)
    sets = [dict(x=r.random((300 + 50 * k, 2 + k % 2)).astype(np.float32),
                 y=r.standard_normal(300 + 50 * k).astype(np.float32)) for k in range(4)]
    bat = []
    for s in sets:
        e = oracle.orthant_sums(s["x"])
        if count_err:
            e = e.copy()
            e[0, 0] += 1
        bat.append((s["x"], s["y"], e, oracle.kde_laplace(s["x"], bench.H, w=s["y"]) * (1 + err)))
    idx = np.array([0, 5, 17, 40])
    xs = x[:, :2].copy()
    ys = np.sin(xs.sum(axis=1))
    vals = {}
    for h in (0.05, 0.1, 0.3):
        for path in ("mixed", "fp64"):
            vals[(h, path)] = (oracle.kde_laplace(xs, h, z=xs[idx]) * (1 + err),
                               oracle.kreg_laplace(xs, ys, h, z=xs[idx]) + err)
    z = xs[[1, 2, 3]] + 0.01
    g = np.array([0.5, -1.0, 2.0])
    hv = np.array([0.1, 0.12])
    rw, rz, rh = oracle.kde_grad(xs, hv, g, z=z)
    sw = np.array([0, 3, 9])
    adj = {"z": z, "g": g, "h": hv, "mixed": (sw, rw[sw], rz, rh * (1 + err)), "fp64": (sw, rw[sw], rz, rh)}
    y3 = r.random(x.shape[0])
    c2 = oracle.orthant_sums(x, y=y3, z=x[idx])
    c5h = np.full(3, 0.5)
    c5 = oracle.kde_at_points(x, c5h, idx, loo=True)
    return {"batched_mixed": bat, "batched_fp64": bat,
            "backward_d3": {"idx": idx, "grad_w": oracle.kde_laplace(x, bench.H, z=x[idx]) * (1 + err)},
            "c3": {"x": xs, "y": ys, "idx": idx, "values": vals, "adjoint": adj},
            "c2w": {"y": y3, "idx": idx, "mixed": c2 * (1 + err), "fp64": c2},
            "c5": {"x": x, "idx": idx, "h": c5h, "mixed": c5 * (1 + err), "fp64": c5}}


def test_other_workloads_report_the_oracle_error(case):
    """Exact values report zero error everywhere; a relative perturbation of
    1e-4 shows in every floating-point entry it touches; a planted count error
    shows as a mismatch."""
    x = case[0][:400]
    a = bench._accuracy_extras(_extra_samples(x), x)
    assert a["batched_mixed"]["count_mismatches"] == 0 and a["batched_mixed"]["kde_err_rel_to_abs_weights"] < 1e-12
    assert a["kde_backward_d3_grad_w"]["max_rel_err"] < 1e-14
    assert all(v["kde_max_rel_err"] < 1e-14 and v["nw_c9"] < 1e-14
               for k, v in a["c3_copula_d2"].items() if k.startswith("h"))
    assert a["c3_copula_d2"]["adjoint_mixed"]["grad_h_err_rel_max"] < 1e-14
    assert a["c2_weighted_d3"]["mixed_max_rel_err"] < 1e-14 and a["c5_loo_d4"]["mixed_loo_density_max_rel_err"] < 1e-14
    b = bench._accuracy_extras(_extra_samples(x, err=1e-4, count_err=True), x)
    assert b["batched_mixed"]["count_mismatches"] == 4
    assert 0.5e-4 < b["batched_mixed"]["kde_err_rel_to_abs_weights"] <= 1.01e-4
    assert abs(b["kde_backward_d3_grad_w"]["max_rel_err"] - 1e-4) < 1e-9
    assert abs(b["c3_copula_d2"]["h0.1_mixed"]["kde_max_rel_err"] - 1e-4) < 1e-9
    assert b["c3_copula_d2"]["h0.1_mixed"]["nw_c9"] > 1e-5
    assert abs(b["c3_copula_d2"]["adjoint_mixed"]["grad_h_err_rel_max"] - 1e-4) < 1e-9
    assert b["c3_copula_d2"]["adjoint_fp64"]["grad_h_err_rel_max"] < 1e-14
    assert abs(b["c2_weighted_d3"]["mixed_max_rel_err"] - 1e-4) < 1e-9 and b["c2_weighted_d3"]["fp64_max_rel_err"] < 1e-14
    assert abs(b["c5_loo_d4"]["mixed_loo_density_max_rel_err"] - 1e-4) < 1e-9


def test_fp32_peak_reads_the_device_sm_count():
    t, desc = bench.fp32_peak(148, 2000.0, "test")
    assert abs(t - 148 * 128 * 2.0e9 / 1e12) < 1e-9 and "148 SMs" in desc
