"""GPU parity of the batched path: many datasets of uneven N and d in one call
(fk_batched) against the single-dataset calls and the oracle, also when the
call is captured in a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu


def _fk():
    import paper_2005_03246_gb300 as fk
    return fk


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _rel_kde(got, ref):
    big = np.abs(ref) >= 1e-6 * np.abs(ref).max()
    return np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big]))


def _sets(count, seed, nmax=3000):
    r = np.random.default_rng(seed)
    xs, ys = [], []
    for b in range(count):
        d = int(r.integers(1, 5))
        n = int(r.integers(0, nmax)) if b % 7 else int(r.integers(1, 4))
        x = r.random((n, d))
        m = r.random((n, d)) < 0.3
        x[m] = np.round(x[m] * 16) / 16
        xs.append(x.astype(np.float32))
        ys.append(r.standard_normal(n).astype(np.float32))
    return xs, ys


@pytest.mark.parametrize("graph", [False, True])
def test_batched_matches_single_calls_and_oracle(graph):
    fk = _fk()
    xs, ys = _sets(40, 1)
    bt = fk.Batched([_t(x) for x in xs], [_t(y) for y in ys], h=0.1, path="mixed", graph=graph)
    for rep in range(2):                       # replays reuse the same buffers
        ecdf, kde = bt.run()
        for b, (x, y) in enumerate(zip(xs, ys)):
            e = ecdf[b].cpu().numpy()
            if x.shape[0] == 0:
                assert e.size == 0 and kde[b].numel() == 0
                continue
            assert np.array_equal(e, fk.ecdf_points(_t(x)).cpu().numpy()), b
            if b % 5 == 0:
                assert np.array_equal(e, oracle.orthant_sums(x)), b
            f = kde[b].cpu().numpy()
            ref = oracle.kde_laplace(x, 0.1, w=y) if b % 5 == 0 else None
            single = fk.kde_laplace(_t(x), 0.1, w=_t(y), path="mixed").cpu().numpy()
            assert np.max(np.abs(f - single)) <= 1e-5 * np.abs(single).max(), b
            if ref is not None:
                # signed weights: compare against the density scale
                assert np.max(np.abs(f - ref)) <= 1e-5 * oracle.kde_laplace(x, 0.1, w=np.abs(y)).max(), b


def test_batched_fp64_path_kde():
    fk = _fk()
    xs, _ = _sets(12, 2, nmax=2000)
    bt = fk.Batched([_t(x) for x in xs], None, h=0.2, ecdf=False, path="fp64", graph=False)
    _, kde = bt.run()
    for b, x in enumerate(xs):
        if x.shape[0] < 2:
            continue
        assert _rel_kde(kde[b].cpu().numpy(), oracle.kde_laplace(x, 0.2)) <= 1e-12, b


def test_batched_config_512_datasets():
    """512 datasets, N log-uniform in [1e3, 1e5], d alternating 2/3 (graph-captured):
    the orthants partition every dataset; sampled datasets and targets match the oracle."""
    fk = _fk()
    sets = datagen.batched()
    xs = [_t(s["x"]) for s in sets]
    ys = [_t(s["y"]) for s in sets]
    bt = fk.Batched(xs, ys, h=0.1, path="mixed", graph=True)
    ecdf, kde = bt.run()
    r = np.random.default_rng(3)
    for b in range(len(sets)):
        e = ecdf[b]
        assert bool((e.sum(dim=0) == sets[b]["n"]).all())
    for b in r.choice(len(sets), size=6, replace=False):
        x, y = sets[b]["x"], sets[b]["y"]
        idx = datagen.sample_targets(x.shape[0], 64, seed=int(b))
        assert np.array_equal(ecdf[b].cpu().numpy()[:, idx], oracle.orthant_sums(x, z=x[idx]))
        ref = oracle.kde_laplace(x, 0.1, w=y, z=x[idx])
        scale = oracle.kde_laplace(x, 0.1, w=np.abs(y), z=x[idx]).max()
        assert np.max(np.abs(kde[b].cpu().numpy()[idx] - ref)) <= 1e-5 * scale


CONFIGS = [
    {"streams": 2, "coarsen": 1, "kernel_tile": 1, "count_tile": 1},
    {"streams": 4, "coarsen": 2, "kernel_tile": 0, "count_tile": 2},
    {"streams": 8, "coarsen": 0, "kernel_tile": 1, "count_tile": 0},
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_batched_configurations_agree(cfg):
    """Every launch configuration (streams, group coarsening, tile sizes) gives
    the default configuration's counts exactly and its KDE within tolerance,
    eagerly and replayed from a CUDA graph."""
    fk = _fk()
    xs, ys = _sets(30, 5, nmax=6000)
    tx, ty = [_t(x) for x in xs], [_t(y) for y in ys]
    e0, k0 = fk.Batched(tx, ty, h=0.1, graph=False).run()
    # signed weights: differences are measured on the density of |y|
    scales = [oracle.kde_laplace(x, 0.1, w=np.abs(y)).max() if x.shape[0] else 0.0 for x, y in zip(xs, ys)]
    for graph in (False, True):
        bt = fk.Batched(tx, ty, h=0.1, graph=graph, config=cfg)
        assert bt.config == cfg
        for rep in range(2):
            e1, k1 = bt.run()
            for b in range(len(xs)):
                assert np.array_equal(e1[b].cpu().numpy(), e0[b].cpu().numpy()), (b, graph)
                if xs[b].shape[0] == 0:
                    continue
                a, r = k1[b].cpu().numpy(), k0[b].cpu().numpy()
                assert np.max(np.abs(a - r)) <= 2e-5 * scales[b], (b, graph)


def test_batched_autotune_512_datasets():
    """The autotuner picks a configuration by measurement on the 512-dataset
    workload; the tuned, graph-captured call matches the default one."""
    fk = _fk()
    sets = datagen.batched()
    xs = [_t(s["x"]) for s in sets]
    ys = [_t(s["y"]) for s in sets]
    e0, k0 = fk.Batched(xs, ys, h=0.1, graph=False).run()
    bt = fk.Batched(xs, ys, h=0.1, graph=True, config="tune")
    c = bt.config
    assert 1 <= c["streams"] <= 8 and 0 <= c["coarsen"] <= 2
    assert c["kernel_tile"] in (0, 1) and c["count_tile"] in (0, 1, 2)
    assert bt.tune_ms is not None and bt.tune_ms > 0
    e1, k1 = bt.run()
    for b in range(0, len(sets), 7):
        assert np.array_equal(e1[b].cpu().numpy(), e0[b].cpu().numpy()), b
        a, r = k1[b].cpu().numpy(), k0[b].cpu().numpy()
        assert np.max(np.abs(a - r)) <= 2e-5 * np.abs(r).max(), b


def test_batched_tune_cache(tmp_path):
    """A second tuned construction with the same cache file skips the tuning,
    takes the stored configuration, and gives the same results."""
    fk = _fk()
    xs, ys = _sets(24, 9, nmax=4000)
    xs, ys = [_t(x) for x in xs], [_t(y) for y in ys]
    path = str(tmp_path / "tune.json")
    b1 = fk.Batched(xs, ys, h=0.1, graph=False, config="tune", tune_cache=path)
    b2 = fk.Batched(xs, ys, h=0.1, graph=False, config="tune", tune_cache=path)
    assert not b1.tune_cached and b2.tune_cached
    assert b2.config == b1.config and b2.tune_ms == b1.tune_ms
    e1, k1 = b1.run()
    e2, k2 = b2.run()
    for b in range(len(xs)):
        assert np.array_equal(e1[b].cpu().numpy(), e2[b].cpu().numpy()), b
        a, r = k1[b].cpu().numpy(), k2[b].cpu().numpy()
        if r.size:
            assert np.max(np.abs(a - r)) <= 2e-5 * np.abs(r).max(), b
