"""GPU parity of the adjoint of the Laplacian KDE and of the leave-one-out
likelihood gradient (exact derivatives of eq. Laplacian kde nD) against the
oracle's brute-force gradients and against central finite differences.

Gradient vectors are signed sums, so the error is measured against the largest
reference entry: max|g - o| <= tol * max|o|, with tol 1e-10 on the FP64 path
and 1e-5 on the mixed path (brute force), and 1e-4 against finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2005_03246_gb300 import datagen

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-5}


def _fk():
    import paper_2005_03246_gb300 as fk
    return fk


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _err(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


def _pts(n, d, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((n, d)) * 0.8).astype(np.float32)


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_backward_explicit_targets(path, d):
    x = _pts(2500, d, 10 + d)
    z = _pts(600, d, 20 + d)
    w = np.random.default_rng(d).random(2500).astype(np.float32) + 0.2
    g = np.random.default_rng(30 + d).standard_normal(600)
    h = np.linspace(0.3, 0.6, d)
    gw, gz, gh = _fk().kde_laplace_backward(_t(x), h, _t(g), w=_t(w), z=_t(z), path=path)
    rw, rz, rh = oracle.kde_grad(x, h, g, w=w, z=z)
    assert _err(gw.cpu().numpy(), rw) <= TOL[path]
    assert _err(gz.cpu().numpy(), rz) <= TOL[path]
    assert _err(gh.cpu().numpy(), rh) <= TOL[path]


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("loo", [False, True])
def test_backward_sample_points(path, loo):
    x = _pts(3000, 3, 5)
    g = np.random.default_rng(6).standard_normal(3000)
    h = [0.4, 0.5, 0.45]
    gw, gz, gh = _fk().kde_laplace_backward(_t(x), h, _t(g), loo=loo, path=path)
    assert gz is None
    rw, _, rh = oracle.kde_grad(x, h, g, loo=loo)
    assert _err(gw.cpu().numpy(), rw) <= TOL[path]
    assert _err(gh.cpu().numpy(), rh) <= TOL[path]


def test_backward_matches_finite_differences_of_the_gpu_forward():
    """Central differences of the FP64-path GPU forward in z and h (targets kept
    away from source coordinates, so no kink is crossed)."""
    import torch
    fk = _fk()
    r = np.random.default_rng(7)
    x = r.standard_normal((800, 2))
    z = r.standard_normal((50, 2)) + 0.013
    h = np.array([0.35, 0.5])
    g = r.standard_normal(50)
    _, gz, gh = fk.kde_laplace_backward(_t(x), h, _t(g), z=_t(z), path="fp64")

    def L(zz, hh):
        return float(np.dot(g, fk.kde_laplace(_t(x), hh, z=_t(zz), path="fp64").cpu().numpy()))

    fz = np.zeros_like(z)
    for j in range(0, 50, 7):
        for k in range(2):
            zp, zm = z.copy(), z.copy()
            zp[j, k] += 1e-6
            zm[j, k] -= 1e-6
            fz[j, k] = (L(zp, h) - L(zm, h)) / 2e-6
            assert abs(fz[j, k] - gz.cpu().numpy()[j, k]) <= 1e-4 * max(abs(fz[j, k]), 1e-3)
    for k in range(2):
        hp, hm = h.copy(), h.copy()
        hp[k] += 1e-6
        hm[k] -= 1e-6
        fh = (L(z, hp) - L(z, hm)) / 2e-6
        assert abs(fh - gh.cpu().numpy()[k]) <= 1e-4 * abs(fh)


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_autograd_function_matches_backward(path):
    """torch.autograd through fk.kde: FP64 tensors, so the gradients are held
    to the adjoint's own tolerance against the oracle."""
    import torch
    fk = _fk()
    x = _pts(1500, 2, 8).astype(np.float64)
    z = _t(_pts(300, 2, 9).astype(np.float64)).requires_grad_(True)
    w = _t(np.random.default_rng(1).random(1500)).requires_grad_(True)
    h = torch.tensor([0.4, 0.7], dtype=torch.float64, requires_grad=True)
    f = fk.kde(_t(x), h, w=w, z=z, path=path)
    loss = (f * torch.linspace(-1, 1, 300, device="cuda:0", dtype=torch.float64)).sum()
    loss.backward()
    g = np.linspace(-1, 1, 300)
    rw, rz, rh = oracle.kde_grad(x, [0.4, 0.7], g, w=w.detach().cpu().numpy(), z=z.detach().cpu().numpy())
    assert _err(w.grad.cpu().numpy(), rw) <= TOL[path]
    assert _err(z.grad.cpu().numpy(), rz) <= TOL[path]
    assert _err(h.grad.cpu().numpy(), rh) <= TOL[path]


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_loo_likelihood_and_gradient(path):
    x = datagen.copula_exp4(n=3000)["x"]
    h = np.array([0.5, 0.45, 0.55, 0.5])
    L, gh = _fk().loo_laplace(_t(x), h, path=path)
    rL, rg = oracle.loo_loglik(x, h)
    assert abs(float(L.item()) - rL) <= TOL[path] * max(1.0, abs(rL))
    assert _err(gh.cpu().numpy(), rg) <= TOL[path]


def test_bandwidth_selection_steps_match_oracle_gradients():
    """20 ascent steps on log h from h=0.5 on a 2e4-point subsample of the d=4
    copula workload (its first 20000 points): at every visited h the
    likelihood and its gradient match the oracle's, and the ascent step taken
    with the oracle's gradient, u <- u + 0.5 sum_k h_k dL/dh_k on u = log h,
    leads to the next visited h."""
    x = datagen.copula_exp4()["x"][:20000]
    hist = _fk().select_bandwidth_loo(_t(x), h0=0.5, steps=20, lr=0.5, path="fp64")
    assert len(hist) == 20
    assert np.array_equal(hist[0][0], np.full(4, 0.5))
    for k, (h, L, g) in enumerate(hist):
        rL, rg = oracle.loo_loglik(x, h)
        assert abs(L - rL) <= TOL["fp64"] * max(1.0, abs(rL))
        assert _err(g, rg) <= TOL["fp64"]
        if k + 1 < len(hist):
            nxt = np.exp(np.log(h) + 0.5 * float(np.sum(h * rg)))
            assert np.max(np.abs(nxt - hist[k + 1][0])) <= 1e-12 * np.max(nxt)
    assert hist[-1][1] >= hist[0][1]           # ascent increased the likelihood


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_backward_unweighted_explicit_targets_d3(path):
    """d=3, N=70000 sources, 300 explicit targets, no weights (the signed-sum
    adjoint on the mixed path): every output against the oracle.  At this
    shape the transposed grad-w pass is the largest part of the plan."""
    r = np.random.default_rng(71)
    x = _pts(70000, 3, 72)
    z = (x[r.choice(70000, 300, replace=False)] + r.normal(0.0, 0.05, (300, 3))).astype(np.float32)
    g = r.standard_normal(300)
    h = np.array([0.1, 0.12, 0.15])
    gw, gz, gh = _fk().kde_laplace_backward(_t(x), h, _t(g), z=_t(z), path=path)
    rw, rz, rh = oracle.kde_grad(x, h, g, z=z)
    assert _err(gw.cpu().numpy(), rw) <= TOL[path]
    assert _err(gz.cpu().numpy(), rz) <= TOL[path]
    assert _err(gh.cpu().numpy(), rh) <= TOL[path]


@pytest.mark.parametrize("path", ["mixed", "fp64"])
@pytest.mark.parametrize("d", [2, 4])
def test_loo_likelihood_with_isolated_points(path, d):
    """Isolated points whose leave-one-out density lies below the FP32 range
    (nearest neighbour 75 to 440 bandwidths away): the likelihood and its
    gradient stay finite and match the oracle on both paths."""
    r = np.random.default_rng(120 + d)
    x = r.standard_normal((3000, d))
    far = np.array([[8.0 + 3.0 * k] * d for k in range(4)])       # 3 apart per axis from each other
    near = np.array([[-6.0] * d, [-2.25] + [-6.0] * (d - 1)])      # 75 bandwidths apart
    x = np.concatenate([x, far, near]).astype(np.float32)
    h = np.full(d, 0.05)
    L, gh = _fk().loo_laplace(_t(x), h, path=path)
    rL, rg = oracle.loo_loglik(x, h)
    assert np.isfinite(rL) and np.isfinite(float(L.item()))
    assert abs(float(L.item()) - rL) <= TOL[path] * max(1.0, abs(rL))
    assert _err(gh.cpu().numpy(), rg) <= TOL[path]
