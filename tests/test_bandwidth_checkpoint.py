"""Host logic of the leave-one-out bandwidth search: checkpoint and resume
(no GPU: the likelihood call is replaced by a deterministic stand-in)."""
import numpy as np
import pytest


def _fake_loo(x, h, w=None, path="mixed", grad=True):
    import torch
    h = np.asarray(h, dtype=np.float64)
    # a smooth concave function of log h with its maximum at h = 0.2
    L = -float(np.sum(np.log(h / 0.2) ** 2))
    g = -2.0 * np.log(h / 0.2) / h
    return torch.tensor([L], dtype=torch.float64), torch.as_tensor(g)


@pytest.fixture
def fk(monkeypatch):
    import paper_2005_03246_gb300 as fk
    monkeypatch.setattr(fk, "loo_laplace", _fake_loo)
    monkeypatch.setattr(fk, "_prep_points", lambda x, d=None: x)
    return fk


def test_resume_equals_uninterrupted(fk, tmp_path):
    import torch
    x = torch.zeros((10, 3), dtype=torch.float64)
    full = fk.select_bandwidth_loo(x, h0=0.5, steps=6, lr=0.3)
    ck = str(tmp_path / "bw.json")
    first = fk.select_bandwidth_loo(x, h0=0.5, steps=3, lr=0.3, checkpoint=ck)
    assert len(first) == 3
    resumed = fk.select_bandwidth_loo(x, h0=0.5, steps=6, lr=0.3, checkpoint=ck)
    assert len(resumed) == 6
    for (h1, l1, g1), (h2, l2, g2) in zip(full, resumed):
        assert np.array_equal(h1, h2) and l1 == l2 and np.array_equal(g1, g2)
    # a finished search resumes to the same answer without further steps
    again = fk.select_bandwidth_loo(x, h0=0.5, steps=6, lr=0.3, checkpoint=ck)
    assert [a[1] for a in again] == [a[1] for a in full]


def test_checkpoint_of_another_search_is_refused(fk, tmp_path):
    import torch
    x = torch.zeros((10, 2), dtype=torch.float64)
    ck = str(tmp_path / "bw.json")
    fk.select_bandwidth_loo(x, steps=2, lr=0.3, checkpoint=ck)
    with pytest.raises(ValueError):
        fk.select_bandwidth_loo(x, steps=4, lr=0.5, checkpoint=ck)
    with pytest.raises(ValueError):
        fk.select_bandwidth_loo(torch.zeros((10, 3), dtype=torch.float64), steps=4, lr=0.3, checkpoint=ck)
