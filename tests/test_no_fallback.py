"""There is no CPU fallback (no GPU needed): the public functions refuse host
tensors instead of computing on the CPU, and a missing library is an error,
not a silent switch to another implementation."""
import numpy as np
import pytest
import torch

import paper_2005_03246_gb300 as fk
from paper_2005_03246_gb300 import _lib

X = torch.rand(50, 2, dtype=torch.float32)
Y = torch.rand(50, dtype=torch.float32)
AXES = [np.linspace(0.0, 1.0, 5)] * 2

CALLS = {
    "ecdf_grid": lambda: fk.ecdf_grid(X, AXES),
    "ecdf_points": lambda: fk.ecdf_points(X),
    "esf_points": lambda: fk.esf_points(X),
    "kde_laplace": lambda: fk.kde_laplace(X, 0.1),
    "kreg_laplace": lambda: fk.kreg_laplace(X, Y, 0.1),
    "kde_grid": lambda: fk.kde_grid(X, 0.1, AXES),
    "kde_uniform": lambda: fk.kde_uniform(X, 0.1),
    "kde_matern32": lambda: fk.kde_matern32(X, 0.1),
    "kde_laplace_hmatrix": lambda: fk.kde_laplace_hmatrix(X, np.eye(2) * 0.01),
    "kreg_loclin": lambda: fk.kreg_loclin(X, Y, 0.1),
    "kde_laplace_backward": lambda: fk.kde_laplace_backward(X, 0.1, torch.ones(50, dtype=torch.float64)),
    "loo_laplace": lambda: fk.loo_laplace(X, 0.1),
    "kde": lambda: fk.kde(X, 0.1),
    "Batched": lambda: fk.Batched([X], [Y]),
}


@pytest.mark.parametrize("name", sorted(CALLS))
def test_host_tensors_are_refused(name):
    with pytest.raises(TypeError, match="CUDA tensor"):
        CALLS[name]()


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libfastecdf.so"))
    from paper_2005_03246_gb300 import build
    monkeypatch.setattr(build, "build", lambda *a, **k: None)     # the build "produces" nothing
    with pytest.raises(OSError):
        _lib.load()
