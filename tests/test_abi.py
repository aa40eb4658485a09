"""Host-only checks of the C-ABI library: it builds, loads, and exports every
symbol that include/fastecdf.h declares (no compute calls: no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "fastecdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fk_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    names = _declared_symbols()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), "missing export %s" % n
    # and the binding knows a signature for each
    for n in names:
        assert n in _lib.SIGNATURES, "binding has no signature for %s" % n


def test_version_and_error_string():
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    assert b"sm_103a" in lib.fk_version()
    assert isinstance(lib.fk_last_error(), bytes)


def test_workspace_queries_are_host_only():
    import ctypes
    import numpy as np
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    M = np.array([256, 256, 256], dtype=np.int64)
    need = lib.fk_ecdf_grid_workspace(1_000_000, 3, M.ctypes.data_as(ctypes.c_void_p), 0, 0)
    cells = 257 ** 3
    assert need >= cells * 4
    bad = np.array([0, 5], dtype=np.int64)
    assert lib.fk_ecdf_grid_workspace(10, 2, bad.ctypes.data_as(ctypes.c_void_p), 0, 0) == 0


def _dummy_sets(lib_mod, sizes):
    """fk_dataset array with placeholder (never dereferenced) device pointers:
    workspace queries only plan on the host."""
    sets = (lib_mod.Dataset * len(sizes))()
    for b, (n, d) in enumerate(sizes):
        sets[b].x = 0x10000 + 256 * b
        sets[b].y = None
        sets[b].N, sets[b].d = n, d
    return sets


def test_batched_config_default_and_validation():
    import ctypes
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    c = _lib.BatchConfig()
    lib.fk_batched_config_default(ctypes.byref(c))
    assert c.as_dict() == {"streams": 1, "coarsen": 0, "kernel_tile": 0, "count_tile": 0}
    sets = _dummy_sets(_lib, [(1000, 2), (20000, 3), (70000, 2), (5, 1)])
    what = _lib.FK_BATCH_ECDF | _lib.FK_BATCH_KDE
    base = lib.fk_batched_workspace_ex(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED, ctypes.byref(c))
    assert base > 0
    assert base == lib.fk_batched_workspace(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED)
    for bad in ({"streams": 0}, {"streams": 9}, {"coarsen": 3}, {"kernel_tile": 2}, {"count_tile": -1}):
        b = _lib.BatchConfig()
        lib.fk_batched_config_default(ctypes.byref(b))
        for k, v in bad.items():
            setattr(b, k, v)
        assert lib.fk_batched_workspace_ex(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED, ctypes.byref(b)) == 0
    # more streams: one workspace slot per stream, never less than one slot
    c.streams = 4
    four = lib.fk_batched_workspace_ex(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED, ctypes.byref(c))
    assert four >= base
    # the autotuner's workspace covers every candidate configuration
    tune = lib.fk_batched_autotune_workspace(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED)
    for s in (1, 2, 4, 8):
        for co in (0, 1, 2):
            for ct in (0, 1, 2):
                for kt in (0, 1):
                    c.streams, c.coarsen, c.count_tile, c.kernel_tile = s, co, ct, kt
                    assert tune >= lib.fk_batched_workspace_ex(sets, 4, _lib.FK_F32, what, _lib.FK_PATH_MIXED,
                                                               ctypes.byref(c))


def test_sample_point_dimension_limits():
    """Counts at the sample points accept d <= 8; weighted sums, the KDE and
    Nadaraya-Watson d <= 6; the adjoint and the leave-one-out likelihood d <= 4."""
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    for d in (5, 6, 8):
        assert lib.fk_ecdf_points_workspace(1000, d, 0, 1, 0, 0) > 0
    for d in (5, 6):
        assert lib.fk_ecdf_points_workspace(1000, d, 0, 1, 1, 0) > 0
        assert lib.fk_kde_laplace_workspace(1000, d, 0, 1, 0, 0) > 0
        assert lib.fk_kreg_laplace_workspace(1000, d, 0, 1, 0) > 0
        assert lib.fk_kde_laplace_backward_workspace(1000, d, 0, 1, 0) == 0
        assert lib.fk_loo_laplace_workspace(1000, d, 0) == 0
    assert lib.fk_ecdf_points_workspace(1000, 7, 0, 1, 1, 0) == 0
    assert lib.fk_ecdf_points_workspace(1000, 9, 0, 1, 0, 0) == 0
    assert lib.fk_kde_laplace_workspace(1000, 7, 0, 1, 0, 0) == 0


def test_extra_kernel_workspaces_and_limits():
    """Workspace queries of the uniform / Matern-3/2 / matrix-bandwidth / local
    linear calls: sizes are positive where the call is supported, 0 where not
    (local linear only on the FP64 path; uniform counts to d = 8)."""
    from paper_2005_03246_gb300 import _lib
    lib = _lib.load()
    for d in (1, 2, 3, 4):
        for path in (0, 1):
            assert lib.fk_kde_uniform_workspace(5000, d, 0, 1, 1, path) > 0
            assert lib.fk_kde_matern32_workspace(5000, d, 300, 0, 0, path) > 0
            assert lib.fk_kde_laplace_hmatrix_workspace(5000, d, 0, 1, path) > 0
        assert lib.fk_kreg_loclin_laplace_workspace(5000, d, 0, 1, 1) > 0
        assert lib.fk_kreg_loclin_laplace_workspace(5000, d, 0, 1, 0) == 0
    assert lib.fk_kde_uniform_workspace(5000, 8, 0, 1, 0, 0) > 0       # counts: d <= 8
    assert lib.fk_kde_uniform_workspace(5000, 5, 0, 1, 1, 0) == 0      # weighted: d <= 4
    assert lib.fk_kde_matern32_workspace(5000, 5, 0, 1, 0, 0) == 0
    # the uniform kernel's 2^d corner targets count against the item limit
    assert lib.fk_kde_uniform_workspace(300_000, 8, 0, 1, 0, 0) == 0


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_hmatrix_factor_host(d):
    """The host factorisation H = R diag(h)^2 R^T: reconstructs H, R orthonormal,
    eigenvalues equal numpy's; non-symmetric / indefinite H are rejected."""
    import numpy as np
    from paper_2005_03246_gb300 import hmatrix_factor, FastEcdfError
    r = np.random.default_rng(70 + d)
    A = r.standard_normal((d, d))
    H = A @ A.T + 0.1 * np.eye(d)
    R, h = hmatrix_factor(H)
    np.testing.assert_allclose(R @ np.diag(h ** 2) @ R.T, H, rtol=0, atol=1e-13 * np.abs(H).max())
    np.testing.assert_allclose(R.T @ R, np.eye(d), rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.sort(h ** 2), np.linalg.eigvalsh(H), rtol=1e-13)
    if d >= 2:
        bad = H.copy()
        bad[0, 1] += 1.0
        with pytest.raises(FastEcdfError):
            hmatrix_factor(bad)
        with pytest.raises(FastEcdfError):
            hmatrix_factor(-H)
