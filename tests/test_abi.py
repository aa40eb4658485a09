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
