"""Argument validation of the C ABI on the host (no GPU): every compute entry
point rejects invalid arguments with the status and message include/fastecdf.h
documents, before any device work, so these calls run on a machine without a
GPU.  Arrays are host memory; each case breaks exactly one argument of an
otherwise valid call."""
import ctypes

import numpy as np
import pytest

from paper_2005_03246_gb300 import _lib

P = ctypes.c_void_p
INVALID, UNSUPPORTED = -1, -2

N, D = 100, 3
X = np.random.default_rng(0).random((N, D)).astype(np.float32)
H = np.full(D, 0.1)
OUT = np.zeros(N)
OUTI = np.zeros((8, N), dtype=np.int64)
M = np.full(D, 4, dtype=np.int64)
Z = np.concatenate([np.linspace(0.0, 1.0, 4)] * D)
G = np.zeros(8 * 64, dtype=np.int64)
F = np.zeros(64)


def p(a):
    return None if a is None else a.ctypes.data_as(P)


def _zbad():
    z = Z.copy()
    z[5] = z[4]                     # axis 1 not strictly increasing
    return z


def _sets(d1=D):
    s = (_lib.Dataset * 2)()
    for k, d in enumerate((D, d1)):
        s[k].x, s[k].N, s[k].d = X.ctypes.data, N, d
    return s


def kde(x=X, xd=_lib.FK_F32, n=N, d=D, z=None, m=0, h=H, flags=0, out=OUT, path=0):
    return _lib.load().fk_kde_laplace(p(x), xd, n, d, None, p(z), m, p(h), flags, p(out), None, path, None, 0, None)


CASES = [
    ("kde dtype", lambda: kde(xd=7), INVALID, "xdtype"),
    ("kde d=0", lambda: kde(d=0), INVALID, "d must be >= 1"),
    ("kde d=7", lambda: kde(d=7), UNSUPPORTED, "d <= 6"),
    ("backward d=5", lambda: _lib.load().fk_kde_laplace_backward(p(X), 0, N // 5, 5, None, None, 0, p(np.full(5, 0.1)),
                                                                 0, p(OUT), p(OUT), None, None, 0, None, 0, None),
     UNSUPPORTED, "d <= 4"),
    ("loo d=5", lambda: _lib.load().fk_loo_laplace(p(X), 0, N // 5, 5, None, p(np.full(5, 0.1)), p(OUT), None, 0,
                                                   None, 0, None), UNSUPPORTED, "d <= 4"),
    ("kde N<0", lambda: kde(n=-1), INVALID, "N must be >= 0"),
    ("kde x NULL", lambda: kde(x=None), INVALID, "x is NULL"),
    ("kde h=0", lambda: kde(h=np.array([0.1, 0.0, 0.1])), INVALID, "h[1] must be finite and > 0"),
    ("kde h nan", lambda: kde(h=np.array([0.1, 0.1, np.nan])), INVALID, "h[2] must be finite and > 0"),
    ("kde h NULL", lambda: kde(h=None), INVALID, "h is NULL"),
    ("kde out NULL", lambda: kde(out=None), INVALID, "out is NULL"),
    ("kde path", lambda: kde(path=5), INVALID, "precision path"),
    ("kde LOO with z", lambda: kde(z=X, m=N, flags=_lib.FK_LOO), INVALID, "FK_LOO needs z == NULL"),
    ("points d=9", lambda: _lib.load().fk_ecdf_points(p(X), 0, N, 9, None, None, 0, None, p(OUTI), 0, None, 0,
                                                      None), UNSUPPORTED, "d <= 8"),
    ("points weighted d=7", lambda: _lib.load().fk_ecdf_points(p(X), 0, 20, 7, p(OUT), None, 0, None, p(OUTI), 0,
                                                               None, 0, None), UNSUPPORTED, "d <= 6"),
    ("points out NULL", lambda: _lib.load().fk_ecdf_points(p(X), 0, N, D, None, None, 0, None, None, 0, None, 0,
                                                           None), INVALID, "out is NULL"),
    ("esf d=9", lambda: _lib.load().fk_esf_points(p(X), 0, N, 9, None, None, 0, p(OUTI), 0, None, 0, None),
     UNSUPPORTED, "d out of range"),
    ("grid axis order", lambda: _lib.load().fk_ecdf_grid(p(X), 0, N, D, None, p(_zbad()), p(M), None, p(G), 0, None,
                                                         0, None), INVALID, "axis 1 not strictly increasing at 1"),
    ("grid M=0", lambda: _lib.load().fk_ecdf_grid(p(X), 0, N, D, None, p(Z), p(np.array([4, 0, 4], dtype=np.int64)),
                                                  None, p(G), 0, None, 0, None), INVALID, "M[1] must be >= 1"),
    ("grid d=9", lambda: _lib.load().fk_ecdf_grid(p(X), 0, N, 9, None, p(Z), p(M), None, p(G), 0, None, 0, None),
     UNSUPPORTED, "d <= 8"),
    ("grid too large", lambda: _lib.load().fk_ecdf_grid(p(X), 0, N, 2, None, p(Z), p(np.array([1 << 21, 1 << 21],
                                                        dtype=np.int64)), None, p(G), 0, None, 0, None),
     UNSUPPORTED, "grid too large"),
    ("noalloc host pointers", lambda: _lib.load().fk_ecdf_grid_counts_noalloc(p(X), 0, N, D, p(Z), p(M), None, p(G),
                                                                               None), INVALID, "device pointers"),
    # cell counts whose int64 product wraps (65536^4 = 2^64, 512^7 = 2^63): refused before any size arithmetic
    ("noalloc cells wrap d=4", lambda: _lib.load().fk_ecdf_grid_counts_noalloc(
        p(X), 0, N, 4, p(Z), p(np.full(4, 65535, dtype=np.int64)), None, p(G), None), UNSUPPORTED, "grid too large"),
    ("noalloc cells wrap d=7", lambda: _lib.load().fk_ecdf_grid_counts_noalloc(
        p(X), 0, N, 7, p(Z), p(np.full(7, 511, dtype=np.int64)), None, p(G), None), UNSUPPORTED, "grid too large"),
    ("noalloc histogram beyond scratch", lambda: _lib.load().fk_ecdf_grid_counts_noalloc(
        p(X), 0, N, 2, p(Z), p(np.array([2048, 2048], dtype=np.int64)), None, p(G), None), UNSUPPORTED,
     "grid too large"),
    ("kde_grid h<0", lambda: _lib.load().fk_kde_grid(p(X), 0, N, D, None, p(Z), p(M), p(np.array([0.1, -1.0, 0.1])),
                                                     p(F), 0, None, 0, None), INVALID, "h[1] must be finite and > 0"),
    ("interp d=9", lambda: _lib.load().fk_grid_interp(p(F), 9, p(Z), p(M), p(X), 0, N, p(OUT), None, 0, None),
     UNSUPPORTED, "d in [1, 8]"),
    ("interp Q<0", lambda: _lib.load().fk_grid_interp(p(F), D, p(Z), p(M), p(X), 0, -1, p(OUT), None, 0, None),
     INVALID, "Q must be >= 0"),
    ("interp f NULL", lambda: _lib.load().fk_grid_interp(None, D, p(Z), p(M), p(X), 0, N, p(OUT), None, 0, None),
     INVALID, "must be given"),
    ("uniform d=9", lambda: _lib.load().fk_kde_uniform(p(X), 0, N, 9, None, None, 0, p(H), 0, p(OUT), 0, None, 0,
                                                       None), UNSUPPORTED, "d <= 8"),
    ("matern d=5", lambda: _lib.load().fk_kde_matern32(p(X), 0, N, 5, None, None, 0, p(H), 0, p(OUT), 0, None, 0,
                                                       None), UNSUPPORTED, "d <= 4"),
    ("loclin mixed path", lambda: _lib.load().fk_kreg_loclin_laplace(p(X), 0, N, D, p(OUT), None, 0, p(H), 0, p(OUT),
                                                                     0, None, 0, None), UNSUPPORTED, "FK_PATH_FP64"),
    ("loclin y NULL", lambda: _lib.load().fk_kreg_loclin_laplace(p(X), 0, N, D, None, None, 0, p(H), 0, p(OUT), 1,
                                                                 None, 0, None), INVALID, "y is NULL"),
    ("hmatrix non-symmetric", lambda: _lib.load().fk_kde_laplace_hmatrix(
        p(X), 0, N, D, None, None, 0, p(np.array([[1.0, 0.5, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])), 0, p(OUT), 0,
        None, 0, None), INVALID, "not symmetric"),
    ("hmatrix indefinite", lambda: _lib.load().fk_hmatrix_factor(p(np.array([[1.0, 2.0], [2.0, 1.0]])), 2,
                                                                  p(np.zeros(4)), p(np.zeros(2))),
     INVALID, "not positive definite"),
    ("loo N=1", lambda: _lib.load().fk_loo_laplace(p(X), 0, 1, D, None, p(H), p(OUT), None, 0, None, 0, None),
     INVALID, "N >= 2"),
    ("kreg y NULL", lambda: _lib.load().fk_kreg_laplace(p(X), 0, N, D, None, None, 0, p(H), 0, p(OUT), 0, None, 0,
                                                        None), INVALID, "y is NULL"),
    ("backward grad_out NULL", lambda: _lib.load().fk_kde_laplace_backward(p(X), 0, N, D, None, None, 0, p(H), 0,
                                                                           None, None, None, None, 0, None, 0, None),
     INVALID, "grad_out is NULL"),
    ("batched d=5", lambda: _lib.load().fk_batched(_sets(5), 2, 0, 3, 0.1, p(OUTI), p(OUT), 0, None, 0, None),
     UNSUPPORTED, "dataset 1: d must be in [1, 4]"),
    ("batched h=0", lambda: _lib.load().fk_batched(_sets(), 2, 0, 3, 0.0, p(OUTI), p(OUT), 0, None, 0, None),
     INVALID, "h must be > 0"),
    ("batched nothing", lambda: _lib.load().fk_batched(_sets(), 2, 0, 0, 0.1, p(OUTI), p(OUT), 0, None, 0, None),
     INVALID, "nothing requested"),
    ("lookback probe n", lambda: _lib.load().fk_debug_lookback_timeout(100, None), INVALID, "probe size"),
    ("batched host data", lambda: _lib.load().fk_batched(_sets(), 2, 0, 3, 0.1, p(OUTI), p(OUT), 0, None, 0, None),
     INVALID, "device"),
]


@pytest.mark.parametrize("name,call,status,msg", CASES, ids=[c[0] for c in CASES])
def test_rejected_on_the_host(name, call, status, msg):
    rc = call()
    err = _lib.load().fk_last_error().decode()
    assert rc == status, (name, _lib.STATUS.get(rc, rc), err)
    assert msg in err, (name, err)


def test_empty_orthant_selection_is_a_no_op():
    """A selection with no orthant has nothing to compute: OK, no device work."""
    mask = np.zeros(1, dtype=np.uint32)
    rc = _lib.load().fk_ecdf_points(p(X), 0, N, D, None, None, 0, p(mask), p(OUTI), 0, None, 0, None)
    assert rc == 0
