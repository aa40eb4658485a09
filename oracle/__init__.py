"""CPU oracle for the fast multivariate ECDF / Laplacian KDE (arXiv 2005.03246).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2005_03246_gb300``) never imports, links or
executes anything here, and this package never imports the product.

Every function is a brute-force restatement of a definition in the paper:

* ``orthant_sums``  -- eqs. (ECDF), (ESF), (ECDFdelta), Sec. 1, in the reflected
  orthant reading of eq. (Laplacian decomposition nD), Sec. 3.1: orthant bit k
  clear means ``x_k <= z_k``, bit k set means ``x_k > z_k``.
* ``ecdf_grid``     -- the same sums evaluated on a rectilinear grid (Sec. 2.1).
* ``kde_laplace``   -- eq. (Laplacian kde nD), Sec. 3.1, term by term.
* ``kreg_laplace``  -- Nadaraya-Watson ratio with the Laplacian kernel (Sec. 4).
* ``kde_uniform``   -- eq. (uniform kde nD), Sec. 3.2, box counts term by term.
* ``kde_matern32``  -- the additive Matern-3/2 kernel, eq. (Matern32 average),
  Appendix C, term by term.
* ``kde_laplace_hmatrix`` -- eq. (kde nD H), Appendix B: Laplacian KDE with a
  full bandwidth matrix H, H^{-1/2} = diag(1/h) R^T from H = R diag(h)^2 R^T.
* ``kreg_loclin``   -- locally linear kernel regression (the weighted least
  squares fit of an affine function around each target; Sec. 4 names it
  beside Nadaraya-Watson), solved target by target.
* ``kde_grad``      -- exact derivatives of eq. (Laplacian kde nD).
* ``loo_loglik``    -- leave-one-out log-likelihood of the KDE and its h-gradient.
* ``fenwick2d``     -- an independent sort + binary-indexed-tree 2D count.

Parity status of each function (what pins it) is listed in ``tests/test_oracle.py``;
no function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "fk_oracle.c")
_LIB = os.path.join(_BUILD, "libfk_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc + OpenMP into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    lib.fko_orthant_sums.argtypes = [P, I64, I, P, P, I64, P, P, P, I]
    lib.fko_kde.argtypes = [P, I64, I, P, P, I64, P, I, P, P, I]
    lib.fko_kreg.argtypes = [P, I64, I, P, P, I64, P, I, P, I]
    lib.fko_kde_grad.argtypes = [P, I64, I, P, P, I64, P, I, P, P, P, P, I]
    lib.fko_loo_loglik.argtypes = [P, I64, I, P, P, P, P, I]
    lib.fko_kde_at.argtypes = [P, I64, I, P, P, I64, P, I, P, I]
    lib.fko_fenwick2d.argtypes = [P, I64, P, I64, P]
    lib.fko_kde_uniform.argtypes = [P, I64, I, P, P, I64, P, I, P, I]
    lib.fko_kde_matern32.argtypes = [P, I64, I, P, P, I64, P, I, P, I]
    lib.fko_max_threads.argtypes = []
    for f in (lib.fko_orthant_sums, lib.fko_kde, lib.fko_kreg, lib.fko_kde_grad,
              lib.fko_loo_loglik, lib.fko_fenwick2d, lib.fko_max_threads, lib.fko_kde_at,
              lib.fko_kde_uniform, lib.fko_kde_matern32):
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def max_threads() -> int:
    return int(_load().fko_max_threads())


def _f64(a, ncols=None):
    """Widen to a C-contiguous float64 array (exact for float32 input)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if ncols is not None:
        a = a.reshape(-1, ncols)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle call failed with status %d" % rc)


def mask_bits(d, mask):
    """Bitset words (uint32) over the 2^d orthant indices."""
    nw = max(1, (1 << d) // 32)
    bits = np.zeros(nw, dtype=np.uint32)
    if mask is None:
        sel = range(1 << d)
    elif isinstance(mask, (int, np.integer)):
        sel = [o for o in range(1 << d) if (int(mask) >> o) & 1]
    else:
        sel = [int(o) for o in mask]
    for o in sel:
        if not 0 <= o < (1 << d):
            raise ValueError("orthant index out of range")
        bits[o >> 5] |= np.uint32(1 << (o & 31))
    return bits


def orthant_sums(x, y=None, z=None, mask=None, threads=0):
    """Brute-force generalized orthant sums.

    x: [N, d] sources; y: [N] weights or None (exact int64 counts);
    z: [M, d] targets or None (the sources themselves).
    mask: which orthants to return: None (all), an int bitset (bit o = orthant o)
    or an iterable of orthant indices.
    Returns an array [popcount(mask), M] (int64 counts or float64 sums), rows in
    increasing orthant index.  Orthant o has bit k set iff the test on axis k is
    ``x_k > z_k`` (else ``x_k <= z_k``).
    """
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    z = x if z is None else _f64(z, d)
    n, m = x.shape[0], z.shape[0]
    bits = mask_bits(d, mask)
    nout = int(sum(bin(int(w)).count("1") for w in bits))
    if y is None:
        out = np.zeros((nout, m), dtype=np.int64)
        rc = _load().fko_orthant_sums(_ptr(x), n, d, None, _ptr(z), m, _ptr(bits),
                                      _ptr(out), None, int(threads))
    else:
        yy = _f64(y).reshape(-1)
        out = np.zeros((nout, m), dtype=np.float64)
        rc = _load().fko_orthant_sums(_ptr(x), n, d, _ptr(yy), _ptr(z), m, _ptr(bits),
                                      None, _ptr(out), int(threads))
    _check(rc)
    return out


def grid_points(axes):
    """Rectilinear grid of Sec. 2.1 as an [M_1*...*M_d, d] array, last axis fastest."""
    mesh = np.meshgrid(*[np.asarray(a, dtype=np.float64) for a in axes], indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


def ecdf_grid(x, axes, y=None, mask=None, threads=0):
    """Orthant sums at every point of the rectilinear grid ``axes`` (Sec. 2.1).

    Returns [popcount(mask), M_1, ..., M_d]."""
    z = grid_points(axes)
    out = orthant_sums(x, y=y, z=z, mask=mask, threads=threads)
    return out.reshape((out.shape[0],) + tuple(len(a) for a in axes))


def kde_laplace(x, h, w=None, z=None, loo=False, terms=False, threads=0):
    """Laplacian KDE by eq. (Laplacian kde nD).  h: scalar or [d].

    With ``terms=True`` also returns the per-orthant pieces [2^d, M]."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    zz = None if z is None else _f64(z, d)
    m = x.shape[0] if zz is None else zz.shape[0]
    out = np.zeros(m, dtype=np.float64)
    tt = np.zeros((1 << d, m), dtype=np.float64) if terms else None
    ww = None if w is None else _f64(w).reshape(-1)
    rc = _load().fko_kde(_ptr(x), x.shape[0], d, _ptr(ww), _ptr(zz), m, _ptr(hh),
                         int(bool(loo)), _ptr(out), _ptr(tt), int(threads))
    _check(rc)
    return (out, tt) if terms else out


def kde_at_points(x, h, idx, w=None, loo=False, threads=0):
    """eq. (Laplacian kde nD) at the sample points x[idx]; with ``loo`` the
    leave-one-out density f_{-j} (drops exactly source idx[j], normalises by
    N-1)."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    ii = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
    out = np.zeros(ii.shape[0], dtype=np.float64)
    ww = None if w is None else _f64(w).reshape(-1)
    rc = _load().fko_kde_at(_ptr(x), x.shape[0], d, _ptr(ww), _ptr(ii), ii.shape[0], _ptr(hh),
                            int(bool(loo)), _ptr(out), int(threads))
    _check(rc)
    return out


def kreg_laplace(x, y, h, z=None, loo=False, threads=0):
    """Nadaraya-Watson regression with the Laplacian kernel."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    zz = None if z is None else _f64(z, d)
    m = x.shape[0] if zz is None else zz.shape[0]
    out = np.zeros(m, dtype=np.float64)
    yy = _f64(y).reshape(-1)
    rc = _load().fko_kreg(_ptr(x), x.shape[0], d, _ptr(yy), _ptr(zz), m, _ptr(hh),
                          int(bool(loo)), _ptr(out), int(threads))
    _check(rc)
    return out


def _kernel_call(fn, x, h, w, z, loo, threads):
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    zz = None if z is None else _f64(z, d)
    m = x.shape[0] if zz is None else zz.shape[0]
    out = np.zeros(m, dtype=np.float64)
    ww = None if w is None else _f64(w).reshape(-1)
    _check(fn(_ptr(x), x.shape[0], d, _ptr(ww), _ptr(zz), m, _ptr(hh), int(bool(loo)), _ptr(out),
              int(threads)))
    return out


def kde_uniform(x, h, w=None, z=None, loo=False, threads=0):
    """Uniform-kernel KDE, eq. (uniform kde nD): the weight in the closed box
    [z - h, z + h] (corners rounded once in FP64) over 2^d N prod h."""
    return _kernel_call(_load().fko_kde_uniform, x, h, w, z, loo, threads)


def kde_matern32(x, h, w=None, z=None, loo=False, threads=0):
    """Additive Matern-3/2 KDE, eq. (Matern32 average) with u = (x - z)/h:
    sum_i w_i (1 + D_i) e^{-D_i} / (2^d (1+d) N prod h), D_i = sum_k |x_ik - z_k|/h_k."""
    return _kernel_call(_load().fko_kde_matern32, x, h, w, z, loo, threads)


def hmatrix_factor(H):
    """H = R diag(h)^2 R^T (numpy's symmetric eigendecomposition).  Returns
    (R, h) with h > 0; raises if H is not symmetric positive definite."""
    H = np.asarray(H, dtype=np.float64)
    if H.ndim != 2 or H.shape[0] != H.shape[1] or not np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max()):
        raise ValueError("H must be a symmetric matrix")
    ev, R = np.linalg.eigh(0.5 * (H + H.T))
    if not np.all(ev > 0):
        raise ValueError("H must be positive definite")
    return R, np.sqrt(ev)


def kde_laplace_hmatrix(x, H, w=None, z=None, chunk=256):
    """eq. (kde nD H), Appendix B, with the Laplacian kernel K(u) = 2^-d e^{-|u|_1}:
    f(z) = 1/(|H|^{1/2} N) sum_i w_i K(H^{-1/2}(x_i - z)), H^{-1/2} = diag(1/h) R^T."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    zz = x if z is None else _f64(z, d)
    ww = np.ones(x.shape[0]) if w is None else _f64(w).reshape(-1)
    R, h = hmatrix_factor(H)
    A = (R / h[None, :]).T                 # diag(1/h) R^T
    c = 1.0 / (2.0 ** d * np.prod(h) * x.shape[0])   # |H|^{1/2} = prod h
    out = np.empty(zz.shape[0])
    for s in range(0, zz.shape[0], chunk):
        diff = x[None, :, :] - zz[s:s + chunk, None, :]          # [c, N, d]
        u = np.einsum("kl,cnl->cnk", A, diff)
        out[s:s + chunk] = c * (np.exp(-np.abs(u).sum(axis=2)) @ ww)
    return out


def kreg_loclin(x, y, h, z=None, loo=False):
    """Locally linear regression with the Laplacian kernel: at each target z,
    the intercept a of the fit minimising sum_i K_i (y_i - a - b.(x_i - z))^2,
    K_i = exp(-(D_i - min D)), D_i = sum_k |x_ik - z_k| / h_k (the shift by the
    minimum cancels in the fit).  NaN where the normal matrix is singular."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    yy = _f64(y).reshape(-1)
    hh = np.broadcast_to(np.asarray(h, dtype=np.float64), (d,))
    zz = x if z is None else _f64(z, d)
    out = np.empty(zz.shape[0])
    for j in range(zz.shape[0]):
        diff = x - zz[j]
        D = (np.abs(diff) / hh).sum(axis=1)
        keep = np.ones(x.shape[0], dtype=bool)
        if loo and z is None:
            keep[j] = False
        K = np.exp(-(D[keep] - D[keep].min()))
        X = np.concatenate([np.ones((int(keep.sum()), 1)), diff[keep]], axis=1)
        A = X.T @ (K[:, None] * X)
        b = X.T @ (K * yy[keep])
        try:
            out[j] = np.linalg.solve(A, b)[0]
        except np.linalg.LinAlgError:
            out[j] = np.nan
    return out


def kde_grad(x, h, g, w=None, z=None, loo=False, threads=0):
    """Adjoint of ``kde_laplace`` for upstream gradient g [M].

    Returns (grad_w [N], grad_z [M, d] or None, grad_h [d])."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    zz = None if z is None else _f64(z, d)
    m = x.shape[0] if zz is None else zz.shape[0]
    gg = _f64(g).reshape(-1)
    assert gg.shape[0] == m
    ww = None if w is None else _f64(w).reshape(-1)
    gw = np.zeros(x.shape[0], dtype=np.float64)
    gz = np.zeros((m, d), dtype=np.float64) if zz is not None else None
    gh = np.zeros(d, dtype=np.float64)
    rc = _load().fko_kde_grad(_ptr(x), x.shape[0], d, _ptr(ww), _ptr(zz), m, _ptr(hh),
                              int(bool(loo)), _ptr(gg), _ptr(gw), _ptr(gz), _ptr(gh),
                              int(threads))
    _check(rc)
    return gw, gz, gh


def loo_loglik(x, h, w=None, threads=0):
    """Leave-one-out log-likelihood L(h) and dL/dh [d]."""
    x = np.asarray(x)
    d = x.shape[1] if x.ndim == 2 else 1
    x = _f64(x, d)
    hh = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)))
    ww = None if w is None else _f64(w).reshape(-1)
    L = np.zeros(1, dtype=np.float64)
    dL = np.zeros(d, dtype=np.float64)
    rc = _load().fko_loo_loglik(_ptr(x), x.shape[0], d, _ptr(ww), _ptr(hh), _ptr(L),
                                _ptr(dL), int(threads))
    _check(rc)
    return float(L[0]), dL


def fenwick2d(x, z=None):
    """All four 2D orthant counts by an independent sort + Fenwick-tree sweep."""
    x = _f64(x, 2)
    zz = None if z is None else _f64(z, 2)
    m = x.shape[0] if zz is None else zz.shape[0]
    out = np.zeros((4, m), dtype=np.int64)
    _check(_load().fko_fenwick2d(_ptr(x), x.shape[0], _ptr(zz), m, _ptr(out)))
    return out


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
