"""GB300 (sm_103a) implementation of the fast exact multivariate ECDF / ESF and
Laplacian KDE / kernel regression of Langrene & Warin (arXiv 2005.03246).

The Python layer only marshals arguments into the C ABI of
``include/fastecdf.h``; every step of the computation runs in the library's
CUDA kernels.  Tensors on a CUDA device are passed as device pointers on the
current stream; numpy arrays are passed as host pointers and staged by the
library.  PyTorch supplies device memory (the workspace) and the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import FastEcdfError

__all__ = ["ecdf_grid", "ecdf_points", "esf_points", "kde_laplace", "kreg_laplace",
           "FastEcdfError", "mask_words"]


def _torch():
    import torch
    return torch


def mask_words(d: int, orthants=None):
    """Bitset (uint32 words) over the 2^d orthant indices; None selects all."""
    nw = max(1, (1 << d) // 32)
    w = np.zeros(nw, dtype=np.uint32)
    sel = range(1 << d) if orthants is None else [int(o) for o in orthants]
    for o in sel:
        if not 0 <= o < (1 << d):
            raise ValueError("orthant index %d out of range for d=%d" % (o, d))
        w[o >> 5] |= np.uint32(1 << (o & 31))
    return w


def _dtype_code(t):
    torch = _torch()
    if t in (torch.float32, np.float32):
        return _lib.FK_F32
    if t in (torch.float64, np.float64):
        return _lib.FK_F64
    raise TypeError("x must be float32 or float64, got %s" % (t,))


def _path_code(path):
    if path in ("mixed", _lib.FK_PATH_MIXED):
        return _lib.FK_PATH_MIXED
    if path in ("fp64", _lib.FK_PATH_FP64):
        return _lib.FK_PATH_FP64
    raise ValueError("path must be 'mixed' or 'fp64'")


def _stream_ptr(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _workspace(nbytes, device):
    torch = _torch()
    if nbytes == 0:
        return None, 0
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device), int(nbytes)


def _prep_points(x, d=None):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("x must be a CUDA tensor")
    if x.dim() == 1:
        x = x[:, None]
    if x.dim() != 2:
        raise ValueError("x must be [N, d]")
    return x.contiguous()


def ecdf_grid(x, axes, y=None, orthants=None, path="mixed"):
    """Orthant sums of the points x [N, d] on the rectilinear grid ``axes``
    (list of d strictly increasing 1-D arrays).  Returns a tensor
    [n_orthants, M_1, ..., M_d]: int64 counts when y is None, else float64.
    Orthant o tests x_k > z_k on the axes whose bit is set in o, x_k <= z_k
    elsewhere (Sec. 1, eq. ECDFdelta; Sec. 2.1, Algorithm 1)."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    M = np.array([len(a) for a in axes], dtype=np.int64)
    z = torch.as_tensor(np.concatenate([np.asarray(a, dtype=np.float64) for a in axes]),
                        device=dev)
    if y is not None:
        y = y.to(device=dev, dtype=x.dtype).contiguous()
    mw = mask_words(d, orthants)
    nsel = int(sum(bin(int(v)).count("1") for v in mw))
    out = torch.empty((nsel,) + tuple(int(m) for m in M),
                      dtype=torch.int64 if y is None else torch.float64, device=dev)
    pc = _path_code(path)
    need = lib.fk_ecdf_grid_workspace(n, d, M.ctypes.data_as(ctypes.c_void_p),
                                      int(y is not None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_ecdf_grid(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(y), _ptr(z),
                          M.ctypes.data_as(ctypes.c_void_p), mw.ctypes.data_as(ctypes.c_void_p),
                          _ptr(out), pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_ecdf_grid")
    return out


def _prep_targets(z, x):
    if z is None:
        return None, 0
    z = z.to(device=x.device, dtype=x.dtype)
    if z.dim() == 1:
        z = z[:, None]
    if z.shape[1] != x.shape[1]:
        raise ValueError("z must be [M, d] with the same d as x")
    z = z.contiguous()
    return z, int(z.shape[0])


def _weights(v, x):
    if v is None:
        return None
    v = v.to(device=x.device, dtype=x.dtype).reshape(-1).contiguous()
    if v.shape[0] != x.shape[0]:
        raise ValueError("weights must have N entries")
    return v


def ecdf_points(x, y=None, z=None, orthants=None, path="mixed"):
    """Orthant sums at the sample points (z None) or at explicit targets z
    [M, d], by rank transform and divide-and-conquer (Sec. 2.2, Appendix D).
    Returns [n_orthants, M']: int64 counts when y is None, else float64."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    y = _weights(y, x)
    z, m = _prep_targets(z, x)
    mw = mask_words(d, orthants)
    nsel = int(sum(bin(int(v)).count("1") for v in mw))
    mo = m if z is not None else n
    out = torch.empty((nsel, mo), dtype=torch.int64 if y is None else torch.float64, device=dev)
    pc = _path_code(path)
    need = lib.fk_ecdf_points_workspace(n, d, m, int(z is None), int(y is not None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_ecdf_points(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(y), _ptr(z), m,
                            mw.ctypes.data_as(ctypes.c_void_p), _ptr(out), pc, _ptr(ws), wsb,
                            _stream_ptr(dev))
    _lib.check(rc, "fk_ecdf_points")
    return out


def esf_points(x, y=None, z=None, path="mixed"):
    """Empirical survival function (eq. ESF): sum of y over x_k > z_k on every axis."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    y = _weights(y, x)
    z, m = _prep_targets(z, x)
    mo = m if z is not None else n
    out = torch.empty((mo,), dtype=torch.int64 if y is None else torch.float64, device=dev)
    pc = _path_code(path)
    need = lib.fk_ecdf_points_workspace(n, d, m, int(z is None), int(y is not None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_esf_points(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(y), _ptr(z), m, _ptr(out), pc,
                           _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_esf_points")
    return out


def _h_array(h, d):
    hh = np.broadcast_to(np.asarray(h, dtype=np.float64), (d,)).copy()
    return hh


def kde_laplace(x, h, w=None, z=None, loo=False, terms=False, path="mixed"):
    """Laplacian KDE (eq. Laplacian kde nD) via the 2^d exponentially weighted
    orthant sums of eq. (Laplacian decomposition nD).  Returns f [M'] (float64),
    and with terms=True also the per-orthant terms [2^d, M']."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    w = _weights(w, x)
    z, m = _prep_targets(z, x)
    hh = _h_array(h, d)
    mo = m if z is not None else n
    out = torch.empty((mo,), dtype=torch.float64, device=dev)
    tt = torch.empty((1 << d, mo), dtype=torch.float64, device=dev) if terms else None
    pc = _path_code(path)
    need = lib.fk_kde_laplace_workspace(n, d, m, int(z is None), int(bool(terms)), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_kde_laplace(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(w), _ptr(z), m,
                            hh.ctypes.data_as(ctypes.c_void_p), _lib.FK_LOO if loo else 0, _ptr(out),
                            _ptr(tt), pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_kde_laplace")
    return (out, tt) if terms else out


def kreg_laplace(x, y, h, z=None, loo=False, path="mixed"):
    """Nadaraya-Watson regression with the Laplacian kernel.  Returns [M'] float64."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    y = _weights(y, x)
    z, m = _prep_targets(z, x)
    hh = _h_array(h, d)
    mo = m if z is not None else n
    out = torch.empty((mo,), dtype=torch.float64, device=dev)
    pc = _path_code(path)
    need = lib.fk_kreg_laplace_workspace(n, d, m, int(z is None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_kreg_laplace(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(y), _ptr(z), m,
                             hh.ctypes.data_as(ctypes.c_void_p), _lib.FK_LOO if loo else 0, _ptr(out),
                             pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_kreg_laplace")
    return out
