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

__all__ = ["ecdf_grid", "ecdf_points", "esf_points", "kde_laplace", "kreg_laplace", "kde", "Batched",
           "kde_grid", "grid_interp", "kde_uniform", "kde_matern32", "kde_laplace_hmatrix", "hmatrix_factor",
           "kreg_loclin",
           "kde_laplace_backward", "loo_laplace", "select_bandwidth_loo",
           "tune_key", "tune_cache_get", "tune_cache_put",
           "FastEcdfError", "mask_words", "device_status"]


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


def device_status(device=None):
    """Synchronise the current stream of `device` and raise FastEcdfError if a
    kernel recorded an error since the last check (for example
    FK_ERR_NONFINITE: a NaN or infinite coordinate in x or z); clears it."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _lib.check(_lib.load().fk_device_status(_stream_ptr(dev)), "fk_device_status")


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


def _axes_tensor(axes, dev):
    M = np.array([len(a) for a in axes], dtype=np.int64)
    z = _torch().as_tensor(np.concatenate([np.asarray(a, dtype=np.float64) for a in axes]), device=dev)
    return M, z


def kde_grid(x, h, axes, w=None, path="mixed"):
    """Laplacian KDE (eq. Laplacian kde nD) at every point of the rectilinear
    grid ``axes`` (list of d strictly increasing 1-D arrays): the grid form of
    eq. Laplacian decomposition nD with per-axis decaying recurrences, exact at
    the grid points.  Returns float64 [M_1, ..., M_d]."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    M, z = _axes_tensor(axes, dev)
    w = _weights(w, x)
    hh = _h_array(h, d)
    out = torch.empty(tuple(int(m) for m in M), dtype=torch.float64, device=dev)
    pc = _path_code(path)
    need = lib.fk_kde_grid_workspace(n, d, M.ctypes.data_as(ctypes.c_void_p), pc)
    if need == 0:
        _lib.check(-1, "fk_kde_grid_workspace")
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_kde_grid(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(w), _ptr(z), M.ctypes.data_as(ctypes.c_void_p),
                         hh.ctypes.data_as(ctypes.c_void_p), _ptr(out), pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_kde_grid")
    return out


def grid_interp(f, axes, q):
    """Multilinear interpolation of the grid function f [M_1, ..., M_d]
    (float64, e.g. kde_grid's output) at the points q [Q, d]; coordinates
    outside the grid box are clamped to it.  Returns float64 [Q]."""
    torch = _torch()
    lib = _lib.load()
    q = _prep_points(q)
    nq, d = q.shape
    dev = q.device
    M, z = _axes_tensor(axes, dev)
    f = f.to(device=dev, dtype=torch.float64).contiguous()
    out = torch.empty((nq,), dtype=torch.float64, device=dev)
    ws, wsb = _workspace(lib.fk_grid_interp_workspace(), dev)
    rc = lib.fk_grid_interp(_ptr(f), d, _ptr(z), M.ctypes.data_as(ctypes.c_void_p), _ptr(q), _dtype_code(q.dtype),
                            nq, _ptr(out), _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_grid_interp")
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
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return out
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
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return out
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
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return (out, tt) if terms else out
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
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return out
    pc = _path_code(path)
    need = lib.fk_kreg_laplace_workspace(n, d, m, int(z is None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_kreg_laplace(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(y), _ptr(z), m,
                             hh.ctypes.data_as(ctypes.c_void_p), _lib.FK_LOO if loo else 0, _ptr(out),
                             pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_kreg_laplace")
    return out


# ----------------------------------------------------------------------------- other kernels


def _kfam_call(name, x, h_or_H, w, z, loo, path, weighted_ws=True, ws_fn=None):
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    w = _weights(w, x)
    z, m = _prep_targets(z, x)
    mo = m if z is not None else n
    out = torch.empty((mo,), dtype=torch.float64, device=dev)
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return out
    pc = _path_code(path)
    if weighted_ws:
        need = getattr(lib, name + "_workspace")(n, d, m, int(z is None), int(w is not None), pc)
    else:
        need = getattr(lib, name + "_workspace")(n, d, m, int(z is None), pc)
    if need == 0 and n > 0 and mo > 0:
        _lib.check(-2, name + "_workspace")
    ws, wsb = _workspace(need, dev)
    rc = getattr(lib, name)(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(w), _ptr(z), m,
                            h_or_H.ctypes.data_as(ctypes.c_void_p), _lib.FK_LOO if loo else 0, _ptr(out), pc,
                            _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, name)
    return out


def kde_uniform(x, h, w=None, z=None, loo=False, path="mixed"):
    """Uniform-kernel KDE (eq. uniform kde nD) by the signed corner
    combination of 2^d ECDFs (eq. uniform decomposition nD).  Returns [M'] float64."""
    x = _prep_points(x)
    return _kfam_call("fk_kde_uniform", x, _h_array(h, x.shape[1]), w, z, loo, path)


def kde_matern32(x, h, w=None, z=None, loo=False, path="mixed"):
    """KDE with the additive Matern-3/2 kernel (eq. Matern32 average,
    Appendix C) from 2^d (d+1) orthant sums (eq. Matern32 decomposition nD)."""
    x = _prep_points(x)
    return _kfam_call("fk_kde_matern32", x, _h_array(h, x.shape[1]), w, z, loo, path)


def kde_laplace_hmatrix(x, H, w=None, z=None, loo=False, path="mixed"):
    """Laplacian KDE with a full bandwidth matrix H (eq. kde nD H, Appendix B):
    points rotated by R^T, H = R diag(h)^2 R^T, then the diagonal KDE."""
    x = _prep_points(x)
    d = x.shape[1]
    HH = np.ascontiguousarray(np.asarray(H, dtype=np.float64).reshape(d, d))
    return _kfam_call("fk_kde_laplace_hmatrix", x, HH, w, z, loo, path, weighted_ws=False)


def hmatrix_factor(H):
    """H = R diag(h)^2 R^T as the library factors it (host only).  Returns (R, h)."""
    lib = _lib.load()
    HH = np.ascontiguousarray(np.asarray(H, dtype=np.float64))
    d = HH.shape[0]
    R = np.zeros((d, d))
    h = np.zeros(d)
    rc = lib.fk_hmatrix_factor(HH.ctypes.data_as(ctypes.c_void_p), d, R.ctypes.data_as(ctypes.c_void_p),
                               h.ctypes.data_as(ctypes.c_void_p))
    _lib.check(rc, "fk_hmatrix_factor")
    return R, h


def kreg_loclin(x, y, h, z=None, loo=False, path="fp64"):
    """Locally linear regression with the Laplacian kernel (the intercept of
    the kernel-weighted affine least-squares fit at each target).  FP64 path
    only.  Returns [M'] float64."""
    x = _prep_points(x)
    return _kfam_call("fk_kreg_loclin_laplace", x, _h_array(h, x.shape[1]), y, z, loo, path, weighted_ws=False)


# ----------------------------------------------------------------------------- adjoints


def kde_laplace_backward(x, h, grad_out, w=None, z=None, loo=False, need_w=True, need_z=True, need_h=True,
                         path="mixed"):
    """Adjoint of ``kde_laplace`` for the upstream gradient ``grad_out`` [M']:
    returns (grad_w [N] or None, grad_z [M, d] or None, grad_h [d] or None),
    float64 tensors on x's device (exact derivatives of eq. Laplacian kde nD)."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    w = _weights(w, x)
    z, m = _prep_targets(z, x)
    hh = _h_array(h, d)
    mo = m if z is not None else n
    g = grad_out.to(device=dev, dtype=torch.float64).reshape(-1).contiguous()
    if g.shape[0] != mo:
        raise ValueError("grad_out must have one entry per target")
    gw = torch.empty((n,), dtype=torch.float64, device=dev) if need_w else None
    gz = torch.empty((mo, d), dtype=torch.float64, device=dev) if (need_z and z is not None) else None
    gh = torch.empty((d,), dtype=torch.float64, device=dev) if need_h else None
    if z is not None and m == 0:      # no targets: nothing to compute (an empty z has no address)
        return (None if gw is None else gw.zero_()), gz, (None if gh is None else gh.zero_())
    pc = _path_code(path)
    need = lib.fk_kde_laplace_backward_workspace(n, d, m, int(z is None), pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_kde_laplace_backward(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(w), _ptr(z), m,
                                     hh.ctypes.data_as(ctypes.c_void_p), _lib.FK_LOO if loo else 0, _ptr(g),
                                     _ptr(gw), _ptr(gz), _ptr(gh), pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_kde_laplace_backward")
    return gw, gz, gh


def loo_laplace(x, h, w=None, path="mixed", grad=True):
    """Leave-one-out log-likelihood L(h) = mean_j log f_{-j}(x_j) of the
    Laplacian KDE and dL/dh [d].  Returns (L as a 0-d float64 tensor, grad_h)."""
    torch = _torch()
    lib = _lib.load()
    x = _prep_points(x)
    n, d = x.shape
    dev = x.device
    w = _weights(w, x)
    hh = _h_array(h, d)
    L = torch.empty((1,), dtype=torch.float64, device=dev)
    gh = torch.empty((d,), dtype=torch.float64, device=dev) if grad else None
    pc = _path_code(path)
    need = lib.fk_loo_laplace_workspace(n, d, pc)
    ws, wsb = _workspace(need, dev)
    rc = lib.fk_loo_laplace(_ptr(x), _dtype_code(x.dtype), n, d, _ptr(w), hh.ctypes.data_as(ctypes.c_void_p),
                            _ptr(L), _ptr(gh), pc, _ptr(ws), wsb, _stream_ptr(dev))
    _lib.check(rc, "fk_loo_laplace")
    return L[0], gh


def _kde_function():
    torch = _torch()

    class KDELaplace(torch.autograd.Function):
        """f = kde_laplace(x, h, w, z) with the hand-written adjoint in w, z and h."""

        @staticmethod
        def forward(ctx, x, w, z, h, loo, path):
            hv = h.detach().to(torch.float64).cpu().numpy()
            f = kde_laplace(x, hv, w=w, z=z, loo=loo, path=path)
            ctx.save_for_backward(x, w if w is not None else torch.empty(0), z if z is not None else torch.empty(0))
            ctx.has_w, ctx.has_z = w is not None, z is not None
            ctx.hv, ctx.loo, ctx.path, ctx.hdev, ctx.hdt = hv, loo, path, h.device, h.dtype
            return f

        @staticmethod
        def backward(ctx, gf):
            x, w, z = ctx.saved_tensors
            w = w if ctx.has_w else None
            z = z if ctx.has_z else None
            nw, nz, nh = ctx.needs_input_grad[1], ctx.needs_input_grad[2], ctx.needs_input_grad[3]
            gw, gz, gh = kde_laplace_backward(x, ctx.hv, gf, w=w, z=z, loo=ctx.loo, need_w=nw, need_z=nz,
                                              need_h=nh, path=ctx.path)
            if gw is not None and w is not None:
                gw = gw.to(w.dtype)
            if gz is not None and z is not None:
                gz = gz.to(z.dtype)
            if gh is not None:
                gh = gh.to(device=ctx.hdev, dtype=ctx.hdt)
            return None, gw, gz, gh, None, None

    return KDELaplace


_KDE_FN = None


def kde(x, h, w=None, z=None, loo=False, path="mixed"):
    """Differentiable Laplacian KDE: gradients flow to w, z and h (a tensor of
    shape [d] or scalar) through the C-ABI adjoint (fk_kde_laplace_backward)."""
    global _KDE_FN
    torch = _torch()
    if _KDE_FN is None:
        _KDE_FN = _kde_function()
    x = _prep_points(x)
    d = x.shape[1]
    if not isinstance(h, torch.Tensor):
        h = torch.tensor(h, dtype=torch.float64)
    hfull = h.reshape(-1).expand(d) if h.numel() == 1 else h.reshape(-1)
    return _KDE_FN.apply(x, w, z, hfull, loo, path)


def select_bandwidth_loo(x, h0=0.5, steps=20, lr=0.5, w=None, path="mixed", per_axis=False, checkpoint=None):
    """Leave-one-out likelihood bandwidth selection: gradient ascent on u = log h,
    u <- u + lr * dL/du (dL/du = h * dL/dh), from h0, for `steps` steps.
    Returns a list of (h, L, dL/dh) per step (h before the step).

    checkpoint: optional path of a JSON file holding the optimiser state (steps
    done, log h and the history so far), rewritten atomically after every step.
    If it exists when the call starts, the search resumes from it (it must come
    from a search with the same d, lr, per_axis and path, else ValueError);
    floats round-trip exactly through the file."""
    import json
    import os
    x = _prep_points(x)
    d = x.shape[1]
    u = np.log(np.broadcast_to(np.asarray(h0, dtype=np.float64), (d,)).copy())
    hist = []
    start = 0
    meta = {"d": int(d), "lr": float(lr), "per_axis": bool(per_axis), "path": str(path)}
    if checkpoint is not None and os.path.exists(checkpoint):
        with open(checkpoint) as f:
            st = json.load(f)
        if {k: st.get(k) for k in meta} != meta:
            raise ValueError("checkpoint %s belongs to another search (%s)" % (checkpoint, {k: st.get(k) for k in meta}))
        u = np.asarray(st["log_h"], dtype=np.float64)
        hist = [(np.asarray(e["h"], dtype=np.float64), float(e["L"]), np.asarray(e["grad_h"], dtype=np.float64))
                for e in st["history"]]
        start = int(st["step"])
    for step in range(start, steps):
        h = np.exp(u)
        L, gh = loo_laplace(x, h, w=w, path=path)
        g = gh.cpu().numpy()
        hist.append((h.copy(), float(L.item()), g.copy()))
        if per_axis:
            u = u + lr * h * g
        else:
            u = u + lr * float(np.sum(h * g))
        if checkpoint is not None:
            st = dict(meta, step=step + 1, log_h=[float(v) for v in u],
                      history=[{"h": [float(v) for v in a], "L": b, "grad_h": [float(v) for v in c]}
                               for a, b, c in hist])
            tmp = "%s.tmp%d" % (checkpoint, os.getpid())
            with open(tmp, "w") as f:
                json.dump(st, f)
            os.replace(tmp, checkpoint)
    return hist


# ----------------------------------------------------------------------------- batching


def tune_key(cc, dtype_code, path_code, what, shapes):
    """Key of a tuned batch configuration: the GPU's compute capability, the
    dtype, the precision path and the request, and the shape of the batch (the
    dataset count, the datasets per dimension, and the power-of-two buckets of
    the total and the largest N).  shapes: iterable of (N_b, d_b)."""
    shapes = [(int(n), int(d)) for n, d in shapes]
    per_d = {}
    for _, d in shapes:
        per_d[d] = per_d.get(d, 0) + 1
    ntot = sum(n for n, _ in shapes)
    nmax = max([n for n, _ in shapes] + [0])
    return "sm%d%d|dtype%d|path%d|what%d|sets%d|%s|ntot~2^%d|nmax~2^%d" % (
        int(cc[0]), int(cc[1]), int(dtype_code), int(path_code), int(what), len(shapes),
        ",".join("d%d:%d" % (d, per_d[d]) for d in sorted(per_d)),
        int(round(np.log2(max(ntot, 1)))), int(round(np.log2(max(nmax, 1)))))


def tune_cache_get(path, key):
    """The cached entry {"config": {...}, "ms": t} for key, or None.  A missing
    or unreadable cache file is a miss."""
    import json
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        return None
    e = cache.get(key) if isinstance(cache, dict) else None
    if not isinstance(e, dict) or not isinstance(e.get("config"), dict):
        return None
    return e


def tune_cache_put(path, key, config, ms):
    """Store a tuned configuration under key (the file is rewritten atomically;
    other keys are kept, an unreadable file is replaced)."""
    import json
    import os
    try:
        with open(path) as f:
            cache = json.load(f)
        if not isinstance(cache, dict):
            cache = {}
    except (OSError, ValueError):
        cache = {}
    cache[key] = {"config": {k: int(v) for k, v in dict(config).items()}, "ms": float(ms)}
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Batched:
    """Many independent datasets in one call (fk_batched): all orthant counts at
    each dataset's sample points and/or its Laplacian KDE (bandwidth h on every
    axis, weights ys[b] or 1).

    xs: list of CUDA tensors [N_b, d_b] of one dtype (1 <= d_b <= 4); ys: list of
    [N_b] tensors or None.  With graph=True the call is captured once in a CUDA
    graph and ``run()`` replays it (the input tensors must keep their storage).
    ``run()`` returns (ecdf, kde): lists of per-dataset views [2^d_b, N_b] int64
    and [N_b] float64 (None for the part not requested).

    config: a dict of fk_batch_config fields (streams, coarsen, kernel_tile,
    count_tile), "tune" to let fk_batched_autotune choose it by measurement on
    these datasets, or None for the default; ``self.config`` holds the one
    used (and ``self.tune_ms`` the tuned time).

    tune_cache: with config="tune", the path of a JSON file of tuned
    configurations keyed by ``tune_key`` (GPU, dtype, path, request and the
    batch's shape buckets).  A hit skips the tuning (``self.tune_cached`` is
    True); a miss tunes and stores the result."""

    def __init__(self, xs, ys=None, h=0.1, ecdf=True, kde=True, path="mixed", graph=True, config=None,
                 tune_cache=None):
        torch = _torch()
        lib = _lib.load()
        if not xs:
            raise ValueError("no datasets")
        self.xs = [_prep_points(x) for x in xs]
        dt = self.xs[0].dtype
        dev = self.xs[0].device
        if any(x.dtype != dt for x in self.xs):
            raise TypeError("all datasets must share one dtype")
        self.ys = [None if (ys is None or ys[b] is None) else _weights(ys[b], self.xs[b])
                   for b in range(len(self.xs))]
        self.what = (_lib.FK_BATCH_ECDF if ecdf else 0) | (_lib.FK_BATCH_KDE if kde else 0)
        self.h = float(h)
        self.path = _path_code(path)
        self.dev = dev
        n = len(self.xs)
        self.sets = (_lib.Dataset * n)()
        ne = nk = 0
        self.shape_e, self.off_e, self.off_k = [], [], []
        for b, x in enumerate(self.xs):
            nb, d = x.shape
            s = self.sets[b]
            s.x = x.data_ptr() if nb else None
            s.y = self.ys[b].data_ptr() if self.ys[b] is not None else None
            s.N, s.d = nb, d
            self.off_e.append(ne)
            self.off_k.append(nk)
            self.shape_e.append((1 << d, nb))
            ne += (1 << d) * nb
            nk += nb
        self.ecdf_out = torch.empty(max(ne, 1), dtype=torch.int64, device=dev) if ecdf else None
        self.kde_out = torch.empty(max(nk, 1), dtype=torch.float64, device=dev) if kde else None
        self.dtype_code = _dtype_code(dt)
        self.cfg = _lib.BatchConfig()
        lib.fk_batched_config_default(ctypes.byref(self.cfg))
        self.tune_ms = None
        self.tune_cached = False
        cached = None
        if config == "tune" and tune_cache is not None:
            key = tune_key(torch.cuda.get_device_capability(dev), self.dtype_code, self.path, self.what,
                           [tuple(x.shape) for x in self.xs])
            cached = tune_cache_get(tune_cache, key)
        if cached is not None:
            fields = [f for f, _ in _lib.BatchConfig._fields_]
            for k in fields:
                if k in cached["config"]:
                    setattr(self.cfg, k, int(cached["config"][k]))
            self.tune_ms = float(cached.get("ms", 0.0))
            self.tune_cached = True
        elif config == "tune":
            need = lib.fk_batched_autotune_workspace(self.sets, n, self.dtype_code, self.what, self.path)
            tws, twsb = _workspace(need, dev)
            ms = ctypes.c_double(0.0)
            rc = lib.fk_batched_autotune(self.sets, n, self.dtype_code, self.what, self.h, _ptr(self.ecdf_out),
                                         _ptr(self.kde_out), self.path, _ptr(tws), twsb, _stream_ptr(dev),
                                         ctypes.byref(self.cfg), ctypes.byref(ms))
            _lib.check(rc, "fk_batched_autotune")
            self.tune_ms = ms.value
            del tws
            if tune_cache is not None:
                tune_cache_put(tune_cache, key, self.cfg.as_dict(), self.tune_ms)
        elif config is not None:
            for k, v in dict(config).items():
                setattr(self.cfg, k, int(v))
        self.config = self.cfg.as_dict()
        need = lib.fk_batched_workspace_ex(self.sets, n, self.dtype_code, self.what, self.path, ctypes.byref(self.cfg))
        if need == 0 and n > 0:
            _lib.check(-1, "fk_batched_workspace_ex")
        self.ws, self.wsb = _workspace(need, dev)
        self.graph = None
        self._call()                         # warm-up (sets kernel attributes, checks errors)
        torch.cuda.synchronize(dev)
        if graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                self._call()
            self.graph = g

    def _call(self):
        lib = _lib.load()
        rc = lib.fk_batched_ex(self.sets, len(self.xs), self.dtype_code, self.what, self.h, _ptr(self.ecdf_out),
                               _ptr(self.kde_out), self.path, ctypes.byref(self.cfg), _ptr(self.ws), self.wsb,
                               _stream_ptr(self.dev))
        _lib.check(rc, "fk_batched_ex")

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._call()
        ecdf = kde = None
        if self.ecdf_out is not None:
            ecdf = [self.ecdf_out[o:o + a * b].view(a, b) for o, (a, b) in zip(self.off_e, self.shape_e)]
        if self.kde_out is not None:
            kde = [self.kde_out[o:o + x.shape[0]] for o, x in zip(self.off_k, self.xs)]
        return ecdf, kde
