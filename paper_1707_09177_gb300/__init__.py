"""Python binding of libgad.so, the GB300 approximate-deconvolution library.

Argument marshalling only: every step of filtering and solving runs in the
library's CUDA kernels. Tensors are torch CUDA tensors (torch provides the
device memory and the stream); the library sees plain device pointers.

    import paper_1707_09177_gb300 as gad
    ubar = gad.filter(u, gamma=0.01)                        # G u (Section 4, Eq. df2)
    res = gad.deconvolve(ubar, gamma=0.01, method="bicgstab", tol=1e-6, maxit=500)
    res.u, res.iterations, res.status, res.history

Fields are C-ordered with x last: (Ny, Nx) or (Nz, Ny, Nx), with optional
leading batch dimensions; pass ``ndim`` when the shape is ambiguous (a 3-axis
tensor may be one 3D field or a batch of 2D fields).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgad.so")

AD_OK, AD_MAXIT, AD_BREAKDOWN = 0, 1, 2
AD_ERR_ARG, AD_ERR_NONFINITE, AD_ERR_CUDA, AD_ERR_TIMEOUT, AD_ERR_NOMEM = -1, -2, -3, -4, -5
AD_SPECTRAL = 4                     # flag: iterate on the half spectra (G a pointwise multiply)
AD_PRECOND = 8                      # flag on AD_CG: preconditioned CG (stencil approximation of G^-1)
METHODS = {"vancittert": 0, "cg": 1, "bicgstab": 2, "sd": 3, "pcg": 1 | AD_PRECOND}
SPACES = ("physical", "spectral")


def method_code(method, space="physical"):
    """The C method value for a method name and iteration space."""
    if method not in METHODS:
        raise ValueError("method must be one of %s" % sorted(METHODS))
    if space not in SPACES:
        raise ValueError("space must be one of %s" % (SPACES,))
    return METHODS[method] | (AD_SPECTRAL if space == "spectral" else 0)
AD_F32, AD_F64 = 0, 1

EXPORTED = ("ad_create", "ad_destroy", "ad_filter", "ad_deconvolve", "ad_deconvolve_batched", "ad_time_pass",
            "ad_autotune", "ad_set_graph_mode", "ad_last_launch_count", "ad_status_str", "ad_last_error",
            "ad_filter_static", "ad_guess_weight_count", "ad_guess_init", "ad_guess_infer", "ad_guess_grad",
            "ad_guess_train", "ad_closure", "ad_spectrum", "ad_histogram", "ad_curl", "ad_set_wait_limit",
            "ad_deconvolve_host", "ad_guess_time_conv", "ad_set_batched_launch")
PASS_KINDS = {0: "xfwd", 1: "xinv", 2: "filt", 3: "yfwd", 4: "yinv", 5: "lfwd", 6: "linv", 7: "spec", 8: "sten"}


class ad_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("dtype", ctypes.c_int),
                ("gamma", ctypes.c_double)]


class GadError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__("libgad status %d: %s" % (status, detail))
        self.status = status


_lib = None
_ctx = {}


def library_path():
    return _LIB_PATH


def load(path=None):
    """Loads libgad.so (building it first if it is missing). Raises if the
    library cannot be loaded: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        from . import build as _b
        _b.build()
    lib = ctypes.CDLL(p)
    c_p, c_i, c_d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ad_create.argtypes = [ctypes.POINTER(c_p), c_i]
    lib.ad_create.restype = c_i
    lib.ad_destroy.argtypes = [c_p]
    lib.ad_destroy.restype = None
    lib.ad_filter.argtypes = [c_p, ctypes.POINTER(ad_grid), c_p, c_p, c_i, c_p]
    lib.ad_filter.restype = c_i
    lib.ad_deconvolve.argtypes = [c_p, ctypes.POINTER(ad_grid), c_p, c_p, c_i, c_i, c_d, c_i, c_p,
                                  c_p, c_p, c_p, c_p, c_p]
    lib.ad_deconvolve.restype = c_i
    lib.ad_deconvolve_host.argtypes = [c_p, ctypes.POINTER(ad_grid), c_p, c_p, c_i, c_i, c_d, c_i, c_p, c_p, c_p,
                                       c_p]
    lib.ad_deconvolve_host.restype = c_i
    lib.ad_deconvolve_batched.argtypes = [c_p, c_i, ctypes.POINTER(ad_grid), c_p, c_p, c_i, c_d, c_i, c_p, c_p,
                                          c_p, c_p]
    lib.ad_deconvolve_batched.restype = c_i
    lib.ad_guess_weight_count.argtypes = []
    lib.ad_guess_weight_count.restype = ctypes.c_int64
    lib.ad_guess_init.argtypes = [c_p, ctypes.c_int64, ctypes.c_uint64, c_i]
    lib.ad_guess_init.restype = c_i
    lib.ad_guess_infer.argtypes = [c_p, ctypes.POINTER(ad_grid), c_p, c_p, c_p, c_i, c_p]
    lib.ad_guess_infer.restype = c_i
    lib.ad_guess_grad.argtypes = [c_p, ctypes.POINTER(ad_grid), c_p, c_p, c_p, c_i, c_p, c_p, c_p]
    lib.ad_guess_grad.restype = c_i
    lib.ad_guess_train.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_p, c_p, c_i, c_i, c_d, ctypes.c_uint64,
                                   c_p, c_p, c_p]
    lib.ad_guess_train.restype = c_i
    lib.ad_autotune.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_i, c_i]
    lib.ad_autotune.restype = c_i
    lib.ad_time_pass.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_i, c_i, c_i, c_p, c_p, c_p, c_p, c_p]
    lib.ad_time_pass.restype = c_i
    lib.ad_set_graph_mode.argtypes = [c_p, c_i]
    lib.ad_set_graph_mode.restype = c_i
    lib.ad_set_batched_launch.argtypes = [c_p, c_i]
    lib.ad_set_batched_launch.restype = c_i
    lib.ad_last_launch_count.argtypes = [c_p]
    lib.ad_last_launch_count.restype = ctypes.c_int64
    lib.ad_status_str.argtypes = [c_i]
    lib.ad_status_str.restype = ctypes.c_char_p
    lib.ad_last_error.argtypes = [c_p]
    lib.ad_last_error.restype = ctypes.c_char_p
    lib.ad_closure.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_i, c_p, c_p, c_p, c_p]
    lib.ad_closure.restype = c_i
    lib.ad_spectrum.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_i, c_p, c_i, c_p, c_p]
    lib.ad_spectrum.restype = c_i
    lib.ad_histogram.argtypes = [c_p, c_i, ctypes.c_int64, c_p, c_d, c_d, c_i, c_p, c_p]
    lib.ad_histogram.restype = c_i
    lib.ad_curl.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_p, c_p, c_p]
    lib.ad_curl.restype = c_i
    lib.ad_guess_time_conv.argtypes = [c_p, ctypes.POINTER(ad_grid), c_i, c_i, c_p, c_p, c_p]
    lib.ad_guess_time_conv.restype = c_i
    lib.ad_set_wait_limit.argtypes = [c_p, ctypes.c_uint64]
    lib.ad_set_wait_limit.restype = c_i
    _lib = lib
    return lib


def context(device=None):
    """The library context for a CUDA device (created on first use)."""
    import torch
    lib = load()
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _ctx:
        h = ctypes.c_void_p()
        st = lib.ad_create(ctypes.byref(h), dev)
        if st != AD_OK:
            raise GadError(st, "ad_create failed on device %d" % dev)
        _ctx[dev] = h
    return _ctx[dev]


def set_graph_mode(enable, device=None):
    load().ad_set_graph_mode(context(device), 1 if enable else 0)


def set_batched_launch(one_launch_per_stage, device=None):
    """Batched solves of several shapes: one graph branch per shape group
    (False, default) or one launch per pass stage over every group (True)."""
    ctx = context(device)
    _check(load().ad_set_batched_launch(ctx, 1 if one_launch_per_stage else 0), ctx)


def set_wait_limit(ns, device=None):
    """Time limit (ns) of the library's bounded device waits; 0 makes each give
    up at once (used to exercise the timeout path)."""
    ctx = context(device)
    _check(load().ad_set_wait_limit(ctx, int(ns)), ctx)


def last_launch_count(device=None):
    return int(load().ad_last_launch_count(context(device)))


def _check(st, ctx, per_field=False):
    # AD_ERR_NONFINITE from a solve is a per-field outcome, reported in status[]
    if st < 0 and not (per_field and st == AD_ERR_NONFINITE):
        lib = load()
        raise GadError(st, "%s (%s)" % (lib.ad_status_str(st).decode(), lib.ad_last_error(ctx).decode()))


def _grid(t, ndim, gamma, host=False):
    import torch
    if t.dtype == torch.float32:
        dt = AD_F32
    elif t.dtype == torch.float64:
        dt = AD_F64
    else:
        raise TypeError("fields must be float32 or float64, got %s" % t.dtype)
    if t.is_cuda == host or not t.is_contiguous():
        raise ValueError("fields must be contiguous %s tensors" % ("CPU" if host else "CUDA"))
    if ndim is None:
        if t.dim() == 2:
            ndim = 2
        elif t.dim() == 4:
            ndim = 3
        else:
            raise ValueError("pass ndim=2 or ndim=3 for a %d-axis tensor" % t.dim())
    if t.dim() < ndim:
        raise ValueError("tensor has fewer axes than ndim")
    shape = tuple(t.shape[t.dim() - ndim:])
    batch = int(np.prod(t.shape[:t.dim() - ndim])) if t.dim() > ndim else 1
    g = ad_grid()
    g.ndim = ndim
    rev = list(reversed(shape)) + [1] * (3 - ndim)
    for i in range(3):
        g.n[i] = int(rev[i])
    g.dtype = dt
    g.gamma = float(gamma)
    return g, batch, shape


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def filter(u, gamma, ndim=None, out=None, stream=None):
    """G u for every field of ``u`` (Section 4, Eq. df/df2, evaluated by FFT)."""
    import torch
    lib = load()
    ctx = context(u.device.index)
    g, batch, _ = _grid(u, ndim, gamma)
    if out is None:
        out = torch.empty_like(u)
    st = lib.ad_filter(ctx, ctypes.byref(g), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                       batch, _stream_ptr(stream))
    _check(st, ctx)
    return out


@dataclass
class Solve:
    u: object                 # torch tensor, same shape as u_bar
    iterations: np.ndarray    # int32 [batch]
    status: np.ndarray        # int32 [batch]
    history: np.ndarray       # float64 [batch, maxit + 1]; h_0 .. h_iterations valid
    true_residual: np.ndarray  # float64 [batch] or None
    launches: int             # kernels the call launched


def deconvolve(ubar, gamma, method="bicgstab", tol=1e-6, maxit=1000, u0=None, ndim=None,
               out=None, history=True, true_residual=False, stream=None, space="physical"):
    """Solves G u = u_bar (Section 3, Eq. tau3) for every field of ``ubar``;
    ``space="spectral"`` iterates on the half spectra (AD_SPECTRAL)."""
    import torch
    lib = load()
    ctx = context(ubar.device.index)
    g, batch, _ = _grid(ubar, ndim, gamma)
    code = method_code(method, space)
    if out is None:
        out = torch.empty_like(ubar)
    if u0 is not None and (u0.shape != ubar.shape or u0.dtype != ubar.dtype or not u0.is_contiguous()):
        raise ValueError("u0 must match u_bar in shape, dtype and layout")
    its = np.zeros(batch, dtype=np.int32)
    sts = np.zeros(batch, dtype=np.int32)
    hist = np.full((batch, int(maxit) + 1), np.nan) if history else None
    tr = np.zeros(batch) if true_residual else None
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p()
    st = lib.ad_deconvolve(ctx, ctypes.byref(g), ctypes.c_void_p(ubar.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                           batch, code, float(tol), int(maxit),
                           ctypes.c_void_p(u0.data_ptr()) if u0 is not None else ctypes.c_void_p(),
                           ptr(its), ptr(sts), ptr(hist), ptr(tr), _stream_ptr(stream))
    _check(st, ctx, per_field=True)
    return Solve(u=out, iterations=its, status=sts, history=hist, true_residual=tr,
                 launches=int(lib.ad_last_launch_count(ctx)))


def deconvolve_host(ubar, gamma, method="bicgstab", tol=1e-6, maxit=1000, ndim=None, out=None, history=True,
                    stream=None, space="physical", device=None):
    """deconvolve() for fields in host memory: ``ubar`` is a contiguous CPU
    tensor (pinned memory copies fastest); the library copies it to the GPU,
    solves and copies u* back into ``out`` (a CPU tensor, may be ``ubar``)."""
    import torch
    lib = load()
    ctx = context(device)
    g, batch, _ = _grid(ubar, ndim, gamma, host=True)
    code = method_code(method, space)
    if out is None:
        out = torch.empty_like(ubar)
    if out.shape != ubar.shape or out.dtype != ubar.dtype or out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CPU tensor like u_bar")
    its = np.zeros(batch, dtype=np.int32)
    sts = np.zeros(batch, dtype=np.int32)
    hist = np.full((batch, int(maxit) + 1), np.nan) if history else None
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p()
    st = lib.ad_deconvolve_host(ctx, ctypes.byref(g), ctypes.c_void_p(ubar.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), batch, code, float(tol), int(maxit), ptr(its),
                                ptr(sts), ptr(hist), _stream_ptr(stream))
    _check(st, ctx, per_field=True)
    return Solve(u=out, iterations=its, status=sts, history=hist, true_residual=None,
                 launches=int(lib.ad_last_launch_count(ctx)))


def time_passes(shape, gamma, batch, method="bicgstab", dtype="f32", reps=20, stream=None, device=None,
                space="physical"):
    """Per-launch time (ms) of every pass kernel of one iteration of ``method``,
    measured by the library with CUDA events in the solve's launch shapes.
    Returns a list of dicts (index, kind, op, ms)."""
    lib = load()
    ctx = context(device)
    g = ad_grid()
    g.ndim = len(shape)
    rev = list(reversed(shape)) + [1] * (3 - len(shape))
    for i in range(3):
        g.n[i] = int(rev[i])
    g.dtype = AD_F32 if dtype == "f32" else AD_F64
    g.gamma = float(gamma)
    cnt = ctypes.c_int(0)
    code = method_code(method, space)
    st = lib.ad_time_pass(ctx, ctypes.byref(g), int(batch), code, -1, 1, _stream_ptr(stream),
                          None, None, None, ctypes.byref(cnt))
    _check(st, ctx)
    out = []
    for i in range(cnt.value):
        ms, kind, op = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
        st = lib.ad_time_pass(ctx, ctypes.byref(g), int(batch), code, i, int(reps), _stream_ptr(stream),
                              ctypes.byref(ms), ctypes.byref(kind), ctypes.byref(op), None)
        _check(st, ctx)
        out.append(dict(index=i, kind=PASS_KINDS[kind.value], op=int(op.value), ms=float(ms.value)))
    return out


def time_body(shape, gamma, batch, method="bicgstab", dtype="f32", reps=10, stream=None, device=None,
              space="physical"):
    """Time (ms) of one whole iteration body of ``method`` (all its pass
    launches in order), measured by the library with CUDA events in the
    solve's launch shapes on its internal buffers."""
    lib = load()
    ctx = context(device)
    g = ad_grid()
    g.ndim = len(shape)
    rev = list(reversed(shape)) + [1] * (3 - len(shape))
    for i in range(3):
        g.n[i] = int(rev[i])
    g.dtype = AD_F32 if dtype == "f32" else AD_F64
    g.gamma = float(gamma)
    ms = ctypes.c_double()
    st = lib.ad_time_pass(ctx, ctypes.byref(g), int(batch), method_code(method, space), -2, int(reps),
                          _stream_ptr(stream), ctypes.byref(ms), None, None, None)
    _check(st, ctx)
    return float(ms.value)


def deconvolve_batched(fields, gammas, method="bicgstab", tol=1e-6, maxit=1000, ndims=None, outs=None,
                       history=True, stream=None, space="physical"):
    """Solves G u = u_bar for a list of fields of uneven size in one library
    call (one CUDA graph). ``fields`` is a list of contiguous CUDA tensors,
    each one field ((Ny, Nx) or (Nz, Ny, Nx)); ``gammas`` a list of filter
    strengths. Returns (outputs, iterations, status, histories)."""
    import torch
    lib = load()
    n = len(fields)
    if n == 0:
        return [], np.zeros(0, np.int32), np.zeros(0, np.int32), []
    ctx = context(fields[0].device.index)
    grids = (ad_grid * n)()
    for i, (t, g) in enumerate(zip(fields, gammas)):
        nd = (ndims[i] if ndims else t.dim())
        gi, b, _ = _grid(t, nd, g)
        if b != 1:
            raise ValueError("deconvolve_batched takes one field per tensor")
        grids[i] = gi
    outs = outs if outs is not None else [torch.empty_like(t) for t in fields]
    pin = (ctypes.c_void_p * n)(*[t.data_ptr() for t in fields])
    pout = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
    its = np.zeros(n, dtype=np.int32)
    sts = np.zeros(n, dtype=np.int32)
    hist = [np.full(int(maxit) + 1, np.nan) for _ in range(n)] if history else None
    phist = (ctypes.c_void_p * n)(*[h.ctypes.data for h in hist]) if history else None
    st = lib.ad_deconvolve_batched(ctx, n, grids, pin, pout, method_code(method, space), float(tol), int(maxit),
                                   ctypes.c_void_p(its.ctypes.data), ctypes.c_void_p(sts.ctypes.data),
                                   phist, _stream_ptr(stream))
    _check(st, ctx, per_field=True)
    return outs, its, sts, hist


def autotune(shape=None, gamma=0.1, batch=1, method="bicgstab", dtype="f32", for_batched=False, device=None,
             space="physical"):
    """Tunes the tile widths of the plan for (shape, batch) by timing every
    admissible width per pass (``shape=None``: only set whether batched solves
    tune their plans)."""
    lib = load()
    ctx = context(device)
    g = None
    if shape is not None:
        g = ad_grid()
        g.ndim = len(shape)
        rev = list(reversed(shape)) + [1] * (3 - len(shape))
        for i in range(3):
            g.n[i] = int(rev[i])
        g.dtype = AD_F32 if dtype == "f32" else AD_F64
        g.gamma = float(gamma)
    st = lib.ad_autotune(ctx, ctypes.byref(g) if g is not None else None, int(batch), method_code(method, space),
                         1 if for_batched else 0)
    _check(st, ctx)


# --- learned initial guess ------------------------------------------------------

def guess_init(seed=0, stencil=True, device=None):
    """Initial network weights as a float32 CUDA tensor: the explicit local
    inverse stencil (default) or He-normal."""
    import torch
    lib = load()
    n = int(lib.ad_guess_weight_count())
    w = np.zeros(n, dtype=np.float32)
    st = lib.ad_guess_init(ctypes.c_void_p(w.ctypes.data), n, int(seed), 1 if stencil else 0)
    if st != AD_OK:
        raise GadError(st, "ad_guess_init")
    return torch.from_numpy(w).to("cuda" if device is None else device)


def _guess_grid(t, gamma):
    g, b, _ = _grid(t, 3, gamma)
    return g, b


def guess_infer(weights, ubar, gamma, out=None, stream=None):
    """u0 = u_bar + sigma A CNN(u_bar / sigma) for 3D float32 fields (batch first)."""
    import torch
    lib = load()
    ctx = context(ubar.device.index)
    g, b = _guess_grid(ubar, gamma)
    out = torch.empty_like(ubar) if out is None else out
    st = lib.ad_guess_infer(ctx, ctypes.byref(g), ctypes.c_void_p(weights.data_ptr()),
                            ctypes.c_void_p(ubar.data_ptr()), ctypes.c_void_p(out.data_ptr()), b, _stream_ptr(stream))
    _check(st, ctx)
    return out


def guess_time_conv(shape, batch, gamma=0.01, reps=5, stream=None, device=None):
    """(ms per launch, ran on tcgen05) of one forward 32 -> 32 layer of the
    learned guess's network for fields of ``shape`` (Z, Y, X) and ``batch``,
    timed by the library with CUDA events in inference's launch shape."""
    lib = load()
    ctx = context(device)
    g = ad_grid()
    g.ndim = 3
    for i, n in enumerate(reversed(shape)):
        g.n[i] = int(n)
    g.dtype = AD_F32
    g.gamma = float(gamma)
    ms, tc = ctypes.c_double(), ctypes.c_int()
    st = lib.ad_guess_time_conv(ctx, ctypes.byref(g), int(batch), int(reps), _stream_ptr(stream), ctypes.byref(ms),
                                ctypes.byref(tc))
    _check(st, ctx)
    return float(ms.value), bool(tc.value)


def guess_grad(weights, ubar, utrue, gamma, stream=None):
    """(loss, gradient) of the batch-mean relative MSE for one batch."""
    import torch
    lib = load()
    ctx = context(ubar.device.index)
    g, b = _guess_grid(ubar, gamma)
    grad = torch.empty_like(weights)
    loss = ctypes.c_double(0.0)
    st = lib.ad_guess_grad(ctx, ctypes.byref(g), ctypes.c_void_p(weights.data_ptr()), ctypes.c_void_p(ubar.data_ptr()),
                           ctypes.c_void_p(utrue.data_ptr()), b, ctypes.c_void_p(grad.data_ptr()), ctypes.byref(loss),
                           _stream_ptr(stream))
    _check(st, ctx)
    return loss.value, grad


def guess_train(weights, ubar, utrue, gamma, epochs=20, batch=8, lr=2e-5, seed=0, stream=None):
    """Trains ``weights`` (updated in place) on pairs [npairs, Z, Y, X]; returns
    the per-epoch mean losses."""
    lib = load()
    ctx = context(ubar.device.index)
    g, n = _guess_grid(ubar, gamma)
    hist = np.zeros(max(int(epochs), 1))
    st = lib.ad_guess_train(ctx, ctypes.byref(g), n, ctypes.c_void_p(ubar.data_ptr()), ctypes.c_void_p(utrue.data_ptr()),
                            int(epochs), int(batch), float(lr), int(seed), ctypes.c_void_p(weights.data_ptr()),
                            ctypes.c_void_p(hist.ctypes.data), _stream_ptr(stream))
    _check(st, ctx)
    return hist[: int(epochs)]


# --- closure and statistics of deconvolved fields ---------------------------

def _velocity_grid(u, ncomp, ndim, gamma=1.0):
    """Grid of a [..., ncomp, *grid] tensor and the number of velocities."""
    g, batch, shape = _grid(u, ndim, gamma)
    if batch % ncomp != 0:
        raise ValueError("the leading axes must hold a multiple of ncomp = %d fields" % ncomp)
    return g, batch // ncomp, shape


def closure(ubar, ustar, gamma, ncomp=None, ndim=None, out=None, stream=None):
    """Sub-filter stress tau_ij = u_bar_i u_bar_j - G(u*_i u*_j), i <= j (Eq.
    fge3 with the deconvolved estimate), for tensors shaped [..., ncomp, *grid]
    (ncomp defaults to ndim). Returns [..., npairs, *grid]."""
    import torch
    lib = load()
    ctx = context(ubar.device.index)
    if ndim is None:
        ndim = 3 if ubar.dim() >= 4 and ubar.shape[-4] == 3 else 2
    ncomp = ndim if ncomp is None else int(ncomp)
    if ustar.shape != ubar.shape or ustar.dtype != ubar.dtype or not ustar.is_contiguous():
        raise ValueError("ustar must match ubar in shape, dtype and layout")
    g, nvel, shape = _velocity_grid(ubar, ncomp, ndim, gamma)
    npairs = ncomp * (ncomp + 1) // 2
    lead = tuple(ubar.shape[:ubar.dim() - ndim - 1])
    if out is None:
        out = torch.empty(lead + (npairs,) + tuple(shape), dtype=ubar.dtype, device=ubar.device)
    st = lib.ad_closure(ctx, ctypes.byref(g), nvel, ncomp, ctypes.c_void_p(ubar.data_ptr()),
                        ctypes.c_void_p(ustar.data_ptr()), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
    _check(st, ctx)
    return out


def spectrum(u, nbins, ncomp=1, ndim=None, stream=None):
    """Shell-summed energy spectrum E[g][k], k < nbins, of the fields of ``u``
    taken in groups of ncomp (float64 numpy array [groups, nbins])."""
    lib = load()
    ctx = context(u.device.index)
    g, batch, _ = _grid(u, ndim, 1.0)
    if batch % ncomp != 0:
        raise ValueError("number of fields must be a multiple of ncomp")
    e = np.zeros((batch // ncomp, int(nbins)), dtype=np.float64)
    st = lib.ad_spectrum(ctx, ctypes.byref(g), batch, int(ncomp), ctypes.c_void_p(u.data_ptr()), int(nbins),
                         ctypes.c_void_p(e.ctypes.data), _stream_ptr(stream))
    _check(st, ctx)
    return e


def histogram(x, lo, hi, nbins, stream=None):
    """Bin counts of the values of ``x`` (float32 or float64 CUDA tensor):
    (counts[nbins], below, above, nan)."""
    import torch
    lib = load()
    ctx = context(x.device.index)
    if x.dtype not in (torch.float32, torch.float64) or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32/float64 CUDA tensor")
    c = np.zeros(int(nbins) + 3, dtype=np.int64)
    st = lib.ad_histogram(ctx, AD_F64 if x.dtype == torch.float64 else AD_F32, x.numel(),
                          ctypes.c_void_p(x.data_ptr()), float(lo), float(hi), int(nbins),
                          ctypes.c_void_p(c.ctypes.data), _stream_ptr(stream))
    _check(st, ctx)
    return c[:nbins], int(c[nbins]), int(c[nbins + 1]), int(c[nbins + 2])


def curl(u, ndim=None, out=None, stream=None):
    """Vorticity of velocities shaped [..., ndim, *grid]: 2D -> [..., *grid]
    (dv/dx - du/dy), 3D -> [..., 3, *grid]."""
    import torch
    lib = load()
    ctx = context(u.device.index)
    if ndim is None:
        ndim = 3 if u.dim() >= 4 and u.shape[-4] == 3 else 2
    g, nvel, shape = _velocity_grid(u, ndim, ndim)
    lead = tuple(u.shape[:u.dim() - ndim - 1])
    if out is None:
        oshape = lead + tuple(shape) if ndim == 2 else lead + (3,) + tuple(shape)
        out = torch.empty(oshape, dtype=u.dtype, device=u.device)
    st = lib.ad_curl(ctx, ctypes.byref(g), nvel, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                     _stream_ptr(stream))
    _check(st, ctx)
    return out
