"""Preconditioned conjugate gradient for G u = u_bar with a local
finite-difference approximation of G^{-1} as the preconditioner.
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves Eq. tau3 with unpreconditioned Krylov methods (Algorithms
1-4). This module adds the preconditioned variant of Algorithm 3; the paper
has no counterpart, so the definitions below are the textbook ones, written
out in full:

  * The filter is G = (I - delta^2 Laplacian)^{-1} with delta = 1/k_c
    (Section 4, Eq. df). Its exact inverse is a differential operator, and the
    preconditioner replaces the Laplacian there by the second-order central
    difference on the 2*pi-periodic grid (h_d = 2*pi/N_d per axis):
        M x = x + sum_d c_d (2 x_i - x_{i+e_d} - x_{i-e_d}),
        c_d = delta^2 / h_d^2 = (N_d / (2 pi k_c))^2.
    M is symmetric positive definite (M >= I) and, on a periodic grid, has the
    Fourier symbol M_hat(k) = 1 + sum_d 4 c_d sin^2(k_d h_d / 2). M and G
    commute (both are diagonal in Fourier space), so M G is symmetric positive
    definite with eigenvalues M_hat(k) G_hat(k) in [(2/pi)^2, 1]: a condition
    number of at most pi^2/4 instead of 1 + max|k|^2/k_c^2.
  * Preconditioned CG (the standard form with an approximate inverse M):
        r_0 = u_bar - G u_0, z_0 = M r_0, p_0 = z_0, rho_0 = (r_0, z_0);
        per pass  d_n = G p_n, alpha_n = rho_n / (p_n, d_n),
                  u_{n+1} = u_n + alpha_n p_n, r_{n+1} = r_n - alpha_n d_n,
                  z_{n+1} = M r_{n+1}, rho_{n+1} = (r_{n+1}, z_{n+1}),
                  beta_n = rho_{n+1} / rho_n, p_{n+1} = z_{n+1} + beta_n p_n.
    With M = I these are exactly the steps of Algorithm 3.
  * precision="f32" evaluates M in float32 as apply_preconditioner_f32
    states (the other float32 rules are those of solvers.py).
  * Stopping, counting and normalisation follow the rules of solvers.py: the
    stop test uses the unpreconditioned recurrence residual,
    h_n = ||r_n|| / ||u_bar - G u_bar||; rho_n <= 0 or a non-finite scalar is a
    breakdown.
"""

from __future__ import annotations

import math

import numpy as np

from .solvers import (STATUS_BREAKDOWN, STATUS_MAXIT, STATUS_OK, _Arith, _finish, _h, _pre_loop, _space,
                      _start)
from .spectral import cutoff_wavenumber


def stencil_coefficients(shape, gamma):
    """c_d = (delta / h_d)^2 = (N_d / (2 pi k_c))^2 per array axis (C order)."""
    kc = cutoff_wavenumber(shape, gamma)
    return tuple((n / (2.0 * math.pi * kc)) ** 2 for n in shape)


def apply_preconditioner(x, gamma):
    """M x = x + sum_d c_d (2 x - x shifted by +1 - x shifted by -1) along each
    axis d, periodic (np.roll), in float64."""
    x = np.asarray(x, dtype=np.float64)
    out = x.copy()
    for d, c in enumerate(stencil_coefficients(x.shape, gamma)):
        out += c * (2.0 * x - np.roll(x, 1, axis=d) - np.roll(x, -1, axis=d))
    return out


def apply_preconditioner_f32(x, gamma):
    """M x in float32 arithmetic, each operation rounded once, in the order
    z = ((x + c_x d_x) + c_y d_y) + c_z d_z with d = (2 x - left) - right along
    each axis (x = last array axis first) and c_d rounded to float32: the
    evaluation order a float32 implementation of M uses, so that the
    float32-storage mode of preconditioned_cg sees the same rounding."""
    x = np.asarray(x, dtype=np.float32)
    cs = stencil_coefficients(x.shape, gamma)
    two = x + x
    z = x.copy()
    for axis in reversed(range(x.ndim)):
        d = (two - np.roll(x, 1, axis=axis)) - np.roll(x, -1, axis=axis)
        z = z + np.float32(cs[axis]) * d
    return z.astype(np.float64)


def preconditioner_symbol(shape, gamma):
    """M_hat(k) = 1 + sum_d 4 c_d sin^2(pi k_d / N_d) on the full FFT grid."""
    cs = stencil_coefficients(shape, gamma)
    axes = [np.fft.fftfreq(n, d=1.0 / n) for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    out = np.ones(tuple(shape))
    for c, k, n in zip(cs, grids, shape):
        out += 4.0 * c * np.sin(math.pi * k / n) ** 2
    return out


def preconditioned_cg(ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, precond=True,
                      space="physical"):
    """The preconditioned CG iteration of the module docstring. precond=False
    uses M = I (Algorithm 3 itself). space="spectral" runs the same steps on
    the half spectra (solvers.py's spectral space): M is circulant, so it
    becomes the pointwise multiply by M_hat, and the iterates equal the
    physical-space ones in exact arithmetic."""
    ar = _Arith(precision)
    shape = np.shape(ubar)
    sp = _space(space, shape, gamma)
    ubar, ref, u, r = _start(ubar, gamma, u0, ar, sp)
    if not precond:
        M = lambda x: np.asarray(x)                            # noqa: E731
    elif space == "spectral":
        mh = preconditioner_symbol(shape, gamma)[..., : shape[-1] // 2 + 1]
        M = lambda x: mh * x                                   # noqa: E731
    elif ar.f32:
        M = lambda x: apply_preconditioner_f32(x, gamma)       # noqa: E731
    else:
        M = lambda x: apply_preconditioner(x, gamma)           # noqa: E731
    rr = sp.inner(r, r)
    status, h0 = _pre_loop(rr, ref, tol, maxit)
    hist = [h0]
    trace = {"r": [r.copy()], "z": [], "p": [], "d": [], "alpha": [], "beta": []} if record else {}
    n = 0
    z = p = None
    rho = 0.0
    if status is None:
        z = ar.vec(M(r))
        rho = sp.inner(r, z)
        p = z.copy()
        if record:
            trace["z"].append(z.copy())
            trace["p"].append(p.copy())
        if not (rho > 0.0) or not math.isfinite(rho):
            status = STATUS_BREAKDOWN
    while status is None:
        d = ar.vec(sp.G(p))
        pd = sp.inner(p, d)
        alpha = rho / pd if pd != 0.0 else float("nan")
        if not math.isfinite(alpha):
            status = STATUS_BREAKDOWN
            break
        a = ar.scal(alpha)
        u = ar.vec(u + a * p)
        r = ar.vec(r - a * d)
        n += 1
        rr = sp.inner(r, r)
        h = _h(rr, ref)
        hist.append(h)
        if record:
            trace["d"].append(d.copy())
            trace["r"].append(r.copy())
            trace["alpha"].append(alpha)
        if not math.isfinite(rr):
            status = STATUS_BREAKDOWN
            break
        if h <= tol:
            status = STATUS_OK
            break
        if n >= maxit:
            status = STATUS_MAXIT
            break
        z = ar.vec(M(r))
        rho_new = sp.inner(r, z)
        if not (rho_new > 0.0) or not math.isfinite(rho_new):
            status = STATUS_BREAKDOWN
            break
        beta = rho_new / rho
        p = ar.vec(z + ar.scal(beta) * p)
        rho = rho_new
        if record:
            trace["z"].append(z.copy())
            trace["p"].append(p.copy())
            trace["beta"].append(beta)
    return _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar)
