"""Iterative solvers for the approximate-deconvolution problem G u = u_bar
(Section 3, Eq. tau3), written step by step in the paper's order and notation.
TEST INFRASTRUCTURE ONLY (see the package docstring).

  van_cittert        -- Algorithm 1 (Van Cittert / Richardson, Eq. adm2, Eq. ric)
  steepest_descent   -- Algorithm 2 (Eq. sd, Eq. sd-a)
  conjugate_gradient -- Algorithm 3 (Eq. cg1 ... Eq. cg-b)
  bicgstab           -- Algorithm 4

Readings of points the paper leaves open (each applies to every method):
  * Inner product (a, b) = integral of a b dx is taken as the plain sum
    sum_i a_i b_i; the cell volume cancels in every ratio (Eq. inner).
  * The residual is normalised by the initial residual of the plain start,
    h_n = ||r_n||_2 / ||u_bar - G u_bar||_2 (Section 4.1: "normalized with
    respect to the initial residual"); with an explicit starting guess u0 the
    denominator stays ||u_bar - G u_bar||_2.
  * The loop "while n < N" is driven by (tol, maxit): h_0 is tested before
    the loop (h_0 <= tol -> 0 iterations); after every completed pass h_{n+1}
    is computed from the recurrence residual and the solve stops at the first
    h <= tol (STATUS_OK) or when maxit passes are done (STATUS_MAXIT).
    Fixed-N runs are tol = 0, maxit = N. ``iterations`` counts completed
    passes; N passes of Algorithm 1 give u_N = sum_{n=0}^{N} (I-G)^n u_bar.
  * BiCGSTAB breakdown (not discussed in the paper): if ||s||/ref <= tol or
    (t, t) = 0, the pass ends with u += alpha p, r = s and the solve returns
    STATUS_OK; if rho_{n+1} = 0, (f0, q) = 0 or a scalar is not finite the
    solve returns STATUS_BREAKDOWN with u from the last full pass.
  * precision="f32" emulates float32 storage of every vector (rounded after
    each update and after each application of G) and float32 scalars where
    they multiply vectors; inner products and scalar recurrences stay in
    float64. precision="f64" is plain float64 throughout.
  * space="spectral" runs the same steps on the half spectra of the vectors
    (numpy rfftn layout): G is diagonal in Fourier space (Eq. df2), so it
    becomes a pointwise multiply by G_hat, and the inner product becomes the
    Parseval sum (a, b) = (1/P) sum_k w(k_x) Re(a_hat conj(b_hat)) with
    w = 1 on the k_x = 0 and k_x = N_x/2 planes and 2 elsewhere. u_bar (and
    u0) are transformed once at the start and u once at the end; the
    iterates equal those of space="physical" in exact arithmetic. In f32
    mode the complex vectors are rounded to complex64.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .spectral import filter_field, transfer_function

STATUS_OK = 0
STATUS_MAXIT = 1
STATUS_BREAKDOWN = 2
STATUS_NONFINITE = -2


@dataclass
class SolveResult:
    u: np.ndarray
    iterations: int
    status: int
    history: np.ndarray          # h_0 .. h_iterations
    true_residual: float         # ||u_bar - G u|| / ref for the returned u
    trace: dict = field(default_factory=dict)


def inner(a, b):
    """(a, b) = sum_i a_i b_i in float64 (Eq. inner, unweighted)."""
    return float(np.dot(np.ravel(a).astype(np.float64), np.ravel(b).astype(np.float64)))


class _Arith:
    """Rounding rules of the chosen storage precision."""

    def __init__(self, precision):
        if precision not in ("f64", "f32"):
            raise ValueError("precision must be 'f64' or 'f32'")
        self.f32 = precision == "f32"

    def vec(self, x):
        x = np.asarray(x)
        if np.iscomplexobj(x):
            x = x.astype(np.complex128)
            return x.astype(np.complex64).astype(np.complex128) if self.f32 else x
        x = x.astype(np.float64)
        return x.astype(np.float32).astype(np.float64) if self.f32 else x

    def scal(self, a):
        return float(np.float32(a)) if self.f32 else float(a)


class _Physical:
    """Vectors are fields on the grid; G by FFT (Eq. df2), plain sums (Eq. inner)."""

    def __init__(self, shape, gamma):
        self.gamma = gamma

    def G(self, x):
        return filter_field(x, self.gamma)

    def inner(self, a, b):
        return inner(a, b)

    def to(self, x):
        return x

    def back(self, x):
        return x


class _Spectral:
    """Vectors are half spectra (rfftn over all axes, last axis halved); G is
    the pointwise multiply by G_hat and (a, b) the weighted Parseval sum."""

    def __init__(self, shape, gamma):
        self.shape = tuple(shape)
        nxh = self.shape[-1] // 2 + 1
        self.gh = transfer_function(self.shape, gamma)[..., :nxh]
        w = np.full(nxh, 2.0)
        w[0] = 1.0
        if self.shape[-1] % 2 == 0:
            w[-1] = 1.0
        self.w = w
        self.p = float(np.prod(self.shape))

    def G(self, x):
        return self.gh * x

    def inner(self, a, b):
        return float(np.sum(self.w * np.real(a * np.conj(b)))) / self.p

    def to(self, x):
        return np.fft.rfftn(np.asarray(x, dtype=np.float64))

    def back(self, x):
        return np.fft.irfftn(x, s=self.shape, axes=tuple(range(len(self.shape))))


def _space(space, shape, gamma):
    if space == "physical":
        return _Physical(shape, gamma)
    if space == "spectral":
        return _Spectral(shape, gamma)
    raise ValueError("space must be 'physical' or 'spectral'")


def _start(ubar, gamma, u0, ar, sp):
    ubar = ar.vec(ubar)
    b = ar.vec(sp.to(ubar))
    g_b = ar.vec(sp.G(b))
    ref = math.sqrt(sp.inner(ar.vec(b - g_b), ar.vec(b - g_b)))
    u = b.copy() if u0 is None else ar.vec(sp.to(ar.vec(u0)))
    r = ar.vec(b - (g_b if u0 is None else ar.vec(sp.G(u))))
    return ubar, ref, u, r


def _h(rr, ref):
    return 0.0 if ref == 0.0 else math.sqrt(max(rr, 0.0)) / ref


def _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar):
    u = ar.vec(sp.back(u))
    res = ubar - filter_field(u, gamma)
    tr = math.sqrt(inner(res, res)) / ref if ref > 0 else math.sqrt(inner(res, res))
    return SolveResult(u=u, iterations=n, status=status,
                       history=np.asarray(hist, dtype=np.float64),
                       true_residual=tr, trace=trace)


def _pre_loop(rr0, ref, tol, maxit):
    """Status decided before the first pass, or None to enter the loop."""
    h0 = _h(rr0, ref)
    if not math.isfinite(rr0) or not math.isfinite(ref):
        return STATUS_NONFINITE, h0
    if h0 <= tol:
        return STATUS_OK, h0
    if maxit <= 0:
        return STATUS_MAXIT, h0
    return None, h0


def van_cittert(ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, space="physical"):
    """Algorithm 1: u_{n+1} = u_n + r_n, d_n = G r_n, r_{n+1} = r_n - d_n,
    starting from u_0 = u_bar, r_0 = u_bar - G u_0 (Eq. adm2, Eq. res, Eq. ric)."""
    ar = _Arith(precision)
    sp = _space(space, np.shape(ubar), gamma)
    ubar, ref, u, r = _start(ubar, gamma, u0, ar, sp)
    rr = sp.inner(r, r)
    status, h0 = _pre_loop(rr, ref, tol, maxit)
    hist = [h0]
    trace = {"r": [r.copy()]} if record else {}
    n = 0
    while status is None:
        u = ar.vec(u + r)                        # u_{n+1} = u_n + r_n
        d = ar.vec(sp.G(r))       # d_n = G r_n
        r = ar.vec(r - d)                        # r_{n+1} = r_n - d_n
        n += 1
        rr = sp.inner(r, r)
        h = _h(rr, ref)
        hist.append(h)
        if record:
            trace["r"].append(r.copy())
        if not math.isfinite(rr):
            status = STATUS_BREAKDOWN
        elif h <= tol:
            status = STATUS_OK
        elif n >= maxit:
            status = STATUS_MAXIT
    return _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar)


def steepest_descent(ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, space="physical"):
    """Algorithm 2: d_n = G r_n, alpha_n = (r_n, r_n)/(r_n, d_n) (Eq. sd-a),
    u_{n+1} = u_n + alpha_n r_n (Eq. sd), r_{n+1} = r_n - alpha_n d_n (Eq. rnew1)."""
    ar = _Arith(precision)
    sp = _space(space, np.shape(ubar), gamma)
    ubar, ref, u, r = _start(ubar, gamma, u0, ar, sp)
    rr = sp.inner(r, r)
    status, h0 = _pre_loop(rr, ref, tol, maxit)
    hist = [h0]
    trace = {"alpha": []} if record else {}
    n = 0
    while status is None:
        d = ar.vec(sp.G(r))
        rd = sp.inner(r, d)
        alpha = rr / rd if rd != 0.0 else float("nan")
        if not math.isfinite(alpha):
            status = STATUS_BREAKDOWN
            break
        a = ar.scal(alpha)
        u = ar.vec(u + a * r)
        r = ar.vec(r - a * d)
        n += 1
        rr = sp.inner(r, r)
        h = _h(rr, ref)
        hist.append(h)
        if record:
            trace["alpha"].append(alpha)
        if not math.isfinite(rr):
            status = STATUS_BREAKDOWN
        elif h <= tol:
            status = STATUS_OK
        elif n >= maxit:
            status = STATUS_MAXIT
    return _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar)


def conjugate_gradient(ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, space="physical"):
    """Algorithm 3: p_0 = r_0, rho_0 = (r_0, r_0); per pass d_n = G p_n,
    alpha_n = rho_n/(p_n, d_n) (Eq. cg-alpha), u_{n+1} = u_n + alpha_n p_n,
    r_{n+1} = r_n - alpha_n d_n (Eq. rnew2), rho_{n+1} = (r_{n+1}, r_{n+1}),
    beta_n = rho_{n+1}/rho_n (Eq. cg-b), p_{n+1} = r_{n+1} + beta_n p_n (Eq. cg4)."""
    ar = _Arith(precision)
    sp = _space(space, np.shape(ubar), gamma)
    ubar, ref, u, r = _start(ubar, gamma, u0, ar, sp)
    p = r.copy()
    rho = sp.inner(r, r)
    status, h0 = _pre_loop(rho, ref, tol, maxit)
    hist = [h0]
    trace = {"r": [r.copy()], "p": [p.copy()], "d": [], "alpha": [], "beta": [], "u": [u.copy()]} if record else {}
    n = 0
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
        rho_new = sp.inner(r, r)
        beta = rho_new / rho
        p = ar.vec(r + ar.scal(beta) * p)
        rho = rho_new
        n += 1
        h = _h(rho, ref)
        hist.append(h)
        if record:
            trace["d"].append(d.copy())
            trace["r"].append(r.copy())
            trace["p"].append(p.copy())
            trace["u"].append(u.copy())
            trace["alpha"].append(alpha)
            trace["beta"].append(beta)
        if not math.isfinite(rho):
            status = STATUS_BREAKDOWN
        elif h <= tol:
            status = STATUS_OK
        elif n >= maxit:
            status = STATUS_MAXIT
    return _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar)


def bicgstab(ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, space="physical"):
    """Algorithm 4: f_0 = r_0, p_0 = q_0 = 0, alpha_0 = omega_0 = rho_0 = 1; per pass
    rho_{n+1} = (f_0, r_n), beta_n = (alpha_n/omega_n)(rho_{n+1}/rho_n),
    p_{n+1} = r_n + beta_n (p_n - omega_n q_n), q_{n+1} = G p_{n+1},
    alpha_{n+1} = rho_{n+1}/(f_0, q_{n+1}), s_n = r_n - alpha_{n+1} q_{n+1},
    t_n = G s_n, omega_{n+1} = (s_n, t_n)/(t_n, t_n),
    u_{n+1} = u_n + alpha_{n+1} p_{n+1} + omega_{n+1} s_n,
    r_{n+1} = s_n - omega_{n+1} t_n."""
    ar = _Arith(precision)
    sp = _space(space, np.shape(ubar), gamma)
    ubar, ref, u, r = _start(ubar, gamma, u0, ar, sp)
    f0 = r.copy()
    p = np.zeros_like(r)
    q = np.zeros_like(r)
    alpha = omega = rho = 1.0
    rr = sp.inner(r, r)
    status, h0 = _pre_loop(rr, ref, tol, maxit)
    hist = [h0]
    trace = {"s": [], "t": [], "r": [r.copy()], "alpha": [], "omega": [], "rho": []} if record else {}
    n = 0
    while status is None:
        rho_new = sp.inner(f0, r)
        if rho_new == 0.0 or not math.isfinite(rho_new):
            status = STATUS_BREAKDOWN
            break
        beta = (alpha / omega) * (rho_new / rho)
        if not math.isfinite(beta):
            status = STATUS_BREAKDOWN
            break
        p = ar.vec(r + ar.scal(beta) * ar.vec(p - ar.scal(omega) * q))
        q = ar.vec(sp.G(p))
        fq = sp.inner(f0, q)
        if fq == 0.0 or not math.isfinite(fq):
            status = STATUS_BREAKDOWN
            break
        alpha = rho_new / fq
        s = ar.vec(r - ar.scal(alpha) * q)
        ss = sp.inner(s, s)
        t = ar.vec(sp.G(s))
        tt = sp.inner(t, t)
        early = _h(ss, ref) <= tol or tt == 0.0
        omega = 0.0 if early else sp.inner(s, t) / tt
        if not math.isfinite(omega):
            status = STATUS_BREAKDOWN
            break
        u = ar.vec(ar.vec(u + ar.scal(alpha) * p) + ar.scal(omega) * s)
        r = ar.vec(s - ar.scal(omega) * t)
        rho = rho_new
        n += 1
        rr = sp.inner(r, r)
        h = _h(rr, ref)
        hist.append(h)
        if record:
            trace["s"].append(s.copy())
            trace["t"].append(t.copy())
            trace["r"].append(r.copy())
            trace["alpha"].append(alpha)
            trace["omega"].append(omega)
            trace["rho"].append(rho_new)
        if not math.isfinite(rr):
            status = STATUS_BREAKDOWN
        elif early or h <= tol:
            status = STATUS_OK
        elif n >= maxit:
            status = STATUS_MAXIT
    return _finish(ubar, gamma, u, ref, n, status, hist, trace, sp, ar)


_METHODS = {
    "vancittert": van_cittert,
    "sd": steepest_descent,
    "cg": conjugate_gradient,
    "bicgstab": bicgstab,
}


def solve(method, ubar, gamma, tol=0.0, maxit=5, u0=None, precision="f64", record=False, space="physical"):
    """Dispatch by method name: 'vancittert', 'sd', 'cg', 'bicgstab', or 'pcg'
    (preconditioned CG, precond.py)."""
    if method == "pcg":
        from .precond import preconditioned_cg
        return preconditioned_cg(ubar, gamma, tol=tol, maxit=maxit, u0=u0, precision=precision, record=record,
                                 space=space)
    return _METHODS[method](ubar, gamma, tol=tol, maxit=maxit, u0=u0,
                            precision=precision, record=record, space=space)
