"""Tolerances for comparing Krylov iterates with the oracle.

A Krylov iterate after several passes, and the number of passes to a
tolerance, depend on rounding: two correct implementations that round
differently drift apart, the more so the more passes and the worse the
conditioning of G. The GPU path evaluates G with FFTs in the field's
precision, so the comparison is made against the oracle run with its G
evaluated in that same precision (a float32 single-precision FFT for float32
fields; numpy's float64 FFT for float64 fields) -- the integer outcome (the
pass count) is then decided in the kernel's precision on both sides. The
oracle's own sensitivity is measured, not guessed: G commutes with periodic
shifts, so G(x) = shift^-1 G(shift x) for every shift, and each shift is an
equally valid evaluation that rounds differently. The spread of the oracle
over a few shifts is its rounding sensitivity at the path's precision.

  * fields: the GPU must agree with the precision-matched oracle to
    max(base, 10 * spread), base = 1e-5 (float32) or 1e-12 (float64);
  * pass counts to a tolerance: exact if every shifted oracle run gives the
    same count; otherwise within the observed range widened by that range on
    each side, [min - R - 1, max + R + 1] with R = max - min (a count that is
    chaotic under rounding -- BiCGSTAB at gamma = 0.01 spans tens of passes --
    cannot be bracketed by the extremes of a few samples).

The oracle's code is not changed: these helpers wrap the filter function the
oracle's solvers call.
"""

import contextlib

import numpy as np
import scipy.fft

import oracle
import oracle.solvers as _osv

BASE = {"f32": 1e-5, "f64": 1e-12}
SHIFTS = [(0, 0, 0), (1, 3, 2), (5, 2, 7), (11, 7, 3)]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _g_f32(x, gamma):
    """Eq. df2 applied with single-precision FFTs (float32 storage of the
    spectrum and of the transfer function)."""
    shape = x.shape
    gh = oracle.transfer_function(shape, gamma)[..., : shape[-1] // 2 + 1].astype(np.float32)
    X = scipy.fft.rfftn(np.asarray(x, dtype=np.float32))
    return scipy.fft.irfftn(X * gh, s=shape).astype(np.float64)


@contextlib.contextmanager
def precision_filter(precision, shift):
    """Within the block the oracle's solvers evaluate G in `precision` on
    the input shifted periodically by `shift` (and shifted back)."""
    clean = _osv.filter_field
    base = _g_f32 if precision == "f32" else clean

    def g(x, gamma):
        ax = tuple(range(x.ndim))
        sh = tuple(shift[: x.ndim])
        return np.roll(base(np.roll(x, sh, ax), gamma), tuple(-s for s in sh), ax)

    _osv.filter_field = g
    try:
        yield
    finally:
        _osv.filter_field = clean


def ensemble_runs(method, ub, gamma, tol, maxit, precision, u0=None, shifts=SHIFTS):
    """The precision-matched oracle (first shift) and its shifted twins."""
    out = []
    for sh in shifts:
        with precision_filter(precision, sh):
            out.append(oracle.solve(method, ub, gamma, tol=tol, maxit=maxit, u0=u0, precision=precision))
    return out[0], out[1:]


def field_tolerance(base, runs, precision):
    spread = max(rel(r.u, base.u) for r in runs)
    return max(BASE[precision], 10.0 * spread), spread


def history_tolerance(base, runs, floor):
    n = len(base.history)
    spread = max(float(np.max(np.abs(r.history[:n] / base.history[: len(r.history)] - 1)))
                 for r in runs if len(r.history) == n)
    return max(floor, 10.0 * spread)


def count_ok(n_gpu, base, runs):
    counts = [base.iterations] + [r.iterations for r in runs]
    lo, hi = min(counts), max(counts)
    if lo == hi:
        return n_gpu == lo, counts
    r = hi - lo
    return lo - r - 1 <= n_gpu <= hi + r + 1, counts


# --- the spectral-space variant ------------------------------------------------
# The oracle's space="spectral" mode stores the half spectra (complex64 in
# float32 mode) but transforms in float64; the GPU transforms in the field's
# precision. These helpers make the transforms precision-matched and build the
# ensemble from periodic shifts of the input itself: a shift is a phase
# rotation of every mode, which changes how each stored coefficient rounds
# (whereas the storage rounding of a real field commutes with shifts).

@contextlib.contextmanager
def spectral_transforms(precision):
    """Within the block the oracle's spectral space transforms u_bar, u0 and
    u with single-precision FFTs when `precision` is f32."""
    if precision != "f32":
        yield
        return
    cls = _osv._Spectral
    to0, back0 = cls.to, cls.back

    def to(self, x):
        return scipy.fft.rfftn(np.asarray(x, dtype=np.float32)).astype(np.complex128)

    def back(self, x):
        y = scipy.fft.irfftn(np.asarray(x).astype(np.complex64), s=self.shape, axes=tuple(range(len(self.shape))))
        return y.astype(np.float64)

    cls.to, cls.back = to, back
    try:
        yield
    finally:
        cls.to, cls.back = to0, back0


# Wider shifts than SHIFTS: a phase rotation by a large shift re-rounds every
# stored coefficient, and at gamma = 0.01 a few samples underestimate how far
# equally valid float32 runs of BiCGSTAB drift apart.
SHIFTS_SPECTRAL = [(0, 0, 0), (1, 3, 2), (5, 2, 7), (11, 7, 3), (37, 101, 13), (64, 17, 29), (90, 211, 5),
                   (123, 45, 61), (200, 133, 77)]


def ensemble_runs_spectral(method, ub, gamma, tol, maxit, precision, u0=None, shifts=SHIFTS_SPECTRAL):
    """The precision-matched spectral-space oracle on u_bar and on shifted
    copies of it (results shifted back)."""
    out = []
    ax = tuple(range(ub.ndim))
    with spectral_transforms(precision):
        for sh in shifts:
            s = tuple(sh[: ub.ndim])
            back = tuple(-x for x in s)
            r = oracle.solve(method, np.roll(ub, s, ax), gamma, tol=tol, maxit=maxit,
                             u0=None if u0 is None else np.roll(u0, s, ax), precision=precision, space="spectral")
            r.u = np.roll(r.u, back, ax)
            out.append(r)
    return out[0], out[1:]
