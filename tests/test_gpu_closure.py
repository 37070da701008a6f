"""GPU parity of the closure and statistics entry points (ad_closure,
ad_spectrum, ad_histogram, ad_curl) against the CPU oracle
(oracle/closure.py) through the C ABI.

Tolerances, derived from the arithmetic:
  * stress: tau_ij = u_bar_i u_bar_j - G(u*_i u*_j) is a difference of
    products; the float32 path rounds the product (1 ulp), evaluates G with
    float32 FFTs (a few ulps times log N of |u*_i u*_j|) and forms the
    difference with one fused multiply-add, so
    ||tau_gpu - tau|| <= 16 eps (||u*_i u*_j|| + ||u_bar_i u_bar_j||) with
    eps = 2^-24 (2^-53 for float64 fields);
  * spectrum: float32 transforms give each shell sum to a relative 1e-5 plus
    an absolute floor of 1e-6 of the total energy (float64: 1e-11, 1e-14);
  * histogram: bit-exact integer counts (the bin is decided in the data's
    precision on both sides);
  * vorticity: 1e-5 relative L2 (float32), 1e-12 (float64).
"""

import numpy as np
import pytest

import oracle
from oracle import closure as oc
from synth import fields

pytestmark = pytest.mark.gpu

EPS = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}


def _to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _velocity(shape, seed):
    if len(shape) == 3:
        return fields.random_velocity_field(shape, seed, fields.spectrum_3d_kolmogorov)
    # 2D: a solenoidal velocity from a stream function with a k^-3 spectrum
    psi = fields.random_scalar_field(shape, seed, fields.spectrum_2d_kraichnan)
    return np.stack([-oc.derivative(psi, 0), oc.derivative(psi, 1)])


def _check_stress(gpu, ub, us, gamma, dtype):
    ref = oc.closure_stress(ub, us, gamma)
    for p, (i, j) in enumerate(oc.pair_list(ub.shape[0])):
        bound = 16 * EPS[dtype] * (np.linalg.norm(us[i] * us[j]) + np.linalg.norm(ub[i] * ub[j]))
        err = np.linalg.norm(gpu[p] - ref[p])
        assert err <= bound, (p, err, bound, np.linalg.norm(ref[p]))


@pytest.mark.parametrize("shape,gamma,dtype", [((32, 32, 32), 0.1, np.float32), ((24, 48, 32), 0.1, np.float32),
                                               ((256, 256), 0.1, np.float32), ((2048, 2048), 0.01, np.float32),
                                               ((64, 64, 64), 0.01, np.float64), ((128, 128), 0.1, np.float64)])
def test_closure_stress(gad, shape, gamma, dtype):
    """tau for the exact field (u* = u), the Layton-Lewandowski model (u* =
    u_bar) and a deconvolved estimate (u* from 3 BiCGSTAB passes)."""
    u = _velocity(shape, 3).astype(dtype)
    ncomp = len(shape)
    ub = np.stack([oracle.filter_field(c, gamma) for c in u]).astype(dtype)
    tub = _to_gpu(ub)
    sol = gad.deconvolve(tub, gamma, method="bicgstab", tol=0.0, maxit=3, ndim=len(shape))
    for us in (u, ub, sol.u.cpu().numpy()):
        tau = gad.closure(tub, _to_gpu(us), gamma, ncomp=ncomp, ndim=len(shape))
        assert tuple(tau.shape) == (ncomp * (ncomp + 1) // 2,) + shape
        _check_stress(tau.cpu().numpy().astype(np.float64), ub.astype(np.float64), us.astype(np.float64), gamma,
                      dtype)


def test_closure_batch_and_scalar(gad):
    """Two velocities in one call equal two calls (bitwise); ncomp = 1 gives
    the scalar variance u_bar^2 - G(u*^2)."""
    shape, gamma = (32, 48, 64), 0.1
    v = np.stack([_velocity(shape, 1), _velocity(shape, 2)]).astype(np.float32)
    vb = np.stack([[oracle.filter_field(c, gamma) for c in w] for w in v]).astype(np.float32)
    both = gad.closure(_to_gpu(vb), _to_gpu(v), gamma, ncomp=3, ndim=3).cpu().numpy()
    one = gad.closure(_to_gpu(vb[1]), _to_gpu(v[1]), gamma, ncomp=3, ndim=3).cpu().numpy()
    np.testing.assert_array_equal(both[1], one)
    s = gad.closure(_to_gpu(vb[0, :1]), _to_gpu(v[0, :1]), gamma, ncomp=1, ndim=3).cpu().numpy()
    _check_stress(s, vb[0, :1].astype(np.float64), v[0, :1].astype(np.float64), gamma, np.float32)


def test_closure_rejects_overlap(gad):
    """The output may not overlap an input: rejected before any launch."""
    shape = (32, 32)
    big = _to_gpu(np.zeros((5,) + shape, dtype=np.float32))
    ub, us = big[:2], _to_gpu(np.zeros((2,) + shape, dtype=np.float32))
    with pytest.raises(gad.GadError):
        gad.closure(ub, us, 0.1, ncomp=2, ndim=2, out=big[1:4])


def _check_spectrum(e, ref, dtype):
    rtol, floor = (1e-5, 1e-6) if dtype == np.float32 else (1e-11, 1e-14)
    tot = ref.sum()
    assert np.all(np.abs(e - ref) <= rtol * ref + floor * tot), np.max(np.abs(e - ref) / (ref + tot))


@pytest.mark.parametrize("shape,dtype", [((256, 256), np.float32), ((2048, 2048), np.float32),
                                         ((96, 128), np.float64), ((32, 32, 32), np.float32),
                                         ((24, 48, 32), np.float32), ((16, 16, 16), np.float64)])
def test_spectrum(gad, shape, dtype):
    if len(shape) == 2:
        u = fields.random_scalar_field(shape, 4, fields.spectrum_2d_kraichnan)[None].astype(dtype)
        ncomp = 1
    else:
        u = fields.random_velocity_field(shape, 4, fields.spectrum_3d_kolmogorov).astype(dtype)
        ncomp = 3
    kmax = int(np.ceil(np.sqrt(sum((n // 2) ** 2 for n in shape)))) + 1
    for nbins in (kmax, max(2, kmax // 3)):
        e = gad.spectrum(_to_gpu(u), nbins, ncomp=ncomp, ndim=len(shape))
        assert e.shape == (1, nbins)
        _check_spectrum(e[0], oc.energy_spectrum(u.astype(np.float64), nbins), dtype)
    full = gad.spectrum(_to_gpu(u), kmax, ncomp=ncomp, ndim=len(shape))[0]
    assert full.sum() == pytest.approx(0.5 * np.mean(np.sum(u.astype(np.float64) ** 2, axis=0)), rel=1e-5)


def test_spectrum_groups_and_single_mode(gad):
    n = 64
    x = 2 * np.pi * np.arange(n) / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    u = np.stack([np.cos(3 * X + 4 * Y), np.sin(X + 2 * Y), 2 * np.cos(X + 2 * Y)]).astype(np.float32)
    e = gad.spectrum(_to_gpu(u), 40, ncomp=1, ndim=2)
    assert e.shape == (3, 40)
    assert e[0, 5] == pytest.approx(0.25, rel=1e-6) and e[0].sum() == pytest.approx(0.25, rel=1e-6)
    assert e[1, 2] + e[2, 2] == pytest.approx(1.25, rel=1e-6)
    with pytest.raises((ValueError, gad.GadError)):
        gad.spectrum(_to_gpu(u), 40, ncomp=2, ndim=2)          # 3 fields are not whole groups of 2
    import ctypes
    lib, ctx = gad.load(), gad.context()
    g, _, _ = gad._grid(_to_gpu(u), 2, 1.0)
    e = np.zeros(80)
    st = lib.ad_spectrum(ctx, ctypes.byref(g), 3, 2, ctypes.c_void_p(_to_gpu(u).data_ptr()), 40,
                         ctypes.c_void_p(e.ctypes.data), None)
    assert st == gad.AD_ERR_ARG                                # the library checks it too


@pytest.mark.parametrize("dtype,prec", [(np.float32, "f32"), (np.float64, "f64")])
def test_histogram_exact(gad, dtype, prec):
    u = fields.random_scalar_field((2048, 2048), 5, fields.spectrum_2d_kraichnan).astype(dtype)
    u[0, :5] = [np.nan, np.inf, -np.inf, 10.0, -10.0]
    sd = float(np.nanstd(u[np.isfinite(u)]))
    for nbins, lo, hi in ((1000, -4 * sd, 4 * sd), (7, -0.5 * sd, 1.3 * sd), (16384, -3.0, 3.0)):
        counts, below, above, nan = gad.histogram(_to_gpu(u), lo, hi, nbins)
        rc, rb, ra, rn = oc.histogram(u, lo, hi, nbins, precision=prec)
        np.testing.assert_array_equal(counts, rc)
        assert (below, above, nan) == (rb, ra, rn)
        assert counts.sum() + below + above + nan == u.size
    with pytest.raises(gad.GadError):
        gad.histogram(_to_gpu(u), 1.0, 1.0, 10)
    c, b, a, n = gad.histogram(_to_gpu(u)[:0], -1.0, 1.0, 4)
    assert c.sum() + b + a + n == 0


@pytest.mark.parametrize("shape,dtype", [((64, 96), np.float32), ((128, 128), np.float64), ((32, 48, 64), np.float32),
                                         ((16, 16, 16), np.float64), ((128, 128, 128), np.float32)])
def test_curl(gad, shape, dtype):
    rng = np.random.default_rng(3)
    v = rng.standard_normal((2, len(shape)) + shape).astype(dtype)     # two velocities
    w = gad.curl(_to_gpu(v), ndim=len(shape)).cpu().numpy().astype(np.float64)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    for i in range(2):
        ref = oc.curl(v[i].astype(np.float64))
        got = w[i] if len(shape) == 3 else w[i][None]
        assert _rel(got, ref) < tol


def test_curl_rejects_overlap(gad):
    big = _to_gpu(np.zeros((3, 32, 32), dtype=np.float32))
    with pytest.raises(gad.GadError):
        gad.curl(big[:2], ndim=2, out=big[1])


def test_curl_of_a_single_mode(gad):
    n = 32
    x = 2 * np.pi * np.arange(n) / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    u = np.stack([np.zeros_like(X), np.sin(3 * X)])
    w = gad.curl(_to_gpu(u), ndim=2).cpu().numpy()
    np.testing.assert_allclose(w, 3 * np.cos(3 * X), atol=1e-12)
