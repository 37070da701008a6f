"""Pins for the oracle's closure and statistics (oracle/closure.py).

The sub-filter stress is checked against hand-worked single-mode values
(where G acts by known fractions) for Eq. fge3 with the true field and for
Eq. tau2, against a dense filter matrix built from explicit DFT matrices, and
against the paper's printed second-order form of Eq. tau3. The spectrum is
checked by Parseval, by single modes landing in their shell, and its shell
rule by brute force. The histogram is checked on values with known bins and
by a scalar float32 loop. The curl is checked on single modes, by
div curl = 0, curl grad = 0, and the stream-function identity omega = lap psi.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import closure
from synth import fields


def _grid2(n):
    x = 2 * np.pi * np.arange(n) / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    return X, Y


def test_stress_single_mode_true_field_hand_values():
    """16^2, gamma = 0.5 (k_c = 4), u = (cos 2x, 0): G_hat(2) = 4/5, G_hat(4) = 1/2,
    tau_11 = (G(2)^2 - 1)/2 + (G(2)^2 - G(4))/2 cos 4x = -9/50 + 7/100 cos 4x,
    tau_12 = tau_22 = 0 (Eq. fge3 with u* = u)."""
    X, _ = _grid2(16)
    u = np.stack([np.cos(2 * X), np.zeros_like(X)])
    ub = np.stack([oracle.filter_field(c, 0.5) for c in u])
    tau = closure.closure_stress(ub, u, 0.5)
    assert tau.shape == (3, 16, 16)
    np.testing.assert_allclose(tau[0], -9.0 / 50 + 7.0 / 100 * np.cos(4 * X), atol=1e-14)
    np.testing.assert_allclose(tau[1], 0.0, atol=1e-14)
    np.testing.assert_allclose(tau[2], 0.0, atol=1e-14)


def test_stress_layton_lewandowski_hand_values():
    """Eq. tau2 (u* = u_bar) for u_bar = (4/5) cos 2x: tau_11 = (8/50) cos 4x."""
    X, _ = _grid2(16)
    ub = np.stack([0.8 * np.cos(2 * X), np.zeros_like(X)])
    tau = closure.closure_stress(ub, ub, 0.5)
    np.testing.assert_allclose(tau[0], 8.0 / 50 * np.cos(4 * X), atol=1e-14)


def _dense_filter(shape, gamma):
    """G as a dense matrix: F^-1 diag(G_hat) F with explicit DFT matrices."""
    mats = []
    for n in shape:
        j = np.arange(n)
        mats.append(np.exp(-2j * np.pi * np.outer(j, j) / n))
    F = mats[0]
    for m in mats[1:]:
        F = np.kron(F, m)
    kc = gamma * min(shape) / 2.0
    ks = [np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n) for n in shape]
    k2 = sum(g ** 2 for g in np.meshgrid(*ks, indexing="ij")).ravel()
    gh = 1.0 / (1.0 + k2 / kc ** 2)
    return np.real(np.conj(F).T @ np.diag(gh) @ F) / F.shape[0]


def test_stress_against_dense_filter_3d():
    shape, gamma = (4, 6, 8), 0.5
    rng = np.random.default_rng(1)
    ub = rng.standard_normal((3,) + shape)
    us = rng.standard_normal((3,) + shape)
    G = _dense_filter(shape, gamma)
    tau = closure.closure_stress(ub, us, gamma)
    for p, (i, j) in enumerate(closure.pair_list(3)):
        expect = ub[i] * ub[j] - (G @ (us[i] * us[j]).ravel()).reshape(shape)
        np.testing.assert_allclose(tau[p], expect, atol=1e-12)
    assert closure.pair_list(3) == [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def test_stress_second_order_van_cittert_form():
    """With the N = 2 estimate u* = 2 u_bar - G u_bar (one pass of Algorithm 1)
    the stress is the paper's printed second-order form of Eq. tau3."""
    gamma = 0.1
    u = fields.random_velocity_field((16, 16, 16), 3, fields.spectrum_3d_kolmogorov)
    ub = np.stack([oracle.filter_field(c, gamma) for c in u])
    us = np.stack([oracle.van_cittert(c, gamma, tol=0.0, maxit=1).u for c in ub])
    tau = closure.closure_stress(ub, us, gamma)
    for p, (i, j) in enumerate(closure.pair_list(3)):
        a = 2 * ub[i] - oracle.filter_field(ub[i], gamma)
        b = 2 * ub[j] - oracle.filter_field(ub[j], gamma)
        np.testing.assert_allclose(tau[p], ub[i] * ub[j] - oracle.filter_field(a * b, gamma), atol=1e-13)


def test_shell_index_brute_force():
    m = np.arange(0, 20000)
    got = closure.shell_index(m)
    for mm, k in zip(m[::7], got[::7]):
        # nearest integer to sqrt(m), halves down: (k - 1/2)^2 < m <= (k + 1/2)^2 in exact arithmetic
        lo = (2 * k - 1) ** 2       # 4 (k - 1/2)^2
        hi = (2 * k + 1) ** 2
        assert (k == 0 and mm == 0) or (lo < 4 * mm <= hi), (mm, k)


def test_spectrum_parseval_and_single_modes():
    X, Y = _grid2(32)
    u = np.stack([np.cos(3 * X + 4 * Y)])                  # |k| = 5: all energy 1/4 in shell 5
    e = closure.energy_spectrum(u, 40)
    assert e[5] == pytest.approx(0.25, rel=1e-13) and abs(e.sum() - 0.25) < 1e-13
    u = np.stack([np.sin(X + 2 * Y), 2 * np.cos(X + 2 * Y)])   # |k|^2 = 5 -> shell 2; (1 + 4)/4
    e = closure.energy_spectrum(u, 40)
    assert e[2] == pytest.approx(1.25, rel=1e-13)
    v = fields.random_velocity_field((24, 24, 24), 4, fields.spectrum_3d_kolmogorov)
    e = closure.energy_spectrum(v, 64)
    assert e.sum() == pytest.approx(0.5 * np.mean(np.sum(v ** 2, axis=0)), rel=1e-12)
    assert e[0] == pytest.approx(0.0, abs=1e-20)           # mean removed by the generator


def test_spectrum_follows_the_generator():
    """The generator prescribes E(k) up to the random amplitudes: octave band
    sums of the shell spectrum of a large 2D draw track the band sums of the
    prescribed E(k) within sampling error (an independent pin of both)."""
    n = 512
    spec = fields.spectrum_2d_kraichnan
    u = fields.random_scalar_field((n, n), 0, spec)
    e = closure.energy_spectrum(u[None], n // 2)
    bands = [(8, 16), (16, 32), (32, 64), (64, 128)]
    got = np.array([e[a:b].sum() for a, b in bands])
    want = np.array([spec(np.arange(a, b, dtype=float)).sum() for a, b in bands])
    ratio = (got / want) / np.median(got / want)
    assert np.all(np.abs(ratio - 1) < 0.15), ratio


def test_histogram_known_bins_and_scalar_loop():
    lo, hi, nb = -1.0, 1.0, 8
    x = np.array([-1.0, -0.75, -0.7499, 0.0, 0.99, 1.0, -1.01, np.nan, 0.125, 0.124], dtype=np.float32)
    counts, below, above, nan = closure.histogram(x, lo, hi, nb)
    assert below == 1 and above == 1 and nan == 1
    assert list(counts) == [1, 2, 0, 0, 3, 0, 0, 1]       # scale 4: t = 0, 1, 1.0004, 4, 7.96, 4.5, 4.496
    assert counts.sum() + below + above + nan == x.size
    rng = np.random.default_rng(5)
    y = (rng.standard_normal(2000) * 0.8).astype(np.float32)
    c2, b2, a2, n2 = closure.histogram(y, lo, hi, 50)
    ref = np.zeros(50, dtype=np.int64)
    rb = ra = 0
    sc = np.float32(50 / (hi - lo))
    for v in y:
        t = np.float32(np.float32(v) - np.float32(lo)) * sc
        b = math.floor(float(np.float32(t)))
        if b < 0:
            rb += 1
        elif b >= 50:
            ra += 1
        else:
            ref[b] += 1
    assert list(c2) == list(ref) and (b2, a2, n2) == (rb, ra, 0)


def test_curl_single_modes_and_identities():
    n = 16
    X, Y = _grid2(n)
    u = np.stack([np.zeros_like(X), np.sin(3 * X)])
    np.testing.assert_allclose(closure.curl(u)[0], 3 * np.cos(3 * X), atol=1e-12)
    psi = np.cos(2 * X + 3 * Y)
    u = np.stack([-closure.derivative(psi, 0), closure.derivative(psi, 1)])
    np.testing.assert_allclose(closure.curl(u)[0], -13 * psi, atol=1e-11)   # omega = lap psi
    # the Nyquist mode has no resolved derivative
    np.testing.assert_allclose(closure.derivative(np.cos(8 * X), 1), 0.0, atol=1e-12)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((3, 8, 12, 16))
    w = closure.curl(v)
    div = sum(closure.derivative(w[c], 2 - c) for c in range(3))       # x = axis 2, y = 1, z = 0
    np.testing.assert_allclose(div, 0.0, atol=1e-10)
    phi = rng.standard_normal((8, 12, 16))
    g = np.stack([closure.derivative(phi, 2), closure.derivative(phi, 1), closure.derivative(phi, 0)])
    np.testing.assert_allclose(closure.curl(g), 0.0, atol=1e-10)
