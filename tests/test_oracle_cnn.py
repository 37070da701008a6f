"""Pins for the oracle's learned-guess network (oracle/cnn.py): the periodic
convolution against an FFT evaluation and shift kernels, and every gradient
against central finite differences."""

import numpy as np
import pytest

from oracle import cnn


def _rng(s=0):
    return np.random.default_rng(s)


def test_conv_single_channel_matches_fft_correlation():
    """C = 1: the periodic cross-correlation is diagonal in Fourier space,
    y_hat(k) = x_hat(k) * sum_taps w e^{+i k . offset}."""
    x = _rng(1).standard_normal((1, 6, 8, 10))
    w = _rng(2).standard_normal((1, 1, 3, 3, 3))
    shape = x.shape[1:]
    k = np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in shape], indexing="ij")
    tf = np.zeros(shape, dtype=complex)
    for (a, b, c) in cnn.TAPS:
        off = (a - 1, b - 1, c - 1)
        phase = sum(2 * np.pi * kk * o / n for kk, o, n in zip(k, off, shape))
        tf += w[0, 0, a, b, c] * np.exp(1j * phase)
    ref = np.real(np.fft.ifftn(np.fft.fftn(x[0]) * tf))
    np.testing.assert_allclose(cnn.conv3d(x, w)[0], ref, atol=1e-12)


def test_conv_delta_kernels_are_shifts_and_channel_mixing():
    x = _rng(3).standard_normal((2, 5, 6, 7))
    w = np.zeros((3, 2, 3, 3, 3))
    w[0, 1, 1, 1, 1] = 1.0          # centre tap: copy channel 1
    w[1, 0, 2, 1, 1] = 1.0          # z + 1
    w[2, 0, 1, 0, 2] = -2.0         # y - 1, x + 1
    y = cnn.conv3d(x, w)
    np.testing.assert_array_equal(y[0], x[1])
    np.testing.assert_array_equal(y[1], np.roll(x[0], -1, axis=0))
    np.testing.assert_array_equal(y[2], -2.0 * np.roll(np.roll(x[0], 1, axis=1), -1, axis=2))


def test_conv_backward_finite_differences():
    x = _rng(4).standard_normal((3, 4, 5, 6))
    w = _rng(5).standard_normal((2, 3, 3, 3, 3))
    dy = _rng(6).standard_normal((2, 4, 5, 6))
    dx, dw = cnn.conv3d_backward(x, w, dy)
    f = lambda xx, ww: float(np.sum(dy * cnn.conv3d(xx, ww)))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (2, 3, 4, 5), (1, 2, 0, 3)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, w) - f(x - e, w)) / (2 * h) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0, 0), (1, 2, 2, 1, 0), (0, 1, 1, 1, 1)]:
        e = np.zeros_like(w); e[idx] = h
        assert abs((f(x, w + e) - f(x, w - e)) / (2 * h) - dw[idx]) < 1e-7


def test_network_gradients_finite_differences():
    ws = cnn.init_weights(channels=3, seed=1, scale_last=1.0)
    ubar = _rng(7).standard_normal((6, 6, 6))
    ut = ubar + 0.3 * _rng(8).standard_normal((6, 6, 6))
    A = 1.7
    L, grads = cnn.loss_and_grads(ws, ubar, ut, A)
    h = 1e-6
    for k in range(4):
        for idx in [tuple(0 for _ in ws[k].shape), tuple(s - 1 for s in ws[k].shape)]:
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[k][idx] += h
            wm[k][idx] -= h
            fd = (cnn.loss(cnn.forward(wp, ubar, A)[0], ut) - cnn.loss(cnn.forward(wm, ubar, A)[0], ut)) / (2 * h)
            assert abs(fd - grads[k][idx]) < 1e-6 * max(1.0, abs(fd)), (k, idx, fd, grads[k][idx])


def test_network_is_positively_homogeneous():
    ws = cnn.init_weights(channels=4, seed=2, scale_last=1.0)
    ubar = _rng(9).standard_normal((6, 6, 6))
    u1 = cnn.forward(ws, ubar)[0]
    u2 = cnn.forward(ws, 3.5 * ubar)[0]
    np.testing.assert_allclose(u2, 3.5 * u1, atol=1e-12)


def test_adam_first_step_is_signed_lr():
    ws = [np.array([1.0, -2.0, 3.0])]
    opt = cnn.Adam(ws, lr=0.01)
    out = opt.step(ws, [np.array([0.5, -4.0, 0.0])])
    np.testing.assert_allclose(out[0], [0.99, -1.99, 3.0], atol=1e-9)


def test_output_scale_is_the_grid_unit_filter_radius():
    """A = (delta/h)^2 with delta = 1/(gamma N/2), h = 2 pi/N, for any N."""
    for gamma, n in [(0.01, 64), (0.1, 256), (0.05, 96)]:
        delta, h = 1.0 / (gamma * n / 2.0), 2.0 * np.pi / n
        assert abs(cnn.output_scale(gamma) - (delta / h) ** 2) < 1e-9 * (delta / h) ** 2
