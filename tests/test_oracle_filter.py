"""Pins for the oracle's filter G (Section 4, Eq. df and Eq. df2).

Each test checks the oracle against something other than itself:
hand-computed transfer values of single Fourier modes, a finite-difference
residual of the Helmholtz equation that defines G, a dense-matrix inverse
of (I - delta^2 Laplacian) built from an explicit DFT matrix, and the
operator's symmetries.
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle


def _grid(shape):
    """Physical coordinates x_d = 2 pi j / N_d, returned in (x, y[, z]) order."""
    axes = [2.0 * np.pi * np.arange(n) / n for n in shape]
    g = np.meshgrid(*axes, indexing="ij")
    return list(reversed(g))           # arrays are (.., y, x): x is last


def _mode(shape, kvec, phase=0.0):
    xs = _grid(shape)
    arg = sum(k * x for k, x in zip(kvec, xs)) + phase
    return np.cos(arg)


# (shape, gamma, wavevector (kx, ky[, kz]), G_hat as an exact fraction)
# k_m = min(N)/2, k_c = gamma k_m, G_hat = 1/(1 + |k|^2/k_c^2), worked by hand.
HAND_VALUES = [
    ((16, 16), 0.5, (0, 0), Fraction(1)),
    ((16, 16), 0.5, (4, 0), Fraction(1, 2)),       # |k|^2/k_c^2 = 16/16
    ((16, 16), 0.5, (0, 4), Fraction(1, 2)),
    ((16, 16), 0.5, (4, 4), Fraction(1, 3)),       # 32/16
    ((16, 16), 0.5, (2, 0), Fraction(4, 5)),       # 4/16
    ((16, 16), 0.5, (8, 0), Fraction(1, 5)),       # Nyquist: 64/16
    ((16, 16), 0.5, (8, 8), Fraction(1, 9)),       # corner: 128/16
    ((16, 16), 0.5, (3, 5), Fraction(8, 25)),      # 34/16
    ((16, 16), 0.25, (2, 2), Fraction(1, 3)),      # k_c = 2: 8/4
    ((12, 16), 0.5, (3, 0), Fraction(1, 2)),       # k_m = 6, k_c = 3: 9/9
    ((12, 16), 0.5, (0, 3), Fraction(1, 2)),
    ((12, 16), 0.5, (6, 0), Fraction(1, 5)),       # 36/9
    ((12, 16), 0.5, (8, 6), Fraction(9, 109)),     # 100/9
    ((8, 8, 8), 0.5, (2, 0, 0), Fraction(1, 2)),   # k_m = 4, k_c = 2
    ((8, 8, 8), 0.5, (2, 2, 2), Fraction(1, 4)),   # 12/4
    ((8, 8, 8), 0.5, (0, 0, 4), Fraction(1, 5)),   # 16/4
    ((8, 8, 8), 0.5, (1, 1, 0), Fraction(2, 3)),   # 2/4
    ((6, 6, 6), 1.0, (1, 2, 3), Fraction(9, 23)),  # k_m = k_c = 3: 14/9
]


@pytest.mark.parametrize("shape,gamma,kvec,ghat", HAND_VALUES)
def test_single_mode_transfer_hand_values(shape, gamma, kvec, ghat):
    for phase in (0.0, 0.7):
        u = _mode(shape, kvec, phase)
        if np.max(np.abs(u)) < 1e-12:
            continue
        out = oracle.filter_field(u, gamma)
        np.testing.assert_allclose(out, float(ghat) * u, atol=1e-13)


def _fd_laplacian(v, h):
    """8th-order central finite-difference Laplacian on a periodic grid."""
    c = [-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0]
    out = np.zeros_like(v)
    for ax in range(v.ndim):
        out += c[0] * v
        for m in range(1, 5):
            out += c[m] * (np.roll(v, m, axis=ax) + np.roll(v, -m, axis=ax))
    return out / (h * h)


@pytest.mark.parametrize("shape,gamma", [((128, 128), 0.1), ((64, 64, 64), 0.1), ((96, 96), 0.05)])
def test_helmholtz_residual_finite_difference(shape, gamma):
    # A smooth field (|k| <= 4) so that the 8th-order stencil is accurate.
    rng = np.random.default_rng(3)
    u = np.zeros(shape)
    for _ in range(6):
        k = rng.integers(-4, 5, size=len(shape))
        u += rng.standard_normal() * _mode(shape, tuple(k), rng.uniform(0, 6.28))
    v = oracle.filter_field(u, gamma)
    n = shape[0]
    delta = 1.0 / (gamma * n / 2.0)             # delta = 1/k_c, k_c = gamma N/2
    h = 2.0 * np.pi / n
    resid = v - delta * delta * _fd_laplacian(v, h) - u    # (I - delta^2 lap) G u = u
    assert np.max(np.abs(resid)) < 1e-7 * np.max(np.abs(u))


def _dft_matrix(n):
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("shape,gamma", [((6, 8), 0.5), ((12, 6), 0.3), ((4, 6, 4), 0.7), ((6, 6, 6), 0.4)])
def test_dense_helmholtz_inverse_brute_force(shape, gamma):
    """G equals the dense inverse of I - delta^2 L, with L the spectral
    Laplacian assembled from explicit DFT matrices (no FFT involved)."""
    P = int(np.prod(shape))
    F = np.ones((1, 1), dtype=complex)
    kk = np.zeros(1)
    for n in shape:                               # Kronecker order matches C order
        F = np.kron(F, _dft_matrix(n))
        k = np.array([j if j < n // 2 else j - n for j in range(n)], dtype=float)
        kk = np.add.outer(kk, k * k).ravel()
    Finv = np.conj(F).T / P
    L = np.real(Finv @ np.diag(-kk) @ F)
    kc = gamma * min(shape) / 2.0
    H = np.eye(P) - L / (kc * kc)
    G_brute = np.linalg.inv(H)
    G_oracle = np.column_stack([oracle.filter_field(e.reshape(shape), gamma).ravel()
                                for e in np.eye(P)])
    np.testing.assert_allclose(G_oracle, G_brute, atol=1e-12)


def _rand(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("shape", [(32, 32), (24, 40), (16, 16, 16), (12, 8, 6)])
def test_symmetries(shape):
    g = 0.2
    u, v = _rand(shape, 1), _rand(shape, 2)
    gu, gv = oracle.filter_field(u, g), oracle.filter_field(v, g)
    # self-adjoint and positive definite, 0 < G_hat <= 1
    assert abs(np.vdot(u, gv) - np.vdot(gu, v)) < 1e-10 * np.linalg.norm(u) * np.linalg.norm(v)
    assert 0.0 < np.vdot(u, gu) <= np.vdot(u, u)
    # mean preserved (G_hat(0) = 1)
    assert abs(gu.mean() - u.mean()) < 1e-13
    # linearity and shift equivariance
    np.testing.assert_allclose(oracle.filter_field(2.0 * u - v, g), 2.0 * gu - gv, atol=1e-12)
    for ax in range(len(shape)):
        np.testing.assert_allclose(oracle.filter_field(np.roll(u, 3, axis=ax), g),
                                   np.roll(gu, 3, axis=ax), atol=1e-12)


def test_rotation_equivariance_square():
    u = _rand((32, 32), 4)
    g = oracle.filter_field(u, 0.15)
    np.testing.assert_allclose(oracle.filter_field(np.rot90(u), 0.15), np.rot90(g), atol=1e-12)
    u3 = _rand((12, 12, 12), 5)
    g3 = oracle.filter_field(u3, 0.15)
    np.testing.assert_allclose(oracle.filter_field(np.transpose(u3, (2, 0, 1)), 0.15),
                               np.transpose(g3, (2, 0, 1)), atol=1e-12)


@pytest.mark.parametrize("shape", [(64, 64), (48, 48), (16, 24, 32)])
def test_exact_inverse_round_trip(shape):
    u = _rand(shape, 7)
    for gamma in (0.1, 0.01):
        ub = oracle.filter_field(u, gamma)
        rel = np.linalg.norm(oracle.exact_inverse(ub, gamma) - u) / np.linalg.norm(u)
        # the inverse amplifies rounding by up to 1/G_hat_min
        assert rel < 1e-15 * (1.0 + (max(shape) / (gamma * min(shape))) ** 2)


def test_transfer_bounds():
    for shape in [(128, 128), (8, 8, 8)]:
        gh = oracle.transfer_function(shape, 0.01)
        assert gh.max() == 1.0 and gh.min() > 0.0
        assert gh.flat[0] == 1.0
