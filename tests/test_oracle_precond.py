"""Pins for the oracle's preconditioned CG (oracle/precond.py).

The preconditioner M is the periodic second-order finite-difference version
of G^{-1} = I - delta^2 Laplacian (Section 4, Eq. df). It is checked against
an independent dense construction (Kronecker sums of circulant difference
matrices), against the closed-form eigenvalues of circulant matrices, and
against the exact inverse symbol it approximates (second-order consistency).
The iteration is checked by reduction to Algorithm 3 (M = I), finite
termination on few-mode fields, the orthogonality relations of
preconditioned CG, and convergence to the exact Fourier inverse.
"""

import math

import numpy as np
import pytest

import oracle
from synth import fields


def _circulant_second_difference(n):
    """Dense n x n matrix of x -> 2 x_i - x_{i+1} - x_{i-1}, periodic."""
    D = 2.0 * np.eye(n)
    for i in range(n):
        D[i, (i + 1) % n] -= 1.0
        D[i, (i - 1) % n] -= 1.0
    return D


def _dense_preconditioner(shape, gamma):
    """I + sum_d c_d (I x ... x D_d x ... x I) as a dense matrix, with
    c_d = (N_d / (2 pi k_c))^2 and k_c = gamma min(N)/2 written out here."""
    kc = gamma * min(shape) / 2.0
    n = int(np.prod(shape))
    M = np.eye(n)
    for d, nd in enumerate(shape):
        c = (nd / (2.0 * math.pi * kc)) ** 2
        term = np.ones((1, 1))
        for e, ne in enumerate(shape):
            term = np.kron(term, _circulant_second_difference(ne) if e == d else np.eye(ne))
        M += c * term
    return M


@pytest.mark.parametrize("shape,gamma", [((8, 12), 0.25), ((6, 8, 10), 0.4)])
def test_stencil_equals_dense_kronecker_construction(shape, gamma):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape)
    M = _dense_preconditioner(shape, gamma)
    np.testing.assert_allclose(oracle.apply_preconditioner(x, gamma).ravel(), M @ x.ravel(), rtol=1e-13, atol=1e-12)


def test_stencil_eigenvalues_are_the_circulant_closed_form():
    """The eigenvalues of a circulant second difference are 2 - 2 cos(2 pi k / n)
    = 4 sin^2(pi k / n); the dense M's spectrum must be their weighted sums."""
    shape, gamma = (8, 12), 0.25
    M = _dense_preconditioner(shape, gamma)
    ev = np.sort(np.linalg.eigvalsh(M))
    np.testing.assert_allclose(ev, np.sort(oracle.preconditioner_symbol(shape, gamma).ravel()), rtol=1e-12)


def test_single_mode_hand_value():
    """8 x 12 grid, gamma = 0.25: k_c = 1, c_y = 16/pi^2, c_x = 36/pi^2. For
    cos(3x + y): M_hat = 1 + (64/pi^2) sin^2(pi/8) + (144/pi^2) sin^2(pi/4)
    = 1 + (64/pi^2)(2 - sqrt 2)/4 + 72/pi^2."""
    ny, nx = 8, 12
    y, x = np.meshgrid(2 * np.pi * np.arange(ny) / ny, 2 * np.pi * np.arange(nx) / nx, indexing="ij")
    f = np.cos(3 * x + y)
    expect = 1.0 + (16.0 / math.pi ** 2) * (2.0 - math.sqrt(2.0)) + 72.0 / math.pi ** 2
    np.testing.assert_allclose(oracle.apply_preconditioner(f, 0.25), expect * f, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("shape,gamma", [((32, 48), 0.01), ((16, 8, 12), 0.1)])
def test_float32_evaluation_within_rounding_bound(shape, gamma):
    """The float32 evaluation differs from the float64 one of the same float32
    input by rounding only: per term at most a few float32 ulps of the
    magnitudes that enter it."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    z64 = oracle.apply_preconditioner(x, gamma)
    z32 = oracle.apply_preconditioner_f32(x, gamma)
    cs = oracle.stencil_coefficients(shape, gamma)
    scale = np.abs(x) + sum(c * (2 * np.abs(x) + np.abs(np.roll(x, 1, a)) + np.abs(np.roll(x, -1, a)))
                            for a, c in enumerate(cs))
    assert np.all(np.abs(z32 - z64) <= 8 * 2.0 ** -24 * scale)
    assert np.max(np.abs(z32 - z64) / scale) > 0           # genuinely float32


def test_second_order_consistency_with_the_exact_inverse():
    """For a fixed smooth mode, M_hat(k) -> 1 + |k|^2/k_c^2 (the symbol of
    G^{-1}) with an error that falls by 4x when the grid is refined 2x at a
    fixed k_c (second-order central differences)."""
    k = (3, 2)
    errs = []
    for n in (32, 64, 128):
        gamma = 8.0 / n                       # k_c = gamma n/2 = 4 at every n
        sym = oracle.preconditioner_symbol((n, n), gamma)
        exact = 1.0 + (k[0] ** 2 + k[1] ** 2) / 16.0
        errs.append(abs(sym[k[0], k[1]] - exact))
    assert 3.9 < errs[0] / errs[1] < 4.1 and 3.9 < errs[1] / errs[2] < 4.1


@pytest.mark.parametrize("shape,gamma", [((64, 64), 0.01), ((64, 64), 0.1), ((16, 16, 16), 0.1)])
def test_preconditioned_spectrum_is_bounded(shape, gamma):
    """M and G commute; the eigenvalues M_hat G_hat of M G lie in [4/pi^2, 1]."""
    lam = oracle.preconditioner_symbol(shape, gamma) * oracle.transfer_function(shape, gamma)
    assert lam.max() <= 1.0 + 1e-12 and lam.min() >= 4.0 / math.pi ** 2 - 1e-12


def test_identity_preconditioner_is_algorithm_3():
    u = fields.random_scalar_field((32, 32), 5, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, 0.1)
    a = oracle.preconditioned_cg(ub, 0.1, tol=0.0, maxit=12, precond=False)
    b = oracle.conjugate_gradient(ub, 0.1, tol=0.0, maxit=12)
    assert a.iterations == b.iterations == 12
    np.testing.assert_allclose(a.u, b.u, rtol=0, atol=1e-13)
    np.testing.assert_allclose(a.history, b.history, rtol=1e-12)


def _cos_mode(shape, kvec):
    axes = [2.0 * np.pi * np.arange(n) / n for n in shape]
    g = list(reversed(np.meshgrid(*axes, indexing="ij")))
    return np.cos(sum(k * x for k, x in zip(kvec, g)))


@pytest.mark.parametrize("nmodes", [1, 2, 3])
def test_finite_termination(nmodes):
    """A field made of m Fourier modes with distinct eigenvalues of M G lies in
    an m-dimensional invariant subspace: preconditioned CG ends in m passes."""
    shape, gamma = (32, 32), 0.25
    modes = [(1, 0), (5, 2), (11, 7)][:nmodes]
    lam = oracle.preconditioner_symbol(shape, gamma) * oracle.transfer_function(shape, gamma)
    assert len({round(lam[k[1], k[0]], 12) for k in modes}) == nmodes
    u = sum((i + 1.0) * _cos_mode(shape, k) for i, k in enumerate(modes))
    ub = oracle.filter_field(u, gamma)
    res = oracle.preconditioned_cg(ub, gamma, tol=1e-11, maxit=50)
    assert res.status == oracle.STATUS_OK and res.iterations == nmodes
    np.testing.assert_allclose(res.u, u, atol=1e-9)


def test_orthogonality_relations():
    """Preconditioned CG keeps (r_{n+1}, z_j) = 0 for j <= n and
    (p_{n+1}, G p_j) = 0 for j <= n."""
    gamma = 0.1
    u = fields.random_scalar_field((32, 32), 9, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, gamma)
    res = oracle.preconditioned_cg(ub, gamma, tol=0.0, maxit=6, record=True)
    tr = res.trace
    for n in range(5):
        r_next = tr["r"][n + 1]
        for j in range(n + 1):
            zr = oracle.inner(r_next, tr["z"][j])
            assert abs(zr) <= 1e-9 * math.sqrt(oracle.inner(r_next, r_next) * oracle.inner(tr["z"][j], tr["z"][j]))
            gp = oracle.filter_field(tr["p"][j], gamma)
            pg = oracle.inner(tr["p"][n + 1], gp)
            assert abs(pg) <= 1e-9 * math.sqrt(oracle.inner(tr["p"][n + 1], tr["p"][n + 1]) * oracle.inner(gp, gp))


@pytest.mark.parametrize("gamma", [0.1, 0.01])
def test_converges_to_exact_inverse_in_few_passes(gamma):
    """The residual bound ||u - u_ex|| <= ||r_true|| / G_hat_min holds, and the
    bounded condition number (<= pi^2/4) caps the pass count far below that of
    plain CG at gamma = 0.01."""
    shape = (64, 64)
    u = fields.random_scalar_field(shape, 2, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, gamma)
    res = oracle.preconditioned_cg(ub, gamma, tol=1e-10, maxit=200)
    assert res.status == oracle.STATUS_OK and res.iterations <= 20
    ex = oracle.exact_inverse(ub, gamma)
    ghmin = oracle.transfer_function(shape, gamma).min()
    r = ub - oracle.filter_field(ub, gamma)
    ref = math.sqrt(oracle.inner(r, r))
    assert np.linalg.norm(res.u - ex) <= res.true_residual * ref / ghmin * (1 + 1e-6) + 1e-12
    cg = oracle.conjugate_gradient(ub, gamma, tol=1e-10, maxit=2000)
    assert cg.iterations > 4 * res.iterations


def test_zero_and_breakdown_rules():
    z = np.zeros((16, 16))
    res = oracle.preconditioned_cg(z, 0.1, tol=1e-6, maxit=10)
    assert res.iterations == 0 and res.status == oracle.STATUS_OK
    res = oracle.preconditioned_cg(np.ones((16, 16)), 0.1, tol=1e-6, maxit=10)
    assert res.iterations == 0 and res.status == oracle.STATUS_OK     # G 1 = 1: r_0 = 0
    res = oracle.preconditioned_cg(z, 0.1, tol=0.0, maxit=3)
    assert res.iterations == 0


@pytest.mark.parametrize("shape,gamma", [((32, 48), 0.01), ((16, 12, 8), 0.1)])
def test_spectral_space_iterates_equal_physical(shape, gamma):
    """M is circulant, so in spectral space it is the pointwise multiply by
    M_hat: the iterates, histories and pass counts equal the physical-space
    ones in float64 (to rounding)."""
    if len(shape) == 3:
        u = fields.random_velocity_field(shape, 1, fields.spectrum_3d_kolmogorov)[0]
    else:
        u = fields.random_scalar_field(shape, 1, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, gamma)
    a = oracle.preconditioned_cg(ub, gamma, tol=0.0, maxit=6)
    b = oracle.preconditioned_cg(ub, gamma, tol=0.0, maxit=6, space="spectral")
    np.testing.assert_allclose(b.u, a.u, atol=1e-12 * np.abs(a.u).max())
    np.testing.assert_allclose(b.history, a.history, rtol=1e-9)
    c = oracle.solve("pcg", ub, gamma, tol=1e-9, maxit=100, space="spectral")
    d = oracle.solve("pcg", ub, gamma, tol=1e-9, maxit=100)
    assert c.iterations == d.iterations and c.status == d.status == oracle.STATUS_OK
