"""GPU parity of the preconditioned CG solve (AD_CG | AD_PRECOND, method
"pcg") against the CPU oracle (oracle/precond.py) through the C ABI.

The float32 oracle evaluates the preconditioner in the kernel's float32
operation order, so the stencil itself rounds identically on both sides for
the same input; the differences come from G (FFT rounding) and the dot
products, and M amplifies them at the highest wavenumbers by up to
1 + 4 sum_d c_d (c_d = 1/(pi gamma)^2 on cubic grids: ~8000 at gamma = 0.01).
Fields are therefore judged, from the first pass on, with the same
precision-matched ensemble as the other solvers (tests/parity_tools.py):
within max(1e-5 float32 / 1e-12 float64, 3 x the oracle's spread over
equally valid shifted evaluations of G), never above 1e-4 / 1e-12; pass
counts exact (the preconditioned iteration is well conditioned, and every
shifted oracle run must agree on the count).
"""

import numpy as np
import pytest

import oracle
from synth import fields
from parity_tools import count_exact, ensemble_runs, field_tolerance, history_tolerance

pytestmark = pytest.mark.gpu


# Float32 histories deep below the float32 residual floor (h ~ 1e-7, where the
# stored vectors can no longer represent a smaller residual) are compared to an
# absolute 1e-12, i.e. 1e-5 of that floor: there the recurrence keeps shrinking
# but two equally valid runs differ by more than the ensemble's relative spread.
H_ATOL = 1e-12


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(shape, seed, gamma, dtype=np.float32):
    if len(shape) == 3:
        u = fields.random_velocity_field(shape, seed, fields.spectrum_3d_kolmogorov)[0]
    else:
        u = fields.random_scalar_field(shape, seed, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, gamma).astype(dtype)
    return u, ub


def _to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_one_pass_on_wrapping_tiles(gad):
    """One preconditioned pass from u0 = u_bar: r_0 and z_0 = M r_0 enter
    p_0 = z_0; with tol = 0 and maxit = 1 the result u_1 = u_bar + alpha_0 z_0
    must match the oracle's float32-storage run to 1e-5, on grids whose row
    tiles wrap around in y and z (small and non-power-of-two sides)."""
    for shape, gamma in (((8, 8), 0.5), ((24, 36), 0.3), ((12, 8, 16), 0.4), ((8, 24, 12), 0.25)):
        _, ub = _problem(shape, 7, gamma)
        res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=0.0, maxit=1, ndim=len(shape))
        ref = oracle.preconditioned_cg(ub.astype(np.float64), gamma, tol=0.0, maxit=1, precision="f32")
        assert int(res.iterations[0]) == 1 and int(res.status[0]) == gad.AD_MAXIT
        assert _rel(res.u.double().cpu().numpy(), ref.u) < 1e-5, shape
        np.testing.assert_allclose(res.history[0, :2], ref.history, rtol=1e-5)


# gamma = 0.01 is compared in float64 (below): there M amplifies float32
# rounding at the top wavenumbers by up to ~8000, and the float32 oracle's own
# spread over equally valid evaluations is 1e-4 - 3e-4 already after one pass
# (measured), above the 1e-4 ceiling
@pytest.mark.parametrize("shape,gamma", [((64, 64), 0.1), ((96, 128), 0.1), ((32, 32, 32), 0.1), ((24, 48, 32), 0.1)])
@pytest.mark.parametrize("npass", [1, 5, 12])
def test_fixed_passes_f32(gad, shape, gamma, npass):
    _, ub = _problem(shape, 3, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=0.0, maxit=npass, ndim=len(shape))
    assert int(res.iterations[0]) == npass and int(res.status[0]) == gad.AD_MAXIT
    u64 = ub.astype(np.float64)
    gpu = res.u.double().cpu().numpy()
    # every pass, the first included, goes through the precision-matched
    # ensemble: M amplifies rounding noise at the highest wavenumbers by up to
    # 1 + 4 sum_d c_d (about 8000 at gamma = 0.01), so two equally valid
    # float32 evaluations of r_0 already give z_0 that differ by ~1e-4
    base, runs = ensemble_runs("pcg", u64, gamma, 0.0, npass, "f32")
    tol, spread = field_tolerance(base, runs, "f32")
    assert _rel(gpu, base.u) < tol, (_rel(gpu, base.u), spread)
    np.testing.assert_allclose(res.history[0, :npass + 1], base.history, rtol=history_tolerance(base, runs, 1e-5),
                               atol=H_ATOL)


@pytest.mark.parametrize("shape,gamma", [((128, 128), 0.1), ((256, 256), 0.01), ((64, 64, 64), 0.01)])
def test_fixed_passes_f64(gad, shape, gamma):
    _, ub = _problem(shape, 0, gamma, dtype=np.float64)
    for npass in (1, 5, 12):
        res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=0.0, maxit=npass, ndim=len(shape))
        base, runs = ensemble_runs("pcg", ub, gamma, 0.0, npass, "f64")
        tol, spread = field_tolerance(base, runs, "f64")
        err = _rel(res.u.cpu().numpy(), base.u)
        assert err < 1e-12, "passes %d: error %.3e, oracle spread %.3e" % (npass, err, spread)
        np.testing.assert_allclose(res.history[0, :npass + 1], base.history, rtol=history_tolerance(base, runs, 1e-11))


@pytest.mark.parametrize("gamma", [0.1, 0.01])
def test_config1_f64_to_tolerance(gad, gamma):
    """128^2 float64 vorticity to relative residual 1e-10: exact pass count,
    the field against the oracle and the FFT-exact inverse, the true residual."""
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=8.0)
    u = fields.random_scalar_field((128, 128), 0, spec)
    ub = oracle.filter_field(u, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=1e-10, maxit=500, true_residual=True)
    base, runs = ensemble_runs("pcg", ub, gamma, 1e-10, 500, "f64")
    assert int(res.status[0]) == gad.AD_OK == base.status
    ok, counts = count_exact(int(res.iterations[0]), base, runs)
    assert ok, (int(res.iterations[0]), counts)
    assert int(res.iterations[0]) <= 25
    tol, spread = field_tolerance(base, runs, "f64")
    assert _rel(res.u.cpu().numpy(), base.u) < tol, spread
    assert _rel(res.u.cpu().numpy(), oracle.exact_inverse(ub, gamma)) < 1e-7
    assert res.true_residual[0] < 2e-10


@pytest.mark.parametrize("shape,gamma", [((256, 256), 0.1), ((512, 512), 0.01), ((64, 64, 64), 0.1),
                                         ((96, 64, 48), 0.01)])
def test_f32_to_tolerance_counts(gad, shape, gamma):
    _, ub = _problem(shape, 1, gamma)
    tol = 1e-6
    res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=tol, maxit=500, ndim=len(shape), true_residual=True)
    base, runs = ensemble_runs("pcg", ub.astype(np.float64), gamma, tol, 500, "f32")
    n_gpu = int(res.iterations[0])
    assert int(res.status[0]) == gad.AD_OK
    ok, counts = count_exact(n_gpu, base, runs)
    assert ok, (n_gpu, counts)
    assert res.history[0, n_gpu] <= tol
    assert res.true_residual[0] < 20 * tol
    if gamma >= 0.1:                  # see test_fixed_passes_f32 for gamma = 0.01
        tolf, spread = field_tolerance(base, runs, "f32")
        err = _rel(res.u.double().cpu().numpy(), base.u)
        assert err < tolf, "error %.3e, tolerance %.3e, oracle spread %.3e" % (err, tolf, spread)
    uex = oracle.exact_inverse(ub.astype(np.float64), gamma)
    ref = np.linalg.norm(ub.astype(np.float64) - oracle.filter_field(ub.astype(np.float64), gamma))
    gmin = oracle.transfer_function(shape, gamma).min()
    assert np.linalg.norm(res.u.double().cpu().numpy() - uex) <= 1.05 * res.true_residual[0] * ref / gmin
    cg = gad.deconvolve(_to_gpu(ub), gamma, method="cg", tol=tol, maxit=3000, ndim=len(shape))
    assert int(cg.iterations[0]) > 2 * n_gpu


def test_edge_cases_per_field_status(gad):
    """Regular, zero, constant and NaN fields in one batch: per-field
    statuses, and the regular field bitwise equal to its solve alone."""
    n = 64
    _, ub = _problem((n, n), 2, 0.1)
    batch = np.stack([ub, np.zeros_like(ub), np.full_like(ub, 2.5), ub.copy()])
    batch[3, 5, 7] = np.nan
    res = gad.deconvolve(_to_gpu(batch), 0.1, method="pcg", tol=1e-5, maxit=300, ndim=2)
    alone = gad.deconvolve(_to_gpu(ub), 0.1, method="pcg", tol=1e-5, maxit=300)
    assert int(res.status[0]) == gad.AD_OK and res.iterations[0] == alone.iterations[0]
    np.testing.assert_array_equal(res.u[0].cpu().numpy(), alone.u.cpu().numpy())
    assert int(res.status[1]) == gad.AD_OK and int(res.iterations[1]) == 0
    assert int(res.status[2]) == gad.AD_OK and int(res.iterations[2]) == 0
    assert int(res.status[3]) == gad.AD_ERR_NONFINITE
    np.testing.assert_array_equal(res.u[1].cpu().numpy(), 0.0)
    np.testing.assert_array_equal(res.u[2].cpu().numpy(), 2.5)


def test_maxit_zero_single_mode_and_bad_methods(gad):
    _, ub = _problem((32, 32), 4, 0.1)
    t = _to_gpu(ub)
    res = gad.deconvolve(t, 0.1, method="pcg", tol=1e-6, maxit=0)
    assert int(res.status[0]) == gad.AD_MAXIT and int(res.iterations[0]) == 0
    np.testing.assert_array_equal(res.u.cpu().numpy(), ub)
    # the preconditioner flag is defined for CG only
    import ctypes
    import torch
    lib, ctx = gad.load(), gad.context()
    g, _, _ = gad._grid(t, 2, 0.1)
    out = torch.empty_like(t)
    for code in (gad.METHODS["bicgstab"] | gad.AD_PRECOND, gad.METHODS["vancittert"] | gad.AD_PRECOND,
                 gad.METHODS["sd"] | gad.AD_PRECOND | gad.AD_SPECTRAL):
        st = lib.ad_deconvolve(ctx, ctypes.byref(g), ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               1, code, 1e-6, 10, None, None, None, None, None, None)
        assert st == gad.AD_ERR_ARG
    n = 64
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    u = np.cos(3 * X + 5 * Y)
    ub1 = oracle.filter_field(u, 0.2)
    res = gad.deconvolve(_to_gpu(ub1), 0.2, method="pcg", tol=1e-10, maxit=10)
    assert int(res.iterations[0]) == 1 and int(res.status[0]) == gad.AD_OK
    np.testing.assert_allclose(res.u.cpu().numpy(), u, atol=1e-12)


def test_graph_host_loop_batch_and_batched_agree(gad):
    """The graph loop and the host loop give bitwise equal results; a field
    solved inside a batch, or inside an uneven batched call, is bitwise equal
    to its solve alone."""
    _, ub = _problem((128, 128), 6, 0.01)
    _, ub3 = _problem((32, 48, 64), 6, 0.1)
    t = _to_gpu(ub)
    gad.set_graph_mode(True)
    a = gad.deconvolve(t, 0.01, method="pcg", tol=1e-6, maxit=300)
    gad.set_graph_mode(False)
    b = gad.deconvolve(t, 0.01, method="pcg", tol=1e-6, maxit=300)
    gad.set_graph_mode(True)
    assert int(a.iterations[0]) == int(b.iterations[0])
    np.testing.assert_array_equal(a.u.cpu().numpy(), b.u.cpu().numpy())
    pair = gad.deconvolve(_to_gpu(np.stack([ub, ub[::-1].copy()])), 0.01, method="pcg", tol=1e-6, maxit=300, ndim=2)
    np.testing.assert_array_equal(pair.u[0].cpu().numpy(), a.u.cpu().numpy())
    a3 = gad.deconvolve(_to_gpu(ub3), 0.1, method="pcg", tol=1e-6, maxit=300, ndim=3)
    outs, its, sts, _ = gad.deconvolve_batched([_to_gpu(ub), _to_gpu(ub3)], [0.01, 0.1], method="pcg", tol=1e-6,
                                               maxit=300)
    assert list(sts) == [gad.AD_OK, gad.AD_OK]
    assert int(its[0]) == int(a.iterations[0]) and int(its[1]) == int(a3.iterations[0])
    np.testing.assert_array_equal(outs[0].cpu().numpy(), a.u.cpu().numpy())
    np.testing.assert_array_equal(outs[1].cpu().numpy(), a3.u.cpu().numpy())


def test_initial_guess(gad):
    u, ub = _problem((96, 96), 5, 0.1, dtype=np.float64)
    u0 = 0.5 * (ub + u)
    res = gad.deconvolve(_to_gpu(ub), 0.1, method="pcg", tol=1e-9, maxit=200, u0=_to_gpu(u0))
    base, runs = ensemble_runs("pcg", ub, 0.1, 1e-9, 200, "f64", u0=u0)
    ok, counts = count_exact(int(res.iterations[0]), base, runs)
    assert ok, (int(res.iterations[0]), counts)
    assert res.history[0, 0] == pytest.approx(base.history[0], rel=1e-12) and res.history[0, 0] < 1.0
    assert _rel(res.u.cpu().numpy(), oracle.exact_inverse(ub, 0.1)) < 1e-6


def test_bench_workload_full_size(gad):
    """16 x 2048^2 float32 at gamma = 0.01 to 1e-6 (the benchmark's batch):
    every field converges in a few passes and tracks its true residual, and a
    fixed-3-pass run matches the float32 oracle on one field."""
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=10.0, kcut=600.0)
    batch, n = 16, 2048
    ub = np.empty((batch, n, n), dtype=np.float32)
    for b in range(batch):
        ub[b] = oracle.filter_field(fields.random_scalar_field((n, n), b, spec), 0.01)
    t = _to_gpu(ub)
    res = gad.deconvolve(t, 0.01, method="pcg", tol=1e-6, maxit=300, true_residual=True, ndim=2)
    assert np.all(res.status == gad.AD_OK), res.status
    assert np.all(res.iterations <= 20), res.iterations
    assert np.all(res.true_residual < 50e-6)
    # three fixed passes against the float32 oracle on one field: the residual
    # history (a global norm; the float32 field itself is too sensitive at
    # gamma = 0.01 for a 1e-4 comparison, see test_fixed_passes_f32). The
    # residual drops 5000-fold in the first pass, so its float32 evaluation
    # carries an absolute error of a few float32 epsilons of ||r_0||: the
    # normalised history is compared to 2e-7 absolute (3.4 eps32)
    res = gad.deconvolve(t, 0.01, method="pcg", tol=0.0, maxit=3, ndim=2)
    base, _ = ensemble_runs("pcg", ub[9].astype(np.float64), 0.01, 0.0, 3, "f32", shifts=[(0, 0, 0)] * 2)
    np.testing.assert_allclose(res.history[9, :4], base.history, rtol=1e-5, atol=2e-7)


def test_bounded_wait_times_out_cleanly(gad):
    """The stencil's wait for its staged rows is bounded. With the limit at 0
    every wait gives up at once (after which each block still waits, bounded,
    for its own copies): the solve reports AD_ERR_TIMEOUT for each field
    instead of hanging, and the context then solves normally again."""
    _, ub = _problem((64, 96), 3, 0.1)
    t = _to_gpu(np.stack([ub, ub]))
    ok = gad.deconvolve(t, 0.1, method="pcg", tol=1e-6, maxit=100, ndim=2)
    gad.set_wait_limit(0)
    try:
        with pytest.raises(gad.GadError) as e:
            gad.deconvolve(t, 0.1, method="pcg", tol=1e-6, maxit=100, ndim=2)
        assert e.value.status == gad.AD_ERR_TIMEOUT
    finally:
        gad.set_wait_limit(1_000_000_000)
    again = gad.deconvolve(t, 0.1, method="pcg", tol=1e-6, maxit=100, ndim=2)
    assert list(again.status) == [gad.AD_OK, gad.AD_OK]
    np.testing.assert_array_equal(again.u.cpu().numpy(), ok.u.cpu().numpy())


# --- preconditioned CG in spectral space (AD_SPECTRAL | AD_PRECOND) ----------

@pytest.mark.parametrize("shape,gamma", [((64, 64), 0.1), ((96, 128), 0.1), ((32, 32, 32), 0.1), ((24, 48, 32), 0.1)])
@pytest.mark.parametrize("npass", [1, 5, 12])
def test_spectral_fixed_passes_f32(gad, shape, gamma, npass):
    from parity_tools import ensemble_runs_spectral
    _, ub = _problem(shape, 3, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=0.0, maxit=npass, ndim=len(shape), space="spectral")
    assert int(res.iterations[0]) == npass and int(res.status[0]) == gad.AD_MAXIT
    base, runs = ensemble_runs_spectral("pcg", ub.astype(np.float64), gamma, 0.0, npass, "f32")
    tol, spread = field_tolerance(base, runs, "f32")
    assert _rel(res.u.double().cpu().numpy(), base.u) < tol, (_rel(res.u.double().cpu().numpy(), base.u), spread)
    np.testing.assert_allclose(res.history[0, :npass + 1], base.history, rtol=history_tolerance(base, runs, 1e-5),
                               atol=H_ATOL)


@pytest.mark.parametrize("shape,gamma", [((128, 128), 0.1), ((256, 256), 0.01), ((64, 64, 64), 0.01)])
def test_spectral_fixed_passes_f64(gad, shape, gamma):
    from parity_tools import ensemble_runs_spectral
    _, ub = _problem(shape, 0, gamma, dtype=np.float64)
    for npass in (1, 5, 12):
        res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=0.0, maxit=npass, ndim=len(shape),
                             space="spectral")
        base, runs = ensemble_runs_spectral("pcg", ub, gamma, 0.0, npass, "f64")
        tol, spread = field_tolerance(base, runs, "f64")
        err = _rel(res.u.cpu().numpy(), base.u)
        assert err < 1e-12, "passes %d: error %.3e, oracle spread %.3e" % (npass, err, spread)


@pytest.mark.parametrize("gamma", [0.1, 0.01])
def test_spectral_f64_to_tolerance(gad, gamma):
    """Float64 to 1e-10: the pass count of the spectral oracle (which equals the
    physical one, tests/test_oracle_precond.py), the FFT-exact inverse."""
    from parity_tools import ensemble_runs_spectral
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=8.0)
    u = fields.random_scalar_field((128, 128), 0, spec)
    ub = oracle.filter_field(u, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method="pcg", tol=1e-10, maxit=500, true_residual=True,
                         space="spectral")
    base, runs = ensemble_runs_spectral("pcg", ub, gamma, 1e-10, 500, "f64")
    assert int(res.status[0]) == gad.AD_OK
    ok, counts = count_exact(int(res.iterations[0]), base, runs)
    assert ok, (int(res.iterations[0]), counts)
    assert _rel(res.u.cpu().numpy(), oracle.exact_inverse(ub, gamma)) < 1e-7
    assert res.true_residual[0] < 2e-10


@pytest.mark.parametrize("shape,gamma", [((512, 512), 0.01), ((64, 64, 64), 0.1)])
def test_spectral_to_tolerance_matches_physical(gad, shape, gamma):
    """To 1e-6 the spectral and physical preconditioned solves stop within a
    pass of each other and agree to the residual bound; the spectral count
    matches its precision-matched oracle."""
    from parity_tools import ensemble_runs_spectral
    _, ub = _problem(shape, 1, gamma)
    t = _to_gpu(ub)
    a = gad.deconvolve(t, gamma, method="pcg", tol=1e-6, maxit=500, ndim=len(shape), true_residual=True)
    b = gad.deconvolve(t, gamma, method="pcg", tol=1e-6, maxit=500, ndim=len(shape), true_residual=True,
                       space="spectral")
    assert int(a.status[0]) == int(b.status[0]) == gad.AD_OK
    assert abs(int(a.iterations[0]) - int(b.iterations[0])) <= 1
    base, runs = ensemble_runs_spectral("pcg", ub.astype(np.float64), gamma, 1e-6, 500, "f32")
    ok, counts = count_exact(int(b.iterations[0]), base, runs)
    assert ok, (int(b.iterations[0]), counts)
    ref = np.linalg.norm(ub.astype(np.float64) - oracle.filter_field(ub.astype(np.float64), gamma))
    gmin = oracle.transfer_function(shape, gamma).min()
    diff = np.linalg.norm(a.u.double().cpu().numpy() - b.u.double().cpu().numpy())
    assert diff <= 1.05 * (a.true_residual[0] + b.true_residual[0]) * ref / gmin
