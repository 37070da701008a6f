"""GPU parity of the solvers (Algorithms 1-4) against the CPU oracle through
the C ABI.

Tolerances (tests/parity_tools.py):
  * one pass: relative L2 <= 1e-5 (float32 fields, against the oracle's
    float32-storage emulation) or <= 1e-12 (float64), outright;
  * more passes: against the oracle with G evaluated in the path's
    precision, within max(1e-5 or 1e-12, 3 x that oracle's spread over
    equally valid (periodically shifted) evaluations of G), never above 1e-4
    (float32) or 1e-12 (float64). The pass counts compared are the ones at
    which that is meaningful, by measurement: float32 Krylov iterates are
    chaotic under rounding (the oracle's own spread after 20 passes is up to
    1.5e-4 for CG and 1e-2 for BiCGSTAB at gamma = 0.1, 64^2), so longer
    float32 runs are compared where the spread stays small and checked
    otherwise by the residual bound against the exact (Fourier) inverse;
  * pass counts to a tolerance: exact where every shifted oracle run gives
    the same count; within the observed range where equally valid float64
    evaluations give different counts (see count_in_range).
"""

import numpy as np
import pytest

import oracle
from synth import fields
from parity_tools import count_exact, count_in_range, ensemble_runs, field_tolerance, history_tolerance, rel, SHIFTS

pytestmark = pytest.mark.gpu

METHODS = ["vancittert", "sd", "cg", "bicgstab"]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _problem(shape, seed, gamma, dtype=np.float32, spectrum=None):
    spectrum = spectrum or fields.spectrum_2d_kraichnan
    if len(shape) == 3:
        u = fields.random_velocity_field(shape, seed, fields.spectrum_3d_kolmogorov)[0]
    else:
        u = fields.random_scalar_field(shape, seed, spectrum)
    ub = oracle.filter_field(u, gamma).astype(dtype)
    return u, ub


def _to_gpu(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("shape,gamma", [((64, 64), 0.1), ((96, 128), 0.1), ((256, 256), 0.01),
                                         ((32, 32, 32), 0.1), ((24, 48, 32), 0.1)])
@pytest.mark.parametrize("npass", [1, 5])
def test_fixed_passes_f32(gad, method, shape, gamma, npass):
    _, ub = _problem(shape, 3, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method=method, tol=0.0, maxit=npass, ndim=len(shape))
    assert int(res.iterations[0]) == npass and int(res.status[0]) == gad.AD_MAXIT
    u64 = ub.astype(np.float64)
    got = res.u.double().cpu().numpy()
    if npass == 1:
        err = _rel(got, oracle.solve(method, u64, gamma, tol=0.0, maxit=npass, precision="f32").u)
        assert err < 1e-5, err
        return
    base, runs = ensemble_runs(method, u64, gamma, 0.0, npass, "f32")
    tol, spread = field_tolerance(base, runs, "f32")
    err = _rel(got, base.u)
    assert err < tol, "error %.3e, tolerance %.3e, oracle spread %.3e" % (err, tol, spread)
    np.testing.assert_allclose(res.history[0, :npass + 1], base.history,
                               rtol=history_tolerance(base, runs, 1e-5))


# (method, shape, gamma, passes) whose float32 iterates stay comparable at the
# 1e-4 ceiling: the oracle's spread over shifted evaluations of G was measured
# at 5, 10, 15 and 20 passes on these problems, and these are the cases where
# 3 x spread stays below 1e-4 (Van Cittert everywhere: no Krylov scalars).
LONG_F32 = ([(m, (64, 64), 0.1, 10) for m in METHODS] + [(m, (96, 128), 0.1, 10) for m in METHODS] +
            [(m, sh, g, 10) for m in ("vancittert", "sd") for sh, g in (((256, 256), 0.01), ((32, 32, 32), 0.1),
                                                                        ((24, 48, 32), 0.1))] +
            [("vancittert", sh, g, 20) for sh, g in (((64, 64), 0.1), ((96, 128), 0.1), ((256, 256), 0.01),
                                                     ((32, 32, 32), 0.1), ((24, 48, 32), 0.1))] +
            [("sd", (64, 64), 0.1, 20), ("sd", (96, 128), 0.1, 20), ("cg", (96, 128), 0.1, 20)])


@pytest.mark.parametrize("method,shape,gamma,npass", LONG_F32)
def test_longer_fixed_passes_f32(gad, method, shape, gamma, npass):
    _, ub = _problem(shape, 3, gamma)
    res = gad.deconvolve(_to_gpu(ub), gamma, method=method, tol=0.0, maxit=npass, ndim=len(shape))
    base, runs = ensemble_runs(method, ub.astype(np.float64), gamma, 0.0, npass, "f32")
    tol, spread = field_tolerance(base, runs, "f32")
    err = _rel(res.u.double().cpu().numpy(), base.u)
    assert err < tol, "error %.3e, tolerance %.3e, oracle spread %.3e" % (err, tol, spread)


F64_PASSES = {"vancittert": (1, 5, 20, 200), "sd": (1, 5, 20, 200), "cg": (1, 5, 20, 200),
              "bicgstab": (1, 5, 12, 200)}


@pytest.mark.parametrize("method", METHODS)
def test_fixed_passes_f64(gad, method):
    """128^2 float64, gamma = 0.1: fields within 1e-12 of the oracle at fixed
    pass counts (BiCGSTAB to 12 passes: its float64 iterates drift 1.3e-11
    apart between equally valid evaluations by pass 20, measured; all
    methods again at 200 passes, past convergence)."""
    _, ub = _problem((128, 128), 0, 0.1, dtype=np.float64)
    for npass in F64_PASSES[method]:
        res = gad.deconvolve(_to_gpu(ub), 0.1, method=method, tol=0.0, maxit=npass)
        base, runs = ensemble_runs(method, ub, 0.1, 0.0, npass, "f64")
        tol, spread = field_tolerance(base, runs, "f64")
        err = _rel(res.u.cpu().numpy(), base.u)
        assert err < 1e-12, "passes %d: error %.3e, oracle spread %.3e" % (npass, err, spread)
        # the histories to 20 passes (beyond, the Krylov residuals wander between
        # equally valid evaluations before they converge)
        n = min(npass, 20)
        np.testing.assert_allclose(res.history[0, :n + 1], base.history[:n + 1], rtol=1e-9)


# the oracle's pass counts to 1e-10 over eight shifted (equally valid) float64
# evaluations of G vary for the Krylov methods (CG 119-120, SD 1422-1424,
# BiCGSTAB 78-85 at four shifts, measured)
SHIFTS8 = SHIFTS + [(2, 9, 4), (17, 4, 1), (29, 13, 6), (40, 21, 8)]


@pytest.mark.parametrize("method", ["vancittert", "cg", "bicgstab", "sd"])
def test_config1_f64_to_tolerance(gad, method):
    """128^2 float64 vorticity, gamma = 0.1, to relative residual 1e-10.
    Van Cittert: pass count exact and field within 1e-12 of the oracle. CG
    and SD: the pass count within the range of equally valid float64
    evaluations and the field within 1e-10 of an oracle run with the same
    count (when one exists). BiCGSTAB: its count and final iterate are chaotic
    even in float64 (78-85 passes over four equally valid evaluations, and
    same-count runs 4e-10 apart, measured), so it is pinned by the rest. For
    all: the history to 20 passes within 1e-9, the recurrence and true
    residuals at the tolerance, and the distance to the FFT-exact inverse
    within the residual bound ||u - u_ex|| <= ||r|| / G_min."""
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=8.0)
    u = fields.random_scalar_field((128, 128), 0, spec)
    ub = oracle.filter_field(u, 0.1)
    maxit = 5000 if method in ("vancittert", "sd") else 1000
    res = gad.deconvolve(_to_gpu(ub), 0.1, method=method, tol=1e-10, maxit=maxit, true_residual=True)
    n_gpu = int(res.iterations[0])
    got = res.u.cpu().numpy()
    assert int(res.status[0]) == gad.AD_OK
    if method == "vancittert":
        base, runs = ensemble_runs(method, ub, 0.1, 1e-10, maxit, "f64")
        ok, counts = count_exact(n_gpu, base, runs)
        assert ok, (n_gpu, counts)
        err = _rel(got, base.u)
        assert err < 1e-12, err
    elif method in ("cg", "sd"):
        base, runs = ensemble_runs(method, ub, 0.1, 1e-10, maxit, "f64", shifts=SHIFTS8)
        ok, counts = count_in_range(n_gpu, base, runs)
        assert ok, (n_gpu, counts)
        same = [_rel(got, r.u) for r in [base] + runs if r.iterations == n_gpu]
        assert all(e < 1e-10 for e in same), same
    else:
        base = oracle.solve(method, ub, 0.1, tol=1e-10, maxit=maxit)
    n = min(n_gpu, base.iterations, 20)
    np.testing.assert_allclose(res.history[0, :n + 1], base.history[:n + 1], rtol=1e-9)
    assert res.history[0, n_gpu] <= 1e-10
    assert res.true_residual[0] < 2e-10
    uex = oracle.exact_inverse(ub, 0.1)
    ref = np.linalg.norm(ub - oracle.filter_field(ub, 0.1))
    gmin = oracle.transfer_function((128, 128), 0.1).min()
    assert np.linalg.norm(got - uex) <= 1.05 * res.true_residual[0] * ref / gmin
    assert _rel(got, uex) < 1e-7


# float32 pass counts to 1e-6 that every shifted oracle run agrees on
# (measured); elsewhere the count is chaotic under rounding (BiCGSTAB at
# 512^2, gamma = 0.01: 303-338 over four equally valid evaluations, the GPU
# 260) and only the convergence and its bounds are checked
EXACT_COUNT_F32 = {("cg", (256, 256), 0.1), ("cg", (64, 64, 64), 0.1)}


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
@pytest.mark.parametrize("shape,gamma", [((256, 256), 0.1), ((512, 512), 0.01), ((64, 64, 64), 0.1)])
def test_f32_to_tolerance_counts(gad, method, shape, gamma):
    _, ub = _problem(shape, 1, gamma)
    tol = 1e-6
    res = gad.deconvolve(_to_gpu(ub), gamma, method=method, tol=tol, maxit=2000, ndim=len(shape),
                         true_residual=True)
    n_gpu = int(res.iterations[0])
    assert int(res.status[0]) == gad.AD_OK
    if (method, shape, gamma) in EXACT_COUNT_F32:
        base, runs = ensemble_runs(method, ub.astype(np.float64), gamma, tol, 2000, "f32")
        ok, counts = count_exact(n_gpu, base, runs)
        assert ok, (n_gpu, counts)
        tolf, spread = field_tolerance(base, runs, "f32")
        err = _rel(res.u.double().cpu().numpy(), base.u)
        assert err < tolf, "error %.3e, tolerance %.3e, oracle spread %.3e" % (err, tolf, spread)
    assert res.history[0, n_gpu] <= tol
    # the recurrence residual tracks the true one to float32 accuracy
    assert res.true_residual[0] < 20 * tol
    # against the exact (Fourier) inverse: ||u - u_ex|| <= ||r_true|| / G_hat_min
    uex = oracle.exact_inverse(ub.astype(np.float64), gamma)
    ref = np.linalg.norm(ub.astype(np.float64) - oracle.filter_field(ub.astype(np.float64), gamma))
    gmin = oracle.transfer_function(shape, gamma).min()
    err = np.linalg.norm(res.u.double().cpu().numpy() - uex)
    assert err <= 1.05 * res.true_residual[0] * ref / gmin


def test_edge_cases_per_field_status(gad):
    """A batch mixing a regular field, a zero field, a constant field and a
    field holding a NaN: per-field statuses, and the regular field's result
    is bitwise the same as when it is solved alone (fields never interact)."""
    n = 64
    _, ub = _problem((n, n), 2, 0.1)
    batch = np.stack([ub, np.zeros_like(ub), np.full_like(ub, 2.5), ub.copy()])
    batch[3, 5, 7] = np.nan
    for method in METHODS:
        res = gad.deconvolve(_to_gpu(batch), 0.1, method=method, tol=1e-5, maxit=3000, ndim=2)
        alone = gad.deconvolve(_to_gpu(ub), 0.1, method=method, tol=1e-5, maxit=3000)
        assert int(res.status[0]) == gad.AD_OK and res.iterations[0] == alone.iterations[0]
        np.testing.assert_array_equal(res.u[0].cpu().numpy(), alone.u.cpu().numpy())
        assert res.history[0, res.iterations[0]] <= 1e-5
        assert int(res.status[1]) == gad.AD_OK and int(res.iterations[1]) == 0
        assert int(res.status[2]) == gad.AD_OK and int(res.iterations[2]) == 0
        assert int(res.status[3]) == gad.AD_ERR_NONFINITE
        np.testing.assert_array_equal(res.u[1].cpu().numpy(), 0.0)
        np.testing.assert_array_equal(res.u[2].cpu().numpy(), 2.5)


def test_maxit_zero_and_bad_arguments(gad):
    import torch
    _, ub = _problem((32, 32), 4, 0.1)
    t = _to_gpu(ub)
    res = gad.deconvolve(t, 0.1, method="cg", tol=1e-6, maxit=0)
    assert int(res.status[0]) == gad.AD_MAXIT and int(res.iterations[0]) == 0
    np.testing.assert_array_equal(res.u.cpu().numpy(), ub)
    with pytest.raises(gad.GadError):
        gad.deconvolve(t, 0.1, method="cg", tol=-1.0, maxit=10)
    with pytest.raises(gad.GadError):
        gad.deconvolve(t, 0.1, method="cg", tol=1e-6, maxit=10, out=t)    # aliasing
    e = gad.deconvolve(torch.zeros((0, 32, 32), device="cuda"), 0.1, ndim=2)
    assert e.iterations.shape == (0,)


def test_single_mode_terminates_in_one_pass(gad):
    n = 64
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    u = np.cos(3 * X + 5 * Y)
    ub = oracle.filter_field(u, 0.2)
    for method in ("sd", "cg", "bicgstab"):
        res = gad.deconvolve(_to_gpu(ub), 0.2, method=method, tol=1e-10, maxit=10)
        assert int(res.iterations[0]) == 1 and int(res.status[0]) == gad.AD_OK, method
        np.testing.assert_allclose(res.u.cpu().numpy(), u, atol=1e-12)


def test_initial_guess_f64(gad):
    u, ub = _problem((96, 96), 5, 0.1, dtype=np.float64)
    u0 = 0.5 * (ub + u)
    res = gad.deconvolve(_to_gpu(ub), 0.1, method="bicgstab", tol=1e-9, maxit=500, u0=_to_gpu(u0))
    # BiCGSTAB's pass count to a tolerance is chaotic even in float64 (see
    # test_config1_f64_to_tolerance): the start and the first passes are
    # compared, then convergence and the distance to the exact inverse
    base = oracle.solve("bicgstab", ub, 0.1, tol=1e-9, maxit=500, u0=u0)
    np.testing.assert_allclose(res.history[0, :13], base.history[:13], rtol=1e-9)
    assert res.history[0, 0] == pytest.approx(base.history[0], rel=1e-12)
    assert res.history[0, 0] < 1.0
    assert res.history[0, int(res.iterations[0])] <= 1e-9
    uex = oracle.exact_inverse(ub, 0.1)
    assert _rel(res.u.cpu().numpy(), uex) < 1e-6
    res1 = gad.deconvolve(_to_gpu(ub), 0.1, method="bicgstab", tol=0.0, maxit=1, u0=_to_gpu(u0))
    ref1 = oracle.bicgstab(ub, 0.1, tol=0.0, maxit=1, u0=u0)
    assert _rel(res1.u.cpu().numpy(), ref1.u) < 1e-12
    np.testing.assert_allclose(res1.history[0], ref1.history, rtol=1e-11)


def test_graph_and_host_loop_agree(gad):
    _, ub = _problem((128, 128), 6, 0.1)
    t = _to_gpu(ub)
    for method in METHODS:
        gad.set_graph_mode(True)
        a = gad.deconvolve(t, 0.1, method=method, tol=1e-6, maxit=3000)
        gad.set_graph_mode(False)
        b = gad.deconvolve(t, 0.1, method=method, tol=1e-6, maxit=3000)
        gad.set_graph_mode(True)
        assert int(a.iterations[0]) == int(b.iterations[0])
        np.testing.assert_array_equal(a.u.cpu().numpy(), b.u.cpu().numpy())


def test_repeat_solves_are_deterministic(gad):
    _, ub = _problem((256, 256), 8, 0.01)
    t = _to_gpu(np.stack([ub, ub]))
    a = gad.deconvolve(t, 0.01, method="bicgstab", tol=1e-6, maxit=2000, ndim=2)
    b = gad.deconvolve(t, 0.01, method="bicgstab", tol=1e-6, maxit=2000, ndim=2)
    np.testing.assert_array_equal(a.u.cpu().numpy(), b.u.cpu().numpy())
    assert list(a.iterations) == list(b.iterations) and a.iterations[0] == a.iterations[1]


def test_bench_workload_full_size(gad):
    """The benchmark's launch configuration (2048^2 float32, batch 16,
    gamma = 0.01, tolerance 1e-6): every field converges, its true residual
    tracks the recurrence, and a fixed-3-pass run matches the oracle
    element by element on one field."""
    import torch
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=10.0, kcut=600.0)
    batch, n = 16, 2048
    ub = np.empty((batch, n, n), dtype=np.float32)
    for b in range(batch):
        ub[b] = oracle.filter_field(fields.random_scalar_field((n, n), b, spec), 0.01)
    t = _to_gpu(ub)
    for method in ("cg", "bicgstab"):
        res = gad.deconvolve(t, 0.01, method=method, tol=1e-6, maxit=3000, true_residual=True, ndim=2)
        assert np.all(res.status == gad.AD_OK), res.status
        assert np.all(res.true_residual < 50e-6)
        for b in range(batch):
            assert res.history[b, res.iterations[b]] <= 1e-6
    res = gad.deconvolve(t, 0.01, method="bicgstab", tol=0.0, maxit=3, ndim=2)
    ref = oracle.bicgstab(ub[5].astype(np.float64), 0.01, tol=0.0, maxit=3, precision="f32")
    assert _rel(res.u[5].double().cpu().numpy(), ref.u) < 1e-5
    # the launch shapes the benchmark times: tile widths picked by the autotuner
    gad.autotune((n, n), 0.01, batch, method="bicgstab")
    res = gad.deconvolve(t, 0.01, method="bicgstab", tol=1e-6, maxit=3000, true_residual=True, ndim=2)
    assert np.all(res.status == gad.AD_OK), res.status
    assert np.all(res.true_residual < 50e-6)
    res = gad.deconvolve(t, 0.01, method="bicgstab", tol=0.0, maxit=3, ndim=2)
    assert _rel(res.u[5].double().cpu().numpy(), ref.u) < 1e-5
