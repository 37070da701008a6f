"""Batched solve of fields of uneven size and the tile autotuner, through the
C ABI. A batch of several shapes runs one graph branch per shape group
(default) or, for float32, one launch per pass stage over the blocks of every
shape group (a device work list); both are compared with the single-field
solves (bitwise) and with the oracle."""

import numpy as np
import pytest

import oracle
from synth import fields
from parity_tools import ensemble_runs, field_tolerance

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _mixed_fields():
    specs = [((64, 64), 0.1, np.float32), ((96, 128), 0.1, np.float32), ((256, 256), 0.01, np.float32),
             ((64, 64), 0.1, np.float32), ((32, 32, 32), 0.1, np.float32), ((24, 48, 32), 0.1, np.float32),
             ((128, 128), 0.1, np.float64), ((32, 32, 32), 0.05, np.float32)]
    out = []
    for i, (shape, gamma, dt) in enumerate(specs):
        if len(shape) == 3:
            u = fields.random_velocity_field(shape, i, fields.spectrum_3d_kolmogorov)[i % 3]
        else:
            u = fields.random_scalar_field(shape, i, fields.spectrum_2d_kraichnan)
        out.append((oracle.filter_field(u, gamma).astype(dt), gamma))
    return out


@pytest.mark.parametrize("method", ["vancittert", "cg", "bicgstab", "sd"])
def test_batched_equals_single_solves(gad, method):
    import torch
    data = _mixed_fields()
    ts = [torch.from_numpy(a).cuda() for a, _ in data]
    maxit = 3000 if method in ("vancittert", "sd") else 800
    outs, its, sts, hist = gad.deconvolve_batched(ts, [g for _, g in data], method=method, tol=1e-6, maxit=maxit)
    for i, (t, (a, g)) in enumerate(zip(ts, data)):
        single = gad.deconvolve(t, g, method=method, tol=1e-6, maxit=maxit, ndim=a.ndim)
        assert its[i] == single.iterations[0] and sts[i] == single.status[0], i
        np.testing.assert_array_equal(outs[i].cpu().numpy(), single.u.cpu().numpy())
        np.testing.assert_array_equal(hist[i][:its[i] + 1], single.history[0, :its[i] + 1])
    # a second call reuses the cached graph and gives the same fields
    outs2, its2, _, _ = gad.deconvolve_batched(ts, [g for _, g in data], method=method, tol=1e-6, maxit=maxit,
                                               outs=outs)
    assert list(its2) == list(its)


@pytest.mark.parametrize("method", ["vancittert", "cg", "bicgstab", "sd"])
def test_batched_fixed_passes_match_oracle(gad, method):
    import torch
    data = _mixed_fields()
    ts = [torch.from_numpy(a).cuda() for a, _ in data]
    outs, its, sts, _ = gad.deconvolve_batched(ts, [g for _, g in data], method=method, tol=0.0, maxit=1)
    assert list(its) == [1] * len(data) and all(s == gad.AD_MAXIT for s in sts)
    for o, (a, g) in zip(outs, data):
        prec = "f64" if a.dtype == np.float64 else "f32"
        ref = oracle.solve(method, a.astype(np.float64), g, tol=0.0, maxit=1, precision=prec)
        assert _rel(o.double().cpu().numpy(), ref.u) < (1e-12 if prec == "f64" else 1e-5)


def test_autotuned_plan_matches_default(gad):
    """Tuned tiles change only which threads do which butterflies and how the
    dot partials are grouped: fields agree to rounding with the default tiles."""
    import torch
    # shapes used by no other test: tuned plans stay in the context
    u = fields.random_scalar_field((384, 384), 3, fields.spectrum_2d_kraichnan)
    ub = torch.from_numpy(oracle.filter_field(u, 0.01).astype(np.float32)).cuda()
    ref = gad.deconvolve(ub, 0.01, method="cg", tol=0.0, maxit=5)
    gad.autotune((384, 384), 0.01, batch=1, method="cg")
    tuned = gad.deconvolve(ub, 0.01, method="cg", tol=0.0, maxit=5)
    assert _rel(tuned.u.cpu().numpy(), ref.u.cpu().numpy()) < 1e-5
    u3 = fields.random_velocity_field((48, 64, 32), 4, fields.spectrum_3d_kolmogorov)[0]
    ub3 = torch.from_numpy(oracle.filter_field(u3, 0.1).astype(np.float32)).cuda()
    ref3 = gad.deconvolve(ub3, 0.1, method="bicgstab", tol=0.0, maxit=3, ndim=3)
    gad.autotune((48, 64, 32), 0.1, batch=1, method="bicgstab")
    tuned3 = gad.deconvolve(ub3, 0.1, method="bicgstab", tol=0.0, maxit=3, ndim=3)
    assert _rel(tuned3.u.cpu().numpy(), ref3.u.cpu().numpy()) < 1e-5


def test_batched_with_autotune_and_bad_arguments(gad):
    import torch
    data = []
    for i, shape in enumerate([(144, 144), (72, 96), (192, 192)]):
        u = fields.random_scalar_field(shape, 20 + i, fields.spectrum_2d_kraichnan)
        data.append((oracle.filter_field(u, 0.1).astype(np.float32), 0.1))
    ts = [torch.from_numpy(a).cuda() for a, _ in data]
    singles = [gad.deconvolve(t, g, method="cg", tol=1e-6, maxit=800) for t, (_, g) in zip(ts, data)]
    gad.autotune(for_batched=True)
    try:
        outs, its, sts, _ = gad.deconvolve_batched(ts, [g for _, g in data], method="cg", tol=1e-6, maxit=800)
    finally:
        gad.autotune(for_batched=False)
    for i, single in enumerate(singles):
        assert sts[i] == gad.AD_OK and abs(int(its[i]) - int(single.iterations[0])) <= 2
        assert _rel(outs[i].cpu().numpy(), single.u.cpu().numpy()) < 1e-4
    with pytest.raises(gad.GadError):
        gad.deconvolve_batched(ts, [0.1, -1.0, 0.1])
    with pytest.raises(gad.GadError):
        gad.deconvolve_batched(ts, [g for _, g in data], outs=ts)     # aliasing
    assert gad.deconvolve_batched([], [])[0] == []


def _f32_fields():
    """Float32 fields of 2D and 3D shapes, with radix-3 lengths (per-thread
    element count 24) beside powers of two, two fields sharing a shape."""
    specs = [((64, 64), 0.1), ((96, 128), 0.1), ((256, 256), 0.01), ((64, 64), 0.1), ((32, 32, 32), 0.1),
             ((24, 48, 32), 0.1), ((48, 36, 24), 0.1), ((128, 384), 0.1)]
    out = []
    for i, (shape, gamma) in enumerate(specs):
        if len(shape) == 3:
            u = fields.random_velocity_field(shape, 40 + i, fields.spectrum_3d_kolmogorov)[i % 3]
        else:
            u = fields.random_scalar_field(shape, 40 + i, fields.spectrum_2d_kraichnan)
        out.append((oracle.filter_field(u, gamma).astype(np.float32), gamma))
    return out


@pytest.mark.parametrize("method", ["vancittert", "cg", "bicgstab", "sd"])
def test_one_launch_per_stage_equals_branches_and_singles(gad, method):
    """The work-list launches run each group's pass code in the group's own
    launch shape: fields, pass counts and histories bitwise equal to the
    per-group branches and to single-field solves."""
    import torch
    data = _f32_fields()
    ts = [torch.from_numpy(a).cuda() for a, _ in data]
    gammas = [g for _, g in data]
    maxit = 3000 if method in ("vancittert", "sd") else 800
    gad.set_batched_launch(True)
    try:
        om, im, sm, hm = gad.deconvolve_batched(ts, gammas, method=method, tol=1e-6, maxit=maxit)
        lm = gad.last_launch_count()
    finally:
        gad.set_batched_launch(False)
    ob, ib, sb, hb = gad.deconvolve_batched(ts, gammas, method=method, tol=1e-6, maxit=maxit)
    assert list(im) == list(ib) and list(sm) == list(sb)
    for i, (t, (a, g)) in enumerate(zip(ts, data)):
        np.testing.assert_array_equal(om[i].cpu().numpy(), ob[i].cpu().numpy())
        np.testing.assert_array_equal(hm[i][:im[i] + 1], hb[i][:ib[i] + 1])
        single = gad.deconvolve(t, g, method=method, tol=1e-6, maxit=maxit, ndim=a.ndim)
        assert im[i] == single.iterations[0] and sm[i] == single.status[0], i
        np.testing.assert_array_equal(om[i].cpu().numpy(), single.u.cpu().numpy())
    # one launch per stage and (element count, block size) class, for as many
    # loop passes as the slowest field needs
    assert 0 < lm <= 64 * (max(im) + 2), lm


@pytest.mark.parametrize("method", ["vancittert", "cg", "bicgstab", "sd"])
def test_one_launch_per_stage_fixed_passes_match_oracle(gad, method):
    """Fixed passes of the work-list batch against the precision-matched
    oracle, every shape (2D, 3D, radix-3 lengths): five, three for BiCGSTAB
    (whose float32 iterates on these grids drift apart by 4e-5 between
    equally valid evaluations at five, measured)."""
    import torch
    data = _f32_fields()
    ts = [torch.from_numpy(a).cuda() for a, _ in data]
    npass = 3 if method == "bicgstab" else 5
    gad.set_batched_launch(True)
    try:
        outs, its, sts, _ = gad.deconvolve_batched(ts, [g for _, g in data], method=method, tol=0.0, maxit=npass)
    finally:
        gad.set_batched_launch(False)
    assert list(its) == [npass] * len(data) and all(x == gad.AD_MAXIT for x in sts)
    for o, (a, g) in zip(outs, data):
        base, runs = ensemble_runs(method, a.astype(np.float64), g, 0.0, npass, "f32")
        tol, spread = field_tolerance(base, runs, "f32")
        err = _rel(o.double().cpu().numpy(), base.u)
        assert err < tol, (a.shape, err, tol, spread)
