"""Batched solve of fields of uneven size (one CUDA graph, one branch per grid
shape) and the tile autotuner, through the C ABI."""

import numpy as np
import pytest

import oracle
from synth import fields

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
