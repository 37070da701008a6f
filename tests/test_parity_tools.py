"""The tolerance model used by the GPU parity tests (CPU only)."""

import numpy as np

import oracle
import oracle.solvers as osv
import pytest

from parity_tools import (CAP, count_exact, count_in_range, ensemble_runs, field_tolerance, history_tolerance,
                          precision_filter, rel)
from synth import fields


def test_precision_filter_is_scoped_and_shift_invariant():
    clean = osv.filter_field
    u = fields.random_scalar_field((32, 48), 1, fields.spectrum_2d_kraichnan)
    exact = oracle.filter_field(u, 0.1)
    with precision_filter("f64", (3, 5, 0)):
        shifted = osv.filter_field(u, 0.1)
    assert osv.filter_field is clean
    assert rel(shifted, exact) < 1e-15
    with precision_filter("f32", (0, 0, 0)):
        single = osv.filter_field(u, 0.1)
    assert osv.filter_field is clean
    assert 1e-9 < rel(single, exact) < 1e-6      # float32 FFT rounding, nothing worse


def test_tolerance_and_counts_rule():
    u = fields.random_scalar_field((32, 32), 2, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, 0.1)
    b64, r64 = ensemble_runs("cg", ub, 0.1, 0.0, 5, "f64")
    b32, r32 = ensemble_runs("cg", ub, 0.1, 0.0, 5, "f32")
    assert field_tolerance(b64, r64, "f64")[1] < field_tolerance(b32, r32, "f32")[1]
    assert 1e-12 <= field_tolerance(b64, r64, "f64")[0] <= CAP["f64"]
    assert field_tolerance(b32, r32, "f32")[0] <= CAP["f32"]

    class R:
        def __init__(self, n):
            self.iterations = n
    assert count_exact(5, R(5), [R(5), R(5)]) == (True, [5, 5, 5])
    assert count_exact(6, R(5), [R(5), R(5)])[0] is False
    with pytest.raises(AssertionError):          # the oracle's count is not unique: no exact comparison
        count_exact(5, R(5), [R(6), R(5)])
    assert count_in_range(6, R(5), [R(7), R(5)]) == (True, [5, 7, 5])
    assert count_in_range(8, R(5), [R(7), R(5)])[0] is False    # no widening beyond the observed range
    assert count_in_range(4, R(5), [R(7), R(5)])[0] is False


def test_tolerances_have_a_ceiling():
    """A case whose oracle spread would need more than the ceiling fails
    instead of widening the tolerance (20 CG passes at 256^2, gamma = 0.01,
    float32: the oracle's own spread is ~1.5e-4)."""
    u = fields.random_scalar_field((64, 64), 3, fields.spectrum_2d_kraichnan)
    ub = oracle.filter_field(u, 0.1)

    class Run:
        def __init__(self, x, h):
            self.u, self.history = x, h
    base = Run(ub, np.ones(3))
    far = Run(ub * (1 + 5e-5), np.ones(3) * (1 + 1e-3))
    with pytest.raises(AssertionError, match="too chaotic"):
        field_tolerance(base, [far], "f32")
    with pytest.raises(AssertionError, match="too chaotic"):
        field_tolerance(base, [Run(ub * (1 + 1e-12), None)], "f64")
    with pytest.raises(AssertionError, match="too chaotic"):
        history_tolerance(base, [far], 1e-5)
    near = Run(ub * (1 + 2e-6), np.ones(3))
    tol, spread = field_tolerance(base, [near], "f32")
    assert abs(spread - 2e-6) < 1e-9 and tol == 1e-5
