"""The tolerance model used by the GPU parity tests (CPU only)."""

import numpy as np

import oracle
import oracle.solvers as osv
from parity_tools import count_ok, ensemble_runs, field_tolerance, precision_filter, rel
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
    b64, r64 = ensemble_runs("cg", ub, 0.1, 0.0, 10, "f64")
    b32, r32 = ensemble_runs("cg", ub, 0.1, 0.0, 10, "f32")
    assert field_tolerance(b64, r64, "f64")[1] < field_tolerance(b32, r32, "f32")[1]
    assert field_tolerance(b64, r64, "f64")[0] >= 1e-12

    class R:
        def __init__(self, n):
            self.iterations = n
    assert count_ok(5, R(5), [R(5), R(5)]) == (True, [5, 5, 5])
    assert count_ok(6, R(5), [R(5), R(5)])[0] is False
    assert count_ok(7, R(5), [R(6), R(5)])[0] is True      # range 1: [3, 8]
    assert count_ok(8, R(5), [R(6), R(5)])[0] is True
    assert count_ok(9, R(5), [R(6), R(5)])[0] is False
