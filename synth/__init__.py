"""Seeded synthetic turbulence-like fields: the inputs shared by the CPU oracle,
the tests and the benchmark.

This module draws random fields with a prescribed isotropic shell spectrum.
It holds none of the deconvolution method's arithmetic (no filter, no
solver): the filtered field that the method consumes is made by whichever
side is under test (the oracle in the tests, the library in the benchmark).
"""

from .fields import (  # noqa: F401
    spectrum_2d_kraichnan,
    spectrum_3d_kolmogorov,
    random_scalar_field,
    random_velocity_field,
    shell_spectrum,
    gamma_for_grid,
    WORKLOADS,
    smooth_sizes,
    uneven_batch,
)
