"""GPU parity on the grids whose transforms take the fixed-plan FFT path
(compile-time radices and strides: 128-, 256- and 1024-point rows, 256-, 512-
and 2048-point filter columns, 256- and 512-point y columns), in 3D where the
other tests stop at 128^3: the filter G (Section 4, Eq. df2) element by
element against the oracle, and one BiCGSTAB pass (Algorithm 4) and one CG
pass (Algorithm 3) against the oracle's float32-storage emulation."""

import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu

TOL_F32 = 3e-6    # as for the filter elsewhere: log2(N) * 2^-24 growth, N <= 4096


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# (Nz, Ny, Nx): every fixed length along each axis it is used on
SHAPES = [(256, 256, 256),   # rows 128 (half of 256), y columns 256, z filter columns 256
          (512, 512, 32),    # y columns 512, z filter columns 512
          (32, 32, 512),     # rows 256
          (16, 16, 2048)]    # rows 1024


@pytest.mark.parametrize("shape", SHAPES)
def test_filter_3d_fixed_lengths(gad, shape):
    import torch
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal((2,) + shape).astype(np.float32)
    gamma = 0.1
    out = gad.filter(torch.from_numpy(u).cuda(), gamma, ndim=3).double().cpu().numpy()
    for b in range(2):
        ref = oracle.filter_field(u[b].astype(np.float64), gamma)
        assert _rel(out[b], ref) < TOL_F32, (shape, b, _rel(out[b], ref))


@pytest.mark.parametrize("method,shape", [("bicgstab", (256, 256, 256)), ("cg", (512, 512, 32))])
def test_one_pass_3d_fixed_lengths(gad, method, shape):
    import torch
    gamma = 0.1
    u = fields.random_velocity_field(shape, 11, fields.spectrum_3d_kolmogorov)[0]
    ub = oracle.filter_field(u, gamma).astype(np.float32)
    res = gad.deconvolve(torch.from_numpy(ub).cuda(), gamma, method=method, tol=0.0, maxit=1, ndim=3)
    assert int(res.iterations[0]) == 1 and int(res.status[0]) == gad.AD_MAXIT
    ref = oracle.solve(method, ub.astype(np.float64), gamma, tol=0.0, maxit=1, precision="f32")
    assert _rel(res.u.double().cpu().numpy(), ref.u) < 1e-5
    np.testing.assert_allclose(res.history[0, :2], ref.history, rtol=1e-5)
