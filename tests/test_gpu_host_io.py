"""ad_deconvolve_host: the solve of ad_deconvolve (Algorithms 1-4) with the
fields in host memory, copied in and out by the library. Its results must be
bitwise those of the device-buffer call (the same kernels on the same values),
for pinned and pageable buffers, in place, and with a non-finite field."""

import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu


def _batch(n, b, gamma, seed=0):
    us = [fields.random_scalar_field((n, n), seed + i, fields.spectrum_2d_kraichnan) for i in range(b)]
    return np.stack([oracle.filter_field(u, gamma) for u in us]).astype(np.float32)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("method,space", [("bicgstab", "physical"), ("cg", "spectral"), ("pcg", "physical")])
def test_host_solve_equals_device_solve(gad, pinned, method, space):
    import torch
    gamma = 0.01
    ub = _batch(256, 3, gamma)
    dev = gad.deconvolve(torch.from_numpy(ub).cuda(), gamma, method=method, tol=1e-6, maxit=3000, ndim=2,
                         space=space)
    h = torch.from_numpy(ub.copy())
    if pinned:
        h = h.pin_memory()
    res = gad.deconvolve_host(h, gamma, method=method, tol=1e-6, maxit=3000, ndim=2, space=space)
    assert not res.u.is_cuda
    np.testing.assert_array_equal(res.u.numpy(), dev.u.cpu().numpy())
    np.testing.assert_array_equal(res.iterations, dev.iterations)
    np.testing.assert_array_equal(res.status, dev.status)
    for b in range(3):
        n = int(res.iterations[b]) + 1
        np.testing.assert_array_equal(res.history[b, :n], dev.history[b, :n])
    assert np.all(res.status == gad.AD_OK)
    np.testing.assert_array_equal(h.numpy(), ub)          # the input is left as it was


def test_host_solve_in_place_and_nonfinite_field(gad):
    import torch
    gamma = 0.1
    ub = _batch(64, 3, gamma, seed=5)
    ub[1, 3, 7] = np.nan
    dev = gad.deconvolve(torch.from_numpy(ub).cuda(), gamma, method="bicgstab", tol=1e-8, maxit=500, ndim=2)
    h = torch.from_numpy(ub.copy())
    res = gad.deconvolve_host(h, gamma, method="bicgstab", tol=1e-8, maxit=500, ndim=2, out=h)
    assert res.u.data_ptr() == h.data_ptr()
    assert int(res.status[1]) == gad.AD_ERR_NONFINITE
    assert int(res.status[0]) == gad.AD_OK and int(res.status[2]) == gad.AD_OK
    for b in (0, 2):
        np.testing.assert_array_equal(h.numpy()[b], dev.u.cpu().numpy()[b])


def test_host_solve_arguments(gad):
    import torch
    with pytest.raises(ValueError):
        gad.deconvolve_host(torch.zeros((2, 16, 16), device="cuda"), 0.1, ndim=2)
    with pytest.raises(ValueError):
        gad.deconvolve_host(torch.zeros((2, 16, 16)), 0.1, ndim=2, out=torch.zeros((2, 16, 8)))
    with pytest.raises(gad.GadError):
        gad.deconvolve_host(torch.zeros((2, 16, 14)), 0.1, ndim=2)      # Nx not a multiple of 4
    r = gad.deconvolve_host(torch.zeros((0, 16, 16)), 0.1, ndim=2)
    assert r.u.shape == (0, 16, 16)
