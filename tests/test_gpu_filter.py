"""GPU parity of the filter G (Section 4, Eq. df2) against the CPU oracle,
through the C ABI: element by element on the same seeded inputs."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

# float32 FFT rounding grows like log2(N) * 2^-24; 3e-6 relative L2 covers N <= 4096
TOL_F32 = 3e-6
TOL_F64 = 1e-13


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES_2D = [(8, 8), (16, 12), (24, 48), (48, 48), (64, 128), (96, 96), (128, 128), (256, 256),
             (384, 384), (512, 512), (1024, 2048)]
SHAPES_3D = [(8, 8, 8), (12, 16, 8), (16, 16, 16), (24, 24, 24), (32, 48, 64), (64, 64, 64),
             (96, 96, 96), (128, 128, 128)]


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_filter_matches_oracle(gad, shape, dtype):
    import torch
    if dtype == "f64" and np.prod(shape) > 2 ** 21:
        pytest.skip("float64 is exercised on small grids")
    rng = np.random.default_rng(abs(hash(shape)) % 2 ** 32)
    batch = 3
    u = rng.standard_normal((batch,) + shape)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    ut = torch.tensor(u, dtype=tdt, device="cuda")
    u_in = ut.double().cpu().numpy()
    gamma = 0.1 if max(shape) < 512 else 0.01
    out = gad.filter(ut, gamma, ndim=len(shape)).double().cpu().numpy()
    for b in range(batch):
        ref = oracle.filter_field(u_in[b], gamma)
        assert _rel(out[b], ref) < (TOL_F32 if dtype == "f32" else TOL_F64), (b, _rel(out[b], ref))


def test_filter_in_place_and_single_mode(gad):
    import torch
    n = 64
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x)                         # Y varies along axis 0
    u = np.cos(4 * X + 4 * Y)                        # |k|^2 = 32, k_c = 0.5 * 32 = 16
    t = torch.tensor(u, dtype=torch.float64, device="cuda")
    gad.filter(t, 0.5, out=t)                        # in place
    np.testing.assert_allclose(t.cpu().numpy(), u / (1 + 32 / 256), atol=1e-14)


def test_filter_batch_zero_and_bad_shapes(gad):
    import torch
    t = torch.zeros((0, 16, 16), device="cuda")
    assert gad.filter(t, 0.1, ndim=2).shape == (0, 16, 16)
    for shape in [(10, 16), (16, 14), (16, 6), (20, 20)]:
        with pytest.raises(gad.GadError):
            gad.filter(torch.zeros(shape, device="cuda"), 0.1)
    with pytest.raises(gad.GadError):
        gad.filter(torch.zeros((16, 16), device="cuda"), 0.0)


def test_filter_full_size_batch_sampled(gad):
    """The benchmark's grid (2048^2 float32, batch 16): every field against
    the oracle at a deterministic sample of points, plus the global mean."""
    import torch
    from synth import fields
    rng = np.random.default_rng(7)
    batch, n = 16, 2048
    u = torch.empty((batch, n, n), dtype=torch.float32, device="cuda")
    u.copy_(torch.from_numpy(rng.standard_normal((batch, n, n)).astype(np.float32)))
    out = gad.filter(u, 0.01, ndim=2).cpu().numpy()
    uh = u.cpu().numpy()
    for b in (0, 7, 15):
        ref = oracle.filter_field(uh[b].astype(np.float64), 0.01)
        assert _rel(out[b], ref) < TOL_F32
    means = out.reshape(batch, -1).astype(np.float64).mean(axis=1)
    np.testing.assert_allclose(means, uh.reshape(batch, -1).astype(np.float64).mean(axis=1), atol=1e-6)
