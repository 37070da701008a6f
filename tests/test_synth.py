"""The seeded input generator: reproducibility, normalisation, spectrum shape
and (3D velocity) discrete incompressibility."""

import numpy as np

from synth import fields


def test_scalar_field_reproducible_and_normalised():
    a = fields.random_scalar_field((64, 48), 3, fields.spectrum_2d_kraichnan)
    b = fields.random_scalar_field((64, 48), 3, fields.spectrum_2d_kraichnan)
    c = fields.random_scalar_field((64, 48), 4, fields.spectrum_2d_kraichnan)
    assert np.array_equal(a, b) and not np.allclose(a, c)
    assert abs(a.mean()) < 1e-14 and abs(np.sqrt(np.mean(a * a)) - 1.0) < 1e-12


def test_scalar_spectrum_follows_target():
    """The ensemble shell spectrum tracks E(k) (k^-3 range) within sampling noise."""
    spec = lambda k: fields.spectrum_2d_kraichnan(k, kp=8.0)
    acc = None
    for s in range(8):
        k, e = fields.shell_spectrum(fields.random_scalar_field((256, 256), s, spec))
        acc = e if acc is None else acc + e
    ks = np.arange(6, 100)
    ratio = acc[ks] / spec(ks)
    ratio /= np.median(ratio)
    assert np.all(np.abs(ratio - 1.0) < 0.25)
    # log-log slope over the inertial range is close to -3
    sl = np.polyfit(np.log(ks[30:]), np.log(acc[ks[30:]]), 1)[0]
    assert -3.4 < sl < -2.6


def test_velocity_solenoidal_and_normalised():
    v = fields.random_velocity_field((24, 16, 32), 2, fields.spectrum_3d_kolmogorov)
    assert v.shape == (3, 24, 16, 32)
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - 1.0) < 1e-12
    kz, ky, kx = np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in (24, 16, 32)], indexing="ij")
    div = kx * np.fft.fftn(v[0]) + ky * np.fft.fftn(v[1]) + kz * np.fft.fftn(v[2])
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(np.fft.fftn(v[0])))


def test_gamma_rule():
    assert fields.gamma_for_grid((2048, 2048)) == 0.01
    assert fields.gamma_for_grid((256, 256)) == 0.1
    assert fields.gamma_for_grid((512, 512, 512)) == 0.01
    assert fields.gamma_for_grid((64, 64, 64)) == 0.1


def test_uneven_batch_sizes():
    shapes = fields.uneven_batch(0)
    assert len(shapes) == 48
    assert all(len(s) == 2 and 256 <= s[0] <= 4096 for s in shapes[:24])
    assert all(len(s) == 3 and 64 <= s[0] <= 384 for s in shapes[24:])
    ok = set(fields.smooth_sizes(64, 4096))
    assert all(s[0] in ok and s[0] % 4 == 0 for s in shapes)
    assert shapes == fields.uneven_batch(0) and shapes != fields.uneven_batch(1)


def test_velocity_torch_recipe_solenoidal_and_normalised():
    import torch
    v = fields.random_velocity_field_torch((24, 16, 32), 2, fields.spectrum_3d_kolmogorov, device="cpu")
    v = v.double().numpy()
    assert v.shape == (3, 24, 16, 32)
    assert abs(np.sqrt(np.mean(np.sum(v * v, axis=0))) - 1.0) < 1e-6
    kz, ky, kx = np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in (24, 16, 32)], indexing="ij")
    div = kx * np.fft.fftn(v[0]) + ky * np.fft.fftn(v[1]) + kz * np.fft.fftn(v[2])
    assert np.max(np.abs(div)) < 1e-5 * np.max(np.abs(np.fft.fftn(v[0])))
    w = fields.random_velocity_field_torch((24, 16, 32), 2, fields.spectrum_3d_kolmogorov, device="cpu")
    assert torch.equal(torch.from_numpy(v).float(), w)
