"""Random periodic fields with isotropic shell spectra (2D scalar, 3D solenoidal
velocity) on a 2*pi-periodic grid with integer wavenumbers.

Recipe (identical for every workload):
  1. draw white noise w ~ N(0, 1) on the grid with numpy's PCG64 generator
     seeded by ``seed``;
  2. shape it in Fourier space: u_hat = w_hat * A(|k|), A = sqrt(E(|k|)/S_d(|k|))
     with the shell area S_2 = 2 pi |k| (2D) or S_3 = 4 pi |k|^2 (3D), so that
     the expected shell spectrum of u is proportional to E; the mean (k = 0)
     is removed;
  3. (3D velocity only) draw the three components in turn from the same
     generator, project onto divergence-free fields,
     u_hat <- u_hat - k (k . u_hat) / |k|^2, and zero every Nyquist plane so that
     the discrete field is exactly solenoidal and Hermitian;
  4. transform back and scale to unit RMS (jointly over components).

The spectra stand in for the paper's DNS snapshots (2D Kraichnan turbulence
with a k^-3 inertial range, 3D Taylor-Green/Kolmogorov turbulence with a
k^-5/3 range), which are not available.

Arrays are C-ordered with x last: (Ny, Nx) in 2D and (Nz, Ny, Nx) in 3D.
"""

from __future__ import annotations

import math

import numpy as np


def spectrum_2d_kraichnan(k, kp=8.0, kcut=None):
    """E(k) ~ (k/kp)^4 / (1 + (k/kp)^2)^(7/2) [* exp(-(k/kcut)^2)]: k^4 at
    large scales, k^-3 in the inertial range."""
    k = np.asarray(k, dtype=np.float64)
    x = k / kp
    e = x ** 4 / (1.0 + x * x) ** 3.5
    if kcut is not None:
        e = e * np.exp(-(k / kcut) ** 2)
    return e


def spectrum_3d_kolmogorov(k, kp=4.0, kcut=100.0):
    """E(k) ~ (k/kp)^4 / (1 + (k/kp)^2)^(17/6) * exp(-(k/kcut)^2): k^4 at large
    scales, k^-5/3 in the inertial range."""
    k = np.asarray(k, dtype=np.float64)
    x = k / kp
    e = x ** 4 / (1.0 + x * x) ** (17.0 / 6.0)
    if kcut is not None:
        e = e * np.exp(-(k / kcut) ** 2)
    return e


def _half_grid_wavenumbers(shape):
    """Integer wavenumber arrays on the rfft half grid (last axis halved)."""
    axes = []
    for d, n in enumerate(shape):
        if d == len(shape) - 1:
            axes.append(np.fft.rfftfreq(n, d=1.0 / n))
        else:
            axes.append(np.fft.fftfreq(n, d=1.0 / n))
    return np.meshgrid(*axes, indexing="ij")


def _amplitude(kmag, ndim, spectrum):
    a = np.zeros_like(kmag)
    nz = kmag > 0
    shell = 2.0 * math.pi * kmag[nz] if ndim == 2 else 4.0 * math.pi * kmag[nz] ** 2
    a[nz] = np.sqrt(spectrum(kmag[nz]) / shell)
    return a


def random_scalar_field(shape, seed, spectrum):
    """One real field of the given shape with shell spectrum ~ ``spectrum``,
    zero mean and unit RMS (float64)."""
    shape = tuple(int(n) for n in shape)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    ks = _half_grid_wavenumbers(shape)
    kmag = np.sqrt(sum(k * k for k in ks))
    uh = np.fft.rfftn(w) * _amplitude(kmag, len(shape), spectrum)
    u = np.fft.irfftn(uh, s=shape, axes=tuple(range(len(shape))))
    u -= u.mean()
    return u / np.sqrt(np.mean(u * u))


def random_velocity_field(shape, seed, spectrum):
    """A 3-component solenoidal velocity on a 3D grid, shape (3, Nz, Ny, Nx),
    unit RMS over all components (float64)."""
    shape = tuple(int(n) for n in shape)
    assert len(shape) == 3
    rng = np.random.default_rng(seed)
    ks = _half_grid_wavenumbers(shape)          # (kz, ky, kx)
    k2 = sum(k * k for k in ks)
    kmag = np.sqrt(k2)
    amp = _amplitude(kmag, 3, spectrum)
    uh = [np.fft.rfftn(rng.standard_normal(shape)) * amp for _ in range(3)]
    # component order (u_x, u_y, u_z) pairs with wavenumbers (kx, ky, kz)
    kvec = (ks[2], ks[1], ks[0])
    safe = np.where(k2 > 0, k2, 1.0)
    kdotu = sum(kvec[i] * uh[i] for i in range(3))
    nyq = np.zeros(k2.shape, dtype=bool)
    for d, n in enumerate(shape):
        nyq |= np.abs(ks[d]) == n // 2
    out = np.empty((3,) + shape)
    for i in range(3):
        v = uh[i] - kvec[i] * kdotu / safe
        v[k2 == 0] = 0.0
        v[nyq] = 0.0
        out[i] = np.fft.irfftn(v, s=shape, axes=(0, 1, 2))
    return out / np.sqrt(np.mean(np.sum(out * out, axis=0)))


def shell_spectrum(u):
    """Shell-summed spectrum E(k) = 1/2 sum_{|k| in [k-1/2, k+1/2)} |u_hat/P|^2
    of one scalar field (used to check the generator)."""
    shape = u.shape
    p = float(np.prod(shape))
    uh = np.fft.fftn(u) / p
    axes = [np.fft.fftfreq(n, d=1.0 / n) for n in shape]
    kmag = np.sqrt(sum(k * k for k in np.meshgrid(*axes, indexing="ij")))
    shell = np.rint(kmag).astype(np.int64)
    e = np.bincount(shell.ravel(), weights=0.5 * np.abs(uh.ravel()) ** 2)
    return np.arange(e.size), e


def gamma_for_grid(shape):
    """Filter strength by grid size: the paper pairs gamma = 0.01 with its fine
    grids (2048^2, 512^3) and gamma = 0.1 with its coarse grids (256^2, 64^3);
    grids with any side >= 512 take 0.01, smaller ones 0.1."""
    return 0.01 if max(shape) >= 512 else 0.1


def smooth_sizes(lo, hi):
    """Even sides of the form 2^a 3^b (a >= 2, b <= 2) in [lo, hi]."""
    out = []
    for b in range(3):
        for a in range(2, 20):
            n = 2 ** a * 3 ** b
            if lo <= n <= hi:
                out.append(n)
    return sorted(out)


def uneven_batch(seed=0, n2d=24, n3d=24):
    """Grid shapes for a batch of uneven fields: sides drawn log-uniformly
    (numpy PCG64, `seed`) in [256, 4096] (2D) and [64, 384] (3D), each
    snapped to the nearest side in log space among smooth_sizes. Returns a
    list of shapes, 2D first, in draw order."""
    rng = np.random.default_rng(seed)
    shapes = []
    for count, lo, hi, nd in ((n2d, 256, 4096, 2), (n3d, 64, 384, 3)):
        cand = np.array(smooth_sizes(lo, hi), dtype=np.float64)
        for _ in range(count):
            x = np.exp(rng.uniform(np.log(lo), np.log(hi)))
            n = int(cand[np.argmin(np.abs(np.log(cand) - np.log(x)))])
            shapes.append((n,) * nd)
    return shapes


# Named workloads (shapes, spectra, filter strengths, solver settings).
WORKLOADS = {
    "vorticity2d_128_f64": dict(
        shape=(128, 128), batch=1, dtype="f64", gamma=0.1,
        spectrum=lambda k: spectrum_2d_kraichnan(k, kp=8.0, kcut=None),
        tol=1e-10, methods=("vancittert", "cg", "bicgstab")),
    "scalar2d_2048_f32_x16": dict(
        shape=(2048, 2048), batch=16, dtype="f32", gamma=0.01,
        spectrum=lambda k: spectrum_2d_kraichnan(k, kp=10.0, kcut=600.0),
        tol=1e-6, methods=("vancittert", "cg", "bicgstab")),
    "velocity3d_256_f32": dict(
        shape=(256, 256, 256), batch=3, dtype="f32", gamma=0.1,
        spectrum=lambda k: spectrum_3d_kolmogorov(k, kp=4.0, kcut=100.0),
        tol=1e-6, methods=("bicgstab",)),
    "velocity3d_512_f32": dict(
        shape=(512, 512, 512), batch=3, dtype="f32", gamma=0.01,
        spectrum=lambda k: spectrum_2d_kraichnan(k, kp=10.0, kcut=600.0),
        tol=1e-6, methods=("bicgstab",)),
}


def random_scalar_field_torch(shape, seed, spectrum, device="cuda"):
    """The recipe of random_scalar_field (white noise shaped to the shell
    spectrum, mean removed, unit RMS) evaluated with torch on a device, for
    benchmark inputs too large to draw on the host. Seeded by a torch
    generator, so the field differs from the NumPy one with the same seed."""
    import torch
    shape = tuple(int(n) for n in shape)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    w = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    axes = []
    for d, n in enumerate(shape):
        f = torch.fft.rfftfreq(n, d=1.0 / n) if d == len(shape) - 1 else torch.fft.fftfreq(n, d=1.0 / n)
        axes.append(f.to(device=device, dtype=torch.float64))
    k2 = None
    for d, f in enumerate(axes):
        view = [1] * len(shape)
        view[d] = -1
        t = f.reshape(view) ** 2
        k2 = t if k2 is None else k2 + t
    kmag = torch.sqrt(k2)
    shell = (2.0 * math.pi * kmag) if len(shape) == 2 else (4.0 * math.pi * kmag * kmag)
    e = torch.as_tensor(spectrum(kmag.cpu().numpy()), device=device)
    amp = torch.where(kmag > 0, torch.sqrt(e / torch.where(kmag > 0, shell, torch.ones_like(shell))),
                      torch.zeros_like(kmag))
    u = torch.fft.irfftn(torch.fft.rfftn(w) * amp, s=shape)
    u = u - u.mean()
    return (u / torch.sqrt(torch.mean(u * u))).float()


def random_velocity_field_torch(shape, seed, spectrum, device="cuda"):
    """The recipe of random_velocity_field (three white-noise components shaped
    to the shell spectrum, Leray projection, Nyquist planes zeroed, joint unit
    RMS) evaluated with torch on a device; float32 result (3, Nz, Ny, Nx).
    Seeded by a torch generator, so it differs from the NumPy field."""
    import torch
    shape = tuple(int(n) for n in shape)
    assert len(shape) == 3
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(device=device, dtype=torch.float64)
    kz = torch.fft.fftfreq(shape[0], d=1.0 / shape[0]).to(**f64).reshape(-1, 1, 1)
    ky = torch.fft.fftfreq(shape[1], d=1.0 / shape[1]).to(**f64).reshape(1, -1, 1)
    kx = torch.fft.rfftfreq(shape[2], d=1.0 / shape[2]).to(**f64).reshape(1, 1, -1)
    k2 = kz * kz + ky * ky + kx * kx
    kmag = torch.sqrt(k2)
    e = torch.as_tensor(spectrum(kmag.cpu().numpy()), device=device)
    amp = torch.where(kmag > 0, torch.sqrt(e / torch.where(kmag > 0, 4.0 * math.pi * k2, torch.ones_like(k2))),
                      torch.zeros_like(kmag))
    del e
    uh = [torch.fft.rfftn(torch.randn(shape, generator=g, **f64)) * amp for _ in range(3)]
    kvec = (kx, ky, kz)
    safe = torch.where(k2 > 0, k2, torch.ones_like(k2))
    kdotu = uh[0] * kx + uh[1] * ky + uh[2] * kz
    keep = (k2 > 0) & (kz.abs() != shape[0] // 2) & (ky.abs() != shape[1] // 2) & (kx.abs() != shape[2] // 2)
    out = torch.empty((3,) + shape, device=device, dtype=torch.float32)
    ss = 0.0
    for i in range(3):
        v = torch.where(keep, uh[i] - kvec[i] * kdotu / safe, torch.zeros_like(uh[i]))
        ui = torch.fft.irfftn(v, s=shape)
        ss += float(torch.sum(ui * ui))
        out[i] = ui.float()
        del v, ui
    return out / math.sqrt(ss / math.prod(shape))
