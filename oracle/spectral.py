"""The paper's filter operator G, evaluated spectrally (Section 4, Eq. df and
Eq. df2). TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions followed here:
  * G = (I - delta^2 Laplacian)^{-1}, delta = 1/k_c, k_c = gamma * k_m
    (Section 4, Eq. df and the text after it);
  * k_m is the highest wavenumber the grid resolves. On a 2*pi-periodic grid
    of N points per side that is N/2; for a grid with unequal sides the
    smallest side sets it (reading: k_m = min_d N_d / 2);
  * transfer function G_hat(k) = 1 / (1 + (k/k_c)^2) (Eq. df2), where k is the
    Euclidean norm of the integer wavenumber vector (reading: corner modes of
    a 2D/3D grid have |k| > k_m, and the Nyquist index -N/2 enters squared);
  * the Laplacian is applied spectrally with a standard FFT, which the paper
    does to avoid discretisation error (Section 4).

Arrays are C-ordered with x last: (Ny, Nx) or (Nz, Ny, Nx). A leading batch
axis is not accepted here; callers loop over fields.
"""

from __future__ import annotations

import numpy as np


def wavenumber_grid(shape):
    """|k|^2 on the full FFT grid, integer wavenumbers k_d in [-N_d/2, N_d/2)."""
    axes = [np.fft.fftfreq(n, d=1.0 / n) for n in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    return sum(g * g for g in grids)


def cutoff_wavenumber(shape, gamma):
    """k_c = gamma * k_m with k_m = min(N)/2 (Section 4, text after Eq. df)."""
    k_m = min(int(n) for n in shape) / 2.0
    return gamma * k_m


def transfer_function(shape, gamma):
    """G_hat(k) = 1/(1 + (|k|/k_c)^2) on the full FFT grid (Eq. df2)."""
    kc = cutoff_wavenumber(shape, gamma)
    return 1.0 / (1.0 + wavenumber_grid(shape) / (kc * kc))


def filter_field(u, gamma):
    """u_bar = G u = F^{-1}[G_hat F u] (Eq. df evaluated spectrally)."""
    u = np.asarray(u, dtype=np.float64)
    gh = transfer_function(u.shape, gamma)
    return np.real(np.fft.ifftn(gh * np.fft.fftn(u)))


def exact_inverse(ubar, gamma):
    """u = G^{-1} u_bar = F^{-1}[(1 + |k|^2/k_c^2) F u_bar]: the solution of
    Eq. tau3 by Fourier division, possible because G is diagonal in Fourier
    space on a periodic grid."""
    ubar = np.asarray(ubar, dtype=np.float64)
    gh = transfer_function(ubar.shape, gamma)
    return np.real(np.fft.ifftn(np.fft.fftn(ubar) / gh))
