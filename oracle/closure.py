"""What the deconvolved field is for: the approximate-deconvolution closure
and the statistics the paper assesses it by. TEST INFRASTRUCTURE ONLY (see
the package docstring).

  closure_stress   -- the sub-filter stress of the structural model,
                      tau_ij = u_bar_i u_bar_j - G(u*_i u*_j): Eq. fge3,
                      tau_ij = u_bar_i u_bar_j - overline(u_i u_j), with the
                      unclosed product of unfiltered velocities replaced by the
                      deconvolved estimate u* (Section 3; with u* = u_bar it is
                      Eq. tau2, with the Van Cittert N = 2 estimate
                      u* = 2 u_bar - G u_bar the second-order form of Eq. tau3).
  energy_spectrum  -- the shell-summed kinetic energy spectrum E(k) (Sections
                      4.1 and 4.2 compare true, filtered and recovered spectra).
  histogram        -- bin counts of a field's values (the PDFs of Sections 4.1
                      and 4.2), with the bin decided in float32.
  curl             -- the vorticity of a velocity field by spectral
                      differentiation (the paper's PDFs and isosurfaces are of
                      vorticity).

Readings (the paper states none of these details):
  * Pairs are ordered (0,0), (0,1), ..., (0,d-1), (1,1), ..., (d-1,d-1), i <= j.
  * E(k) = sum over components and over wavevectors k' whose shell index is k
    of |u_hat(k')|^2 / 2, with u_hat = FFT(u) / P (Fourier coefficients, so
    sum_k E(k) = mean(|u|^2) / 2 by Parseval). The shell index of an integer
    wavevector with |k'|^2 = m is the nearest integer to sqrt(m), halves
    rounded down: the smallest k >= 0 with k^2 + k >= m (exact in integers).
  * Histogram: with lo and scale = nbins / (hi - lo) rounded to the data's
    precision (float32 for float32 fields), the bin of x is
    floor((x - lo) * scale) computed in that precision (each operation
    rounded once); bins < 0 count as "below", >= nbins as "above", NaN as
    "nan". The PDF is count / (n * (hi - lo) / nbins).
  * Spectral derivative: d/dx_d multiplies the Fourier coefficient by i k_d,
    with k_d = 0 at the Nyquist index N_d/2 (its derivative is not resolved).
"""

from __future__ import annotations

import numpy as np

from .spectral import filter_field, wavenumber_grid


def pair_list(ncomp):
    """(i, j) with i <= j in the order stated in the module docstring."""
    return [(i, j) for i in range(ncomp) for j in range(i, ncomp)]


def closure_stress(ubar, ustar, gamma):
    """tau[p] = ubar_i ubar_j - G(ustar_i ustar_j) for the p-th pair (i, j);
    ubar and ustar have shape (ncomp, *grid)."""
    ubar = np.asarray(ubar, dtype=np.float64)
    ustar = np.asarray(ustar, dtype=np.float64)
    return np.stack([ubar[i] * ubar[j] - filter_field(ustar[i] * ustar[j], gamma)
                     for i, j in pair_list(ubar.shape[0])])


def shell_index(m):
    """Smallest integer k >= 0 with k^2 + k >= m, elementwise for integer m >= 0."""
    m = np.asarray(m, dtype=np.int64)
    k = np.floor(np.sqrt(m.astype(np.float64))).astype(np.int64)
    k = np.where(k * k + k < m, k + 1, k)
    k = np.where((k > 0) & ((k - 1) * (k - 1) + (k - 1) >= m), k - 1, k)
    return k


def energy_spectrum(u, nbins):
    """E[k], k = 0 .. nbins-1, of u with shape (ncomp, *grid); wavevectors
    whose shell index is >= nbins are not counted."""
    u = np.asarray(u, dtype=np.float64)
    shape = u.shape[1:]
    P = float(np.prod(shape))
    m = np.rint(wavenumber_grid(shape)).astype(np.int64)
    k = shell_index(m).ravel()
    e = np.zeros(nbins)
    for c in range(u.shape[0]):
        uh = np.fft.fftn(u[c]) / P
        w = 0.5 * (uh.real ** 2 + uh.imag ** 2).ravel()
        keep = k < nbins
        e += np.bincount(k[keep], weights=w[keep], minlength=nbins)[:nbins]
    return e


def histogram(x, lo, hi, nbins, precision="f32"):
    """(counts[nbins], below, above, nan) with the bin rule evaluated in
    float32 (precision="f32") or float64 ("f64")."""
    dt = np.float32 if precision == "f32" else np.float64
    x = np.asarray(x, dtype=dt).ravel()
    lo_t = dt(lo)
    scale = dt(nbins / (float(hi) - float(lo)))
    t = (x - lo_t) * scale
    nan = np.isnan(t)
    b = np.floor(t[~nan])
    below = int(np.count_nonzero(b < 0))
    above = int(np.count_nonzero(b >= nbins))
    inside = b[(b >= 0) & (b < nbins)].astype(np.int64)
    return np.bincount(inside, minlength=nbins).astype(np.int64), below, above, int(np.count_nonzero(nan))


def _ik(shape, axis):
    """i k_d on the full FFT grid for array axis `axis` (Nyquist index -> 0)."""
    n = shape[axis]
    k = np.fft.fftfreq(n, d=1.0 / n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    sh = [1] * len(shape)
    sh[axis] = n
    return 1j * k.reshape(sh)


def derivative(f, axis):
    """d f / d x_axis on the 2*pi-periodic grid by FFT."""
    f = np.asarray(f, dtype=np.float64)
    return np.real(np.fft.ifftn(_ik(f.shape, axis) * np.fft.fftn(f)))


def curl(u):
    """Vorticity of u. 2D: u = (u_x, u_y) on (Ny, Nx) -> omega = dv/dx - du/dy
    (shape (1, Ny, Nx)). 3D: u = (u_x, u_y, u_z) on (Nz, Ny, Nx) -> (omega_x,
    omega_y, omega_z). Array axes: x = -1, y = -2, z = -3."""
    u = np.asarray(u, dtype=np.float64)
    nd = u.ndim - 1
    ax = {"x": nd - 1, "y": nd - 2, "z": nd - 3}
    if nd == 2:
        return np.stack([derivative(u[1], ax["x"]) - derivative(u[0], ax["y"])])
    return np.stack([derivative(u[2], ax["y"]) - derivative(u[1], ax["z"]),
                     derivative(u[0], ax["z"]) - derivative(u[2], ax["x"]),
                     derivative(u[1], ax["x"]) - derivative(u[0], ax["y"])])
