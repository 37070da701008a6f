// Statistics of deconvolved fields: the shell-summed energy spectrum, value
// histograms (PDFs) and the vorticity by spectral differentiation -- the
// assessments the paper makes of recovered fields (energy spectra and PDFs of
// vorticity, Sections 4.1 and 4.2).
//
// The spectrum and the curl read half spectra in the layout of the last-axis
// transform (2D [kx][ky], 3D [kx][ky][kz], unscaled forward transforms).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace gad {

// Signed wavenumber of FFT index i on an axis of n points.
__device__ __forceinline__ int signed_k(int i, int n) { return i < (n >> 1) ? i : i - n; }

// Shell index of an integer wavevector with |k|^2 = m: the nearest integer
// to sqrt(m), halves rounded down, i.e. the smallest k >= 0 with k^2 + k >= m.
__device__ __forceinline__ int shell_of(long long m) {
  long long k = (long long)sqrt((double)m);
  while (k * k + k < m) ++k;
  while (k > 0 && (k - 1) * (k - 1) + (k - 1) >= m) --k;
  return (int)k;
}

// E[g][k] += |X|^2 w(kx) / (2 P^2) over the half spectrum X of field f
// (g = f / ncomp), w = 1 on the kx = 0 and kx = nx/2 planes and 2 elsewhere
// (each stored coefficient stands for itself and its conjugate twin).
// Per-block shared-memory bins, then one atomic add per nonzero bin.
template <typename T>
__global__ void __launch_bounds__(256) k_shell(const typename cpx<T>::t* __restrict__ X, int nx, int ny, int nz,
                                               long long SP, int ncomp, int nbins, double scale, double* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* bins = reinterpret_cast<double*>(smem_raw);
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) bins[b] = 0.0;
  __syncthreads();
  const int f = blockIdx.y;
  const auto* Xf = X + (long long)f * SP;
  const int kxn = nx / 2 + 1;
  (void)kxn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < SP; i += (long long)gridDim.x * blockDim.x) {
    int kx, ky, kz = 0;
    if (nz > 1) {
      const long long seq = i / nz;
      kz = signed_k((int)(i - seq * nz), nz);
      kx = (int)(seq / ny);
      ky = signed_k((int)(seq - (long long)kx * ny), ny);
    } else {
      kx = (int)(i / ny);
      ky = signed_k((int)(i - (long long)kx * ny), ny);
    }
    const long long m = (long long)kx * kx + (long long)ky * ky + (long long)kz * kz;
    const int b = shell_of(m);
    if (b < nbins) {
      const auto x = Xf[i];
      const double w = (kx == 0 || 2 * kx == nx) ? 0.5 : 1.0;
      const double re = (double)x.x, im = (double)x.y;
      atomicAdd(&bins[b], w * (re * re + im * im) * scale);
    }
  }
  __syncthreads();
  double* og = out + (long long)(f / ncomp) * nbins;
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (bins[b] != 0.0) atomicAdd(&og[b], bins[b]);
}

__device__ __forceinline__ float hist_t(float x, float lo, float sc) { return __fmul_rn(__fsub_rn(x, lo), sc); }
__device__ __forceinline__ double hist_t(double x, double lo, double sc) { return __dmul_rn(__dsub_rn(x, lo), sc); }

// counts[0 .. nbins-1] per bin, counts[nbins] below, [nbins + 1] above,
// [nbins + 2] NaN: the bin of x is floor((x - lo) * scale), each operation
// rounded once in T.
template <typename T>
__global__ void __launch_bounds__(256) k_hist(const T* __restrict__ x, long long n, T lo, T scale, int nbins,
                                              unsigned long long* counts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned* bins = reinterpret_cast<unsigned*>(smem_raw);
  for (int b = threadIdx.x; b < nbins + 3; b += blockDim.x) bins[b] = 0u;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T t = hist_t(x[i], lo, scale);
    int b;
    if (t != t) b = nbins + 2;
    else {
      const T fl = floor(t);
      b = fl < T(0) ? nbins : (fl >= T(nbins) ? nbins + 1 : (int)fl);
    }
    atomicAdd(&bins[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins + 3; b += blockDim.x)
    if (bins[b]) atomicAdd(&counts[b], (unsigned long long)bins[b]);
}

// i k X for a wavenumber k (Nyquist index already mapped to 0 by the caller).
template <typename C> __device__ __forceinline__ C ikx(int k, C v) { return C{-k * v.y, k * v.x}; }

// Half spectra of the vorticity from those of the velocity, velocity v of
// the batch: 2D (ncomp = 2) omega_hat = i kx v_hat - i ky u_hat; 3D
// (ncomp = 3) omega_hat = i k x u_hat componentwise. Derivatives of the
// Nyquist index are zero. U: [v][ncomp][SP], W: [v][nout][SP].
template <typename T>
__global__ void __launch_bounds__(256) k_curl(const typename cpx<T>::t* __restrict__ U, typename cpx<T>::t* W, int nx,
                                              int ny, int nz, long long SP, int ncomp) {
  using C = typename cpx<T>::t;
  const int v = blockIdx.y;
  const int nout = ncomp == 2 ? 1 : 3;
  const C* u = U + (long long)v * ncomp * SP;
  C* w = W + (long long)v * nout * SP;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < SP; i += (long long)gridDim.x * blockDim.x) {
    int kx, ky, kz = 0;
    if (nz > 1) {
      const long long seq = i / nz;
      const int izi = (int)(i - seq * nz);
      kz = 2 * izi == nz ? 0 : signed_k(izi, nz);
      kx = (int)(seq / ny);
      const int iyi = (int)(seq - (long long)kx * ny);
      ky = 2 * iyi == ny ? 0 : signed_k(iyi, ny);
    } else {
      kx = (int)(i / ny);
      const int iyi = (int)(i - (long long)kx * ny);
      ky = 2 * iyi == ny ? 0 : signed_k(iyi, ny);
    }
    if (2 * kx == nx) kx = 0;
    if (ncomp == 2) {
      const C a = ikx(kx, u[SP + i]), b = ikx(ky, u[i]);
      w[i] = C{a.x - b.x, a.y - b.y};
    } else {
      const C ux = u[i], uy = u[SP + i], uz = u[2 * SP + i];
      C a = ikx(ky, uz), b = ikx(kz, uy);
      w[i] = C{a.x - b.x, a.y - b.y};
      a = ikx(kz, ux); b = ikx(kx, uz);
      w[SP + i] = C{a.x - b.x, a.y - b.y};
      a = ikx(kx, uy); b = ikx(ky, ux);
      w[2 * SP + i] = C{a.x - b.x, a.y - b.y};
    }
  }
}

}  // namespace gad
