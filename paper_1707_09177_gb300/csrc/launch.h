// Host-side launchers for the pass kernels, instantiated per precision in
// kernels_f32.cu and kernels_f64.cu (compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "args.h"

namespace gad {

enum PassKind : int {
  PK_XFWD = 0, PK_XINV = 1, PK_FILT = 2, PK_YFWD = 3, PK_YINV = 4,
  PK_LFWD = 5,   // forward FFT along the last axis, S1 (2D) / S2 (3D) -> spectral vector O1
  PK_LINV = 6,   // inverse FFT along the last axis, spectral vector A (scaled by 1/P) -> S1 / S2
  PK_SPEC = 7,   // spectral-space Krylov pass (SpOp), 256 threads, no shared memory
  PK_STEN = 8,   // preconditioner z = M r with the dot (r, z), W rows per block (stencil.cuh)
};

// Launches pass `kind` with per-thread element count E (16 or 24). Returns the
// launch error (cudaSuccess when enqueued).
template <typename T>
cudaError_t launch_pass(int kind, int E, dim3 grid, int threads, size_t smem, cudaStream_t s,
                        const PassArgs<T>& a);

// One pass kind over several shape groups (k_multi): `args` (device) holds
// each group's PassArgs (vgx, vgy its own launch shape), `start` (device,
// ngroups + 1 entries) the first block of each group; blocks = start[ngroups].
template <typename T>
cudaError_t launch_multi(int kind, int E, int blocks, int threads, size_t smem, cudaStream_t s,
                         const PassArgs<T>* args, const int* start, int ngroups);

template <typename T>
cudaError_t launch_cg_finish(T* u, const T* p, const FieldState* st, long long P, int batch, cudaStream_t s);

cudaError_t launch_reset_state(FieldState* st, int batch, cudaStream_t s);

// Statistics (stats.cuh). X, U, W are half spectra of the field's precision.
template <typename T>
cudaError_t launch_shell(const void* X, int nx, int ny, int nz, long long SP, int batch, int ncomp, int nbins,
                         double scale, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_hist(const T* x, long long n, double lo, double scale, int nbins, unsigned long long* counts,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_curl(const void* U, void* W, int nx, int ny, int nz, long long SP, int nvel, int ncomp,
                        cudaStream_t s);

}  // namespace gad
