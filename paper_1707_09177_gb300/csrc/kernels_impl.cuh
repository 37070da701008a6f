// Definition of the launchers for one precision; included by kernels_f32.cu
// and kernels_f64.cu with GAD_REAL set to float or double.
#pragma once

#include "launch.h"
#include "passes.cuh"
#include "spectral.cuh"

namespace gad {

template <typename T, int E>
static cudaError_t launch_pass_e(int kind, dim3 grid, int threads, size_t smem, cudaStream_t s,
                                 const PassArgs<T>& a) {
  void (*fn)(PassArgs<T>) = nullptr;
  switch (kind) {
    case PK_XFWD: fn = k_xfwd<T, E>; break;
    case PK_XINV: fn = k_xinv<T, E>; break;
    case PK_FILT: fn = k_filt<T, E>; break;
    case PK_YFWD: fn = k_yfwd<T, E>; break;
    case PK_YINV: fn = k_yinv<T, E>; break;
    case PK_LFWD: fn = k_lfwd<T, E>; break;
    case PK_LINV: fn = k_linv<T, E>; break;
    default: return cudaErrorInvalidValue;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pass(int kind, int E, dim3 grid, int threads, size_t smem, cudaStream_t s,
                        const PassArgs<T>& a) {
  if (kind == PK_SPEC) return launch_spec<T>(grid, s, a);
  if (E == 16) return launch_pass_e<T, 16>(kind, grid, threads, smem, s, a);
  if (E == 24) return launch_pass_e<T, 24>(kind, grid, threads, smem, s, a);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cg_finish(T* u, const T* p, const FieldState* st, long long P, int batch, cudaStream_t s) {
  const long long n4 = P / 4;
  int blocks = (int)((n4 + 255) / 256);
  if (blocks > 1184) blocks = 1184;   // 8 waves of 148-152 SMs are plenty for a single axpy
  if (blocks < 1) blocks = 1;
  k_cg_finish<T><<<dim3(blocks, batch), 256, 0, s>>>(u, p, st, P, batch);
  return cudaGetLastError();
}

template cudaError_t launch_pass<GAD_REAL>(int, int, dim3, int, size_t, cudaStream_t, const PassArgs<GAD_REAL>&);
template cudaError_t launch_cg_finish<GAD_REAL>(GAD_REAL*, const GAD_REAL*, const FieldState*, long long, int,
                                                cudaStream_t);

}  // namespace gad
