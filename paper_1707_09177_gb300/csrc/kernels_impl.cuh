// Definition of the launchers for one precision; included by kernels_f32.cu
// and kernels_f64.cu with GAD_REAL set to float or double.
#pragma once

#include <algorithm>

#include "launch.h"
#include "passes.cuh"
#include "spectral.cuh"
#include "stencil.cuh"
#include "stats.cuh"

namespace gad {

// Dynamic shared memory above 48 KB per block needs an opt-in; the kernels'
// static shared memory (reduction scratch, mbarrier: under 1 KB) counts
// against the same limit, so the opt-in is made with this margin.
constexpr size_t kStaticSmemMargin = 4096;

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
  if (smem + kStaticSmemMargin > 48 * 1024) {
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
  if (kind == PK_STEN) {
    if (smem + kStaticSmemMargin > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_sten<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_sten<T><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
  }
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

template <typename T>
cudaError_t launch_shell(const void* X, int nx, int ny, int nz, long long SP, int batch, int ncomp, int nbins,
                         double scale, double* out, cudaStream_t s) {
  const size_t smem = (size_t)nbins * sizeof(double);
  if (smem + kStaticSmemMargin > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_shell<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  long long bx = (SP + 1023) / 1024;
  bx = std::min<long long>(bx, std::max<long long>(1, (1216 + batch - 1) / batch));
  k_shell<T><<<dim3((unsigned)std::max<long long>(bx, 1), batch), 256, smem, s>>>(
      reinterpret_cast<const typename cpx<T>::t*>(X), nx, ny, nz, SP, ncomp, nbins, scale, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hist(const T* x, long long n, double lo, double scale, int nbins, unsigned long long* counts,
                        cudaStream_t s) {
  const size_t smem = (size_t)(nbins + 3) * sizeof(unsigned);
  if (smem + kStaticSmemMargin > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_hist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = std::max<long long>(1, std::min<long long>((n + 2047) / 2048, 1216));
  k_hist<T><<<(unsigned)blocks, 256, smem, s>>>(x, n, (T)lo, (T)scale, nbins, counts);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_curl(const void* U, void* W, int nx, int ny, int nz, long long SP, int nvel, int ncomp,
                        cudaStream_t s) {
  using C = typename cpx<T>::t;
  long long bx = (SP + 255) / 256;
  bx = std::min<long long>(bx, std::max<long long>(1, (4864 + nvel - 1) / nvel));
  k_curl<T><<<dim3((unsigned)std::max<long long>(bx, 1), nvel), 256, 0, s>>>(
      reinterpret_cast<const C*>(U), reinterpret_cast<C*>(W), nx, ny, nz, SP, ncomp);
  return cudaGetLastError();
}

template cudaError_t launch_shell<GAD_REAL>(const void*, int, int, int, long long, int, int, int, double, double*,
                                            cudaStream_t);
template cudaError_t launch_hist<GAD_REAL>(const GAD_REAL*, long long, double, double, int, unsigned long long*,
                                           cudaStream_t);
template cudaError_t launch_curl<GAD_REAL>(const void*, void*, int, int, int, long long, int, int, cudaStream_t);
template cudaError_t launch_pass<GAD_REAL>(int, int, dim3, int, size_t, cudaStream_t, const PassArgs<GAD_REAL>&);
template cudaError_t launch_cg_finish<GAD_REAL>(GAD_REAL*, const GAD_REAL*, const FieldState*, long long, int,
                                                cudaStream_t);

}  // namespace gad
