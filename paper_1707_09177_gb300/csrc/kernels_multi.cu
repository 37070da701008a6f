// float32 instantiation of the multi-group pass kernels (k_multi): one launch
// per pass stage over the blocks of several shape groups of a batched solve.
// A translation unit of its own so that it compiles in parallel with the
// single-group kernels.
#include <algorithm>

#include "launch.h"
#include "passes.cuh"

namespace gad {

constexpr size_t kMultiStaticSmemMargin = 4096;

template <typename T, int E, int KIND>
static cudaError_t launch_multi_k(int blocks, int threads, size_t smem, cudaStream_t s, const PassArgs<T>* args,
                                  const int* start, int ngroups) {
  if (smem + kMultiStaticSmemMargin > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_multi<T, E, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_multi<T, E, KIND><<<blocks, threads, smem, s>>>(args, start, ngroups);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t launch_multi_e(int kind, int blocks, int threads, size_t smem, cudaStream_t s,
                                  const PassArgs<T>* args, const int* start, int ngroups) {
  switch (kind) {
    case PK_XFWD: return launch_multi_k<T, E, 0>(blocks, threads, smem, s, args, start, ngroups);
    case PK_XINV: return launch_multi_k<T, E, 1>(blocks, threads, smem, s, args, start, ngroups);
    case PK_FILT: return launch_multi_k<T, E, 2>(blocks, threads, smem, s, args, start, ngroups);
    case PK_YFWD: return launch_multi_k<T, E, 3>(blocks, threads, smem, s, args, start, ngroups);
    case PK_YINV: return launch_multi_k<T, E, 4>(blocks, threads, smem, s, args, start, ngroups);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_multi(int kind, int E, int blocks, int threads, size_t smem, cudaStream_t s,
                         const PassArgs<T>* args, const int* start, int ngroups) {
  if (E == 16) return launch_multi_e<T, 16>(kind, blocks, threads, smem, s, args, start, ngroups);
  if (E == 24) return launch_multi_e<T, 24>(kind, blocks, threads, smem, s, args, start, ngroups);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_multi<float>(int, int, int, int, size_t, cudaStream_t, const PassArgs<float>*, const int*,
                                         int);

}  // namespace gad
