// float32 instantiation of the pass kernels.
#define GAD_REAL float
#include "kernels_impl.cuh"

namespace gad {
cudaError_t launch_reset_state(FieldState* st, int batch, cudaStream_t s) {
  k_reset_state<<<(batch + 127) / 128, 128, 0, s>>>(st, batch);
  return cudaGetLastError();
}
}  // namespace gad
