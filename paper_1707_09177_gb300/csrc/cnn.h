// Buffers and host drivers of the learned-guess network (cnn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace gad {

// float32 master weight layout (see cnn.cu)
constexpr int kW1 = 0;                       // [27][32]
constexpr int kW2 = kW1 + 27 * 32;           // [27][32][32]
constexpr int kW3 = kW2 + 27 * 32 * 32;      // [27][32][32]
constexpr int kW4 = kW3 + 27 * 32 * 32;      // [27][32]
constexpr int kCnnWeights = kW4 + 27 * 32;
constexpr int kSmallBlocks = 456;            // blocks of the 1-channel weight-gradient kernel (3 per SM)
constexpr int kWgradBlocks = 304;            // blocks of the 32x32 weight-gradient kernel

struct CnnBuffers {
  float* master = nullptr;     // weights
  float* m = nullptr;          // Adam moments
  float* v = nullptr;
  float* grad = nullptr;
  uint2* frag2 = nullptr;      // layer 2/3 weights in mma fragment order (forward)
  uint2* frag3 = nullptr;
  uint2* frag2t = nullptr;     // flipped, channel-swapped (backward data)
  uint2* frag3t = nullptr;
  uint2* frag4 = nullptr;      // layer 4 weights as one n8 tile (column 0) in mma fragment order
  __nv_bfloat16* H1 = nullptr; // activations [B][P][32]
  __nv_bfloat16* H2 = nullptr;
  __nv_bfloat16* H3 = nullptr;
  __nv_bfloat16* dA = nullptr; // gradient scratch [B][P][32]
  __nv_bfloat16* dB = nullptr;
  float* g = nullptr;          // dL/dy of the last layer [B][P]
  double* sumsq = nullptr;     // [B] sum u_bar^2, [B] sum u_true^2, [1] loss
  float* part = nullptr;       // weight-gradient partials
  __nv_bfloat16* umma2 = nullptr;   // layer 2/3 weights as tcgen05 B operands in shared-memory order (forward)
  __nv_bfloat16* umma3 = nullptr;
  __nv_bfloat16* umma2t = nullptr;  // flipped, channel-swapped (backward data)
  __nv_bfloat16* umma3t = nullptr;
  int* flag = nullptr;              // set to 1 by a tensor-core kernel whose bounded wait ran out
  unsigned long long wait_ns = 1000000000ull;   // limit of those waits
};

// floats of the weight-gradient partial buffer
constexpr long long kCnnPartFloats = (long long)kWgradBlocks * 27 * 32 * 32 > (long long)kSmallBlocks * 27 * 32
                                         ? (long long)kWgradBlocks * 27 * 32 * 32
                                         : (long long)kSmallBlocks * 27 * 32;

bool cnn_shape_ok(int X, int Y, int Z);
cudaError_t cnn_pack(const CnnBuffers& w, cudaStream_t s);
// ascale = A = 1/(pi gamma)^2, the fixed output scale
cudaError_t cnn_forward(const CnnBuffers& w, const float* ubar, float* u0, const float* utrue, int X, int Y, int Z,
                        int B, double ascale, cudaStream_t s);
cudaError_t cnn_backward(const CnnBuffers& w, const float* ubar, int X, int Y, int Z, int B, cudaStream_t s);
cudaError_t cnn_adam(const CnnBuffers& w, int step, float lr, cudaStream_t s);
// one forward 32 -> 32 layer H2 = ReLU(conv(H1, W2)) in inference's launch shape (timing)
cudaError_t cnn_conv_layer(const CnnBuffers& w, int X, int Y, int Z, int B, cudaStream_t s, bool* tensor_cores);

// 32 -> 32 layers on the tcgen05 tensor cores (conv_tc.cu): grids whose x side
// is a multiple of 128; others use the warp-level kernels of cnn.cu.
bool conv_tc_shape_ok(int X, int Y, int Z);
size_t conv_tc_image_bytes();
cudaError_t conv_tc_pack(const float* W, __nv_bfloat16* img, int transposed, cudaStream_t s);
// Hout = epilogue(conv(Hin, W)); mode 0: ReLU, mode 1: zero where Hmask <= 0
cudaError_t conv_tc_forward(const __nv_bfloat16* Hin, const __nv_bfloat16* Wimg, __nv_bfloat16* Hout,
                            const __nv_bfloat16* Hmask, int X, int Y, int Z, int B, int mode, int* flag,
                            unsigned long long wait_ns, cudaStream_t s);

}  // namespace gad
